"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every entry point include/bec.h declares, and rejects invalid arguments before
any CUDA call."""
import ctypes
import os
import re

import pytest

from paper_2002_01108_gb300 import build as bec_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    bec_build.build()
    from paper_2002_01108_gb300 import bec
    return bec.load()


def _declared():
    text = open(os.path.join(ROOT, "include", "bec.h")).read()
    return set(re.findall(r"^(?:bec_status|long long|const char\*)\s+(bec_\w+)\s*\(", text, re.M))


def test_header_declares_the_documented_entry_points():
    names = _declared()
    for core in ("bec_allocate_problem", "bec_set_eps", "bec_apply_A", "bec_apply_Pinv",
                 "bec_gmres_solve"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2002_01108_gb300 import bec
    names = _declared()
    assert names == set(bec.EXPORTED)
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.bec_status_string(0) == b"BEC_OK"
    assert lib.bec_status_string(1) == b"BEC_EINVAL"
    assert lib.bec_status_string(4) == b"BEC_ENOTCONV"
    assert lib.bec_status_string(99) == b"BEC_UNKNOWN"


@pytest.mark.parametrize("field,value", [
    ("dim", 4), ("nx", 254), ("nx", 2), ("nx", 2047), ("N", 100), ("N", 1), ("N", 2048),
    ("T", 0.0), ("T", float("nan")), ("a", -1.0), ("precision", 7), ("max_restart", 61),
])
def test_allocate_rejects_invalid_descriptions(lib, field, value):
    from paper_2002_01108_gb300.bec import ProblemDesc
    d = ProblemDesc(2, 63, 63, 64, 1.0, 1.0, 0, 0, 10, 0, 0)
    setattr(d, field, value)
    out = ctypes.c_void_p()
    st = lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out))
    assert st == 1, (field, value, lib.bec_last_error())
    assert out.value is None
    assert lib.bec_last_error() != b""


def test_allocate_rejects_mismatched_ny_and_unknown_route(lib):
    from paper_2002_01108_gb300.bec import ProblemDesc
    out = ctypes.c_void_p()
    d = ProblemDesc(2, 63, 31, 64, 1.0, 1.0, 0, 0, 10, 0, 0)
    assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1
    d = ProblemDesc(2, 63, 63, 64, 1.0, 1.0, 5, 0, 10, 0, 0)
    assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1


def test_allocate_rejects_invalid_multigrid_requests(lib):
    import numpy as np
    from paper_2002_01108_gb300.bec import ProblemDesc
    out = ctypes.c_void_p()
    a = np.ones(65 * 65)
    # a variable coefficient needs the multigrid route
    d = ProblemDesc(2, 63, 63, 64, 1.0, 1.0, 0, 0, 10, 0, 0, a.ctypes.data)
    assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1
    # the multigrid route is 2D, N <= 512, omega in [0, 2), sweeps in [0, 8]
    for dim, N, pre, omega in ((1, 64, 0, 0.0), (2, 1024, 0, 0.0), (2, 64, 9, 0.0), (2, 64, 0, 2.5)):
        d = ProblemDesc(dim, 63, 63, N, 1.0, 1.0, 1, 0, 10, 0, 0, None, pre, 0, omega)
        assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1, (dim, N, pre, omega)


def test_allocate_rejects_invalid_space_requests(lib):
    from paper_2002_01108_gb300.bec import ProblemDesc
    out = ctypes.c_void_p()
    # an unknown discretisation, and Q1 elements off the sine-transform route
    for route, space in ((0, 2), (0, -1), (1, 1), (2, 1)):
        d = ProblemDesc(2, 63, 63, 64, 1.0, 1.0, route, 1 if route == 2 else 0, 10, 0, 0, None,
                        0, 0, 0.0, 0, 0, space)
        assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1, (route, space)
        assert out.value is None


def test_allocate_rejects_invalid_time_schemes(lib):
    from paper_2002_01108_gb300.bec import ProblemDesc
    out = ctypes.c_void_p()
    # an unknown scheme; BDF2 off the sine-transform route, in 3D, or with N < 4
    for dim, N, route, scheme in ((2, 64, 0, 2), (2, 64, 0, -1), (2, 64, 1, 1), (3, 64, 0, 1),
                                  (2, 2, 0, 1)):
        d = ProblemDesc(dim, 63, 63, N, 1.0, 1.0, route, 0, 10, 0, 0, None,
                        0, 0, 0.0, 0, 0, 0, scheme)
        assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1, (dim, N, scheme)
        assert out.value is None
        assert b"BDF2" in lib.bec_last_error() or b"time_scheme" in lib.bec_last_error()


def test_allocate_rejects_invalid_convection_requests(lib):
    import numpy as np
    from paper_2002_01108_gb300.bec import ProblemDesc
    out = ctypes.c_void_p()
    w = np.zeros(2 * 65 * 65)
    # a wind, a side length or the ILU smoother off the multigrid route; an
    # unknown smoother; a negative side
    for route, wind, side, smoother in ((0, w.ctypes.data, 0.0, 0), (0, None, 2.0, 0),
                                        (0, None, 0.0, 1), (1, None, 0.0, 5), (1, None, -1.0, 0),
                                        (2, None, 0.0, 1)):
        d = ProblemDesc(2, 63, 63, 64, 1.0, 1.0, route, 1 if route == 2 else 0, 10, 0, 0, None,
                        0, 0, 0.0, 0, 0, 0, 0, wind, side, smoother)
        assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1, (route, side)
        assert out.value is None
    # the FP64 ILU smoother stages its operands in shared memory: nx <= 511
    d = ProblemDesc(2, 1023, 1023, 64, 1.0, 1.0, 1, 0, 10, 0, 0, None,
                    0, 0, 0.0, 0, 0, 0, 0, None, 0.0, 1)
    assert lib.bec_allocate_problem(ctypes.byref(d), None, ctypes.byref(out)) == 1
    assert b"511" in lib.bec_last_error()


def test_null_arguments_are_rejected(lib):
    assert lib.bec_set_eps(None, 0.5) == 1
    assert lib.bec_build_rhs_dirichlet(None, None, None, None, None) == 1
    assert lib.bec_apply_A(None, None, None) == 1
    assert lib.bec_apply_Pinv(None, None, None) == 1
    assert lib.bec_gmres_solve(None, None, None, None, None) == 1
    assert lib.bec_free_problem(None) == 0
    assert lib.bec_problem_size(None) == 0
    assert lib.bec_allocate_problem(None, None, None) == 1
