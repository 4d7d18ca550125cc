"""bec_relres_noalloc: the relative residual RES of Sec. 5 computed without any
device allocation, for callers that cannot allocate device memory when they
check a solution (memory owned by another allocator, a fixed budget, a
no-allocation-after-start-up rule, a nearly full device).

The entry point is called through the C ABI twice in a row on different
inputs and compared with the problem-based bec_true_relres; it keeps its
partial sums in a static device array shared by all calls, so the second call
also shows that nothing is left over from the first.  This file is collected
last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest

import oracle as O
from workloads import heat_case_2d

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def lib():
    from paper_2002_01108_gb300 import build
    build.build()
    from paper_2002_01108_gb300 import bec
    return bec.load()


def _noalloc(lib, case, f, u, out, stream):
    return lib.bec_relres_noalloc(case.dim, case.m, case.N, case.T, case.a,
                                  ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))


def test_relres_noalloc_matches_bec_true_relres_on_two_calls(lib):
    import torch
    from paper_2002_01108_gb300 import Problem
    case = heat_case_2d(seed=12, m=63, N=32, eps=0.1)
    f_np = O.build_rhs(case.u0, case.fsrc, case.tau)
    rng = np.random.default_rng(13)
    f = torch.from_numpy(f_np).cuda()
    # two different iterates: a perturbed solution and a random vector
    with Problem(case.dim, case.m, case.N, T=case.T) as p:
        p.set_eps(case.eps)
        sol, _ = p.gmres_solve(f, rtol=1e-6)
        u1 = sol + 1e-3 * torch.from_numpy(rng.standard_normal(f_np.shape)).cuda()
        u2 = torch.from_numpy(rng.standard_normal(f_np.shape)).cuda()
        stream = torch.cuda.current_stream()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        tol = 16 * U64 * math.log2(p.U)
        for u in (u1, u2):
            ref = p.true_relres(f, u)
            assert _noalloc(lib, case, f, u, out, stream) == 0, lib.bec_last_error()
            torch.cuda.synchronize()
            got = float(out.item())
            assert abs(got - ref) <= tol * ref, (got, ref)


def test_relres_noalloc_rejects_sizes_beyond_its_static_scratch(lib):
    import torch
    stream = torch.cuda.current_stream()
    f = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 1023^2 x 1024 needs far more than 16384 partial sums
    st = lib.bec_relres_noalloc(2, 1023, 1024, 1.0, 1.0, ctypes.c_void_p(f.data_ptr()),
                                ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(stream.cuda_stream))
    assert st == 1
    assert b"too large" in lib.bec_last_error()
    assert lib.bec_relres_noalloc(2, 100, 8, 1.0, 1.0, None, None, None, None) == 1
