"""bec_relres_noalloc: the relative residual RES of Sec. 5 computed without any
device allocation, for callers that cannot allocate device memory when they
check a solution (memory owned by another allocator, a fixed budget, a
no-allocation-after-start-up rule, a nearly full device).

The entry point keeps its block partial sums in one static device array that
every call shares.  The calls below run back to back on different
geometries: first a large 2D problem (2040 partial sums), then a small 2D one
(64) and a 1D one (8), so a later call reads only slots that an earlier,
larger call also wrote.  Every result is compared with the oracle's RES of
the assembled all-at-once matrix and with the problem-based bec_true_relres.
This file is collected last on purpose: a run that stops at the first
failure has then already run every other test.
"""
import ctypes
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import heat_case_1d, heat_case_2d

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


def test_relres_noalloc_matches_the_oracle_and_bec_true_relres_on_calls_in_a_row(lib):
    """Large 2D, small 2D, then 1D; two iterates each (a perturbed solution and
    a random vector), so the static array is reused by six calls in a row.
    Tolerance: 16 u log2(U) relative, the rounding of two FP64 sums of U
    squares in a fixed order plus the stencil's few operations per term."""
    import torch
    from paper_2002_01108_gb300 import Problem
    cases = [heat_case_2d(seed=21, m=255, N=64, eps=0.1),
             heat_case_2d(seed=12, m=63, N=32, eps=0.1),
             heat_case_1d(seed=13, m=63, N=64)]
    rng = np.random.default_rng(13)
    stream = torch.cuda.current_stream()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for case in cases:
        f_np = O.build_rhs(case.u0, case.fsrc, case.tau)
        K = O.fd_stiffness(case.dim, case.m, case.a)
        L = O.assemble_L(case.N, sp.identity(K.shape[0], format="csr"), K, case.tau)
        u_sol = O.timestep_solve(f_np, sp.identity(K.shape[0], format="csr"), K, case.tau)
        f = torch.from_numpy(f_np).cuda()
        iterates = [u_sol + 1e-3 * rng.standard_normal(f_np.shape), rng.standard_normal(f_np.shape)]
        with Problem(case.dim, case.m, case.N, T=case.T, max_restart=2) as p:
            tol = 16 * U64 * math.log2(p.U)
            for u_np in iterates:
                u = torch.from_numpy(u_np).cuda()
                ref = O.relative_residual(L, u_np, f_np)
                lib_ref = p.true_relres(f, u)
                out.fill_(float("nan"))
                assert _noalloc(lib, case, f, u, out, stream) == 0, lib.bec_last_error()
                torch.cuda.synchronize()
                got = float(out.item())
                assert abs(got - ref) <= tol * ref, (case.name, got, ref)
                assert abs(got - lib_ref) <= tol * ref, (case.name, got, lib_ref)


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
    # dim 3 is outside the operator it covers
    assert lib.bec_relres_noalloc(3, 7, 8, 1.0, 1.0, ctypes.c_void_p(f.data_ptr()),
                                  ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream.cuda_stream)) == 1
