"""The multigrid route on the GPU (variable coefficient a = exp(g), g a
Gaussian random field) against the oracle: the variable-coefficient operator
L, one V-cycle per shifted system inside P_eps^{-1} (same algorithm as the
oracle's: bilinear prolongation, full weighting, Galerkin coarse operators,
damped Jacobi), and FGMRES reaching the sequential-stepping solution.

Tolerance of the V-cycle parity: the transforms contribute 16 u log2(N n^2)
/ eps as on the sine-transform route; each of the L levels adds O(1) stable
operations (smoothing, residual, transfers) whose rounding is amplified by at
most the same 1/eps, so the bound used is 16 u (log2(N n^2) + 8 L) / eps."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import grf_log_coefficient, heat_case_2d

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2002_01108_gb300 import build
    build.build()


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def setup(m, seed=5):
    a = O.node_coefficient(grf_log_coefficient(seed=seed, m=m))
    K = O.fd_stiffness_varcoef(a)
    return a, K, sp.identity(K.shape[0], format="csr")


def levels(m):
    return int(math.log2(m + 1))


def tol(eps, N, m, unit):
    return 16 * unit * (math.log2(N * (m + 1) ** 2) + 8 * levels(m)) / eps


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("m,N", [(15, 8), (63, 32)])
def test_apply_A_variable_coefficient(m, N):
    from paper_2002_01108_gb300 import Problem
    a, K, M = setup(m)
    v = np.random.default_rng(3).uniform(-1, 1, (N, m, m))
    with Problem(2, m, N, route="mg", a_nodes=a) as p:
        y = host(p.apply_A(dev(v)))
    ref = (O.assemble_L(N, M, K, 1.0 / N) @ v.reshape(-1)).reshape(v.shape)
    kmax = abs(K).max() / N
    assert np.max(np.abs(y - ref)) <= 16 * U64 * (1 + 4 * kmax) * np.max(np.abs(v))


@pytest.mark.parametrize("m,N,eps,pre,post", [(31, 16, 0.0625, 1, 1), (63, 32, 1.0, 1, 1),
                                              (63, 32, 1e-3, 1, 1), (31, 8, 0.2, 2, 3),
                                              (127, 4, 0.5, 1, 1)])
def test_mg_apply_Pinv_fp64_matches_oracle_vcycle(m, N, eps, pre, post):
    from paper_2002_01108_gb300 import Problem
    a, K, M = setup(m)
    h = O.MGHierarchy(K, m)
    y = np.random.default_rng(4).uniform(-1, 1, (N, m, m))
    with Problem(2, m, N, route="mg", a_nodes=a, mg_pre=pre, mg_post=post) as p:
        p.set_eps(eps)
        z = host(p.apply_Pinv(dev(y)))
    ref = O.apply_Pinv_mg(y, h, 1.0 / N, eps, nu1=pre, nu2=post)
    assert max_rel(z, ref) <= tol(eps, N, m, U64)


@pytest.mark.parametrize("m,N,eps", [(31, 16, 0.0625), (63, 32, 0.01)])
def test_mg_apply_Pinv_fp32_within_single_precision_bound(m, N, eps):
    from paper_2002_01108_gb300 import Problem
    a, K, M = setup(m)
    h = O.MGHierarchy(K, m)
    y = np.random.default_rng(5).uniform(-1, 1, (N, m, m))
    with Problem(2, m, N, route="mg", a_nodes=a, precision="fp32") as p:
        p.set_eps(eps)
        z = host(p.apply_Pinv(dev(y)))
    ref = O.apply_Pinv_mg(y, h, 1.0 / N, eps)
    err = max_rel(z, ref)
    assert 1e-12 < err <= tol(eps, N, m, U32)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mg_fgmres_reaches_time_stepping_solution(precision):
    from paper_2002_01108_gb300 import Problem
    m, N = 63, 32
    a, K, M = setup(m)
    case = heat_case_2d(seed=6, m=m, N=N, eps=math.sqrt(1.0 / N) / 2)
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    u_ref = O.timestep_solve(f, M, K, case.tau)
    with Problem(2, m, N, route="mg", a_nodes=a, precision=precision, flexible=True) as p:
        p.set_eps(case.eps)
        u, info = p.gmres_solve(dev(f), restart=30, rtol=1e-8, flexible=True)
        assert info["converged"] == 1 and info["true_relres"] <= 1.01e-8 and info["iters"] <= 20
        u, info = p.gmres_solve(dev(f), restart=30, rtol=1e-11, flexible=True)
        err = float(np.linalg.norm(host(u) - u_ref) / np.linalg.norm(u_ref))
    assert err <= 1e-8


def test_mg_route_with_constant_coefficient_matches_fst_solution():
    """With a constant a both routes solve the same L u = f."""
    from paper_2002_01108_gb300 import Problem
    m, N = 31, 16
    case = heat_case_2d(seed=7, m=m, N=N, eps=0.1)
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    sols = []
    for route in ("fst", "mg"):
        with Problem(2, m, N, route=route, flexible=True) as p:
            p.set_eps(case.eps)
            u, info = p.gmres_solve(dev(f), rtol=1e-12, flexible=True)
            sols.append(host(u))
    assert np.linalg.norm(sols[0] - sols[1]) / np.linalg.norm(sols[0]) < 1e-10


def test_mg_grf_255_N256_workload():
    """The variable-coefficient workload: 255^2 grid, N = 256, a = exp(GRF,
    l = 0.1, sigma = 1), eps = sqrt(tau)/2, FP32 multigrid preconditioner in
    FP64 FGMRES reaching RES <= 1e-8."""
    from paper_2002_01108_gb300 import Problem
    m, N = 255, 256
    a = O.node_coefficient(grf_log_coefficient(seed=5, m=m))
    case = heat_case_2d(seed=6, m=m, N=N, eps=math.sqrt(1.0 / N) / 2)
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    for precision in ("fp32", "fp64"):
        with Problem(2, m, N, route="mg", a_nodes=a, precision=precision, flexible=True) as p:
            p.set_eps(case.eps)
            u, info = p.gmres_solve(dev(f), restart=30, rtol=1e-8, flexible=True)
            assert info["converged"] == 1 and info["true_relres"] <= 1.01e-8, info
            assert info["iters"] <= 25, info
