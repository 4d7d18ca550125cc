"""Convection-diffusion (Example 3 of Sec. 5: nu = 1/200, the circulating
wind on (-1, 1)^2, the hot wall) on the multigrid route with the ILU
smoother, against the oracle: the operator L with the upwind convection,
the right-hand side with the wall data, P_eps^{-1} with one ILU-smoothed
V-cycle per frequency element by element, and FGMRES reaching the
sequential-stepping solution.

Tolerance of the P_eps^{-1} parity: the transforms contribute
16 u log2(N n^2) / eps as on the other routes, each of the L levels O(1)
stable passes (16 u 8 L / eps, as for damped Jacobi), and the two triangular
recurrences of each ILU step run over 3 (m - 1) + 1 wavefronts of a
diagonally dominant factor, adding at most 16 u 6 m / eps."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import circulating_wind_case

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53
U32 = 2.0 ** -24
NU = 1.0 / 200.0


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


def problem(m, N, wind, precision="fp64", **kw):
    from paper_2002_01108_gb300 import Problem
    return Problem(2, m, N, a=NU, route="mg", precision=precision, wind=wind, side=2.0,
                   mg_smoother="ilu", flexible=True, **kw)


def max_rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def levels(m):
    n = 1
    while m > 1:
        m = (m - 1) // 2
        n += 1
    return n


@pytest.mark.parametrize("m,N", [(31, 8), (63, 16)])
def test_convection_apply_A_matches_assembled_L(m, N):
    wind, _, _, _ = circulating_wind_case(m, N)
    K, _ = O.fd_convection_diffusion(NU, wind)
    tau = 1.0 / N
    v = np.random.default_rng(70 + m).uniform(-1, 1, (N, m, m))
    with problem(m, N, wind) as p:
        y = host(p.apply_A(dev(v)))
    I = sp.identity(m * m, format="csr")
    ref = (O.assemble_L(N, I, K, tau) @ v.reshape(-1)).reshape(v.shape)
    wsum = abs(I + tau * K).sum(axis=1).max() + 1.0
    assert np.max(np.abs(y - ref)) <= 8 * U64 * wsum * np.max(np.abs(v))


def test_convection_right_hand_side_with_wall_data():
    m, N = 31, 8
    wind, g, _, fs = circulating_wind_case(m, N)
    rng = np.random.default_rng(71)
    u0 = rng.uniform(-1, 1, (m, m))
    fs = rng.uniform(-1, 1, (N, m, m))
    K, Kb = O.fd_convection_diffusion(NU, wind)
    ref = O.build_rhs_dirichlet(u0, fs, g, 1.0 / N, Kb)
    with problem(m, N, wind) as p:
        f = host(p.build_rhs_dirichlet(dev(u0), dev(fs), dev(g)))
    assert np.max(np.abs(f - ref)) <= 16 * U64 * np.max(np.abs(ref)) * 4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("m,N,eps", [(31, 16, 0.05), (63, 8, 0.0625)])
def test_ilu_multigrid_apply_Pinv_matches_oracle(precision, m, N, eps):
    wind, _, _, _ = circulating_wind_case(m, N)
    K, _ = O.fd_convection_diffusion(NU, wind)
    tau = 1.0 / N
    y = np.random.default_rng(72).uniform(-1, 1, (N, m, m))
    with problem(m, N, wind, precision) as p:
        p.set_eps(eps)
        z = host(p.apply_Pinv(dev(y)))
    ref = O.apply_Pinv_mg(y, O.MGHierarchy(K, m), tau, eps, smoother="ilu")
    u = U64 if precision == "fp64" else U32
    tol = 16 * u * (math.log2(N * (m + 1) ** 2) + 8 * levels(m) + 6 * m) / eps
    err = max_rel(z, ref)
    assert err <= tol, (err, tol)
    if precision == "fp32":
        assert err > 1e-12          # the FP32 V-cycle really ran in single precision


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_convection_fgmres_reaches_the_stepping_solution(precision):
    """Example 3 (hot wall, u0 = 0, eps = min(0.5, 0.5 tau)) at m = 63, N = 32:
    FGMRES with the ILU multigrid preconditioner reaches the backward-Euler
    solution in few iterations."""
    m, N = 63, 32
    tau = 1.0 / N
    wind, g, u0, fs = circulating_wind_case(m, N)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    f = O.build_rhs_dirichlet(u0, fs, g, tau, Kb)
    ref = O.timestep_solve(f, sp.identity(m * m, format="csr"), K, tau)
    with problem(m, N, wind, precision) as p:
        p.set_eps(min(0.5, 0.5 * tau))
        fd = p.build_rhs_dirichlet(dev(u0), dev(fs), dev(g))
        u, info = p.gmres_solve(fd, restart=30, rtol=1e-10, flexible=True)
        u = host(u)
    print(f"convection-diffusion m={m} N={N} {precision}: {info['iters']} FGMRES iterations, "
          f"RES {info['true_relres']:.2e}")
    assert info["converged"] == 1 and info["true_relres"] <= 1e-10 * (1 + 1e-6)
    assert float(np.linalg.norm(u - ref) / np.linalg.norm(ref)) <= 1e-7
    assert info["iters"] <= 12, info


def test_convection_at_the_workload_size():
    """Example 3 at the size bench.py times (255^2 x 256, FP32 ILU multigrid,
    FGMRES(30) to RES 1e-8): converged in at most 10 iterations and equal to
    sequential stepping."""
    m, N = 255, 256
    tau = 1.0 / N
    wind, g, u0, fs = circulating_wind_case(m, N)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    f = O.build_rhs_dirichlet(u0, fs, g, tau, Kb)
    ref = O.timestep_solve(f, sp.identity(m * m, format="csr"), K, tau)
    with problem(m, N, wind, "fp32") as p:
        p.set_eps(min(0.5, 0.5 * tau))
        fd = p.build_rhs_dirichlet(dev(u0), dev(fs), dev(g))
        assert max_rel(host(fd), f) <= 64 * U64
        u, info = p.gmres_solve(fd, restart=30, rtol=1e-8, flexible=True)
        u = host(u)
    assert info["converged"] == 1 and info["true_relres"] <= 1.01e-8 and info["iters"] <= 10, info
    assert float(np.linalg.norm(u - ref) / np.linalg.norm(ref)) <= 1e-5
