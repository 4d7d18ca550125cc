"""Pins of the oracle's multigrid route (one V-cycle per shifted system,
Sec. 4 and Example 2 of Sec. 5) against independent facts: the bilinear
interpolant evaluated point by point, Galerkin consistency with -div(a grad)
on smooth functions, convergence of repeated V-cycles to a direct solve,
linearity, and the all-at-once solution by sequential stepping."""
import math

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O
from workloads import grf_log_coefficient, heat_case_2d


def test_prolongation_is_the_bilinear_interpolant():
    mc = 7
    mf = 2 * mc + 1
    rng = np.random.default_rng(0)
    c = rng.standard_normal((mc, mc))
    cz = np.zeros((mc + 2, mc + 2))          # with the zero boundary
    cz[1:-1, 1:-1] = c
    H = 1.0 / (mc + 1)
    fine = np.zeros((mf, mf))
    for iy in range(mf):
        for ix in range(mf):
            x, y = (ix + 1) / (mf + 1), (iy + 1) / (mf + 1)
            gx, gy = x / H, y / H
            jx, jy = int(math.floor(gx)), int(math.floor(gy))
            tx, ty = gx - jx, gy - jy
            fine[iy, ix] = ((1 - tx) * (1 - ty) * cz[jy, jx] + tx * (1 - ty) * cz[jy, jx + 1]
                            + (1 - tx) * ty * cz[jy + 1, jx] + tx * ty * cz[jy + 1, jx + 1])
    P = O.mg_prolongation(mc)
    np.testing.assert_allclose((P @ c.reshape(-1)).reshape(mf, mf), fine, atol=1e-14)


def test_restriction_is_full_weighting():
    P = O.mg_prolongation(7)
    R = (P.T / 4.0).tocsr()
    rows = np.asarray(R.sum(axis=1)).ravel()
    # an interior coarse point weighs its 3x3 fine neighbourhood 1/4, 1/8, 1/16
    assert abs(rows.reshape(7, 7)[3, 3] - 1.0) < 1e-15
    w = R[3 * 7 + 3].toarray().reshape(15, 15)
    assert w[7, 7] == 0.25 and w[7, 6] == 0.125 and w[6, 6] == 0.0625


@pytest.mark.parametrize("const_a", [True, False])
def test_galerkin_coarse_operators_are_consistent(const_a):
    """K_l = R K_{l-1} P stays a consistent discretisation of -div(a grad u),
    and M_l = R M_{l-1} P of the identity, on a smooth function."""
    m = 63
    if const_a:
        a_nodes = np.full((m + 2, m + 2), 2.0)
    else:
        xs = np.arange(m + 2) / (m + 1)
        X, Y = np.meshgrid(xs, xs)
        a_nodes = 1.0 + 0.5 * np.sin(np.pi * X) * np.cos(np.pi * Y)
    h = O.MGHierarchy(O.fd_stiffness_varcoef(a_nodes), m)
    for l in (1, 2):
        ml = h.sizes[l]
        xs = np.arange(1, ml + 1) / (ml + 1)
        X, Y = np.meshgrid(xs, xs)
        u = np.sin(np.pi * X) * np.sin(np.pi * Y)
        Mu = h.M[l] @ u.reshape(-1)
        Ku = h.K[l] @ u.reshape(-1)
        if const_a:
            exact = 2.0 * 2 * np.pi ** 2 * u
        else:
            a = 1.0 + 0.5 * np.sin(np.pi * X) * np.cos(np.pi * Y)
            ax = 0.5 * np.pi * np.cos(np.pi * X) * np.cos(np.pi * Y)
            ay = -0.5 * np.pi * np.sin(np.pi * X) * np.sin(np.pi * Y)
            ux = np.pi * np.cos(np.pi * X) * np.sin(np.pi * Y)
            uy = np.pi * np.sin(np.pi * X) * np.cos(np.pi * Y)
            exact = -(ax * ux + ay * uy) + a * 2 * np.pi ** 2 * u
        inner = (slice(2, -2), slice(2, -2))
        relK = np.abs(Ku.reshape(ml, ml) - exact)[inner].max() / np.abs(exact).max()
        relM = np.abs(Mu.reshape(ml, ml) - u)[inner].max()
        assert relK < 0.02 * 4 ** l and relM < 0.01 * 4 ** l, (l, relK, relM)
        assert abs(h.K[l] - h.K[l].T).max() < 1e-9 * abs(h.K[l]).max()


@pytest.mark.parametrize("eps,k", [(0.0625, 0), (0.0625, 16), (1.0, 0), (1e-4, 32)])
def test_repeated_vcycles_converge_to_the_direct_solve(eps, k):
    m, N = 31, 64
    a = O.node_coefficient(grf_log_coefficient(seed=5, m=m))
    h = O.MGHierarchy(O.fd_stiffness_varcoef(a), m)
    tau = 1.0 / N
    lam = O.eps_circulant_eigs(N, eps)[k]
    rng = np.random.default_rng(1)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    xs = spla.spsolve(h.op(0, lam, tau).tocsc(), b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(12):
        x = O.mg_vcycle(h, lam, tau, b, x0=x)
        errs.append(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    assert errs[-1] < 1e-5
    assert (errs[-1] / errs[1]) ** (1 / 10) < 0.6


def test_vcycle_is_linear():
    m = 15
    a = O.node_coefficient(grf_log_coefficient(seed=2, m=m))
    h = O.MGHierarchy(O.fd_stiffness_varcoef(a), m)
    rng = np.random.default_rng(2)
    b1, b2 = rng.standard_normal((2, m * m))
    lam = 0.3 - 0.2j
    lhs = O.mg_vcycle(h, lam, 0.1, 2.0 * b1 - 3.0 * b2)
    rhs = 2.0 * O.mg_vcycle(h, lam, 0.1, b1) - 3.0 * O.mg_vcycle(h, lam, 0.1, b2)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-14)


def test_fgmres_with_multigrid_preconditioner_reaches_the_solution():
    m, N = 31, 32
    a = O.node_coefficient(grf_log_coefficient(seed=5, m=m))
    K = O.fd_stiffness_varcoef(a)
    M = sp.identity(K.shape[0], format="csr")
    h = O.MGHierarchy(K, m)
    tau = 1.0 / N
    eps = math.sqrt(tau) / 2
    case = heat_case_2d(seed=6, m=m, N=N, eps=eps)
    f = O.build_rhs(case.u0, case.fsrc, tau)
    L = O.assemble_L(N, M, K, tau)
    Minv = lambda v: O.apply_Pinv_mg(v.reshape(N, m, m), h, tau, eps).reshape(-1)
    u, info = O.fgmres(lambda v: L @ v, f.reshape(-1), Minv, restart=30, tol=1e-10)
    assert info["converged"] and info["iters"] <= 20
    uref = O.timestep_solve(f, M, K, tau)
    assert np.linalg.norm(u - uref.reshape(-1)) / np.linalg.norm(uref) < 1e-8
