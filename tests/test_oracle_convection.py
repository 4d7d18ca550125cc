"""Pins of the oracle's convection-diffusion operator (Example 3 of Sec. 5:
-nu Lap u + w . grad u with the circulating wind on (-1, 1)^2, here by
central diffusion and first-order upwind convection) against facts that do
not depend on how it is assembled: the pure-diffusion case, exactness on
constants and linear functions, the upwind (not downwind) first-order error
on x^2 and y^2, the sign pattern of an M-matrix, the steady state of the
all-at-once system with constant wall data, and the contraction of the
multigrid V-cycle on its shifted systems."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle as O
from workloads import circulating_wind_case

NU = 1.0 / 200.0


def _nodes(m, side=2.0):
    s = -side / 2 + side * np.arange(m + 2) / (m + 1)
    X, Y = np.meshgrid(s, s)
    return X, Y


def _apply_full(K, Kb, u_nodes):
    """Rows of the operator at the interior nodes for a field given on all nodes."""
    m = u_nodes.shape[0] - 2
    return (K @ u_nodes[1:-1, 1:-1].reshape(-1) + Kb @ u_nodes.reshape(-1)).reshape(m, m)


def test_zero_wind_is_the_scaled_laplacian():
    m = 7
    K, Kb = O.fd_convection_diffusion(NU, np.zeros((2, m + 2, m + 2)), side=2.0)
    # h = 2/(m+1) = 2 x the unit-square spacing
    np.testing.assert_allclose(K.toarray(), NU / 4.0 * O.fd_stiffness(2, m).toarray(), rtol=1e-14)
    h = 2.0 / (m + 1)
    assert np.allclose(Kb.data, -NU / h ** 2)
    # every boundary-adjacent row couples to its 1 or 2 wall neighbours
    counts = np.diff(Kb.indptr).reshape(m, m)
    assert counts[0, 0] == 2 and counts[3, 3] == 0 and counts[0, 3] == 1


@pytest.mark.parametrize("m", [7, 15])
def test_constants_and_linear_functions_are_exact(m):
    wind, _, _, _ = circulating_wind_case(m, 4)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    X, Y = _nodes(m)
    np.testing.assert_allclose(_apply_full(K, Kb, np.ones_like(X)), 0.0, atol=1e-10)
    np.testing.assert_allclose(_apply_full(K, Kb, X), wind[0, 1:-1, 1:-1], rtol=1e-12, atol=1e-11)
    np.testing.assert_allclose(_apply_full(K, Kb, Y), wind[1, 1:-1, 1:-1], rtol=1e-12, atol=1e-11)


def test_upwind_error_on_quadratics():
    """On x^2 the upwind difference gives 2 x w_x - |w_x| h (a downwind one
    would give + |w_x| h), and the diffusion gives -2 nu."""
    m = 15
    h = 2.0 / (m + 1)
    wind, _, _, _ = circulating_wind_case(m, 4)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    X, Y = _nodes(m)
    wx, wy = wind[0, 1:-1, 1:-1], wind[1, 1:-1, 1:-1]
    xi, yi = X[1:-1, 1:-1], Y[1:-1, 1:-1]
    np.testing.assert_allclose(_apply_full(K, Kb, X * X), -2 * NU + 2 * xi * wx - np.abs(wx) * h,
                               rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(_apply_full(K, Kb, Y * Y), -2 * NU + 2 * yi * wy - np.abs(wy) * h,
                               rtol=1e-11, atol=1e-11)


def test_m_matrix_sign_pattern():
    """Coarse grid, cell Peclet number up to |w| h / (2 nu) = 25: still no
    positive off-diagonal entry, and weak diagonal dominance."""
    m = 15
    wind, _, _, _ = circulating_wind_case(m, 4)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    A = K.toarray()
    off = A - np.diag(np.diag(A))
    assert off.max() <= 0.0 and Kb.toarray().max() <= 0.0
    rowsum = np.abs(off).sum(axis=1) + np.abs(Kb.toarray()).sum(axis=1)
    assert np.all(np.diag(A) >= rowsum * (1 - 1e-14))


def test_steady_wall_data_give_a_constant_trajectory():
    """With wall data g constant in time and u^0 the discrete steady state
    u* (K u* = -Kb g), u^n = u* for every n solves L u = f."""
    m, N = 15, 6
    wind, g, _, fs = circulating_wind_case(m, N)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    G = g[-1]
    gs = np.repeat(G[None], N, axis=0)
    ustar = spla.spsolve(K.tocsc(), -(Kb @ G.reshape(-1)))
    f = O.build_rhs_dirichlet(ustar.reshape(m, m), fs, gs, 1.0 / N, Kb)
    import scipy.sparse as sp
    L = O.assemble_L(N, sp.identity(m * m, format="csr"), K, 1.0 / N)
    np.testing.assert_allclose(L @ np.tile(ustar, N), f.reshape(-1), rtol=1e-12, atol=1e-12)
    u = O.timestep_solve(f, sp.identity(m * m, format="csr"), K, 1.0 / N)
    np.testing.assert_allclose(u.reshape(N, -1), np.tile(ustar, (N, 1)), rtol=1e-10, atol=1e-12)


def _dilu_matrix(A, d):
    import scipy.sparse as sp
    L = sp.tril(A, -1)
    U = sp.triu(A, 1)
    D = sp.diags(d)
    Dinv = sp.diags(1.0 / d)
    return ((D + L) @ Dinv @ (D + U)).toarray()


def test_dilu_is_ilu0_on_the_five_point_operator():
    """On the 5-point shifted operator lambda I + tau K the factorisation
    (D + L) D^{-1} (D + U) equals A on every entry of A's pattern (ILU(0)),
    and the solve inverts it."""
    m, N = 7, 8
    wind, _, _, _ = circulating_wind_case(m, N)
    K, _ = O.fd_convection_diffusion(NU, wind)
    lam = O.eps_circulant_eigs(N, 0.05)[3]
    import scipy.sparse as sp
    A = (lam * sp.identity(m * m) + K / N).tocsr()
    d = O.dilu_diagonal(A)
    M = _dilu_matrix(A, d)
    Ad = A.toarray()
    mask = Ad != 0
    np.testing.assert_allclose(M[mask], Ad[mask], rtol=1e-13, atol=1e-13)
    r = np.random.default_rng(60).standard_normal(m * m) + 0j
    np.testing.assert_allclose(M @ O.dilu_solve(A, d, r), r, rtol=1e-12, atol=1e-12)


def test_dilu_keeps_the_diagonal_of_the_nine_point_coarse_operators():
    m, N = 15, 8
    wind, _, _, _ = circulating_wind_case(m, N)
    K, _ = O.fd_convection_diffusion(NU, wind)
    h = O.MGHierarchy(K, m)
    lam = O.eps_circulant_eigs(N, 0.05)[1]
    A = h.op(1, lam, 1.0 / N)
    d = O.dilu_diagonal(A)
    M = _dilu_matrix(A, d)
    np.testing.assert_allclose(np.diag(M), A.diagonal(), rtol=1e-12, atol=1e-12)
    r = np.random.default_rng(61).standard_normal(A.shape[0]) + 0j
    np.testing.assert_allclose(M @ O.dilu_solve(A, d, r), r, rtol=1e-11, atol=1e-11)


@pytest.mark.parametrize("k", [0, 5, 16])
def test_ilu_vcycle_contracts_on_the_convection_diffusion_shifted_systems(k):
    """Repeated V-cycles with the ILU smoother (1+1 sweeps, Galerkin coarse
    grids) on lambda_k I + tau K reduce the residual by a steady factor and
    reach the direct solution.  (Damped Jacobi does not: on this recirculating
    wind its cycles stall near a factor 1, which is why Examples 2 and 3 of
    Sec. 5 smooth with ILU.)"""
    m, N = 31, 32
    tau, eps = 1.0 / N, 0.05
    wind, _, _, _ = circulating_wind_case(m, N)
    K, _ = O.fd_convection_diffusion(NU, wind)
    h = O.MGHierarchy(K, m)
    lam = O.eps_circulant_eigs(N, eps)[k]
    rng = np.random.default_rng(50 + k)
    b = rng.standard_normal(m * m) + 1j * rng.standard_normal(m * m)
    A = h.op(0, lam, tau)
    x = np.zeros_like(b)
    res = [np.linalg.norm(b)]
    cache = {}
    for _ in range(5):
        x = x + O.mg_vcycle(h, lam, tau, b - A @ x, smoother="ilu", dcache=cache)
        res.append(np.linalg.norm(b - A @ x))
    rates = np.array(res[1:]) / np.array(res[:-1])
    assert rates.max() < 0.2, rates
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-5


def test_fgmres_with_the_ilu_multigrid_reaches_the_stepping_solution():
    """Example 3's all-at-once system (hot wall, u0 = 0) at m = 31, N = 16:
    FGMRES preconditioned by P_eps^{-1} with one ILU-smoothed V-cycle per
    frequency reaches the sequential backward-Euler solution in a handful of
    iterations (the paper reports 5 with its ILU multigrid)."""
    import scipy.sparse as sp
    m, N = 31, 16
    tau = 1.0 / N
    eps = min(0.5, 0.5 * tau)
    wind, g, u0, fs = circulating_wind_case(m, N)
    K, Kb = O.fd_convection_diffusion(NU, wind)
    f = O.build_rhs_dirichlet(u0, fs, g, tau, Kb)
    I = sp.identity(m * m, format="csr")
    ref = O.timestep_solve(f, I, K, tau)
    L = O.assemble_L(N, I, K, tau)
    h = O.MGHierarchy(K, m)
    caches = {}
    shape = (N, m, m)
    x, info = O.fgmres(lambda v: L @ v, f.reshape(-1),
                       lambda r: O.apply_Pinv_mg(r.reshape(shape), h, tau, eps, smoother="ilu",
                                                 dcaches=caches).reshape(-1),
                       restart=30, tol=1e-10)
    assert info["converged"] and info["iters"] <= 10, info["iters"]
    assert np.linalg.norm(x - ref.reshape(-1)) / np.linalg.norm(ref) < 1e-7
