"""Pins of the FP64 oracle against things other than itself: matrices built
entry by entry from the paper's definitions, closed forms, library routines,
the theorems of Sec. 3 and the iteration counts printed in Table table1."""
import math
import os

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle as O


# ---------------------------------------------------------------- helpers
def _stencil_K_bruteforce(dim, m, a):
    """FD stiffness from the stencil, one entry at a time (h = 1/(m+1))."""
    h = 1.0 / (m + 1)
    J = m ** dim
    K = np.zeros((J, J))
    if dim == 1:
        for i in range(m):
            K[i, i] = 2 * a / h ** 2
            if i > 0:
                K[i, i - 1] = -a / h ** 2
            if i < m - 1:
                K[i, i + 1] = -a / h ** 2
        return K
    for iy in range(m):
        for ix in range(m):
            r = iy * m + ix
            K[r, r] = 4 * a / h ** 2
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                jy, jx = iy + dy, ix + dx
                if 0 <= jy < m and 0 <= jx < m:
                    K[r, jy * m + jx] = -a / h ** 2
    return K


def _q1_bruteforce(m, a):
    """Q1 mass/stiffness by element assembly with 2x2 Gauss quadrature."""
    n = m + 1
    h = 1.0 / n
    nodes = (m + 2)
    gp = np.array([-1, 1]) / math.sqrt(3.0)
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]          # (ix, iy) offsets

    def phi(c, xi, eta):
        sx = xi if c[0] else 1 - xi
        sy = eta if c[1] else 1 - eta
        return sx * sy

    def dphi(c, xi, eta):
        dx = (1 if c[0] else -1) * (eta if c[1] else 1 - eta) / h
        dy = (1 if c[1] else -1) * (xi if c[0] else 1 - xi) / h
        return dx, dy

    Me = np.zeros((4, 4))
    Ke = np.zeros((4, 4))
    for gx in gp:
        for gy in gp:
            xi, eta = 0.5 * (gx + 1), 0.5 * (gy + 1)
            wgt = 0.25 * h * h                          # Gauss weights 1, Jacobian h^2/4
            for p, cp in enumerate(corners):
                for q, cq in enumerate(corners):
                    Me[p, q] += wgt * phi(cp, xi, eta) * phi(cq, xi, eta)
                    dp, dq = dphi(cp, xi, eta), dphi(cq, xi, eta)
                    Ke[p, q] += wgt * (dp[0] * dq[0] + dp[1] * dq[1])
    Mg = np.zeros((nodes * nodes, nodes * nodes))
    Kg = np.zeros_like(Mg)
    for ey in range(n):
        for ex in range(n):
            ids = [(ey + c[1]) * nodes + (ex + c[0]) for c in corners]
            for p in range(4):
                for q in range(4):
                    Mg[ids[p], ids[q]] += Me[p, q]
                    Kg[ids[p], ids[q]] += a * Ke[p, q]
    interior = [iy * nodes + ix for iy in range(1, m + 1) for ix in range(1, m + 1)]
    return Mg[np.ix_(interior, interior)], Kg[np.ix_(interior, interior)]


def _L_bruteforce(N, M, K, tau, eps=None):
    """Block matrix of Sec. 2 (eps=None) or P_eps of Sec. 3, block by block."""
    M = np.asarray(M.todense()) if sp.issparse(M) else M
    K = np.asarray(K.todense()) if sp.issparse(K) else K
    J = M.shape[0]
    L = np.zeros((N * J, N * J))
    A0 = M + tau * K
    for n in range(N):
        L[n * J:(n + 1) * J, n * J:(n + 1) * J] = A0
        if n > 0:
            L[n * J:(n + 1) * J, (n - 1) * J:n * J] = -M
    if eps is not None:      # for N = 1 the corner block is the diagonal block itself
        L[0:J, (N - 1) * J:N * J] += -eps * M
    return L


def _fd_problem(dim, m, N, a=1.0):
    K = O.fd_stiffness(dim, m, a)
    M = sp.identity(K.shape[0], format="csr")
    return M, K, 1.0 / N


# ---------------------------------------------------------------- spatial
@pytest.mark.parametrize("dim,m,a", [(1, 5, 1.0), (2, 4, 2.5), (2, 3, 1e-5)])
def test_fd_stiffness_is_the_stencil(dim, m, a):
    K = O.fd_stiffness(dim, m, a).toarray()
    np.testing.assert_allclose(K, _stencil_K_bruteforce(dim, m, a), rtol=1e-15, atol=0)


def test_fd_varcoef_constant_a_reduces_to_laplacian():
    m = 5
    a_nodes = np.full((m + 2, m + 2), 3.0)
    K = O.fd_stiffness_varcoef(a_nodes).toarray()
    np.testing.assert_allclose(K, _stencil_K_bruteforce(2, m, 3.0), rtol=1e-14, atol=0)


def test_fd_varcoef_is_symmetric_and_conservative():
    m = 6
    rng = np.random.default_rng(0)
    a_nodes = np.exp(rng.standard_normal((m + 2, m + 2)))
    K = O.fd_stiffness_varcoef(a_nodes).toarray()
    np.testing.assert_allclose(K, K.T, rtol=0, atol=1e-12 * np.abs(K).max())
    assert np.all(np.linalg.eigvalsh(K) > 0)
    # one interior node: diagonal = sum of its four face coefficients / h^2
    h = 1.0 / (m + 1)
    iy, ix = 2, 3
    gy, gx = iy + 1, ix + 1
    faces = sum(0.5 * (a_nodes[gy, gx] + a_nodes[gy + dy, gx + dx])
                for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)))
    assert math.isclose(K[iy * m + ix, iy * m + ix], faces / h ** 2, rel_tol=1e-14)


def test_q1_matrices_match_element_assembly():
    m, a = 4, 0.7
    M, K = O.q1_mass_stiffness(m, a)
    Mb, Kb = _q1_bruteforce(m, a)
    np.testing.assert_allclose(M.toarray(), Mb, rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(K.toarray(), Kb, rtol=1e-13, atol=1e-14)


def test_dst_diagonalises_fd_laplacian():
    m = 7
    S = O.dst_matrix(m)
    # S from its definition, entry by entry
    for j in range(m):
        for k in range(m):
            assert math.isclose(S[j, k], math.sqrt(2 / (m + 1)) * math.sin(math.pi * (j + 1) * (k + 1) / (m + 1)),
                                rel_tol=1e-15, abs_tol=1e-16)
    np.testing.assert_allclose(S @ S, np.eye(m), atol=1e-14)
    K1 = _stencil_K_bruteforce(1, m, 1.0)
    mu = O.fd_dst_eigs(m)
    np.testing.assert_allclose(K1 @ S, S @ np.diag(mu), atol=1e-11 * mu.max())
    np.testing.assert_allclose(np.sort(mu), np.linalg.eigvalsh(K1), rtol=1e-12)
    x = np.random.default_rng(1).standard_normal(m)
    np.testing.assert_allclose(S @ x, sfft.dst(x, type=1, norm="ortho"), atol=1e-14)


# ---------------------------------------------------------------- all-at-once system
@pytest.mark.parametrize("dim,m,N", [(1, 4, 3), (2, 3, 4)])
def test_L_and_P_match_block_definitions(dim, m, N):
    M, K, tau = _fd_problem(dim, m, N)
    np.testing.assert_allclose(O.assemble_L(N, M, K, tau).toarray(), _L_bruteforce(N, M, K, tau), atol=1e-13)
    for eps in (1.0, 0.3, 1e-4):
        np.testing.assert_allclose(O.assemble_P(N, M, K, tau, eps).toarray(),
                                   _L_bruteforce(N, M, K, tau, eps), atol=1e-13)


def test_L_and_P_with_q1_mass():
    m, N = 3, 4
    M, K = O.q1_mass_stiffness(m, 1e-2)
    tau = 1.0 / N
    np.testing.assert_allclose(O.assemble_P(N, M, K, tau, 0.2).toarray(),
                               _L_bruteforce(N, M, K, tau, 0.2), atol=1e-15)


def test_pstep_eps_circulant_layout_bdf2():
    """R_eps of eq. pstepbecpreconditioner for p = 2: first row (r0, 0, .., eps r2, eps r1)."""
    N, eps = 5, 0.1
    r0, r1, r2 = O.BDF2
    R = O.time_eps_circulant(N, eps, O.BDF2).toarray()
    expect = np.zeros((N, N))
    for n in range(N):
        expect[n, n] = r0
        if n >= 1:
            expect[n, n - 1] = r1
        if n >= 2:
            expect[n, n - 2] = r2
    expect[0, N - 1] = eps * r1
    expect[0, N - 2] = eps * r2
    expect[1, N - 1] = eps * r2
    np.testing.assert_array_equal(R, expect)


def test_build_rhs_first_slice_carries_u0():
    m, N = 4, 3
    M, K = O.q1_mass_stiffness(m)
    rng = np.random.default_rng(2)
    u0 = rng.standard_normal((m, m))
    fs = rng.standard_normal((N, m, m))
    f = O.build_rhs(u0, fs, 0.25, M)
    np.testing.assert_allclose(f[0].reshape(-1), 0.25 * fs[0].reshape(-1) + M @ u0.reshape(-1), rtol=1e-14)
    np.testing.assert_allclose(f[1:], 0.25 * fs[1:], rtol=0)


@pytest.mark.parametrize("dim,m,N", [(1, 9, 7), (2, 5, 6)])
def test_timestep_solve_equals_direct_solve_of_L(dim, m, N):
    M, K, tau = _fd_problem(dim, m, N)
    f = np.random.default_rng(3).standard_normal((N,) + (m,) * dim)
    u = O.timestep_solve(f, M, K, tau)
    L = O.assemble_L(N, M, K, tau)
    ud = spla.spsolve(L.tocsc(), f.reshape(-1))
    np.testing.assert_allclose(u.reshape(-1), ud, rtol=1e-12, atol=1e-14)


def test_timestep_solve_single_mode_closed_form():
    """One DST mode, zero source: u^n = (1 + tau mu)^{-n} u^0 (backward Euler)."""
    m, N, k = 15, 10, 3
    M, K, tau = _fd_problem(1, m, N)
    S = O.dst_matrix(m)
    u0 = S[:, k - 1]
    f = O.build_rhs(u0, np.zeros((N, m)), tau)
    u = O.timestep_solve(f, M, K, tau)
    mu = O.fd_dst_eigs(m)[k - 1]
    for n in range(N):
        np.testing.assert_allclose(u[n], (1 + tau * mu) ** (-(n + 1)) * u0, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- p-step (BDF2) system
@pytest.mark.parametrize("dim,m,N,space", [(1, 9, 7, "fd"), (2, 5, 6, "fd"), (2, 4, 5, "q1")])
def test_pstep_stepping_equals_direct_solve_of_L(dim, m, N, space):
    """Stepping the BDF2 rows one after another gives the solution of the
    assembled all-at-once matrix R (x) M + tau I (x) K (eq. pstepscheme)."""
    if space == "fd":
        M, K, tau = _fd_problem(dim, m, N)
    else:
        M, K = O.q1_mass_stiffness(m, 0.3)
        tau = 1.0 / N
    f = np.random.default_rng(31).standard_normal((N,) + (m,) * dim)
    u = O.timestep_solve_pstep(f, M, K, tau, O.BDF2)
    ud = spla.spsolve(O.assemble_L(N, M, K, tau, O.BDF2).tocsc(), f.reshape(-1))
    np.testing.assert_allclose(u.reshape(-1), ud, rtol=1e-11, atol=1e-13)


def test_pstep_with_bdf1_is_backward_euler():
    M, K, tau = _fd_problem(2, 5, 6)
    rng = np.random.default_rng(32)
    u0, fs = rng.standard_normal((5, 5)), rng.standard_normal((6, 5, 5))
    np.testing.assert_array_equal(O.build_rhs_pstep(u0, fs, tau, O.BDF1), O.build_rhs(u0, fs, tau))
    f = O.build_rhs(u0, fs, tau)
    np.testing.assert_allclose(O.timestep_solve_pstep(f, M, K, tau, O.BDF1),
                               O.timestep_solve(f, M, K, tau), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("k", [1, 4, 15])
def test_bdf2_single_mode_closed_form(k):
    """One DST mode, zero source, pre-start value u^{-1} = u^0: u^n = a_n u^0
    with (r0 + tau mu) a_n + r1 a_{n-1} + r2 a_{n-2} = 0, a_0 = a_{-1} = 1,
    i.e. a_n = A z1^n + B z2^n over the roots of (r0 + tau mu) z^2 + r1 z + r2."""
    m, N = 15, 12
    M, K, tau = _fd_problem(1, m, N)
    S = O.dst_matrix(m)
    u0 = S[:, k - 1]
    f = O.build_rhs_pstep(u0, np.zeros((N, m)), tau, O.BDF2)
    u = O.timestep_solve_pstep(f, M, K, tau, O.BDF2)
    mu = (4.0 * (m + 1) ** 2) * math.sin(k * math.pi / (2 * (m + 1))) ** 2
    r0, r1, r2 = O.BDF2
    z1, z2 = np.roots([r0 + tau * mu, r1, r2]).astype(complex)
    # A + B = 1 and A / z1 + B / z2 = 1
    A, B = np.linalg.solve(np.array([[1, 1], [1 / z1, 1 / z2]]), np.array([1, 1], dtype=complex))
    for n in range(1, N + 1):
        an = (A * z1 ** n + B * z2 ** n).real
        np.testing.assert_allclose(u[n - 1], an * u0, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("space", ["fd", "q1"])
def test_pstep_steady_state_with_constant_pre_history(space):
    """With every pre-start value equal to u^0 and the source K w, the constant
    trajectory u^n = w solves L u = f: the rows of R sum to zero."""
    m, N = 5, 6
    if space == "fd":
        M, K, tau = _fd_problem(2, m, N)
    else:
        M, K = O.q1_mass_stiffness(m, 0.2)
        tau = 1.0 / N
    w = np.random.default_rng(33).standard_normal(m * m)
    fs = np.tile((K @ w).reshape(m, m), (N, 1, 1))
    f = O.build_rhs_pstep(w.reshape(m, m), fs, tau, O.BDF2, M=None if space == "fd" else M)
    L = O.assemble_L(N, M, K, tau, O.BDF2)
    np.testing.assert_allclose(L @ np.tile(w, N), f.reshape(-1), rtol=1e-12, atol=1e-13)


# ---------------------------------------------------------------- diagonalisation
def test_fourier_matrix_is_unitary_and_an_inverse_dft():
    N = 8
    F = O.fourier_matrix(N)
    np.testing.assert_allclose(F @ F.conj().T, np.eye(N), atol=1e-14)
    x = np.random.default_rng(4).standard_normal(N)
    np.testing.assert_allclose(F @ x, math.sqrt(N) * np.fft.ifft(x), atol=1e-14)
    assert abs(F[1, 1] - np.exp(2j * np.pi / N) / math.sqrt(N)) < 1e-15


@pytest.mark.parametrize("N,eps,r", [(6, 0.3, O.BDF1), (8, 1.0, O.BDF1), (7, 1e-3, O.BDF2)])
def test_eps_circulant_diagonalisation(N, eps, r):
    """R_eps = D^{-1} F^* Lambda F D with lambda_k = sum_j r_j eps^{j/N} theta^{kj}."""
    R = O.time_eps_circulant(N, eps, r).toarray()
    F = O.fourier_matrix(N)
    D = np.diag(O.eps_scaling(N, eps))
    lam = O.eps_circulant_eigs(N, eps, r)
    recon = np.linalg.inv(D) @ F.conj().T @ np.diag(lam) @ F @ D
    np.testing.assert_allclose(recon, R, atol=1e-12)
    ev = np.linalg.eigvals(R)
    for lk in lam:
        assert np.min(np.abs(ev - lk)) < 1e-7
    if r == O.BDF1:     # closed form 1 - eps^{1/N} theta^k
        k = np.arange(N)
        np.testing.assert_allclose(lam, 1 - eps ** (1 / N) * np.exp(2j * np.pi * k / N), atol=1e-15)


# ---------------------------------------------------------------- P_eps^{-1}
_PINV_CASES = [
    (1, 7, 8, 0.05), (1, 5, 3, 1.0), (1, 6, 5, 1e-4),
    (2, 3, 4, 0.5), (2, 7, 5, 1e-4), (2, 7, 8, 1.0), (2, 5, 2, 0.2), (2, 3, 1, 0.7),
]


@pytest.mark.parametrize("dim,m,N,eps", _PINV_CASES)
def test_apply_Pinv_routes_agree_with_dense_inverse(dim, m, N, eps):
    M, K, tau = _fd_problem(dim, m, N)
    y = np.random.default_rng(5).standard_normal((N,) + (m,) * dim)
    P = _L_bruteforce(N, M, K, tau, eps)
    zd = np.linalg.solve(P, y.reshape(-1)).reshape(y.shape)
    tol = 1e-13 / min(eps, 1.0) ** 0.5 * 10
    n = np.linalg.norm(zd)
    for z in (O.apply_Pinv_lu(y, M, K, tau, eps), O.apply_Pinv_woodbury(y, M, K, tau, eps),
              O.apply_Pinv_fst(y, dim, 1.0, tau, eps)):
        assert np.linalg.norm(z - zd) / n < tol
    # P z = y for the routes
    zf = O.apply_Pinv_fst(y, dim, 1.0, tau, eps)
    Ps = O.assemble_P(N, M, K, tau, eps)
    assert np.linalg.norm(Ps @ zf.reshape(-1) - y.reshape(-1)) / np.linalg.norm(y) < tol


@pytest.mark.parametrize("dim,m,N,eps", [(1, 7, 8, 0.05), (2, 5, 4, 1e-3), (2, 3, 6, 1.0)])
def test_apply_Pinv_fst_bdf2_agrees_with_dense_inverse(dim, m, N, eps):
    """The sine-transform route with the BDF2 eigenvalues
    lambda_k = r0 + r1 eps^{1/N} theta^k + r2 eps^{2/N} theta^{2k} inverts
    R_eps (x) I + tau I (x) K (eq. pstepbecpreconditioner)."""
    M, K, tau = _fd_problem(dim, m, N)
    y = np.random.default_rng(34).standard_normal((N,) + (m,) * dim)
    P = O.assemble_P(N, M, K, tau, eps, O.BDF2).toarray()
    zd = np.linalg.solve(P, y.reshape(-1))
    z = O.apply_Pinv_fst(y, dim, 1.0, tau, eps, O.BDF2).reshape(-1)
    assert np.linalg.norm(z - zd) / np.linalg.norm(zd) < 1e-11


def test_apply_Pinv_lu_with_q1_and_bdf2():
    m, N, eps = 4, 6, 0.05
    M, K = O.q1_mass_stiffness(m, 0.1)
    tau = 1.0 / N
    y = np.random.default_rng(6).standard_normal((N, m, m))
    for r in (O.BDF1, O.BDF2):
        P = O.assemble_P(N, M, K, tau, eps, r).toarray()
        zd = np.linalg.solve(P, y.reshape(-1))
        zl = O.apply_Pinv_lu(y, M, K, tau, eps, r).reshape(-1)
        assert np.linalg.norm(zl - zd) / np.linalg.norm(zd) < 1e-12
    zw = O.apply_Pinv_woodbury(y, M, K, tau, eps).reshape(-1)
    zd = np.linalg.solve(O.assemble_P(N, M, K, tau, eps).toarray(), y.reshape(-1))
    assert np.linalg.norm(zw - zd) / np.linalg.norm(zd) < 1e-13


def test_half_spectrum_symmetry():
    """Sec. 4: conj(y~^{k+1}) = y~^{N-k+1} and conj(B_k) = B_{N-k}, so the solves
    for k > N/2 are conjugates of those below."""
    N, eps, m = 8, 0.1, 5
    y = np.random.default_rng(7).standard_normal((N, m))
    yt = math.sqrt(N) * np.fft.ifft(O.eps_scaling(N, eps)[:, None] * y, axis=0)
    lam = O.eps_circulant_eigs(N, eps)
    for k in range(1, N):
        np.testing.assert_allclose(np.conj(yt[k]), yt[N - k], atol=1e-14)
        assert abs(np.conj(lam[k]) - lam[N - k]) < 1e-15


# ---------------------------------------------------------------- Sec. 3 theorems
@pytest.mark.parametrize("dim,m,N,eps", [(1, 6, 5, 0.1), (2, 3, 4, 0.05), (1, 5, 6, 0.5)])
def test_preconditioned_spectrum(dim, m, N, eps):
    """Theorem preconditionedspectrum: rank(P^{-1}L - I) = J; (N-1)J eigenvalues
    equal to 1; the other J are lambda^N/(lambda^N - eps), lambda in sigma(I + tau K);
    |lambda - 1| <= eps/(1 - eps)."""
    M, K, tau = _fd_problem(dim, m, N)
    J = K.shape[0]
    L = _L_bruteforce(N, M, K, tau)
    P = _L_bruteforce(N, M, K, tau, eps)
    G = np.linalg.solve(P, L)
    sv = np.linalg.svd(G - np.eye(N * J), compute_uv=False)
    assert int(np.sum(sv > 1e-10 * sv[0])) == J
    ev = np.linalg.eigvals(G)
    ones = np.abs(ev - 1) < 1e-9
    assert int(ones.sum()) == (N - 1) * J
    lamK = 1 + tau * np.linalg.eigvalsh(K.toarray())
    pred = lamK ** N / (lamK ** N - eps)
    rest = np.sort(ev[~ones].real)
    np.testing.assert_allclose(rest, np.sort(pred), rtol=1e-9)
    assert np.max(np.abs(ev - 1)) <= eps / (1 - eps) + 1e-12


@pytest.mark.parametrize("eps", [0.3, 0.05, 1e-3])
def test_norm_bound_lemma(eps):
    """Lemma preconditionedmatapproximateidlem: ||P^{-1}L - I||_2 <= eps c0 sqrt(N)/(1-eps),
    c0 = sqrt(kappa(M)) (= 1 for finite differences)."""
    N, m = 6, 4
    M, K, tau = _fd_problem(2, m, N)
    L = _L_bruteforce(N, M, K, tau)
    P = _L_bruteforce(N, M, K, tau, eps)
    nrm = np.linalg.norm(np.linalg.solve(P, L) - np.eye(L.shape[0]), 2)
    assert nrm <= eps * math.sqrt(N) / (1 - eps)
    Mq, Kq = O.q1_mass_stiffness(m, 0.5)
    c0 = math.sqrt(np.linalg.cond(Mq.toarray()))
    Lq = _L_bruteforce(N, Mq, Kq, tau)
    Pq = _L_bruteforce(N, Mq, Kq, tau, eps)
    nq = np.linalg.norm(np.linalg.solve(Pq, Lq) - np.eye(Lq.shape[0]), 2)
    assert nq <= eps * c0 * math.sqrt(N) / (1 - eps)


# ---------------------------------------------------------------- Krylov
def test_gmres_unrestarted_terminates_within_J_plus_1():
    """Consequence of Theorem preconditionedspectrum (i): at most J+1 iterations."""
    dim, m, N, eps = 1, 6, 16, 1.0
    M, K, tau = _fd_problem(dim, m, N)
    L = O.assemble_L(N, M, K, tau)
    f = np.random.default_rng(8).standard_normal(N * m)
    Minv = lambda v: O.apply_Pinv_fst(v.reshape(N, m), dim, 1.0, tau, eps).reshape(-1)
    u, info = O.gmres(lambda v: L @ v, f, Minv, restart=200, tol=1e-12)
    assert info["converged"] and info["iters"] <= m + 1
    np.testing.assert_allclose(u, O.timestep_solve(f.reshape(N, m), M, K, tau).reshape(-1), rtol=1e-9, atol=1e-11)


def test_gmres_rate_bound_theorem():
    """Theorem gmrescvgthm: for eps <= b_tau = delta sqrt(tau)/(delta sqrt(tau) + c0 sqrt(T)),
    ||r_k|| <= (2 sqrt(delta)/(1+delta))^k ||r_0||."""
    dim, m, N, T, delta = 2, 7, 16, 1.0, 0.5
    M, K, tau = _fd_problem(dim, m, N)
    b_tau = delta * math.sqrt(tau) / (delta * math.sqrt(tau) + math.sqrt(T))
    L = O.assemble_L(N, M, K, tau)
    f = np.random.default_rng(9).standard_normal(N * m * m)
    Minv = lambda v: O.apply_Pinv_fst(v.reshape(N, m, m), dim, 1.0, tau, b_tau).reshape(-1)
    _, info = O.gmres(lambda v: L @ v, f, Minv, restart=50, tol=1e-14)
    rate = 2 * math.sqrt(delta) / (1 + delta)
    rv = info["resvec"]
    for k in range(1, len(rv)):
        assert rv[k] <= rate ** k * rv[0] * (1 + 1e-9)


def test_fgmres_right_preconditioned_reaches_true_residual():
    dim, m, N, eps = 2, 7, 8, 0.05
    M, K, tau = _fd_problem(dim, m, N)
    L = O.assemble_L(N, M, K, tau)
    f = np.random.default_rng(10).standard_normal(N * m * m)
    Minv = lambda v: O.apply_Pinv_fst(v.reshape(N, m, m), dim, 1.0, tau, eps).reshape(-1)
    u, info = O.fgmres(lambda v: L @ v, f, Minv, restart=10, tol=1e-12)
    assert info["converged"]
    assert O.relative_residual(L, u, f) < 1e-11
    np.testing.assert_allclose(u, O.timestep_solve(f.reshape(N, m, m), M, K, tau).reshape(-1), rtol=1e-9, atol=1e-11)
    # left GMRES reaches the same solution
    u2, _ = O.gmres(lambda v: L @ v, f, Minv, restart=10, tol=1e-13)
    np.testing.assert_allclose(u2, u, rtol=1e-9, atol=1e-11)


def test_fgmres_with_varying_inexact_preconditioner():
    """A preconditioner that changes between iterations still yields the solution."""
    dim, m, N, eps = 1, 15, 8, 0.1
    M, K, tau = _fd_problem(dim, m, N)
    L = O.assemble_L(N, M, K, tau)
    f = np.random.default_rng(11).standard_normal(N * m)
    rng = np.random.default_rng(12)

    def Minv(v):
        z = O.apply_Pinv_fst(v.reshape(N, m), dim, 1.0, tau, eps).reshape(-1)
        return z * (1 + 1e-3 * rng.standard_normal(z.size))

    u, info = O.fgmres(lambda v: L @ v, f, Minv, restart=20, tol=1e-12)
    assert info["converged"] and O.relative_residual(L, u, f) < 1e-11


# ---------------------------------------------------------------- the paper's Table table1
def _table1_rows(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table1_bdf1.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                N, n, it, res, bit, bres = line.split()[:6]
                rows.append((int(N), int(n), int(it), float(res), int(bit), float(bres)))
    return rows


def _example1(N, n):
    m = n - 1
    M, K = O.q1_mass_stiffness(m, 1e-5)
    tau = 1.0 / N
    x = np.arange(1, m + 1) / (m + 1)
    X, Y = np.meshgrid(x, x)
    f = O.build_rhs(X * (X - 1) * Y * (Y - 1), np.zeros((N, m, m)), tau, M)
    return M, K, tau, f


def _table1_row(golden_dir, N, n):
    return next(r for r in _table1_rows(golden_dir) if r[0] == N and r[1] == n)


@pytest.mark.parametrize("N", [64, 128])
def test_table1_bec_iterations_and_res(golden_dir, N):
    N, n, it, res, _, _ = _table1_row(golden_dir, N, 64)
    M, K, tau, f = _example1(N, n)
    m = n - 1
    eps = min(0.5, 0.5 * tau)
    L = O.assemble_L(N, M, K, tau)
    Minv = lambda v: O.apply_Pinv_lu(v.reshape(N, m, m), M, K, tau, eps).reshape(-1)
    u, info = O.gmres(lambda v: L @ v, f.reshape(-1), Minv, restart=50, tol=1e-7)
    assert info["iters"] == it
    assert abs(O.relative_residual(L, u, f) / res - 1) < 0.01     # printed to 3 digits


@pytest.mark.slow
def test_table1_bc_iterations_and_res(golden_dir):
    N, n, _, _, bit, bres = _table1_row(golden_dir, 64, 64)
    M, K, tau, f = _example1(N, n)
    m = n - 1
    L = O.assemble_L(N, M, K, tau)
    Minv = lambda v: O.apply_Pinv_lu(v.reshape(N, m, m), M, K, tau, 1.0).reshape(-1)
    u, info = O.gmres(lambda v: L @ v, f.reshape(-1), Minv, restart=50, tol=1e-7)
    assert info["iters"] == bit
    assert abs(O.relative_residual(L, u, f) / bres - 1) < 0.05


# ---------------------------------------------------------------- 3D domains
def test_fd_stiffness_3d_is_the_7_point_laplacian():
    """Brute force on a 4^3 grid: (K u)_p = a/h^2 (6 u_p - sum of the 6
    neighbours), zero outside the cube."""
    m, a = 4, 0.7
    h = 1.0 / (m + 1)
    K = O.fd_stiffness(3, m, a).toarray()
    rng = np.random.default_rng(31)
    u = rng.standard_normal((m, m, m))
    up = np.zeros((m + 2, m + 2, m + 2))
    up[1:-1, 1:-1, 1:-1] = u
    ref = 6 * u
    for ax in range(3):
        for sgn in (-1, 1):
            sl = [slice(1, -1)] * 3
            sl[ax] = slice(1 + sgn, m + 1 + sgn)
            ref = ref - up[tuple(sl)]
    np.testing.assert_allclose((K @ u.reshape(-1)).reshape(m, m, m), a / h ** 2 * ref, rtol=1e-13)


def test_fd_stiffness_3d_eigenpairs_are_tensor_sine_modes():
    """K S = S diag(mu_i + mu_j + mu_k) with S the 3D orthonormal DST-I."""
    m, a = 7, 1.3
    K = O.fd_stiffness(3, m, a)
    mu1 = O.fd_dst_eigs(m, a)
    rng = np.random.default_rng(32)
    c = rng.standard_normal((m, m, m))
    mu = mu1[:, None, None] + mu1[None, :, None] + mu1[None, None, :]
    u = sfft.dstn(c, type=1, norm="ortho")
    Ku = (K @ u.reshape(-1)).reshape(m, m, m)
    np.testing.assert_allclose(Ku, sfft.dstn(mu * c, type=1, norm="ortho"), rtol=1e-10, atol=1e-9)


@pytest.mark.parametrize("eps", [0.1, 1e-3])
def test_apply_Pinv_fst_3d_equals_banded_lu(eps):
    """The sine-transform route and the banded-LU route of P_eps^{-1} agree in 3D."""
    m, N, a = 7, 8, 0.9
    K = O.fd_stiffness(3, m, a)
    M = sp.identity(m ** 3, format="csr")
    tau = 1.0 / N
    y = np.random.default_rng(33).uniform(-1, 1, (N, m, m, m))
    z1 = O.apply_Pinv_fst(y, 3, a, tau, eps)
    z2 = O.apply_Pinv_lu(y.reshape(N, m ** 3), M, K, tau, eps).reshape(y.shape)
    np.testing.assert_allclose(z1, z2, rtol=1e-9, atol=1e-11 * np.abs(z2).max())
