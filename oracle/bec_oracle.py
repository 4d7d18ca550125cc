"""Plain FP64 CPU oracle for the block epsilon-circulant (BEC) preconditioner of
Lin & Ng, "An all-at-once preconditioner for evolutionary PDEs" (arXiv 2002.01108).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The GPU library never uses it.

Everything is written for clarity, not speed: sparse matrices from
``scipy.sparse``, FFTs from ``numpy.fft`` and DSTs from ``scipy.fft`` serve as
library steps; no blocking or fusion beyond what the paper states.

Conventions (Sec. 2): u = (u^1; u^2; ...; u^N), each u^n a spatial vector of
length J; a 2D spatial vector is stored [ny][nx] (x fastest), so the 2D FD
stiffness is kron(I, K1) + kron(K1, I).  tau = T/N.

Every function below is pinned by a test in tests/test_oracle_pins.py against
something other than itself (brute-force matrices built from the definitions,
closed forms, library routines, the paper's printed iteration counts).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

__all__ = [
    "BDF1", "BDF2",
    "fd_stiffness_1d", "fd_stiffness", "fd_stiffness_varcoef", "q1_mass_stiffness",
    "fd_convection_diffusion", "build_rhs_dirichlet",
    "time_toeplitz", "time_eps_circulant", "assemble_L", "assemble_P",
    "build_rhs", "timestep_solve", "build_rhs_pstep", "timestep_solve_pstep",
    "fourier_matrix", "eps_scaling", "eps_circulant_eigs", "dst_matrix", "fd_dst_eigs",
    "apply_Pinv_dense", "apply_Pinv_lu", "apply_Pinv_woodbury", "apply_Pinv_fst",
    "gmres", "fgmres", "relative_residual",
    "mg_prolongation", "MGHierarchy", "mg_vcycle", "apply_Pinv_mg", "node_coefficient",
    "dilu_diagonal", "dilu_solve",
]

#: backward Euler, r_0 = 1, r_1 = -1 (Sec. 4, remark after eq. pstepscheme)
BDF1 = (1.0, -1.0)
#: two-step backward difference, r = (3/2, -2, 1/2) (Sec. 5, Example 1)
BDF2 = (1.5, -2.0, 0.5)


# --------------------------------------------------------------------------
# Spatial matrices M, K (Sec. 2: K discretises -div(a grad .); FD gives M = I)
# --------------------------------------------------------------------------
def fd_stiffness_1d(m: int, a: float = 1.0) -> sp.csr_matrix:
    """3-point central difference for -a u_xx on m interior nodes, h = 1/(m+1),
    zero Dirichlet data (eq. dtbc with g = 0)."""
    h = 1.0 / (m + 1)
    off = np.full(m - 1, -1.0)
    return ((a / h ** 2) * sp.diags([off, np.full(m, 2.0), off], [-1, 0, 1])).tocsr()


def fd_stiffness(dim: int, m: int, a: float = 1.0) -> sp.csr_matrix:
    """3-point (1D), 5-point (2D) or 7-point (3D) FD Laplacian times a on the
    unit interval, square or cube (the domain of eq. heateq is in R^2 or R^3);
    ordering [ny][nx] and [nz][ny][nx], x fastest."""
    K1 = fd_stiffness_1d(m, a)
    if dim == 1:
        return K1
    I = sp.identity(m, format="csr")
    if dim == 2:
        return (sp.kron(I, K1) + sp.kron(K1, I)).tocsr()
    return (sp.kron(sp.kron(I, I), K1) + sp.kron(sp.kron(I, K1), I)
            + sp.kron(sp.kron(K1, I), I)).tocsr()


def fd_stiffness_varcoef(a_nodes: np.ndarray) -> sp.csr_matrix:
    """Conservative 5-point FD for -div(a grad u) on the unit square (eq. heateq
    with variable a).  ``a_nodes`` holds a on all (m+2)^2 nodes [iy][ix],
    boundary included; the coefficient on a cell face is the mean of its two
    node values.  Interior unknowns are ordered [ny][nx]."""
    n2 = a_nodes.shape[0]
    m = n2 - 2
    h = 1.0 / (m + 1)
    rows, cols, vals = [], [], []

    def idx(iy, ix):
        return iy * m + ix

    for iy in range(m):
        for ix in range(m):
            gy, gx = iy + 1, ix + 1
            ac = a_nodes[gy, gx]
            diag = 0.0
            for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0)):
                af = 0.5 * (ac + a_nodes[gy + dy, gx + dx])
                diag += af
                ny, nx = iy + dy, ix + dx
                if 0 <= ny < m and 0 <= nx < m:
                    rows.append(idx(iy, ix))
                    cols.append(idx(ny, nx))
                    vals.append(-af / h ** 2)
            rows.append(idx(iy, ix))
            cols.append(idx(iy, ix))
            vals.append(diag / h ** 2)
    return sp.csr_matrix((vals, (rows, cols)), shape=(m * m, m * m))


def fd_convection_diffusion(nu: float, wind: np.ndarray, side: float = 2.0):
    """5-point FD for -nu Lap u + w . grad u on a square of side ``side``
    (Example 3 of Sec. 5: nu = 1/200 on (-1, 1)^2 with the circulating wind),
    m interior points per direction, h = side/(m+1).  The diffusion takes
    central second differences; the convection takes first-order upwind
    differences, w_x (u_i - u_{i-1})/h where w_x > 0 and w_x (u_{i+1} - u_i)/h
    where w_x < 0 (likewise in y).  This stands in for the paper's SUPG Q1
    elements: both stabilise the convection, and upwinding keeps every
    off-diagonal entry <= 0.  ``wind`` holds (w_x, w_y) on all nodes,
    [2][m+2][m+2] ([iy][ix]), evaluated at the node of the row.

    Returns (K, Kb): K (J x J) acts on the interior unknowns [ny][nx], Kb
    (J x (m+2)^2) on the values at all nodes of which only the boundary ones
    are used, so that a row of the operator is (K u + Kb g) with g the
    Dirichlet data."""
    n2 = wind.shape[1]
    m = n2 - 2
    h = side / (m + 1)
    rows, cols, vals = [], [], []
    brows, bcols, bvals = [], [], []
    for iy in range(m):
        for ix in range(m):
            gy, gx = iy + 1, ix + 1
            wx, wy = wind[0, gy, gx], wind[1, gy, gx]
            row = iy * m + ix
            # (dy, dx): diffusion -nu/h^2 plus the upwind convection weight
            nbrs = {(0, -1): -nu / h ** 2 - max(wx, 0.0) / h,
                    (0, 1): -nu / h ** 2 + min(wx, 0.0) / h,
                    (-1, 0): -nu / h ** 2 - max(wy, 0.0) / h,
                    (1, 0): -nu / h ** 2 + min(wy, 0.0) / h}
            diag = 4.0 * nu / h ** 2 + (abs(wx) + abs(wy)) / h
            rows.append(row)
            cols.append(row)
            vals.append(diag)
            for (dy, dx), v in nbrs.items():
                ny, nx = iy + dy, ix + dx
                if 0 <= ny < m and 0 <= nx < m:
                    rows.append(row)
                    cols.append(ny * m + nx)
                    vals.append(v)
                else:
                    brows.append(row)
                    bcols.append((gy + dy) * n2 + (gx + dx))
                    bvals.append(v)
    K = sp.csr_matrix((vals, (rows, cols)), shape=(m * m, m * m))
    Kb = sp.csr_matrix((bvals, (brows, bcols)), shape=(m * m, n2 * n2))
    return K, Kb


def build_rhs_dirichlet(u0: np.ndarray, fsrc: np.ndarray, g: np.ndarray, tau: float,
                        Kb) -> np.ndarray:
    """f of the all-at-once system (Sec. 2, M = I) when the boundary values
    are prescribed: f^n = tau (fsrc^n - Kb g^n) plus u^0 in slice 1, with g^n
    the node values [m+2][m+2] at t_n (only the boundary ones enter)."""
    N = fsrc.shape[0]
    f = tau * np.asarray(fsrc, dtype=np.float64).reshape(N, -1).copy()
    for n in range(N):
        f[n] -= tau * (Kb @ np.asarray(g[n], dtype=np.float64).reshape(-1))
    f[0] += np.asarray(u0, dtype=np.float64).reshape(-1)
    return f.reshape(fsrc.shape)


def q1_mass_stiffness(m: int, a: float = 1.0):
    """Consistent bilinear (Q1) finite-element mass and stiffness matrices on a
    uniform mesh of the unit square with m interior nodes per side (Sec. 5).
    On a tensor mesh M = M1 (x) M1 and K = a (M1 (x) K1 + K1 (x) M1) with the 1D
    linear-element matrices M1 = h/6 tridiag(1,4,1), K1 = 1/h tridiag(-1,2,-1)."""
    h = 1.0 / (m + 1)
    o = np.ones(m - 1)
    M1 = (h / 6.0) * sp.diags([o, np.full(m, 4.0), o], [-1, 0, 1])
    K1 = (1.0 / h) * sp.diags([-o, np.full(m, 2.0), -o], [-1, 0, 1])
    M = sp.kron(M1, M1).tocsr()
    K = (a * (sp.kron(M1, K1) + sp.kron(K1, M1))).tocsr()
    return M, K


# --------------------------------------------------------------------------
# All-at-once system (Sec. 2 eq. allatoncesystem; Sec. 4 eqs. pstepscheme and
# pstepbecpreconditioner)
# --------------------------------------------------------------------------
def time_toeplitz(N: int, r=BDF1) -> sp.csr_matrix:
    """R: lower-triangular Toeplitz with R[n, n-j] = r_j, j = 0..p."""
    R = sp.lil_matrix((N, N))
    for n in range(N):
        for j, rj in enumerate(r):
            if n - j >= 0:
                R[n, n - j] = rj
    return R.tocsr()


def time_eps_circulant(N: int, eps: float, r=BDF1) -> sp.csr_matrix:
    """R_eps: R with the wrapped-around entries eps * r_j in the top-right corner,
    R_eps[n, n-j+N] = eps r_j for j > n."""
    R = sp.lil_matrix((N, N))
    for n in range(N):
        for j, rj in enumerate(r):
            if n - j >= 0:
                R[n, n - j] += rj
            else:
                R[n, n - j + N] += eps * rj
    return R.tocsr()


def assemble_L(N: int, M, K, tau: float, r=BDF1) -> sp.csr_matrix:
    """L = R (x) M + tau I_N (x) K.  For BDF1 this is the block lower-bidiagonal
    matrix of Sec. 2 with A_0 = M + tau K on the diagonal and -M below it."""
    return (sp.kron(time_toeplitz(N, r), M) + tau * sp.kron(sp.identity(N), K)).tocsr()


def assemble_P(N: int, M, K, tau: float, eps: float, r=BDF1) -> sp.csr_matrix:
    """P_eps = R_eps (x) M + tau I_N (x) K; for BDF1 it is L with -eps M in block
    (1, N) (definition at the start of Sec. 3)."""
    return (sp.kron(time_eps_circulant(N, eps, r), M)
            + tau * sp.kron(sp.identity(N), K)).tocsr()


def build_rhs(u0: np.ndarray, fsrc: np.ndarray, tau: float, M=None) -> np.ndarray:
    """f = (tau f^1 + M u^0; tau f^2; ...; tau f^N) (Sec. 2), same shape as fsrc."""
    f = tau * np.asarray(fsrc, dtype=np.float64)
    flat0 = np.asarray(u0, dtype=np.float64).reshape(-1)
    mu0 = flat0 if M is None else M @ flat0
    f[0] += mu0.reshape(f[0].shape)
    return f


def timestep_solve(f: np.ndarray, M, K, tau: float) -> np.ndarray:
    """u = L^{-1} f by sequential backward-Euler stepping (eq. stepsystem):
    A_0 u^1 = f^1 and A_0 u^n = f^n + M u^{n-1}, A_0 = M + tau K, one sparse LU of
    A_0.  This is the block lower-triangular Toeplitz inverse of eq.
    elinvlttexpres applied slice by slice."""
    N = f.shape[0]
    F = f.reshape(N, -1)
    lu = spla.splu((M + tau * K).tocsc())
    u = np.empty_like(F)
    prev = None
    for n in range(N):
        rhs = F[n] if prev is None else F[n] + M @ prev
        u[n] = lu.solve(rhs)
        prev = u[n]
    return u.reshape(f.shape)


def build_rhs_pstep(u0: np.ndarray, fsrc: np.ndarray, tau: float, r=BDF1, M=None) -> np.ndarray:
    """Right-hand side of the p-step all-at-once system L u = f with
    L = R (x) M + tau I_N (x) K (eq. pstepscheme).  Block row n of R u reaches
    back to u^{n-p}; the terms r_j M u^{n-j} with n - j <= 0 are known and move
    to the right: f^n = tau f^n - sum_{j=n}^{p} r_j M u^{n-j}, n = 1..p.
    The paper does not state the values before u^0; this reading takes them
    all equal to u^0, so f^n = tau f^n - (r_n + ... + r_p) M u^0.  For BDF1
    it is build_rhs."""
    f = tau * np.asarray(fsrc, dtype=np.float64)
    flat0 = np.asarray(u0, dtype=np.float64).reshape(-1)
    mu0 = (flat0 if M is None else M @ flat0).reshape(f[0].shape)
    p = len(r) - 1
    for n in range(1, min(p, f.shape[0]) + 1):     # 1-based block row n
        f[n - 1] -= sum(r[n:]) * mu0
    return f


def timestep_solve_pstep(f: np.ndarray, M, K, tau: float, r=BDF1) -> np.ndarray:
    """u = L^{-1} f for L = R (x) M + tau I_N (x) K (eq. pstepscheme) by
    stepping block row after block row of the lower-triangular Toeplitz R:
    (r_0 M + tau K) u^n = f^n - sum_{j=1}^{min(p, n-1)} r_j M u^{n-j},
    one sparse LU of r_0 M + tau K."""
    N = f.shape[0]
    F = f.reshape(N, -1)
    lu = spla.splu((r[0] * M + tau * K).tocsc())
    u = np.empty_like(F)
    for n in range(N):
        rhs = F[n].copy()
        for j in range(1, len(r)):
            if n - j >= 0:
                rhs -= r[j] * (M @ u[n - j])
        u[n] = lu.solve(rhs)
    return u.reshape(f.shape)


# --------------------------------------------------------------------------
# The epsilon-circulant diagonalisation (Sec. 4, eq. repsdiagform)
# --------------------------------------------------------------------------
def fourier_matrix(N: int) -> np.ndarray:
    """F_N = N^{-1/2} [theta^{(i-1)(j-1)}], theta = exp(2 pi i / N) (eq. fouriermatdef)."""
    k = np.arange(N)
    return np.exp(2j * np.pi * np.outer(k, k) / N) / math.sqrt(N)


def eps_scaling(N: int, eps: float) -> np.ndarray:
    """Diagonal of D_eps = diag(eps^{0/N}, eps^{1/N}, ..., eps^{(N-1)/N})."""
    return eps ** (np.arange(N) / N)


def eps_circulant_eigs(N: int, eps: float, r=BDF1) -> np.ndarray:
    """lambda_k = sum_{j=0}^{p} r_j eps^{j/N} theta^{kj}, k = 0..N-1."""
    k = np.arange(N)
    lam = np.zeros(N, dtype=np.complex128)
    for j, rj in enumerate(r):
        lam += rj * eps ** (j / N) * np.exp(2j * np.pi * k * j / N)
    return lam


def dst_matrix(m: int) -> np.ndarray:
    """Orthonormal DST-I matrix S[j, k] = sqrt(2/(m+1)) sin(pi (j+1)(k+1)/(m+1));
    S is symmetric and S @ S = I."""
    j = np.arange(1, m + 1)
    return math.sqrt(2.0 / (m + 1)) * np.sin(np.pi * np.outer(j, j) / (m + 1))


def fd_dst_eigs(m: int, a: float = 1.0) -> np.ndarray:
    """Eigenvalues of the 1D FD stiffness: mu_k = (4a/h^2) sin^2(k pi h / 2),
    k = 1..m, with eigenvectors the columns of dst_matrix(m)."""
    h = 1.0 / (m + 1)
    k = np.arange(1, m + 1)
    return (4.0 * a / h ** 2) * np.sin(k * np.pi * h / 2.0) ** 2


# --------------------------------------------------------------------------
# Applying P_eps^{-1}
# --------------------------------------------------------------------------
def apply_Pinv_dense(P, y: np.ndarray) -> np.ndarray:
    """z = P_eps^{-1} y by a dense solve (tiny sizes only)."""
    Pd = P.toarray() if sp.issparse(P) else np.asarray(P)
    return np.linalg.solve(Pd, y.reshape(-1)).reshape(y.shape)


def _band_storage(A: sp.spmatrix, bw: int) -> np.ndarray:
    """LAPACK band storage ab[bw + i - j, j] = A[i, j] for lower = upper = bw."""
    C = A.tocoo()
    ab = np.zeros((2 * bw + 1, A.shape[0]), dtype=np.float64)
    ab[bw + C.row - C.col, C.col] = C.data
    return ab


def _bandwidth(A: sp.spmatrix) -> int:
    C = A.tocoo()
    return int(np.max(np.abs(C.row - C.col))) if C.nnz else 0


def apply_Pinv_lu(y: np.ndarray, M, K, tau: float, eps: float, r=BDF1,
                  freqs=None) -> np.ndarray:
    """z = P_eps^{-1} y by the three steps of Sec. 4 (eqs. ytild, blockdiaginv,
    zcompt), every one of the N shifted systems B_k = lambda_k M + tau K solved
    by complex banded LU (LAPACK gbsv through scipy.linalg.solve_banded).

    Step 1: y~ = [(F_N D_eps) (x) I_J] y;  Step 2: B_k z~^{k+1} = y~^{k+1};
    Step 3: z = [(D_eps^{-1} F_N^*) (x) I_J] z~.  F_N x = sqrt(N) ifft(x) and
    F_N^* x = fft(x)/sqrt(N) under eq. fouriermatdef.

    ``freqs`` (optional) restricts Step 2 to those k and returns the
    partial spectrum z~ (used to time a bounded sample)."""
    N = y.shape[0]
    Y = y.reshape(N, -1).astype(np.float64)
    d = eps_scaling(N, eps)
    yt = math.sqrt(N) * np.fft.ifft(d[:, None] * Y, axis=0)          # Step 1
    lam = eps_circulant_eigs(N, eps, r)
    bw = max(_bandwidth(M), _bandwidth(K))
    Mb, Kb = _band_storage(M, bw), _band_storage(K, bw)
    ks = range(N) if freqs is None else freqs
    zt = np.zeros_like(yt)
    for k in ks:                                                      # Step 2
        ab = lam[k] * Mb + tau * Kb
        zt[k] = sla.solve_banded((bw, bw), ab, yt[k], check_finite=False)
    if freqs is not None:
        return zt
    z = (np.fft.fft(zt, axis=0) / math.sqrt(N)) / d[:, None]           # Step 3
    return z.real.reshape(y.shape)


def apply_Pinv_woodbury(y: np.ndarray, M, K, tau: float, eps: float) -> np.ndarray:
    """z = P_eps^{-1} y by Theorem pinvertibility (BDF1):
    P_eps^{-1} = L^{-1} + L^{-1} E_1 Z_eps^{-1} E_N^T L^{-1},
    Z_eps = eps^{-1} [I - eps (A_0^{-1} M)^N] M^{-1}.
    Uses no Fourier or sine transform: w = L^{-1} y by stepping, x = Z_eps^{-1} w^N,
    then z = w + L^{-1} E_1 x (stepping from the single slice x)."""
    N = y.shape[0]
    Y = y.reshape(N, -1).astype(np.float64)
    J = Y.shape[1]
    A0 = (M + tau * K).tocsc()
    lu = spla.splu(A0)
    w = timestep_solve(Y, M, K, tau)
    wN = w[N - 1]

    def G_pow_N(v):
        for _ in range(N):
            v = lu.solve(M @ v)
        return v

    # Z_eps x = w^N  <=>  [I - eps G^N] q = eps w^N with q = M^{-1} x, G = A_0^{-1} M
    if J <= 1024:
        GN = np.column_stack([G_pow_N(e) for e in np.eye(J)])
        q = np.linalg.solve(np.eye(J) - eps * GN, eps * wN)
    else:
        op = spla.LinearOperator((J, J), matvec=lambda v: v - eps * G_pow_N(v), dtype=np.float64)
        q, info = spla.gmres(op, eps * wN, rtol=1e-15, atol=0.0, restart=60, maxiter=200)
        if info != 0:
            raise RuntimeError("Woodbury inner solve did not converge")
    x = M @ q
    corr = np.zeros_like(Y)
    corr[0] = x
    z = w + timestep_solve(corr, M, K, tau)
    return z.reshape(y.shape)


def _dst_spatial(x: np.ndarray, dim: int) -> np.ndarray:
    """Orthonormal DST-I over the spatial axes of [N][...] data (S is its own inverse)."""
    axes = tuple(range(1, dim + 1))
    if np.iscomplexobj(x):
        return (sfft.dstn(x.real, type=1, axes=axes, norm="ortho")
                + 1j * sfft.dstn(x.imag, type=1, axes=axes, norm="ortho"))
    return sfft.dstn(x, type=1, axes=axes, norm="ortho")


def apply_Pinv_fst(y: np.ndarray, dim: int, a: float, tau: float, eps: float,
                   r=BDF1) -> np.ndarray:
    """z = P_eps^{-1} y for the FD Laplacian with constant a (M = I): the three
    steps of Sec. 4 where every B_k = lambda_k I + tau K is diagonalised by the
    1D, 2D or 3D sine transform (remark after eq. zcompt): B_k^{-1} = S
    diag(1/(lambda_k + tau mu)) S with mu the FD eigenvalues (sums of the 1D
    ones over the axes).  All N frequencies are solved."""
    N = y.shape[0]
    m = y.shape[1]
    d = eps_scaling(N, eps)
    shape_b = (N,) + (1,) * dim
    yt = math.sqrt(N) * np.fft.ifft(d.reshape(shape_b) * y, axis=0)  # Step 1
    mu1 = fd_dst_eigs(m, a)
    if dim == 1:
        mu = mu1
    elif dim == 2:
        mu = mu1[:, None] + mu1[None, :]
    else:
        mu = mu1[:, None, None] + mu1[None, :, None] + mu1[None, None, :]
    lam = eps_circulant_eigs(N, eps, r)
    yh = _dst_spatial(yt, dim)                                         # Step 2
    zh = yh / (lam.reshape(shape_b) + tau * mu[None, ...])
    zt = _dst_spatial(zh, dim)
    z = (np.fft.fft(zt, axis=0) / math.sqrt(N)) / d.reshape(shape_b)  # Step 3
    return z.real


# --------------------------------------------------------------------------
# Krylov solvers (Sec. 5: restarted GMRES, x0 = 0, tolerance relative to r0)
# --------------------------------------------------------------------------
def _givens(a: float, b: float):
    if b == 0.0:
        return 1.0, 0.0
    t = math.hypot(a, b)
    return a / t, b / t


def gmres(Aop, b: np.ndarray, Minv=None, restart: int = 50, tol: float = 1e-7,
          maxiter: int = 1000, x0=None, left: bool = True):
    """Restarted GMRES(restart) with modified Gram-Schmidt Arnoldi and Givens
    rotations.  With ``left=True`` it solves Minv(A x) = Minv(b) and stops when
    the preconditioned residual satisfies ||r_k|| <= tol ||r_0|| (Sec. 5);
    with ``left=False`` it is right-preconditioned (A Minv w = b, x = Minv w) and
    the monitored residual is the true one.  Returns (x, info) where info has
    'iters' (total inner iterations), 'resvec' (monitored residual norms,
    starting with ||r_0||) and 'converged'."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = b.size
    ident = (lambda v: v)
    P = Minv if Minv is not None else ident
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()

    def residual(xv):
        r = b - Aop(xv)
        return P(r) if left else r

    r = residual(x)
    beta = float(np.linalg.norm(r))
    r0 = beta
    resvec = [beta]
    iters = 0
    converged = beta == 0.0
    while not converged and iters < maxiter:
        V = np.zeros((restart + 1, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            w = P(Aop(V[j])) if left else Aop(P(V[j]))
            iters += 1
            for i in range(j + 1):                    # modified Gram-Schmidt
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                        # previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            resvec.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * r0 or iters >= maxiter:
                converged = abs(g[j + 1]) <= tol * r0
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        upd = V[:k].T @ y
        x = x + (upd if left else P(upd))
        if converged or iters >= maxiter:
            break
        r = residual(x)
        beta = float(np.linalg.norm(r))
        if beta <= tol * r0:
            converged = True
            break
    return x, {"iters": iters, "resvec": np.array(resvec), "converged": converged,
               "r0": r0}


def fgmres(Aop, b: np.ndarray, Minv, restart: int = 30, tol: float = 1e-8,
           maxiter: int = 1000, x0=None):
    """Right-preconditioned flexible GMRES(restart): z_j = Minv(v_j) may change
    from one iteration to the next (inexact or non-linear inner solves), the
    basis Z is kept, x += Z y.  Stops when the true-residual estimate satisfies
    ||b - A x|| <= tol ||b - A x0||."""
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    n = b.size
    x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(-1).copy()
    r = b - Aop(x)
    beta = float(np.linalg.norm(r))
    r0 = beta
    resvec = [beta]
    iters = 0
    converged = beta == 0.0
    while not converged and iters < maxiter:
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(restart):
            Z[j] = Minv(V[j])
            w = Aop(Z[j])
            iters += 1
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            resvec.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * r0 or iters >= maxiter:
                converged = abs(g[j + 1]) <= tol * r0
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        x = x + Z[:k].T @ y
        if converged or iters >= maxiter:
            break
        r = b - Aop(x)
        beta = float(np.linalg.norm(r))
        if beta <= tol * r0:
            converged = True
            break
    return x, {"iters": iters, "resvec": np.array(resvec), "converged": converged,
               "r0": r0}


def relative_residual(L, u: np.ndarray, f: np.ndarray) -> float:
    """RES = ||f - L u||_2 / ||f||_2 (Sec. 5)."""
    fv = f.reshape(-1)
    return float(np.linalg.norm(fv - L @ u.reshape(-1)) / np.linalg.norm(fv))


# --------------------------------------------------------------------------
# Multigrid route for variable coefficients (Sec. 4: "a multigrid method as
# inner spatial solver"; Sec. 5, Example 2: one V-cycle per shifted system,
# one pre- and one post-smoothing step, piecewise-linear interpolation and its
# transpose).  Readings: bilinear prolongation P, restriction R = P^T / 4,
# Galerkin coarse operators, damped Jacobi (omega = 0.8) in place of ILU.
# --------------------------------------------------------------------------
def mg_prolongation(mc: int) -> sp.csr_matrix:
    """Bilinear interpolation from the (mc x mc) interior grid of spacing 2h to
    the (2mc+1)^2 fine interior grid, zero Dirichlet data.  1D factor:
    fine 2i+1 <- coarse i (weight 1), fine 2i <- coarse i-1, i (weights 1/2)."""
    mf = 2 * mc + 1
    P1 = sp.lil_matrix((mf, mc))
    for i in range(mc):
        P1[2 * i + 1, i] = 1.0
        P1[2 * i, i] += 0.5
        P1[2 * i + 2, i] += 0.5
    P1 = P1.tocsr()
    return sp.kron(P1, P1).tocsr()


class MGHierarchy:
    """Grids m_0 = m > m_1 = (m-1)/2 > ... > 1, with P_l, R_l = P_l^T/4 and the
    Galerkin pairs (M_l, K_l): M_0 = I, K_0 = K, M_{l+1} = R_l M_l P_l,
    K_{l+1} = R_l K_l P_l.  B_k on level l is lambda M_l + tau K_l."""

    def __init__(self, K: sp.spmatrix, m: int):
        self.sizes = [m]
        while self.sizes[-1] > 1:
            self.sizes.append((self.sizes[-1] - 1) // 2)
        self.P, self.R, self.M, self.K = [], [], [sp.identity(m * m, format="csr")], [K.tocsr()]
        for l in range(len(self.sizes) - 1):
            P = mg_prolongation(self.sizes[l + 1])
            R = (P.T / 4.0).tocsr()
            self.P.append(P)
            self.R.append(R)
            self.M.append((R @ self.M[l] @ P).tocsr())
            self.K.append((R @ self.K[l] @ P).tocsr())

    def op(self, l: int, lam: complex, tau: float):
        return (lam * self.M[l] + tau * self.K[l]).tocsr()


def dilu_diagonal(A) -> np.ndarray:
    """The diagonal D of the incomplete factorisation M = (D + L) D^{-1} (D + U)
    of A = L + diag(A) + U (L, U its strictly lower and upper parts) that
    makes diag(M) = diag(A): d_i = a_ii - sum_{j < i} a_ij a_ji / d_j over the
    neighbours j of i.  On a 5-point matrix this M is ILU(0) (M = A on the
    pattern of A).  This is the ILU smoother of the multigrid route (Example 2
    and 3 of Sec. 5 smooth with ILU); the sum runs row by row in order."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    d = np.array(A.diagonal(), dtype=np.complex128)
    for i in range(n):
        acc = 0.0 + 0.0j
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            if j < i:
                aji = A[j, i]
                if aji != 0:
                    acc += A.data[p] * aji / d[j]
        d[i] = d[i] - acc
    return d


def dilu_solve(A, d: np.ndarray, r: np.ndarray) -> np.ndarray:
    """z = M^{-1} r for M = (D + L) D^{-1} (D + U): forward (D + L) y = r, then
    backward (D + U) z = D y, both by plain row loops."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    y = np.zeros(n, dtype=np.complex128)
    for i in range(n):
        acc = r[i]
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            if j < i:
                acc -= A.data[p] * y[j]
        y[i] = acc / d[i]
    z = np.zeros(n, dtype=np.complex128)
    for i in range(n - 1, -1, -1):
        acc = 0.0 + 0.0j
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            if j > i:
                acc += A.data[p] * z[j]
        z[i] = y[i] - acc / d[i]
    return z


def mg_vcycle(h: MGHierarchy, lam: complex, tau: float, b: np.ndarray, omega: float = 0.8,
              nu1: int = 1, nu2: int = 1, l: int = 0, x0=None, smoother: str = "jacobi",
              dcache=None) -> np.ndarray:
    """One V-cycle for (lam M_l + tau K_l) x = b from x0 (zero if None): nu1
    smoothing sweeps, residual, restriction, recursive coarse correction,
    prolongation, nu2 sweeps.  The 1 x 1 coarsest grid is solved exactly.
    smoother="jacobi": x <- x + omega D^{-1} (b - A x); smoother="ilu":
    x <- x + M^{-1} (b - A x) with M the incomplete factorisation of
    dilu_diagonal (``dcache`` may hold its diagonals per level)."""
    A = h.op(l, lam, tau)
    if h.sizes[l] == 1:
        return b / A.toarray()[0, 0]
    if smoother == "ilu":
        if dcache is None:
            dcache = {}
        if l not in dcache:
            dcache[l] = dilu_diagonal(A)
        dl = dcache[l]

        def sweep(v, rr):
            return v + dilu_solve(A, dl, rr)
    else:
        dinv = 1.0 / A.diagonal()

        def sweep(v, rr):
            return v + omega * dinv * rr
    x = np.zeros_like(b, dtype=np.complex128) if x0 is None else x0.astype(np.complex128)
    for _ in range(nu1):
        x = sweep(x, b - A @ x)
    r = b - A @ x
    ec = mg_vcycle(h, lam, tau, h.R[l] @ r, omega, nu1, nu2, l + 1, smoother=smoother,
                   dcache=dcache)
    x = x + h.P[l] @ ec
    for _ in range(nu2):
        x = sweep(x, b - A @ x)
    return x


def apply_Pinv_mg(y: np.ndarray, h: MGHierarchy, tau: float, eps: float, r=BDF1,
                  omega: float = 0.8, nu1: int = 1, nu2: int = 1, smoother: str = "jacobi",
                  dcaches=None) -> np.ndarray:
    """Approximate P_eps^{-1} y by the three steps of Sec. 4 with Step 2 done
    by one V-cycle per shifted system (all N frequencies).  ``dcaches`` (a
    dict, optional) keeps the ILU diagonals per frequency across calls."""
    N = y.shape[0]
    Y = y.reshape(N, -1).astype(np.float64)
    d = eps_scaling(N, eps)
    yt = math.sqrt(N) * np.fft.ifft(d[:, None] * Y, axis=0)          # Step 1
    lam = eps_circulant_eigs(N, eps, r)
    zt = np.empty_like(yt)
    for k in range(N):                                                # Step 2
        dc = None if dcaches is None else dcaches.setdefault(k, {})
        zt[k] = mg_vcycle(h, lam[k], tau, yt[k], omega, nu1, nu2, smoother=smoother, dcache=dc)
    z = (np.fft.fft(zt, axis=0) / math.sqrt(N)) / d[:, None]           # Step 3
    return z.real.reshape(y.shape)


def node_coefficient(g: np.ndarray) -> np.ndarray:
    """a = exp(g) on all (m+2)^2 nodes (the variable diffusion coefficient)."""
    return np.exp(g)
