"""Q1 (bilinear) finite elements on the sine-transform route (Sec. 5, Example
1): the all-at-once operator L and P_eps with the 9-point mass and
stiffness stencils, the right-hand side with M u0, and P_eps^{-1} with the
divide by lambda_k mu^M + tau mu^K, against the oracle's assembled sparse
matrices and banded LU; then the paper's own Table table1 rows, solved on
the GPU with left-preconditioned GMRES(50) exactly as printed (iteration
counts equal, RES to the printed 3 digits).

Tolerances: the stencil output is a sum of 18 products (9 of M + tau K, 9 of
M), each rounded once: 16 u (sum of |weights|) max|v|.  P_eps^{-1} as on the
finite-difference route: 16 u log2(N n^2) / eps for the transforms plus
16 u max_k cond(lambda_k M + tau K) for the oracle's banded LU."""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O

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


def q1_1d(m, a):
    h = 1.0 / (m + 1)
    o = np.ones(m - 1)
    M1 = (h / 6.0) * sp.diags([o, np.full(m, 4.0), o], [-1, 0, 1])
    K1 = (a / h) * sp.diags([-o, np.full(m, 2.0), -o], [-1, 0, 1])
    return M1.tocsr(), K1.tocsr()


def mats(dim, m, a):
    return O.q1_mass_stiffness(m, a) if dim == 2 else q1_1d(m, a)


@pytest.mark.parametrize("dim,m,N,a", [(2, 31, 8, 1e-2), (2, 63, 4, 1.0), (1, 63, 16, 0.5)])
def test_q1_apply_A_and_P(dim, m, N, a):
    from paper_2002_01108_gb300 import Problem
    M, K = mats(dim, m, a)
    tau = 1.0 / N
    shape = (N, m, m) if dim == 2 else (N, m)
    v = np.random.default_rng(1).uniform(-1, 1, shape)
    with Problem(dim, m, N, a=a, space="q1") as p:
        p.set_eps(0.3)
        y = host(p.apply_A(dev(v)))
        z = host(p.apply_P(dev(v)))
    refL = (O.assemble_L(N, M, K, tau) @ v.reshape(-1)).reshape(shape)
    refP = (O.assemble_P(N, M, K, tau, 0.3) @ v.reshape(-1)).reshape(shape)
    wsum = abs(M + tau * K).sum(axis=1).max() + abs(M).sum(axis=1).max()
    bound = 16 * U64 * wsum * np.max(np.abs(v))
    assert np.max(np.abs(y - refL)) <= bound
    assert np.max(np.abs(z - refP)) <= bound


def test_q1_right_hand_side_has_M_u0():
    from paper_2002_01108_gb300 import Problem
    m, N, a = 31, 8, 0.1
    M, K = O.q1_mass_stiffness(m, a)
    rng = np.random.default_rng(2)
    u0 = rng.uniform(-1, 1, (m, m))
    fs = rng.uniform(-1, 1, (N, m, m))
    with Problem(2, m, N, a=a, space="q1") as p:
        f = host(p.build_rhs(dev(u0), dev(fs)))
    ref = O.build_rhs(u0, fs, 1.0 / N, M)
    assert np.max(np.abs(f - ref)) <= 16 * U64 * np.max(np.abs(ref)) * 2


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dim,m,N,eps,a", [(2, 31, 16, 0.1, 1e-2), (2, 63, 8, 0.0625, 1e-5),
                                           (1, 127, 32, 0.05, 1.0), (2, 31, 256, 0.1, 1e-2)])
def test_q1_apply_Pinv_matches_banded_lu(precision, dim, m, N, eps, a):
    from paper_2002_01108_gb300 import Problem
    M, K = mats(dim, m, a)
    tau = 1.0 / N
    shape = (N, m, m) if dim == 2 else (N, m)
    y = np.random.default_rng(3).uniform(-1, 1, shape)
    with Problem(dim, m, N, a=a, space="q1", precision=precision, flexible=True) as p:
        p.set_eps(eps)
        z = host(p.apply_Pinv(dev(y)))
    ref = O.apply_Pinv_lu(y, M, K, tau, eps)
    u = U64 if precision == "fp64" else U32
    n = m + 1
    # condition of the shifted systems lambda_k M + tau K: both diagonal in the
    # sine basis, eigenvalues lambda_k mu^M + tau mu^K
    lam = O.eps_circulant_eigs(N, eps)
    j = np.arange(1, m + 1)
    mM = (1.0 / n / 3.0) * (2 + np.cos(j * np.pi / n))
    mK = a * 4.0 * n * np.sin(j * np.pi / (2 * n)) ** 2
    if dim == 2:
        muM = np.outer(mM, mM).reshape(-1)
        muK = (np.outer(mM, mK) + np.outer(mK, mM)).reshape(-1)
    else:
        muM, muK = mM, mK
    kappa = max(np.abs(lk * muM + tau * muK).max() / np.abs(lk * muM + tau * muK).min() for lk in lam)
    tol = 16 * u * math.log2(N * n ** dim) / eps + 16 * U64 * kappa
    err = float(np.max(np.abs(z - ref)) / np.max(np.abs(ref)))
    assert err <= tol, (err, tol)


def _table1_rows():
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_bdf1.txt")
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                cols = line.split()
                N, n, it, res, bit, bres = cols[:6]
                flag = cols[6] if len(cols) > 6 else ""
                rows.append((int(N), int(n), int(it), float(res), int(bit), float(bres), flag))
    return rows


@pytest.mark.parametrize("row", range(16))
def test_table1_on_the_gpu(row):
    """Example 1 of Sec. 5: Q1, a = 1e-5, u0 = x(x-1)y(y-1), f = 0, BDF1,
    eps = min(0.5, 0.5 tau), GMRES(50) with left preconditioning, stop at
    1e-7 on the preconditioned residual, x0 = 0: the BEC iteration counts and
    RES of every row of Table table1, and the same for the Strang-type BC
    preconditioner (eps = 1).  No solve reaches 20 iterations, so a Krylov
    basis of 20 vectors gives exactly the GMRES(50) iterates.

    BEC: iterations exact, RES to the 3 printed digits.  BC: iterations exact,
    RES within 10 %: after 13 iterations the stop is a threshold decision and
    RES follows the preconditioned residual at that point.  The entries the
    golden file flags as misprints are checked against the rest of the table
    instead (the rows with the same n, whose BC values do not depend on N,
    and the monotone rise of BEC RES with n)."""
    import torch
    from paper_2002_01108_gb300 import Problem
    rows = _table1_rows()
    N, n, it, res, bit, bres, flag = rows[row]
    same_n = [r for r in rows if r[1] == n and r[0] != N and not r[6]]
    m = n - 1
    x = np.arange(1, m + 1) / (m + 1)
    X, Y = np.meshgrid(x, x)
    u0 = X * (X - 1) * Y * (Y - 1)
    with Problem(2, m, N, a=1e-5, space="q1", max_restart=20) as p:
        f = p.build_rhs(dev(u0), torch.zeros((N, m, m), dtype=torch.float64, device="cuda"))
        p.set_eps(min(0.5, 0.5 / N))
        _, info = p.gmres_solve(f, restart=20, rtol=1e-7, left_pc=True, maxit=500)
        torch.cuda.synchronize()
        assert info["iters"] == it, ("BEC", info)
        if flag == "bec_res":
            lo = next(r[3] for r in rows if r[0] == N and r[1] == n // 2)
            hi = next(r[3] for r in rows if r[0] == N and r[1] == 2 * n)
            assert lo < info["true_relres"] < hi, ("BEC", info["true_relres"], lo, hi)
        else:
            assert abs(info["true_relres"] / res - 1) < 0.01, ("BEC", info["true_relres"], res)
        p.set_eps(1.0)
        _, info = p.gmres_solve(f, restart=20, rtol=1e-7, left_pc=True, maxit=500)
        torch.cuda.synchronize()
        if flag in ("bc", "bc_res"):
            bit, bres = same_n[0][4], same_n[0][5]
        assert info["iters"] == bit, ("BC", info)
        assert abs(info["true_relres"] / bres - 1) < 0.10, ("BC", info["true_relres"], bres)
