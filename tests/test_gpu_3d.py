"""3D domains (the PDE of Sec. 2 is posed in R^2 or R^3) on the sine-transform
route: the 7-point all-at-once operator against the oracle's assembled
matrix; P_eps^{-1} (x-, y- and z-DST, time pass) against the oracle's
sine-transform and banded-LU routes, in FP64 and FP32; and GMRES / FGMRES
reaching the sequential-stepping solution.

Tolerances as in 2D: the stencil 8 u (1 + 2 dim c) max|v|; P_eps^{-1} 16 u
log2(N n^dim) / eps (one more transform axis)."""
import math

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


@pytest.mark.parametrize("m,N,a", [(7, 8, 1.0), (15, 16, 0.3), (31, 4, 2.0)])
def test_apply_A_3d(m, N, a):
    from paper_2002_01108_gb300 import Problem
    K = O.fd_stiffness(3, m, a)
    tau = 1.0 / N
    v = np.random.default_rng(1).uniform(-1, 1, (N, m, m, m))
    with Problem(3, m, N, a=a) as p:
        y = host(p.apply_A(dev(v)))
    ref = (O.assemble_L(N, sp.identity(m ** 3, format="csr"), K, tau) @ v.reshape(-1)).reshape(v.shape)
    c = tau * a * (m + 1) ** 2
    assert np.max(np.abs(y - ref)) <= 8 * U64 * (1 + 6 * c) * np.max(np.abs(v))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("m,N,eps", [(7, 8, 0.1), (15, 32, 0.0625), (31, 16, 1e-3), (63, 8, 0.5),
                                     (15, 256, 0.0625)])
def test_apply_Pinv_3d_matches_oracle(precision, m, N, eps):
    from paper_2002_01108_gb300 import Problem
    a = 1.0
    y = np.random.default_rng(2).uniform(-1, 1, (N, m, m, m))
    with Problem(3, m, N, a=a, precision=precision, flexible=True) as p:
        p.set_eps(eps)
        z = host(p.apply_Pinv(dev(y)))
    ref = O.apply_Pinv_fst(y, 3, a, 1.0 / N, eps)
    u = U64 if precision == "fp64" else U32
    tol = 16 * u * math.log2(N * (m + 1) ** 3) / eps
    err = float(np.max(np.abs(z - ref)) / np.max(np.abs(ref)))
    assert err <= tol, (err, tol)
    if m == 7:   # the banded-LU route as well (independent of any transform)
        K = O.fd_stiffness(3, m, a)
        lu = O.apply_Pinv_lu(y.reshape(N, -1), sp.identity(m ** 3, format="csr"), K, 1.0 / N,
                             eps).reshape(y.shape)
        assert float(np.max(np.abs(z - lu)) / np.max(np.abs(lu))) <= tol + 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gmres_3d_reaches_time_stepping(precision):
    import torch
    from paper_2002_01108_gb300 import Problem
    m, N, a = 31, 32, 1.0
    tau = 1.0 / N
    rng = np.random.default_rng(3)
    u0 = rng.uniform(-1, 1, (m, m, m))
    fs = rng.uniform(-1, 1, (N, m, m, m))
    f = O.build_rhs(u0, fs, tau)
    K = O.fd_stiffness(3, m, a)
    u_ref = O.timestep_solve(f, sp.identity(m ** 3, format="csr"), K, tau)
    with Problem(3, m, N, a=a, precision=precision, flexible=precision == "fp32") as p:
        p.set_eps(math.sqrt(tau))
        fd = p.build_rhs(dev(u0), dev(fs))
        assert np.max(np.abs(host(fd) - f)) <= 4 * U64 * np.max(np.abs(f))
        u, info = p.gmres_solve(fd, restart=20, rtol=1e-12, flexible=precision == "fp32")
        torch.cuda.synchronize()
    err = float(np.linalg.norm(host(u) - u_ref) / np.linalg.norm(u_ref))
    assert info["converged"] and info["true_relres"] <= 1.01e-12 and err <= 1e-9, (info, err)
