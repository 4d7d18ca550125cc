"""The precision workload: 2D heat on a 511 x 511 grid with N = 512 steps
(133.7M space-time unknowns), eps = sqrt(tau).  The FP32/complex64
preconditioner inside FP64 flexible GMRES(20) and the plain FP64 form both
reach RES <= 1e-8; solved to 1e-10 both match the oracle's sequential
backward-Euler solution to relative error <= 1e-8."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import oracle as O
from workloads import heat_case_2d

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    from paper_2002_01108_gb300 import build
    build.build()
    case = heat_case_2d(seed=3, m=511, N=512, eps=math.sqrt(1.0 / 512))
    f = O.build_rhs(case.u0, case.fsrc, case.tau)
    K = O.fd_stiffness(2, case.m)
    u_ref = O.timestep_solve(f, sp.identity(K.shape[0], format="csr"), K, case.tau)
    return case, f, u_ref


@pytest.mark.parametrize("form", ["fp32", "fp64"])
def test_precision_workload_511_N512(workload, form):
    import torch
    from paper_2002_01108_gb300 import Problem
    case, f, u_ref = workload
    with Problem(2, case.m, case.N, precision=form, flexible=True, max_restart=20) as p:
        p.set_eps(case.eps)
        fd = torch.from_numpy(f).cuda()
        u, info = p.gmres_solve(fd, restart=20, rtol=1e-8, flexible=True)
        assert info["converged"] == 1 and info["true_relres"] <= 1.01e-8, info
        u, info = p.gmres_solve(fd, u, restart=20, rtol=1e-10, flexible=True)
        assert info["true_relres"] <= 1.01e-10, info
        torch.cuda.synchronize()
        err = float(np.linalg.norm(u.cpu().numpy() - u_ref) / np.linalg.norm(u_ref))
        del fd, u
    assert err <= 1e-8, err
