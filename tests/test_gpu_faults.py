"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported to the host as BEC_ETIMEOUT and leaves the context usable.  The
failure is injected on the host (bec_inject_fault): the next tensor-core
convolution, or the next TMA-staged FP32 preconditioner pass, withholds its
tile loads, so its waits run out after about 0.2 s and the kernel tears down
with nothing in flight.  No trap,
assert, bad address or endless loop is involved."""
import ctypes

import numpy as np
import pytest

import oracle as O
from workloads import grf_log_coefficient

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2002_01108_gb300 import build
    build.build()


def test_withheld_loads_time_out_and_the_context_survives():
    import torch
    from paper_2002_01108_gb300 import BecError, Problem, load
    from paper_2002_01108_gb300.bec import BEC_ETIMEOUT
    lib = load()
    m, N = 63, 16
    a = O.node_coefficient(grf_log_coefficient(seed=5, m=m))
    rng = np.random.default_rng(4)
    r = torch.from_numpy(rng.standard_normal((4, m, m)) + 1j * rng.standard_normal((4, m, m))).cuda()
    mc = (m - 1) // 2
    e = torch.from_numpy(rng.standard_normal((4, mc, mc)) + 1j * rng.standard_normal((4, mc, mc))).cuda()
    with Problem(2, m, N, route="learned", precision="fp32", a_nodes=a, flexible=True) as p:
        p.set_eps(0.1)
        loss0, _ = p.learned_loss_grad([0, 2, 4, 6], r, e)
        assert lib.bec_inject_fault(1) == 0
        with pytest.raises(BecError) as info:
            p.learned_loss_grad([0, 2, 4, 6], r, e)
        assert info.value.status == BEC_ETIMEOUT
        assert b"ran out" in lib.bec_last_error()
        # one-shot: the next call runs normally and gives the same loss
        loss1, _ = p.learned_loss_grad([0, 2, 4, 6], r, e)
        assert loss1 == loss0
    assert lib.bec_inject_fault(0) == 0
    assert lib.bec_inject_fault(7) == 1          # unknown kind: BEC_EINVAL


@pytest.mark.parametrize("m,N", [(255, 8), (31, 256)])
def test_withheld_tma_tiles_time_out_and_the_context_survives(m, N):
    """The TMA-staged FP32 passes (the n = 256 column pass at 255^2 x 8, the
    N = 256 time pass at 31^2 x 256): with the next launch's tile loads
    withheld, every block's bounded wait runs out, the blocks return without
    writing, and the solve reports BEC_ETIMEOUT; the next solve on the same
    problem equals the one before the injection bit for bit."""
    import torch
    from paper_2002_01108_gb300 import BecError, Problem, load
    from paper_2002_01108_gb300.bec import BEC_ETIMEOUT
    lib = load()
    f = torch.from_numpy(np.random.default_rng(8).uniform(-1, 1, (N, m, m))).cuda()
    with Problem(2, m, N, precision="fp32", flexible=True, max_restart=10) as p:
        p.set_eps(0.05)
        u0, i0 = p.gmres_solve(f, restart=10, rtol=1e-10, flexible=True)
        assert i0["converged"] == 1
        assert lib.bec_inject_fault(3) == 0
        with pytest.raises(BecError) as info:
            p.gmres_solve(f, restart=10, rtol=1e-10, flexible=True)
        assert info.value.status == BEC_ETIMEOUT
        assert b"ran out" in lib.bec_last_error()
        u1, i1 = p.gmres_solve(f, restart=10, rtol=1e-10, flexible=True)
        torch.cuda.synchronize()
        assert i1["iters"] == i0["iters"] and torch.equal(u1, u0)
