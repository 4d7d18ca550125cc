"""Failure detection without a GPU fault: a bounded device wait that runs out
is reported to the host as BEC_ETIMEOUT and leaves the context usable.  The
failure is injected on the host (bec_inject_fault): the next tensor-core
convolution withholds its tile loads, so its MMA and epilogue waits run out
after about 0.2 s and the kernel tears down with nothing in flight.  No trap,
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
