"""Tile shapes of the P_eps^{-1} passes: every block width gives the same
result bit for bit (the width only regroups lines into blocks), bec_autotune
picks widths from the candidates and caches them per shape, and invalid
widths are refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2002_01108_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("m,N", [(63, 64), (255, 32), (127, 256)])
def test_every_block_width_gives_the_same_result(precision, m, N):
    import torch
    from paper_2002_01108_gb300 import Problem
    y = torch.from_numpy(np.random.default_rng(3).uniform(-1, 1, (N, m, m))).cuda()
    with Problem(2, m, N, precision=precision, flexible=precision == "fp32") as p:
        p.set_eps(0.05)
        ref = p.apply_Pinv(y).clone()
        for rows, cols, time in [(4, 4, 4), (16, 16, 16), (4, 16, 8), (8, 8, 16)]:
            p.set_tiles(rows, cols, time)
            z = p.apply_Pinv(y)
            torch.cuda.synchronize()
            assert torch.equal(z, ref), (rows, cols, time)
        p.set_tiles(0, 0, 0)
        assert torch.equal(p.apply_Pinv(y), ref)


def test_autotune_picks_candidates_and_caches_the_shape():
    import torch
    from paper_2002_01108_gb300 import Problem
    m, N = 127, 64
    y = torch.from_numpy(np.random.default_rng(4).uniform(-1, 1, (N, m, m))).cuda()
    with Problem(2, m, N, precision="fp32", flexible=True) as p:
        p.set_eps(0.1)
        ref = p.apply_Pinv(y).clone()
        r = p.autotune(force=True)
        assert not r["cached"]
        for k in ("rows", "cols", "time"):
            assert r[k + "_warps"] in (4, 8, 16)
            ms = r[k + "_ms"]
            assert all(t > 0 for t in ms) and min(ms) == ms[(4, 8, 16).index(r[k + "_warps"])]
        assert torch.equal(p.apply_Pinv(y), ref)
    with Problem(2, m, N, precision="fp32", flexible=True) as q:
        q.set_eps(0.1)
        r2 = q.autotune()
        assert r2["cached"] and all(r2[k] == r[k] for k in ("rows_warps", "cols_warps", "time_warps"))


def test_invalid_widths_are_refused():
    from paper_2002_01108_gb300 import BecError, Problem
    with Problem(2, 63, 16, precision="fp64") as p:
        p.set_eps(0.1)
        for bad in [(3, 0, 0), (0, 32, 0), (0, 0, 4)]:   # N = 16 < 32: the time pass is not tunable
            with pytest.raises(BecError):
                p.set_tiles(*bad)
    with Problem(2, 63, 1024, precision="fp64") as p:    # 16 warps x N = 1024 in FP64 needs > 227 KB
        p.set_eps(0.1)
        with pytest.raises(BecError):
            p.set_tiles(0, 0, 16)
        p.set_tiles(0, 0, 8)
