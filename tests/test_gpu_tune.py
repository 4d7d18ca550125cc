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


def test_tune_cache_file_is_written_and_read(tmp_path):
    """BEC_TUNE_CACHE: a forced tuning appends the shape's choice to the file,
    and a process that starts with the file takes the choice from it,
    skipping lines it cannot use."""
    import os
    import subprocess
    import sys
    path = tmp_path / "tune.txt"
    code = (
        "import torch, sys\n"
        "from paper_2002_01108_gb300 import Problem\n"
        "with Problem(2, 63, 32, precision='fp32', flexible=True) as p:\n"
        "    p.set_eps(0.1)\n"
        "    r = p.autotune(force=len(sys.argv) > 1)\n"
        "    print(int(r['cached']), r['rows_warps'], r['cols_warps'], r['time_warps'])\n")
    env = dict(os.environ, BEC_TUNE_CACHE=str(path))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    first = subprocess.run([sys.executable, "-c", code, "force"], env=env, cwd=root,
                           capture_output=True, text=True, check=True).stdout.split()
    text = path.read_text()
    assert text.split()[:4] == ["0", "2", "63", "32"]
    # a malformed line and a line with invalid widths for the same shape are skipped
    path.write_text("not a tuning line\n" + text + "0 2 63 32 3 3 3\n")
    second = subprocess.run([sys.executable, "-c", code], env=env, cwd=root,
                            capture_output=True, text=True, check=True).stdout.split()
    assert first[0] == "0" and second[0] == "1" and second[1:] == first[1:]
