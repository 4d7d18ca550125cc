"""The integer FP64 <-> FP32 conversions of the FP32 preconditioner passes
against the hardware conversion (torch's .to(), round to nearest even), bit
for bit: random values over the whole exponent range, exact ties with even
and odd mantissas, the edges of the float range (largest finite, rounding
to infinity, smallest normal, subnormal results), signed zeros, infinities
and NaN."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2002_01108_gb300 import build
    build.build()


def _doubles():
    rng = np.random.default_rng(1)
    parts = [rng.standard_normal(100000) * np.exp2(rng.integers(-160, 160, 100000)),
             rng.uniform(-1, 1, 100000)]
    # exact midpoints between adjacent floats (ties), even and odd mantissas
    f = rng.standard_normal(20000).astype(np.float32)
    g = np.nextafter(f, np.float32(np.inf))
    parts.append((f.astype(np.float64) + g.astype(np.float64)) / 2)
    # one ulp of the double on either side of a tie
    t = parts[-1]
    parts += [np.nextafter(t, np.inf), np.nextafter(t, -np.inf)]
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    edges = [0.0, -0.0, np.inf, -np.inf, np.nan, fmax, -fmax, np.nextafter(fmax, np.inf),
             fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24), tiny, -tiny, tiny / 2, tiny * 0.75,
             np.nextafter(tiny, 0.0), 1e-45, 1e-50, 1e300, -1e300, 2.0 ** 127, 2.0 ** 128, 2.0 ** -126,
             2.0 ** -127, 2.0 ** -149, 2.0 ** -150, 1.0, -1.0, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24]
    parts.append(np.array(edges))
    return np.concatenate(parts)


def test_double_to_float_matches_the_hardware_bit_for_bit():
    import torch
    from paper_2002_01108_gb300 import convert
    x = torch.from_numpy(_doubles()).cuda()
    y = convert(x)
    ref = x.to(torch.float32)
    torch.cuda.synchronize()
    a = y.view(torch.int32).cpu().numpy()
    b = ref.view(torch.int32).cpu().numpy()
    nan = np.isnan(ref.cpu().numpy())
    assert np.array_equal(np.isnan(y.cpu().numpy()), nan)
    bad = np.nonzero((a != b) & ~nan)[0]
    assert bad.size == 0, (x.cpu().numpy()[bad[:5]], a[bad[:5]], b[bad[:5]])


def test_float_to_double_matches_the_hardware_bit_for_bit():
    import torch
    from paper_2002_01108_gb300 import convert
    rng = np.random.default_rng(2)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    x = torch.from_numpy(bits.view(np.float32).copy()).cuda()
    y = convert(x)
    ref = x.to(torch.float64)
    torch.cuda.synchronize()
    a = y.view(torch.int64).cpu().numpy()
    b = ref.view(torch.int64).cpu().numpy()
    nan = np.isnan(ref.cpu().numpy())
    assert np.array_equal(np.isnan(y.cpu().numpy()), nan)
    assert np.array_equal(a[~nan], b[~nan])


def test_fp64_reciprocal_of_the_smoother_is_within_one_ulp():
    """The FP64 multigrid smoother's reciprocal (float reciprocal plus two
    Newton-Raphson steps) against IEEE division: within one unit in the last
    place over the fast range [2^-120, 2^120] in magnitude, both signs, exact
    powers of two and values next to them; the values outside that range,
    zeros, infinities and NaN take the division and agree exactly."""
    import torch
    from paper_2002_01108_gb300 import reciprocal_fp64
    rng = np.random.default_rng(5)
    x = rng.uniform(1, 2, 200000) * np.exp2(rng.integers(-119, 119, 200000))
    x *= np.where(rng.random(200000) < 0.5, -1.0, 1.0)
    p2 = np.exp2(np.arange(-119, 120, dtype=np.float64))
    x = np.concatenate([x, p2, np.nextafter(p2, np.inf), np.nextafter(p2, 0.0), -p2])
    y = reciprocal_fp64(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = 1.0 / x
    ulp = np.spacing(np.abs(ref))
    assert np.max(np.abs(y - ref) / ulp) <= 1.0
    slow = np.array([2.0 ** -125, -2.0 ** 125, 1e-300, 1e300, 0.0, -0.0, np.inf, -np.inf])
    ys = reciprocal_fp64(torch.from_numpy(slow).cuda()).cpu().numpy()
    with np.errstate(divide="ignore"):
        np.testing.assert_array_equal(ys, 1.0 / slow)
    yn = reciprocal_fp64(torch.tensor([np.nan], dtype=torch.float64).cuda()).cpu().numpy()
    assert np.isnan(yn[0])
