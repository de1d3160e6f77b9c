"""The FP64 step kernels' exact integer-pipe arithmetic against IEEE FP64.

The FP64 kernels replace FP64 operations by operations on the bit patterns
(the FP64 pipe of a GB300 runs at 1/64 of the FP32 rate): halving (0.5 x in
the PPM interface values, the MC slope's |a + b|/2 and the limiter's
(p + m)/2, the flux's rho/2), and in the MC-limited slope also the minima,
the doubling and the sign (Sec. III-B; Colella & Woodward 1984).  Each must
give the FP64 operations' bits for every input, including zeros of both
signs, subnormals, the halving's rounding at the subnormal boundary and
products within a factor of a few of the underflow threshold (the slope's
sign test).  numpy's float64 operations are the IEEE reference.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2107_10987_gb300 import _build, hydro
    _build.build()
    return hydro


def _specials():
    tiny = np.float64(5e-324)
    mn = np.float64(2.0 ** -1022)
    v = [0.0, tiny, 3 * tiny, 2 * tiny, np.nextafter(mn, 0.0), mn, np.nextafter(mn, 1.0), 1.5 * mn, 2.0 ** -1021,
         np.nextafter(2.0 ** -1021, 0.0), np.nextafter(2.0 ** -1021, 1.0), 2.0 ** -1020, 2.0 ** -538,
         1.5 * 2.0 ** -538, 2.0 ** -537, np.nextafter(2.0 ** -537, 1.0), 2.0 ** -536, 0.1, 1.0, 3.0,
         1e300, 1e308, np.finfo(np.float64).max]
    v = np.array(v, dtype=np.float64)
    return np.concatenate([v, -v])


def _pairs(seed):
    s = _specials()
    a, b = np.meshgrid(s, s, indexing="ij")
    rng = np.random.default_rng(seed)
    n = 200_000
    # random magnitudes over the whole exponent range, random signs
    ea = rng.integers(-1074, 1024, n)
    eb = rng.integers(-1074, 1024, n)
    ra = np.ldexp(rng.uniform(1.0, 2.0, n), ea - 1) * rng.choice([-1.0, 1.0], n)
    rb = np.ldexp(rng.uniform(1.0, 2.0, n), eb - 1) * rng.choice([-1.0, 1.0], n)
    # products straddling the underflow threshold 2^-1075
    m = 50_000
    e1 = rng.integers(-600, -470, m)
    e2 = -1075 - e1 + rng.integers(-4, 5, m)
    ua = np.ldexp(rng.uniform(1.0, 2.0, m), e1) * rng.choice([-1.0, 1.0], m)
    ub = np.ldexp(rng.uniform(1.0, 2.0, m), e2) * rng.choice([-1.0, 1.0], m)
    x = np.concatenate([a.ravel(), ra, ua])
    y = np.concatenate([b.ravel(), rb, ub])
    return x, y


def test_halving_and_slope_match_ieee_fp64(H):
    x, y = _pairs(7)
    with np.errstate(over="ignore", under="ignore"):
        half = 0.5 * x
        prod = x * y
        pos = prod > 0
        ax, ay = np.abs(x), np.abs(y)
        slope = np.where(pos, np.copysign(np.minimum(2.0 * np.minimum(ax, ay), 0.5 * np.abs(x + y)), y), 0.0)
    dev = torch.device("cuda")
    tx = torch.tensor(x, device=dev)
    ty = torch.tensor(y, device=dev)
    out = torch.full((2 * x.size,), float("nan"), dtype=torch.float64, device=dev)
    H.hydro_selftest_arith(tx, ty, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy().reshape(-1, 2)
    assert np.array_equal(o[:, 0].view(np.int64), half.view(np.int64)), "halving"
    assert np.array_equal(o[:, 1].view(np.int64), slope.view(np.int64)), "MC slope"
    # the underflow band was reached: some products there round to zero, some not
    band = np.abs(np.log2(np.abs(x[-50_000:])) + np.log2(np.abs(y[-50_000:])) + 1075) < 4
    assert (pos[-50_000:][band]).any() and (~pos[-50_000:][band] & (prod[-50_000:][band] == 0)).any()


def test_halving_of_infinities(H):
    x = np.array([np.inf, -np.inf], dtype=np.float64)
    dev = torch.device("cuda")
    out = torch.zeros(4, dtype=torch.float64, device=dev)
    t = torch.tensor(x, device=dev)
    H.hydro_selftest_arith(t, torch.ones_like(t), out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy()[0::2], x)
