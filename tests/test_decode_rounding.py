"""The neighbour decode writes the displacement of a pair without a periodic image as one
FP32 subtraction plus a signed zero, and relies on that being bit-identical to the FP64
form the pair predicate uses (the difference and the image term in FP64, rounded once to
float).  Checked here in IEEE arithmetic (numpy) over ordinary, tiny, subnormal, zero and
signed-zero coordinates and over every sign pattern of the cell components."""
import numpy as np


def _coords(rng, n):
    kind = rng.integers(0, 6, size=n)
    v = rng.uniform(-60, 60, size=n)
    v = np.where(kind == 1, rng.uniform(-1e-6, 1e-6, size=n), v)
    v = np.where(kind == 2, rng.choice([0.0, -0.0], size=n), v)
    v = np.where(kind == 3, rng.uniform(-1e-30, 1e-30, size=n), v)
    v = np.where(kind == 4, np.ldexp(rng.uniform(-1, 1, size=n), rng.integers(-149, 20, size=n)), v)
    return v.astype(np.float32)


def test_fp32_difference_matches_fp64_form():
    rng = np.random.default_rng(0)
    n = 400_000
    pi, pj = _coords(rng, n), _coords(rng, n)
    pj[:1000] = pi[:1000]
    pj[1000:2000] = np.nextafter(pi[1000:2000], np.float32(1e9))
    h = rng.choice([1.5, -2.5, 0.0, -0.0], size=(n, 3))  # h_a, h_b, h_c components along one axis
    with np.errstate(all="ignore"):
        # FP64 form: (p_j - p_i) + ((0 h_a + 0 h_b) + 0 h_c), rounded once to float
        rel = pj.astype(np.float64) - pi.astype(np.float64)
        sh = (0.0 * h[:, 0] + 0.0 * h[:, 1]) + 0.0 * h[:, 2]
        d64 = (rel + sh).astype(np.float32)
        # decode: FP32 difference plus a zero that is negative only when all three h are
        neg = np.signbit(h[:, 0]) & np.signbit(h[:, 1]) & np.signbit(h[:, 2])
        d32 = (pj - pi) + np.where(neg, np.float32(-0.0), np.float32(0.0))
    assert d32.dtype == np.float32
    assert np.array_equal(d64.view(np.uint32), d32.view(np.uint32))
    assert np.signbit(d64[d64 == 0]).any() and (~np.signbit(d64[d64 == 0])).any()  # both zero signs occur
