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


# --------------------------------------------------------------------------------------
# Pairs with a periodic image: the decode forms X = (p_j - p_i) + S.h per component as an
# exact float expansion (TwoSum, TwoProduct), rounds once to c and keeps c only when a
# bound shows that both X and the FP64 form lie in the rounding interval of c (else the
# FP64 form is taken).  The same float steps, emulated here in numpy (float32 arithmetic;
# the fused multiply-add of TwoProduct as an exact double product rounded once), must give
# the FP64-formed float bit for bit whenever they keep c.

def _two_sum(a, b):
    s = (a + b).astype(np.float32)
    bb = (s - a).astype(np.float32)
    e = ((a - (s - bb)) + (b - bb)).astype(np.float32)
    return s, e


def _two_prod(a, b):
    p = (a * b).astype(np.float32)
    e = (a.astype(np.float64) * b.astype(np.float64) - p.astype(np.float64)).astype(np.float32)
    return p, e


def _decode_fp32(pi, pj, h, S):
    """Per component: (c, kept) of the FP32 form; h [n, 3] the three cell components along
    this axis (rows a, b, c of the cell), S [n, 3]."""
    f = S.astype(np.float32)
    s0, e0 = _two_sum(pj, -pi)
    p1, e1 = _two_prod(f[:, 0], h[:, 0])
    p2, e2 = _two_prod(f[:, 1], h[:, 1])
    p3, e3 = _two_prod(f[:, 2], h[:, 2])
    h1, t1 = _two_sum(s0, p1)
    h2, t2 = _two_sum(h1, p2)
    h3, t3 = _two_sum(h2, p3)
    lo = (((e0 + e1) + (e2 + e3)) + ((t1 + t2) + t3)).astype(np.float32)
    c, rr = _two_sum(h3, lo)
    M = (np.abs(s0) + np.abs(p1) + np.abs(p2) + np.abs(p3) + np.abs(h1) + np.abs(h2) + np.abs(h3)).astype(np.float32)
    zero = c == 0
    allzero = zero & (M == 0) & (lo == 0) & (rr == 0)
    bits = c.view(np.uint32)
    ec = ((bits >> 23) & 0xFF).astype(np.int64)
    hg = np.ldexp(np.float32(1.0), ec - 127 - 24).astype(np.float32)
    hg_small = np.where((bits & 0x7FFFFF) != 0, hg, np.ldexp(np.float32(1.0), ec - 127 - 25)).astype(np.float32)
    up, down = np.where(c > 0, hg, hg_small), np.where(c > 0, hg_small, hg)
    B = (np.float32(2.0 ** -44) * M + np.float32(2.0 ** -51) * np.abs(c) + np.float32(2.0 ** -110)).astype(np.float32)
    inside = ((rr + B).astype(np.float32) < up) & ((rr - B).astype(np.float32) > -down)
    # near a boundary: kept when lo's sum was exact and every FP64 partial sum is exact
    a1, r1 = _two_sum(e0, e1)
    a2, r2 = _two_sum(e2, e3)
    a3, r3 = _two_sum(a1, a2)
    b1, r4 = _two_sum(t1, t2)
    b2, r5 = _two_sum(b1, t3)
    _, r6 = _two_sum(a3, b2)
    lo_exact = (r1 == 0) & (r2 == 0) & (r3 == 0) & (r4 == 0) & (r5 == 0) & (r6 == 0)

    def lsb(v):
        ev = ((v.view(np.uint32) >> 23) & 0xFF).astype(np.int64)
        return np.where(v != 0, np.maximum(ev, 1) - 150, 1000)

    q = np.minimum.reduce([lsb(pj), lsb(pi), np.where(S[:, 0] != 0, lsb(h[:, 0]), 1000),
                           np.where(S[:, 1] != 0, lsb(h[:, 1]), 1000), np.where(S[:, 2] != 0, lsb(h[:, 2]), 1000)])
    eM = ((M.view(np.uint32) >> 23) & 0xFF).astype(np.int64) - 127
    exact = lo_exact & (eM + 2 <= q + 52)
    ok = ~zero & (ec >= 40) & (ec != 255) & (inside | exact)
    zsum = (s0 + ((p1 + p2).astype(np.float32) + p3)).astype(np.float32)
    out = np.where(allzero, zsum, c)
    return out, ok | allzero


def _decode_fp64(pi, pj, h, S):
    rel = pj.astype(np.float64) - pi.astype(np.float64)
    sh = (S[:, 0] * h[:, 0].astype(np.float64) + S[:, 1] * h[:, 1].astype(np.float64)) \
        + S[:, 2] * h[:, 2].astype(np.float64)
    return (rel + sh).astype(np.float32)


def test_fp32_image_displacement_matches_fp64_form():
    rng = np.random.default_rng(1)
    n = 600_000
    pi = rng.uniform(-80, 80, n).astype(np.float32)
    pj = rng.uniform(-80, 80, n).astype(np.float32)
    h = rng.uniform(-40, 40, (n, 3)).astype(np.float32)
    S = rng.integers(-127, 128, (n, 3))
    # structured cases: orthorhombic cells (zero off-diagonals), the same atom (self images),
    # cancelling images, tiny and huge magnitudes, exact zeros of both signs
    k = n // 8
    h[:k, 1:] = rng.choice([0.0, -0.0], (k, 2))
    pj[k:2 * k] = pi[k:2 * k]
    S[2 * k:3 * k, 1] = -S[2 * k:3 * k, 0]
    h[2 * k:3 * k, 1] = h[2 * k:3 * k, 0]
    pi[3 * k:4 * k] = np.ldexp(rng.uniform(-1, 1, k), rng.integers(-60, 10, k)).astype(np.float32)
    pj[3 * k:4 * k] = np.ldexp(rng.uniform(-1, 1, k), rng.integers(-60, 10, k)).astype(np.float32)
    pi[4 * k:5 * k] = rng.choice([0.0, -0.0], k)
    pj[4 * k:5 * k] = rng.choice([0.0, -0.0], k)
    h[4 * k:5 * k] = rng.choice([0.0, -0.0, 1.5], (k, 3))
    S[5 * k:6 * k] = rng.integers(-2, 3, (k, 3))
    pi[6 * k:7 * k] = np.float32(3.0) + rng.integers(-3, 4, k).astype(np.float32) * np.float32(2.0 ** -20)
    with np.errstate(all="ignore"):
        c, ok = _decode_fp32(pi, pj, h, S)
        d = _decode_fp64(pi, pj, h, S)
    assert np.array_equal(c[ok].view(np.uint32), d[ok].view(np.uint32))
    assert ok.mean() > 0.995  # the FP64 fallback is rare
    z = ok & (d == 0)
    assert np.signbit(d[z]).any() and (~np.signbit(d[z])).any()  # both zero signs occur and agree


def test_fp32_image_displacement_near_rounding_boundaries():
    """Displacements placed at and around float midpoints: the FP32 form either keeps the
    FP64-formed float or declines."""
    rng = np.random.default_rng(2)
    n = 200_000
    base = rng.uniform(1, 8, n).astype(np.float32)
    ulp = np.spacing(base)
    h = np.ones((n, 3), np.float32) * np.float32(0.0)
    h[:, 0] = rng.uniform(2, 10, n).astype(np.float32)
    S = np.zeros((n, 3), np.int64)
    S[:, 0] = 1
    # p_j - p_i + h_a close to base + ulp/2 (a midpoint)
    pj = (base.astype(np.float64) + ulp.astype(np.float64) / 2 - h[:, 0].astype(np.float64)).astype(np.float32)
    pi = np.zeros(n, np.float32) + rng.choice([0.0, 2.0 ** -30, -2.0 ** -30], n).astype(np.float32)
    with np.errstate(all="ignore"):
        c, ok = _decode_fp32(pi, pj, h, S)
        d = _decode_fp64(pi, pj, h, S)
    assert np.array_equal(c[ok].view(np.uint32), d[ok].view(np.uint32))
