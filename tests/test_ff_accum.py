"""Host replay of the float-float accumulation of weighted counts and of the
adjoint (count_impl.cuh, Sec. 3.4 weighted pairs): the FP32 product split
a * b = ph + pl (exact), ff_add = TwoSum then FastTwoSum into a lane's
(hi, lo) column, the take-back of a flagged pair by the negated addition,
the flush that adds the 32 lane columns of a bin by ff_add and converts
hi + lo to FP64, and the FP64 sum of the flushes.  Replayed with IEEE FP32
operations (numpy float32 scalars) and compared with exactly rounded sums
(math.fsum of the exact FP64 products): a column of n terms stays within
n * 2^-46 of the sum of |terms|, so one work item's columns (a few thousand
products per lane) carry about 1e-11 relative error and the weighted
results sit two orders of magnitude inside the 1e-9 relative tolerance of
the weighted parity tests."""
import math

import numpy as np

f32 = np.float32


def _two_sum(a, b):
    s = f32(a + b)
    bp = f32(s - a)
    return s, f32(f32(a - f32(s - bp)) + f32(b - bp))


def _ff_add(hi, lo, ph, pl):
    s, e = _two_sum(hi, ph)
    t = f32(lo + f32(e + pl))
    h = f32(s + t)
    return h, f32(t - f32(h - s))


def _split(a, b):
    """ph = fl(a b), pl = a b - ph (the kernel's FMA; exact in FP64)."""
    ph = f32(a * b)
    return ph, f32(float(a) * float(b) - float(ph))


def _column(a, b, take_back=()):
    hi = lo = f32(0.0)
    for k, (x, y) in enumerate(zip(a, b)):
        ph, pl = _split(x, y)
        hi, lo = _ff_add(hi, lo, ph, pl)
        if k in take_back:
            hi, lo = _ff_add(hi, lo, f32(-ph), f32(-pl))
    return hi, lo


def _weights(rng, n):
    return np.exp(0.3 * rng.normal(size=n)).astype(np.float32)


def test_weighted_column_error_within_bound():
    rng = np.random.default_rng(301)
    for n in (100, 2000, 20000):
        a, b = _weights(rng, n), _weights(rng, n)
        hi, lo = _column(a, b)
        exact = math.fsum(float(x) * float(y) for x, y in zip(a, b))
        err = abs((float(hi) + float(lo)) - exact)
        assert err <= n * 2.0**-46 * exact, (n, err / exact)
        if n == 2000:
            assert err <= 1e-11 * exact


def test_take_back_removes_the_product():
    """A flagged pair's product is added and then taken back by the negated
    addition (its exact value goes to the FP64 re-test instead): the column
    ends within its rounding of the sum of the other products."""
    rng = np.random.default_rng(302)
    n = 3000
    a, b = _weights(rng, n), _weights(rng, n)
    back = set(rng.choice(n, 40, replace=False).tolist())
    hi, lo = _column(a, b, back)
    exact = math.fsum(float(a[k]) * float(b[k]) for k in range(n) if k not in back)
    scale = math.fsum(float(x) * float(y) for x, y in zip(a, b))
    assert abs((float(hi) + float(lo)) - exact) <= (n + len(back)) * 2.0**-46 * scale


def test_flush_and_fp64_sum_of_items():
    """32 lane columns per item, each of a few hundred products, added by
    ff_add at the flush and converted to FP64; 50 items summed in FP64 (the
    output's atomic adds, in any order)."""
    rng = np.random.default_rng(303)
    total, exact_parts = 0.0, []
    for _ in range(50):
        H = L = f32(0.0)
        for _lane in range(32):
            m = int(rng.integers(50, 300))
            a, b = _weights(rng, m), _weights(rng, m)
            hi, lo = _column(a, b)
            H, L = _ff_add(H, L, hi, lo)
            exact_parts.extend(float(x) * float(y) for x, y in zip(a, b))
        total += float(H) + float(L)
    exact = math.fsum(exact_parts)
    assert abs(total - exact) <= 1e-10 * exact


def test_adjoint_signed_terms_against_absolute_scale():
    """The adjoint sums w_j G[bin] with G of either sign: the error is
    bounded against the sum of |terms| (the scale the adjoint parity tests
    use), not against the possibly cancelling sum.  G enters as a
    float-float pair (gh, gl); the kernel forms th = fl(b gh),
    tl = b gl + (b gh - th)."""
    rng = np.random.default_rng(304)
    n = 5000
    w = _weights(rng, n)
    G = rng.normal(size=n)
    gh = G.astype(np.float32)
    gl = (G - gh.astype(np.float64)).astype(np.float32)
    hi = lo = f32(0.0)
    for b, x, y in zip(w, gh, gl):
        th = f32(b * x)
        # the kernel's two FMAs, here in FP64 then rounded (a double rounding
        # at most, far below the bound)
        tl = f32(float(b) * float(y) + (float(b) * float(x) - float(th)))
        hi, lo = _ff_add(hi, lo, th, tl)
    terms = [float(b) * (float(x) + float(y)) for b, x, y in zip(w, gh, gl)]
    exact = math.fsum(terms)
    scale = math.fsum(abs(t) for t in terms)
    assert abs((float(hi) + float(lo)) - exact) <= n * 2.0**-44 * scale
