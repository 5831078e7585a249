"""The exactness claims behind the even-odd form of the FP32-pair element kernel, checked in
plain IEEE float32 arithmetic on the CPU (no GPU code involved):

* alignment: for tau a power of two and |h| <= tau/2, h' = fl(fl(h + tau) - tau) is a
  multiple of 2^-24 tau, |h - h'| <= 2^-24 tau (one grid unit: h + tau >= tau rounds on the
  coarser 2^-23 tau spacing) and fl(h - h') is the exact remainder;
* folds: aligned hi parts a, b (|a|, |b| <= tau/2) add and subtract exactly in float32;
* unfolds: grid parts X = A - sigma of two splitter accumulators (A in [sigma/2, 3 sigma/2],
  so X is a multiple of 2^-24 sigma of at most sigma/2) add and subtract exactly, and
  A - sigma itself is exact.
Each claim is checked on many random values across exponents and at the boundary cases."""
import numpy as np

f32 = np.float32
RNG = np.random.default_rng(20040672)


def _taus():
    return [f32(2.0) ** k for k in (-60, -20, -3, 0, 1, 7, 40)]


def _hi_values(tau, n=4000):
    # magnitudes spread over 2^-30..1 of tau/2, both signs, plus the boundary tau/2
    mags = (tau / 2) * f32(2.0) ** (-RNG.uniform(0, 30, n)).astype(f32)
    vals = (mags * RNG.choice([-1, 1], n)).astype(f32)
    return np.concatenate([vals, np.array([tau / 2, -tau / 2, 0.0], dtype=f32)])


def _align(h, tau):
    return (h + tau) - tau  # float32 operations (numpy keeps the dtype)


def test_alignment_puts_hi_on_the_grid_with_an_exact_remainder():
    for tau in _taus():
        h = _hi_values(tau)
        ha = _align(h, tau)
        assert ha.dtype == np.float32
        unit = np.float64(tau) * 2.0 ** -24
        q = ha.astype(np.float64) / unit
        assert np.all(q == np.round(q))                                        # on the grid
        assert np.all(np.abs(h.astype(np.float64) - ha) <= unit)             # moved by <= one unit
        assert np.any(np.abs(h.astype(np.float64) - ha) > unit / 2)          # (and more than half, sometimes)
        rem32 = (h - ha).astype(np.float64)
        assert np.all(rem32 == h.astype(np.float64) - ha.astype(np.float64))  # remainder exact
        assert np.all(np.abs(ha) <= tau / 2)


def test_folds_of_aligned_values_are_exact():
    for tau in _taus():
        a = _align(_hi_values(tau), tau)
        b = _align(_hi_values(tau)[::-1].copy(), tau)
        s32 = (a + b).astype(np.float64)
        d32 = (a - b).astype(np.float64)
        assert np.all(s32 == a.astype(np.float64) + b.astype(np.float64))
        assert np.all(d32 == a.astype(np.float64) - b.astype(np.float64))


def test_unfolds_of_splitter_grid_parts_are_exact():
    for sigma in _taus():
        # accumulator values A in [sigma/2, 3 sigma/2] as float32
        n = 4000
        A = (sigma * RNG.uniform(0.5, 1.5, (2, n))).astype(f32)
        A[:, :4] = np.array([[sigma / 2, 3 * sigma / 2, sigma, sigma / 2],
                             [3 * sigma / 2, sigma / 2, sigma, sigma / 2]], dtype=f32)
        X = A - sigma                                            # float32
        assert np.all(X.astype(np.float64) == A.astype(np.float64) - np.float64(sigma))  # exact
        unit = np.float64(sigma) * 2.0 ** -24
        q = X.astype(np.float64) / unit
        assert np.all(q == np.round(q)) and np.all(np.abs(X) <= sigma / 2)
        s32, d32 = (X[0] + X[1]).astype(np.float64), (X[1] - X[0]).astype(np.float64)
        assert np.all(s32 == X[0].astype(np.float64) + X[1].astype(np.float64))
        assert np.all(d32 == X[1].astype(np.float64) - X[0].astype(np.float64))


def test_a_value_off_the_grid_would_round():
    """The claims need the alignment: unaligned hi parts of different exponents round."""
    a, b = f32(1.0) + f32(2.0) ** -23, f32(2.0) ** -25 * f32(3.0)
    assert np.float64(a + b) != np.float64(a) + np.float64(b)
