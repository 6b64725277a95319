"""Host-side checks of the fixed-point spread arithmetic (csrc/node_dev.cuh), restated in
NumPy. CPU only.

The spread rounds each term (w, w d / h, times the node weight) to an int32 multiple of
2^-(27 - shift) and sums in int64, so its sums do not depend on the order of the nodes in
a box. Two claims carry that design:

- every term fits in int32: a 1D Lagrange weight over the k interior nodes of a unit
  box is at most 1.875 in magnitude (k <= 3), so |w| <= 3.52 and |w d / h| <= 5.3 for
  |d| <= 1.5 h, i.e. below 2^30 at scale 2^27;
- int64 -> FP32 in 32-bit pieces is the correctly rounded conversion: for |v| < 2^48,
  v = h 2^24 + lo with h = floor(v / 2^24) and 0 <= lo < 2^24 both exact in FP32, and
  one FP32 addition of h 2^24 and lo rounds the exact sum once.
"""
import numpy as np
import pytest


def lagrange(k, u):
    """Weights of the k interior nodes (l + 1/2)/k of a unit box at u, as in the kernels."""
    if k == 1:
        return np.ones((1,) + np.shape(u))
    if k == 2:
        return np.stack([1.5 - 2.0 * u, 2.0 * u - 0.5])
    v = 3.0 * u - 1.5
    return np.stack([0.5 * v * (v - 1.0), 1.0 - v * v, 0.5 * v * (v + 1.0)])


@pytest.mark.parametrize("k", [1, 2, 3])
def test_lagrange_weights_bounded_and_partition_of_unity(k):
    u = np.linspace(0.0, 1.0, 100001, endpoint=False)
    w = lagrange(k, u)
    assert np.allclose(w.sum(axis=0), 1.0)
    assert np.abs(w).max() <= 1.875 + 1e-12
    # interpolation nodes reproduce themselves
    for l in range(k):
        wl = lagrange(k, np.array([(l + 0.5) / k]))
        assert np.allclose(wl[:, 0], np.eye(k)[l])


def test_spread_terms_fit_in_int32():
    q = 2.0 ** 27
    w_max = 1.875 ** 2                 # product of the two axes' weights
    assert w_max * q < 2 ** 30
    assert w_max * 1.5 * q < 2 ** 31   # moment term w d / h with |d| <= 1.5 h


def ll2f_rn(v):
    """The kernels' int64 -> FP32 conversion in 32-bit pieces (|v| < 2^48)."""
    v = np.asarray(v, dtype=np.int64)
    lo32 = (v & 0xFFFFFFFF).astype(np.uint64)
    hi32 = (v >> 32).astype(np.int64)
    # funnel shift right by 24 of (hi32:lo32), low 32 bits, as int32
    h = ((((hi32.astype(np.uint64) & np.uint64(0xFFFFFFFF)) << np.uint64(32)) | lo32) >> np.uint64(24))
    h = (h & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32)
    lo = (lo32 & np.uint64(0xFFFFFF)).astype(np.int32)
    hf = h.astype(np.float32) * np.float32(16777216.0)   # exact: |h| <= 2^24
    return hf + lo.astype(np.float32)                     # one FP32 rounding


def exact_f32(v):
    # |v| < 2^53: float64 holds v exactly, and float64 -> float32 rounds it once
    return np.asarray(v, dtype=np.int64).astype(np.float64).astype(np.float32)


def test_ll2f_matches_correct_rounding_on_random_and_boundary_values():
    rng = np.random.default_rng(5)
    lim = 1 << 48
    vals = [rng.integers(-lim, lim, size=200_000, dtype=np.int64)]
    for e in range(0, 48):  # every magnitude, both signs
        vals.append(rng.integers(-(1 << e), 1 << e, size=2000, dtype=np.int64))
    # exact ties and their neighbours at every exponent above 2^24
    t = []
    for e in range(25, 48):
        half = 1 << (e - 24)  # half an FP32 ulp at magnitude 2^e
        for m in (1 << 23, (1 << 23) + 1, (1 << 24) - 1):
            base = m << (e - 23)
            for d in (-1, 0, 1):
                t += [base + half + d, -(base + half + d)]
    vals.append(np.array(t, dtype=np.int64))
    vals.append(np.array([lim - 1, -lim, -1, 0, 1, (1 << 24) + 1, -(1 << 24) - 1], dtype=np.int64))
    v = np.concatenate(vals)
    got = ll2f_rn(v)
    ref = exact_f32(v)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


def test_fixed_point_sum_is_order_independent():
    # the property the spread relies on: int64 sums of rounded terms do not depend on order
    rng = np.random.default_rng(6)
    terms = np.rint(rng.uniform(-3.5, 3.5, size=5000) * 2.0 ** 27).astype(np.int64)
    a = ll2f_rn(np.sum(terms))
    b = ll2f_rn(np.sum(rng.permutation(terms)))
    assert a == b
