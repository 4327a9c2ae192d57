"""Integer identities the fixed-point kernels rely on, checked on the host with int16 lane
arithmetic (wrapping adds, lane min/max, bitwise not), independent of any GPU:

lambda = sat(s - eta) with sat to [-32767, 32767] equals (s + 1) + ~clamp(eta, L, U) in
wrapping int16 arithmetic, where L = max(s, 0) - 32767 and U = min(s, 0) + 32767, for every
s and eta in [-32767, 32767] (the range every stored value has)."""
import numpy as np

LIM = 32767


def wrap16(x):
    return ((np.asarray(x, np.int64) + 32768) % 65536 - 32768).astype(np.int64)


def clamp_add_lambda(s, eta):
    lo = wrap16(np.maximum(s, 0) + (-LIM))
    hi = wrap16(np.minimum(s, 0) + LIM)
    s1 = wrap16(s + 1)
    e = np.minimum(np.maximum(eta, lo), hi)
    return wrap16(s1 + wrap16(~e))


def test_clamp_and_wrapping_add_equals_saturated_difference():
    s = np.arange(-LIM, LIM + 1, dtype=np.int64)
    edges = [-LIM, -LIM + 1, -32766, -16384, -2, -1, 0, 1, 2, 16384, 32766, LIM - 1, LIM]
    etas = np.unique(np.concatenate([np.array(edges), np.linspace(-LIM, LIM, 301).astype(np.int64),
                                     np.random.default_rng(3).integers(-LIM, LIM + 1, 200)]))
    for eta in etas:
        want = np.clip(s - eta, -LIM, LIM)
        got = clamp_add_lambda(s, np.full_like(s, eta))
        assert np.array_equal(got, want), int(eta)


def test_bounds_are_representable_and_ordered():
    s = np.arange(-LIM, LIM + 1, dtype=np.int64)
    lo, hi = np.maximum(s, 0) - LIM, np.minimum(s, 0) + LIM
    assert lo.min() >= -LIM and hi.max() <= LIM and (lo <= 0).all() and (hi >= 0).all()
