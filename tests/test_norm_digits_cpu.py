"""CPU emulation of the digit split of the tensor-core MC normalisation kernel.

The kernel writes each float amplitude x of wave a as five fixed-point digits
t_s = c_s 2^(r_a - 8s) by the float32 steps t = (z + S_s) - S_s, z -= t with
S_s = 1.5 2^(r_a - 8s + 23), starting from z = x, where 2^r_a > 2 max|A_a|_1.
These tests redo those float32 steps with numpy (each operation rounded to
nearest, as on the GPU) and check the claims the kernel's exactness rests on:
every digit is an integer multiple of its quantum with |c_s| <= 128 (so it is
an exact BF16 value), the digits plus the remainder give x back exactly, the
remainder is at most half the last quantum and zero for |x| >= 2^(r_a - 17),
the sum over 512 events of one digit pair's products stays below 2^23 quanta
(an exact FP32 sum), and the kept pairs (all but (5,5)) reproduce x_p x_q
within the stated bound, where dropping the pair (4,4) as well would leave a
positive bias on the diagonal. A split that truncated instead of rounding, or
that dropped the 1.5 factor, fails.
"""
import numpy as np

import synth

f32 = np.float32


def exponent(amax):
    r = np.where(amax > 0, np.floor(np.log2(np.maximum(amax, 1e-38))).astype(np.int64) + 2, 0)
    return np.maximum(r, -35)


def split(x, r, digits=5, factor=1.5):
    """float32 emulation of the kernel's split of the columns of x (wave scale r)."""
    z = x.astype(f32)
    S = (f32(factor) * np.ldexp(f32(1), (r + 15).astype(np.int32))).astype(f32)
    out = []
    for _ in range(digits):
        t = ((z + S).astype(f32) - S).astype(f32)
        z = (z - t).astype(f32)
        out.append(t)
        S = (S * f32(2.0 ** -8)).astype(f32)
    return out, z


def bf16_exact(t):
    """True where t (float32) has at most 8 significant bits."""
    bits = t.astype(f32).view(np.uint32)
    return (bits & 0xFFFF) == 0


def sample():
    wl = synth.mixture_workload("d", synth.waves_linear(20), 10, 20000, seed_mc=3)
    A = wl.A_mc.astype(np.complex64)
    X = np.empty((A.shape[0], 40), f32)
    X[:, 0::2] = A.real
    X[:, 1::2] = A.imag
    amax = (np.abs(A.real) + np.abs(A.imag)).max(axis=0).astype(f32)
    r = np.repeat(exponent(amax), 2)
    return X, r


def test_digits_exact_and_bounded():
    X, r = sample()
    ts, rest = split(X, r)
    acc = np.zeros(X.shape, np.float64)
    for s, t in enumerate(ts, start=1):
        c = t.astype(np.float64) / np.ldexp(1.0, r - 8 * s)
        assert np.array_equal(c, np.round(c)), "digit is an integer multiple of its quantum"
        assert np.abs(c).max() <= 128
        assert bf16_exact(t).all(), "digit is an exact BF16 value"
        acc += t.astype(np.float64)
    acc += rest.astype(np.float64)
    assert np.array_equal(acc, X.astype(np.float64)), "digits + remainder = x exactly"
    assert np.all(np.abs(rest.astype(np.float64)) <= np.ldexp(1.0, r - 41))
    big = np.abs(X.astype(np.float64)) >= np.ldexp(1.0, r - 17)
    assert np.all(rest[big] == 0)


def test_pair_sums_stay_exact_over_512_events():
    X, r = sample()
    ts, _ = split(X[:512], r)
    for s in range(5):
        cs = ts[s].astype(np.float64) / np.ldexp(1.0, r - 8 * (s + 1))
        for t in range(5):
            ct = ts[t].astype(np.float64) / np.ldexp(1.0, r - 8 * (t + 1))
            G = np.abs(cs).T @ np.abs(ct)     # sum over the 512 events of |c_s c_t| per entry
            assert G.max() < 2 ** 23


def kept_sum(ts, drop):
    ld = np.longdouble
    G = np.zeros((ts[0].shape[1],) * 2, ld)
    for s in range(5):
        for t in range(5):
            if (s + 1, t + 1) not in drop:
                G += ts[s].astype(ld).T @ ts[t].astype(ld)
    return G


def test_kept_pairs_reproduce_products():
    X, r = sample()
    ts, _ = split(X, r)
    n = X.shape[0]
    G = kept_sum(ts, {(5, 5)})
    Gx = X.astype(np.longdouble).T @ X.astype(np.longdouble)
    sc = np.ldexp(1.0, r)
    ax = np.abs(X.astype(np.float64))
    small = ax < np.ldexp(1.0, r - 17)
    bound = 2.0 ** -41 * ((ax.T @ small) * sc[None, :] + (small.T @ ax) * sc[:, None]) \
        + 2.0 ** -61 * n * np.outer(sc, sc)
    # rounding of the extended-precision sums themselves (25 of them)
    slack = 25 * n * float(np.finfo(np.longdouble).eps) * (ax.T @ ax)
    err = np.abs((G - Gx).astype(np.float64))
    assert np.all(err <= bound + slack)
    d = np.sqrt(np.diag(Gx).astype(np.float64))
    assert err.max() <= 1e-13 * float(np.abs(Gx).max())
    assert np.max(err / np.outer(d, d)) <= 1e-12
    # the diagonal has no bias: relative errors ~1e-17 of either sign
    rel = np.diag((G - Gx).astype(np.float64)) / np.diag(Gx).astype(np.float64)
    assert np.abs(rel).max() <= 1e-15
    # without the pair (4,4) it would keep a negative bias (the dropped
    # squares t_4^2 are positive), up to ~1e-12 of the diagonal
    rel44 = np.diag((kept_sum(ts, {(5, 5), (4, 4)}) - Gx).astype(np.float64)) \
        / np.diag(Gx).astype(np.float64)
    assert np.all(rel44 < 0) and np.abs(rel44).max() > 100 * np.abs(rel).max()


def test_wrong_splits_fail():
    X, r = sample()
    # truncation instead of rounding: a digit of 256 appears or the remainder
    # exceeds half a quantum
    z = X.astype(f32)
    q = np.ldexp(f32(1), (r - 8).astype(np.int32)).astype(f32)
    t = (np.trunc(z / q) * q).astype(f32)
    rest = (z - t).astype(f32)
    assert np.any(np.abs(rest.astype(np.float64)) > 0.5 * q)
    # without the 1.5 factor the rounding constant is a power of two and
    # negative remainders round at half the quantum: digits come out wrong
    ts, rest = split(X, r, factor=1.0)
    ok = all(np.array_equal(t.astype(np.float64) / np.ldexp(1.0, r - 8 * (s + 1)),
                            np.round(t.astype(np.float64) / np.ldexp(1.0, r - 8 * (s + 1))))
             for s, t in enumerate(ts))
    assert not (ok and np.all(np.abs(rest.astype(np.float64)) <= np.ldexp(1.0, r - 49)))
