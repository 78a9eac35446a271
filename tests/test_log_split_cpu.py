"""The per-event logarithm of the FP32 kernels, emulated on the CPU in
float32: I = f 2^e with f in [2^-1/2, 2^1/2] (subnormal I scaled into the
normal range first), y = 2^23 ln f rounded to float, then y = k + r split
exactly with t = y + 1.5 2^23 (k = bits(t) - bits(1.5 2^23) an integer,
r = y - (t - 1.5 2^23) a float with |r| <= 1/2). The sums of e and k are
exact integers and only r is summed in floating point, so

  sum_i ln I_i = ln 2 sum_i e_i + 2^-23 (sum_i k_i + sum_i r_i)

holds up to the rounding of each ln f (one float each, |ln f| <= 0.35)
and of the remainder sum: no error grows with the magnitude of the total.
"""
import numpy as np

F32 = np.float32


def split_exponent(x):
    """(f, e) with x = f 2^e, f in [2^-1/2, 2^1/2], as the kernels form it."""
    x = F32(x)
    bits = int(np.array(x).view(np.int32))
    ex = (bits >> 23) & 0xFF
    adj = 0
    if ex == 0:
        x = F32(x * F32(16777216.0))
        bits = int(np.array(x).view(np.int32))
        ex = (bits >> 23) & 0xFF
        adj = -24
    k = ex - 127
    f = np.array((bits & 0x007FFFFF) | 0x3F800000, dtype=np.int32).view(np.float32)[()]
    if f > F32(1.41421356):
        f = F32(f * F32(0.5))
        k += 1
    return F32(f), k + adj


def log_split(I):
    f, e = split_exponent(I)
    y = F32(F32(np.log(np.float64(f))) * F32(8388608.0))   # 2^23 ln f, one rounding
    t = F32(y + F32(12582912.0))                             # 1.5 2^23
    k = int(np.array(t).view(np.int32)) - 0x4B400000
    r = F32(y - F32(t - F32(12582912.0)))
    return e, k, r, y


def split_sum(I):
    """(sum as the kernels form it, float32 sum of ln I, exact FP64 sum, bound)."""
    e_sum = k_sum = 0
    r_sum = naive = F32(0.0)
    for x in I:
        e, k, r, y = log_split(x)
        assert abs(float(r)) <= 0.5
        assert float(k) + float(r) == float(y)                 # the split loses nothing
        f = float(x) / 2.0 ** e
        assert 2 ** -0.5 <= f <= 2 ** 0.5 * (1 + 2 ** -23)
        e_sum += e
        k_sum += k
        r_sum = F32(r_sum + r)
        naive = F32(naive + F32(np.log(np.float64(x))))
    total = np.log(2.0) * e_sum + (k_sum + float(r_sum)) / 8388608.0
    exact = float(np.sum(np.log(np.asarray(I, dtype=np.float64))))
    # per event: the rounding of 2^23 ln f (|ln f| <= 0.35); plus the float sum
    # of the remainders (each |r| <= 1/2)
    n = len(I)
    bound = n * (0.35 * 2.0 ** -24 + 2.0 ** -24) + n ** 2 * 2.0 ** -24 / 8388608.0
    return total, float(naive), exact, bound


def test_split_is_exact_and_the_sum_keeps_its_digits():
    rng = np.random.default_rng(7)
    # intensities over many decades, including subnormal floats
    I = np.concatenate([np.exp(rng.uniform(-80.0, 80.0, 20000)),
                        np.array([1.0, 2.0, 0.5, 1.5e-40, 3e-44, 3.0e38])]).astype(np.float32)
    total, _, exact, bound = split_sum(I)
    assert abs(total - exact) <= bound, (total - exact, bound)


def test_a_float32_sum_of_logs_does_not():
    """Large intensities (a total near 9e5): the kernels' sum stays within the
    bound, a float32 running sum of ln I misses it by orders of magnitude."""
    rng = np.random.default_rng(8)
    I = np.exp(rng.uniform(30.0, 60.0, 20000)).astype(np.float32)
    total, naive, exact, bound = split_sum(I)
    assert abs(total - exact) <= bound, (total - exact, bound)
    assert abs(naive - exact) > 100 * bound, (naive - exact, bound)
