"""The exact product split that forms S = sum_a V_a A_a in the FP32 kernels,
emulated on the CPU in float32 (FMAs evaluated exactly with rationals and
rounded once): each product c a is split against sigma = 1.5 2^k, chosen so
that 2^(k-1) >= 1.25 sum_a |V_a|_1 max |A_a|_1, into a high part (the bits
of t = fma(c, a, sigma), summed as wrapping 32-bit integers) and a remainder
fma(c, a, sigma - t) summed in float32; V is a float pair Vhi + Vlo.

Claim pinned here: S is correct to about one float rounding of |S| however
small |S| is against B = sum_a |V_a|_1 |A_a|_1, i.e.
|S - S_exact| <= 2^-23 |S_exact| + 2N 2^-24 u_k,   u_k = 2^(k-23),
the second term from the float32 sums of the 2N remainders (each below
u_k / 2); it is below 10 N 2^-47 B_max, B_max = sum_a |V_a|_1 max |A_a|_1
(the bound sigma is chosen from, 2^k < 5 B_max). A plain float32 dot
product misses the same bound by orders of magnitude on events with
destructive interference.
"""
from fractions import Fraction

import numpy as np

F32 = np.float32


def rn32(q):
    """A rational rounded to the nearest float32 (ties to even); normal range."""
    if q == 0:
        return F32(0.0)
    sign = -1 if q < 0 else 1
    q = abs(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    scaled = q / Fraction(2) ** (e - 23)
    m = scaled.numerator // scaled.denominator
    rem = scaled - m
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and m % 2 == 1):
        m += 1
    return F32(sign * float(Fraction(m) * Fraction(2) ** (e - 23)))


def fma(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def bits(x):
    return int(np.array(x, dtype=F32).view(np.uint32))


def split_pair(v):
    hi = F32(v)
    return hi, F32(v - float(hi))


def exact_split_S(A, V, sigma, unit):
    """S of one event as the kernel forms it (real and imaginary parts)."""
    N = len(A)
    hR = hI = 0
    lR = lRm = lI = F32(0.0)
    sg = F32(sigma)
    for w in range(N):
        ar, ai = F32(A[w].real), F32(A[w].imag)
        vr, lr = split_pair(V[w].real)
        vi, li = split_pair(V[w].imag)

        def extract(c, a):
            t = fma(c, a, sg)
            return fma(c, a, F32(sg - t)), bits(t)

        r, x = extract(vr, ar)
        lR = F32(lR + r)
        hR += x
        r, x = extract(vi, ai)
        lRm = F32(lRm + r)
        hR -= x
        r, x = extract(vr, ai)
        lI = F32(lI + r)
        hI += x
        r, x = extract(vi, ar)
        lI = F32(lI + r)
        hI += x
        lR = fma(lr, ar, lR)
        lRm = fma(li, ai, lRm)
        lI = fma(lr, ai, fma(li, ar, lI))
    im_offset = 2 * N * bits(sg)

    def as_int32(u):
        u &= 0xFFFFFFFF
        return u - (1 << 32) if u >= (1 << 31) else u

    hr = F32(F32(as_int32(hR)) * F32(unit))
    hi = F32(F32(as_int32(hI - im_offset)) * F32(unit))
    return float(F32(hr + F32(lR - lRm))), float(F32(hi + lI))


def plain_S(A, V):
    """A float32 dot product (V rounded to float, one FMA chain)."""
    sr = si = F32(0.0)
    for w in range(len(A)):
        ar, ai = F32(A[w].real), F32(A[w].imag)
        vr, vi = F32(V[w].real), F32(V[w].imag)
        sr = fma(vr, ar, fma(-vi, ai, sr))
        si = fma(vr, ai, fma(vi, ar, si))
    return float(sr), float(si)


def exact_S(A, V):
    sr = si = Fraction(0)
    for w in range(len(A)):
        ar, ai = Fraction(float(F32(A[w].real))), Fraction(float(F32(A[w].imag)))
        vr, vi = Fraction(float(V[w].real)), Fraction(float(V[w].imag))
        sr += vr * ar - vi * ai
        si += vr * ai + vi * ar
    return sr, si


def sample(n, N, seed):
    """Events with random amplitudes; every other event is made to cancel
    (its last wave chosen so that S is near zero before rounding)."""
    rng = np.random.default_rng(seed)
    V = rng.normal(size=N) + 1j * rng.normal(size=N)
    A = (rng.normal(size=(n, N)) + 1j * rng.normal(size=(n, N))).astype(np.complex64)
    for i in range(0, n, 2):
        partial = (V[:-1] * A[i, :-1].astype(np.complex128)).sum()
        A[i, -1] = np.complex64(-partial / V[-1])
    return A, V


def sigma_for(A, V):
    amax = np.max(np.abs(A.real) + np.abs(A.imag), axis=0)
    b = float(np.sum((np.abs(V.real) + np.abs(V.imag)) * amax))
    k = int(np.floor(np.log2(2.5 * b))) + 1          # 2.5 b < 2^k
    return 1.5 * 2.0 ** k, 2.0 ** (k - 23)


def test_exact_split_within_one_rounding():
    for N, seed in ((4, 1), (20, 2)):
        A, V = sample(60, N, seed)
        sigma, unit = sigma_for(A, V)
        amax = np.max(np.abs(A.real) + np.abs(A.imag), axis=0)
        B_max = float(np.sum((np.abs(V.real) + np.abs(V.imag)) * amax))
        assert 2 * N * 2.0 ** -24 * unit <= 10 * N * 2.0 ** -47 * B_max
        worst = 0.0
        for i in range(A.shape[0]):
            er, ei = exact_S(A[i], V)
            sr, si = exact_split_S(A[i], V, sigma, unit)
            for s, e in ((sr, er), (si, ei)):
                err = abs(Fraction(s) - e)
                bound = Fraction(2.0 ** -23) * abs(e) + Fraction(2 * N * 2.0 ** -24 * unit)
                assert err <= bound, (N, i, float(err), float(bound))
                worst = max(worst, float(err / bound))
        assert worst > 0.0


def test_plain_float32_dot_fails_under_cancellation():
    A, V = sample(60, 20, 3)
    _, unit = sigma_for(A, V)
    misses = 0
    for i in range(0, A.shape[0], 2):          # the cancelling events
        er, _ = exact_S(A[i], V)
        sr, _ = plain_S(A[i], V)
        if abs(Fraction(sr) - er) > 100 * (Fraction(2.0 ** -23) * abs(er) + Fraction(40 * 2.0 ** -24 * unit)):
            misses += 1
    assert misses >= 20
