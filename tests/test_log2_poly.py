"""The log2 polynomial of the tensor-core epilogue: the constants compiled
into the kernel are the ones the generator script produces, the polynomial's
error is within its stated bound on the whole interval, and the kernel's
fixed-point evaluation (float32 Horner with fused multiply-adds, exponent
split, rounding to 2^-19) has no bias beyond that bound on log-uniform
inputs."""
import os
import re
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1108_5673_gb300", "csrc")
sys.path.insert(0, CSRC)
import log2_poly  # noqa: E402


def kernel_constants():
    src = open(os.path.join(CSRC, "k_batched.cu")).read()
    body = src[src.index("log2_fixed2(f2 z)"):]
    body = body[:body.index("}")]
    vals = [float(v) for v in re.findall(r"pk2\(([-0-9.e+]+)f,", body)]
    return vals  # highest degree first, then the 1.5 * 2^23 rounding constant


def test_constants_match_generator():
    coef = log2_poly.coefficients()
    vals = kernel_constants()
    assert vals[-1] == 12582912.0
    got = np.array(vals[:-1][::-1], dtype=np.float32)
    want = np.array([np.float32(a * log2_poly.SCALE) for a in coef], dtype=np.float32)
    assert np.array_equal(got, want)


def test_error_bound():
    assert log2_poly.max_error(log2_poly.coefficients()) < 8e-10


def _fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def test_fixed_point_path_unbiased():
    """Emulates the kernel: I = 2^k (1 + z), 2^19 log2 I to the nearest integer."""
    rng = np.random.Generator(np.random.Philox(5))
    I = np.exp2(rng.uniform(-30.0, 45.0, 2_000_000)).astype(np.float32)
    bits = I.view(np.int32).astype(np.int64)
    k = (bits - 0x3F3504F3) >> 23
    z = ((bits - (k << 23)).astype(np.int32).view(np.float32) - np.float32(1)).astype(np.float32)
    c = np.array(kernel_constants(), dtype=np.float32)
    p = np.full_like(z, c[0])
    for v in c[1:-1]:
        p = _fma32(p, z, np.full_like(z, v))
    y = _fma32(p, z, np.full_like(z, c[-1]))
    l = y.view(np.int32).astype(np.int64) - 0x4B400000 + (k << 19)
    err = l / 2.0 ** 19 - np.log2(I.astype(np.float64))
    assert np.abs(err).max() <= 2.0 ** -20 + 1e-7          # rounding to 2^-19 plus evaluation
    # the rounding to nearest averages out; what remains must be far below 1e-8 per event
    assert abs(err.mean()) < 2e-9, err.mean()
