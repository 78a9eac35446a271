"""GPU parity of the MC normalisation matrix M (the bracket of Eq. 3's second
term) against the FP64 oracle, for the tensor-core kernel (up to 20 waves)
and the FP64 kernel (more waves, or PWA_NORM_KERNEL=fp64).

The tensor-core kernel writes every float amplitude as five fixed-point digits
under one power of two 2^r_a > 2 max|A_a|_1 per wave and keeps every digit
pair but (5,5), the leading blocks with exact tensor-core sums; the error is
that of the dropped remainders and pair: per event and real entry of
G = X X^T at most 2^-41 (|x_p| 2^r_q [|x_q| < 2^(r_q - 17)] + |x_q| 2^r_p
[|x_p| < 2^(r_p - 17)]) + 2^(r_p + r_q - 61), the float-float and FP64 sums
adding ~1e-15 relative. The tests hold M to that bound (computed from the
sample) and to 1e-12 of its largest entry, the tolerance of the FP64 kernel
(exact products, FP64 sums); measured, the two kernels agree to ~1e-15.
"""
import os

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pwa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_5673_gb300 as pkg
    return pkg


def build_M(pwa, A_mc, n_gen, kernel=None):
    N = A_mc.shape[1]
    old = os.environ.get("PWA_NORM_KERNEL")
    if kernel:
        os.environ["PWA_NORM_KERNEL"] = kernel
    try:
        with pwa.Likelihood(N) as L:
            L.load_events(A_mc[:1], A_mc, n_gen)
            return L.build_norm()
    finally:
        if kernel:
            if old is None:
                del os.environ["PWA_NORM_KERNEL"]
            else:
                os.environ["PWA_NORM_KERNEL"] = old


def oracle_M(A_mc, n_gen):
    N = A_mc.shape[1]
    if A_mc.shape[0] * N * N < 2e8:
        return oracle.norm_matrix(A_mc, n_gen)
    return oracle.norm_matrix_blas(A_mc, n_gen)


def digit_bound(A_mc, n_gen):
    """Entrywise bound on |M_tc - M| from the digit truncation (see the header)."""
    A = A_mc.astype(np.complex64)
    X = np.empty((A.shape[0], 2 * A.shape[1]), np.float64)
    X[:, 0::2] = A.real
    X[:, 1::2] = A.imag
    amax = (np.abs(A.real) + np.abs(A.imag)).max(axis=0).astype(np.float32)
    r = np.where(amax > 0, np.floor(np.log2(np.maximum(amax, np.float32(1e-38)))) + 2, 0)
    r = np.repeat(np.maximum(r, -35), 2)
    s = 2.0 ** r
    ax = np.abs(X)
    small = (ax < 2.0 ** (r - 17)).astype(np.float64)
    n = A.shape[0]
    BG = 2.0 ** -41 * ((ax.T @ small) * s[None, :] + (small.T @ ax) * s[:, None]) \
        + 2.0 ** -61 * n * np.outer(s, s)
    # Re and Im of M_ab each combine two entries of G
    B = BG[0::2, 0::2] + BG[1::2, 1::2] + BG[0::2, 1::2] + BG[1::2, 0::2]
    return B / n_gen


@pytest.mark.parametrize("N,n_mc", [(1, 1), (3, 63), (4, 64), (4, 65), (7, 1000), (8, 4097),
                                    (12, 30001), (13, 777), (16, 100003), (19, 5000),
                                    (20, 200000)])
def test_norm_tc_vs_oracle(pwa, N, n_mc):
    wl = synth.mixture_workload("n", synth.waves_linear(N), 10, n_mc, seed_mc=900 + N)
    M = build_M(pwa, wl.A_mc, wl.n_gen)
    Mo = oracle_M(wl.A_mc, wl.n_gen)
    err = np.abs(M - Mo)
    assert np.all(err <= digit_bound(wl.A_mc, wl.n_gen) + 1e-14 * np.abs(Mo).max())
    assert err.max() <= 1e-12 * np.abs(Mo).max(), err.max() / np.abs(Mo).max()
    # Hermitian exactly, real diagonal
    assert np.array_equal(M, M.conj().T)


def test_norm_tc_vs_fp64_kernel_and_determinism(pwa):
    wl = synth.mixture_workload("n", synth.waves_linear(20), 10, 300000, seed_mc=77)
    M1 = build_M(pwa, wl.A_mc, wl.n_gen)
    M2 = build_M(pwa, wl.A_mc, wl.n_gen)
    Mf = build_M(pwa, wl.A_mc, wl.n_gen, kernel="fp64")
    assert np.array_equal(M1, M2), "run-to-run bitwise"
    assert np.max(np.abs(M1 - Mf)) <= 1e-13 * np.abs(Mf).max()


def test_norm_tc_bench_size(pwa):
    """The headline sample's MC: 5M accepted events x 20 waves."""
    wl = synth.paper_scale()
    M = build_M(pwa, wl.A_mc, wl.n_gen)
    Mo = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    err = np.abs(M - Mo)
    assert np.all(err <= digit_bound(wl.A_mc, wl.n_gen) + 1e-14 * np.abs(Mo).max())
    assert err.max() <= 1e-12 * np.abs(Mo).max(), err.max() / np.abs(Mo).max()


def test_norm_tc_scales(pwa):
    """Waves of very different sizes in one sample: a zero wave, waves scaled
    by 2^-30 and 2^40, random signs and phases; and a wave beyond the tensor-
    core kernel's range (2^60), which falls back to the FP64 kernel."""
    rng = np.random.default_rng(5)
    n, N = 20000, 8
    A = (rng.standard_normal((n, N)) + 1j * rng.standard_normal((n, N))).astype(np.complex64)
    A[:, 1] = 0
    A[:, 2] *= np.float32(2.0 ** -30)
    A[:, 3] *= np.float32(2.0 ** 40)
    A[::3, 4] *= np.float32(2.0 ** -20)      # a wave whose events span 20 binary orders
    M = build_M(pwa, A, 1.7 * n)
    Mo = oracle.norm_matrix(A, 1.7 * n)
    err = np.abs(M - Mo)
    assert np.all(err <= digit_bound(A, 1.7 * n) + 1e-14 * np.abs(Mo).max())
    # entrywise relative to the geometric scale of the two waves
    d = np.sqrt(np.abs(np.diag(Mo)))
    scale = np.outer(d, d) + 1e-300
    assert np.max((err / scale)[scale > 1e-250]) <= 1e-12
    assert np.all(M[1, :] == 0) and np.all(M[:, 1] == 0)
    A[:, 5] *= np.float32(2.0 ** 60)
    M = build_M(pwa, A, 1.7 * n)
    Mo = oracle.norm_matrix(A, 1.7 * n)
    d = np.sqrt(np.abs(np.diag(Mo)))
    assert np.max(np.abs(M - Mo) / (np.outer(d, d) + 1e-300)) <= 1e-12


def test_norm_fp64_kernel_many_waves(pwa):
    """More than 20 waves: the FP64 kernel."""
    wl = synth.mixture_workload("n", synth.waves_linear(33), 10, 20001, seed_mc=33)
    M = build_M(pwa, wl.A_mc, wl.n_gen)
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    assert np.max(np.abs(M - Mo)) <= 1e-12 * np.abs(Mo).max()
