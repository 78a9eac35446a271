"""GPU parity of the batched tensor-core form against the FP64 oracle.

Identical inputs: the tensor-core form consumes the amplitudes in block
floating point (one exponent per event, integer slices; see include/pwa.h),
so the oracle is evaluated on exactly those values, rebuilt here from the
complex64 amplitudes by the rounding rule the header states (round to
nearest even at each slice), and with the exact V. Every sum on the tensor
cores is an exact integer sum; what remains per event is FP32 rounding to
nearest (the slice combination, |Q|^2, the log polynomial's evaluation) and
the 2^-19 fixed-point resolution of the log sums, all unbiased with a
per-event spread below 1e-6 in ln I, plus the log polynomial's error (below
8e-10, the only possibly coherent part). Hence the NLL bound
3e-3 sqrt(n / 1e6) + 1e-9 n + 1e-5 (so 4e-3 at one million events, inside the
1e-2 stated for BF16 operands). The gradient uses R = S / I rounded to BF16
(relative 2^-9 per event, random), so ||dg|| / ||g_data|| <= 2e-3.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from grad_bound import term_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pwa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_5673_gb300 as pkg
    return pkg


def bfp_amplitudes(A, xs):
    """The values the tensor-core form consumes: per event E = exponent of the
    largest |Re|, |Im| (max = m 2^E, m in [1/2, 1)); x = A 2^(8-E);
    x0 = rint(x), x1 = rint((x - x0) 256); A' = 2^(E-8) (x0 + x1 / 256)."""
    A = np.asarray(A, dtype=np.complex64)
    n, N = A.shape
    X = np.empty((n, 2 * N), np.float32)
    X[:, 0::2] = A.real
    X[:, 1::2] = A.imag
    m = np.abs(X).max(axis=1)
    _, E = np.frexp(m)
    E = np.where(m > 0, E, 0).astype(np.int32)
    x = np.ldexp(X, (8 - E)[:, None]).astype(np.float32)
    x0 = np.rint(x)
    x1 = np.rint((x - x0) * np.float32(256)) if xs == 2 else np.zeros_like(x0)
    Ap = np.ldexp(x0.astype(np.float64) + x1.astype(np.float64) / 256.0, (E - 8)[:, None])
    return Ap[:, 0::2] + 1j * Ap[:, 1::2]


def nll_tol(n):
    return 3e-3 * math.sqrt(n / 1e6) + 1e-9 * n + 1e-5


GRAD_TOL = 2e-3


def case(N, n_data, n_mc, seed=0):
    return synth.mixture_workload("t", synth.waves_linear(N), n_data, n_mc, seed_data=400 + seed,
                                  seed_mc=500 + seed, seed_v=600 + seed)


def run_tc(pwa, wl, Vs, precision, max_k=None):
    N = wl.A_data.shape[1]
    Vs = np.asarray(Vs)
    with pwa.Likelihood(N, forms=pwa.PWA_FORM_TC | pwa.PWA_FORM_AMP, max_k=max_k or len(Vs),
                        precision=precision) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        L.set_form(pwa.PWA_FORM_TC)
        nll, g = L.nll_grad(Vs)
        status = L.last_status
        nll2, g2 = L.nll_grad(Vs)
    assert np.array_equal(nll, nll2) and np.array_equal(g, g2), "not reproducible"
    return nll, g, status


def check(pwa, wl, Vs, precision, idx=None):
    xs = 1 if precision == pwa.PWA_PREC_BFP8 else 2
    nll, g, status = run_tc(pwa, wl, Vs, precision)
    assert status == pwa.PWA_OK
    Ap = bfp_amplitudes(wl.A_data, xs)
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen) if wl.A_mc.shape[0] * wl.A_mc.shape[1] ** 2 < 2e8 \
        else oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    n = wl.A_data.shape[0]
    for k in (range(len(Vs)) if idx is None else idx):
        no, go, bad = oracle.nll_amp(Ap, Mo, Vs[k])
        assert bad == 0
        gd = go - oracle.norm_term(Mo, Vs[k])[1]
        assert abs(nll[k] - no) <= nll_tol(n), (k, nll[k], no, nll[k] - no)
        err = np.linalg.norm(g[k] - go) / np.linalg.norm(gd)
        assert err <= GRAD_TOL, (k, err)
        c = term_scale(Ap, Vs[k])
        assert np.all(np.abs(g[k] - go) <= 3e-3 * c), (k, np.max(np.abs(g[k] - go) / c))


PRECISIONS = ["BFP16", "BFP8"]


def prec(pwa, name):
    return getattr(pwa, "PWA_PREC_" + name)


@pytest.mark.parametrize("p", PRECISIONS)
@pytest.mark.parametrize("N", [1, 4, 8, 13, 20, 24, 32, 40, 48])
def test_waves_sweep(pwa, N, p):
    wl = case(N, 3000, 4000, seed=N)
    Vs = [synth.random_V(N, 31 + N + j) * (0.5 + j) for j in range(5)]
    check(pwa, wl, Vs, prec(pwa, p))


@pytest.mark.parametrize("p", PRECISIONS)
@pytest.mark.parametrize("K", [1, 31, 33, 64, 65, 128, 129, 200, 300])
def test_parameter_set_counts(pwa, K, p):
    """Half chunks, chunks, launch limits and splitting into several launches."""
    N = 20
    wl = case(N, 2000, 3000, seed=K)
    Vs = [synth.random_V(N, 1000 + j) for j in range(K)]
    check(pwa, wl, Vs, prec(pwa, p), idx=sorted({0, K // 2, K - 1, min(K - 1, 64), min(K - 1, 130)}))


@pytest.mark.parametrize("n_data", [1, 63, 127, 129, 1000, 19455, 19457, 40001])
def test_ragged_event_counts(pwa, n_data):
    """Partial tiles and idle CTAs (fewer tiles than SMs)."""
    wl = case(16, n_data, 700, seed=n_data % 89)
    Vs = [synth.random_V(16, 7 + j) for j in range(3)]
    check(pwa, wl, Vs, pwa.PWA_PREC_BFP16)


def test_degenerate_set_flagged(pwa):
    """A parameter set with V = 0 has I = 0 everywhere: its NLL is +inf and its
    gradient 0 (EDOMAIN); the other sets of the same call stay valid."""
    N = 8
    wl = case(N, 5000, 3000, seed=3)
    Vs = [synth.random_V(N, 1), np.zeros(N, complex), synth.random_V(N, 2)]
    nll, g, status = run_tc(pwa, wl, Vs, pwa.PWA_PREC_BFP16)
    assert status == pwa.PWA_EDOMAIN
    assert np.isinf(nll[1]) and not np.any(g[1])
    Ap = bfp_amplitudes(wl.A_data, 2)
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    for k in (0, 2):
        no, _, _ = oracle.nll_amp(Ap, Mo, Vs[k])
        assert abs(nll[k] - no) <= nll_tol(5000)


def test_scale_invariant_encoding(pwa):
    """The encoding has one exponent per event and per set: scaling all
    amplitudes or all of V by a power of two changes the NLL exactly as Eq. 3
    says (ln I shifts by a constant per event, V^H M V scales)."""
    N = 12
    wl = case(N, 4000, 3000, seed=5)
    V = synth.random_V(N, 9)
    nll1, _, _ = run_tc(pwa, wl, [V], pwa.PWA_PREC_BFP16)
    nll2, _, _ = run_tc(pwa, wl, [V * 4.0], pwa.PWA_PREC_BFP16)
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    nv = oracle.norm_term(Mo, V)[0]
    expect = nll1[0] - 4000 * math.log(16.0) + 15.0 * nv
    assert abs(nll2[0] - expect) <= 1e-7 * abs(expect)


@pytest.mark.slow
@pytest.mark.parametrize("p", PRECISIONS)
def test_multistart_scale(pwa, p):
    """400k events, 32 waves, 128 parameter sets: the batched workload shape."""
    wl = synth.mixture_workload("ms", synth.waves_linear(32), 400_000, 50_000)
    Vs = synth.start_points(32, 128) * 2.0
    check(pwa, wl, Vs, prec(pwa, p), idx=[0, 1, 63, 64, 127])


@pytest.mark.slow
def test_bench_configuration(pwa):
    """The bench configuration: 4M events x 32 waves, 256 parameter sets in
    one call (BFP16); five of the sets against the oracle."""
    wl = synth.multistart_scale(n_mc_acc=1_000_000)
    Vs = synth.start_points(32, 256) * 2.0
    check(pwa, wl, Vs, pwa.PWA_PREC_BFP16, idx=[0, 1, 127, 128, 255])


@pytest.mark.slow
def test_paper_scale_one_million(pwa):
    """1M events, 20 waves (the headline sample), 64 parameter sets."""
    wl = synth.paper_scale(n_mc_acc=300_000)
    Vs = synth.start_points(20, 64) * 2.0
    check(pwa, wl, Vs, pwa.PWA_PREC_BFP16, idx=[0, 31, 63])
