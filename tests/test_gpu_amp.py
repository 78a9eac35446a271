"""GPU parity of the direct amplitude form against the FP64 oracle.

The CUDA path and the oracle get identical inputs: complex64 amplitudes from
the seeded generator (promoted exactly to complex128 for the oracle) and the
same V. Tolerances follow the per-event FP32 rounding budget: random per-event
errors of ~1e-7 in ln I add up as sqrt(N_data), so |dNLL| <= 1e-3 at one
million events, scaled as sqrt(N_data / 1e6) below that; the gradient's
relative error ||dg|| / ||g_data|| <= 1e-5; the normalisation matrix, formed
from exact float products summed in double, to 1e-12 of its largest entry.
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


def nll_tol(n):
    return max(1e-3 * math.sqrt(n / 1e6), 2e-6)


def case(N, n_data, n_mc, seed=0):
    waves = synth.waves_linear(N)
    return synth.mixture_workload("t", waves, n_data, n_mc, seed_data=100 + seed,
                                  seed_mc=200 + seed, seed_v=300 + seed)


def check(pwa, wl, Vs, M_tol=1e-12, forms=None):
    N = wl.A_data.shape[1]
    with pwa.Likelihood(N, max_k=len(Vs)) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        M = L.build_norm()
        nll, g = L.nll_grad(np.array(Vs))
        nll_only = L.nll(np.array(Vs))
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen) if wl.A_mc.shape[0] * N * N < 2e8 \
        else oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    assert np.max(np.abs(M - Mo)) <= M_tol * np.abs(Mo).max()
    n = wl.A_data.shape[0]
    for k, V in enumerate(Vs):
        no, go, bad = oracle.nll_amp(wl.A_data, Mo, V)
        assert bad == 0
        gd = go - oracle.norm_term(Mo, V)[1]
        assert abs(nll[k] - no) <= nll_tol(n), (k, nll[k], no, nll[k] - no)
        assert nll_only[k] == nll[k]
        err = np.linalg.norm(g[k] - go) / np.linalg.norm(gd)
        assert err <= 1e-5, (k, err)
        c = term_scale(wl.A_data, V)
        assert np.all(np.abs(g[k] - go) <= 1e-5 * c), (k, np.max(np.abs(g[k] - go) / c))
    return nll, g


def scaled_truth(wl):
    Mo = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    nv = oracle.norm_term(Mo, wl.V_true)[0]
    return wl.V_true * math.sqrt(wl.A_data.shape[0] / nv)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 13, 20, 24, 25, 32, 40, 48])
def test_waves_sweep(pwa, N):
    wl = case(N, 3000, 4000, seed=N)
    check(pwa, wl, [scaled_truth(wl), synth.random_V(N, 11 + N)])


@pytest.mark.parametrize("n_data", [1, 7, 127, 129, 255, 256, 257, 511, 1000, 10007])
def test_ragged_event_counts(pwa, n_data):
    wl = case(20, n_data, 513, seed=n_data % 97)
    check(pwa, wl, [synth.random_V(20, n_data)])


def test_small_four_wave_model(pwa):
    waves = synth.waves_small()
    ev, n_gen = synth.mc_sample(30_000, seed=synth.SEED_MC)
    A_mc = synth.amplitudes(ev, waves)
    V = synth.random_V(4)
    ev_d = synth.data_sample_mixture(10_000, waves, V)
    wl = synth.Workload("four", waves, synth.amplitudes(ev_d, waves), A_mc, n_gen, V)
    check(pwa, wl, [scaled_truth(wl), V, synth.random_V(4, 9)])


def test_many_parameter_sets_and_determinism(pwa):
    wl = case(20, 20_000, 20_000, seed=5)
    Vs = list(synth.start_points(20, 6))
    n1, g1 = check(pwa, wl, Vs)
    n2, g2 = check(pwa, wl, Vs)
    assert np.array_equal(n1, n2) and np.array_equal(g1, g2)


def test_zero_V_is_a_domain_error(pwa):
    wl = case(4, 500, 500)
    with pwa.Likelihood(4, max_k=2) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        nll, g = L.nll_grad(np.array([np.zeros(4), synth.random_V(4, 1)]))
        assert L.last_status == pwa.PWA_EDOMAIN
    assert math.isinf(nll[0]) and np.all(g[0] == 0)
    assert math.isfinite(nll[1])


def test_call_order_and_bad_arguments(pwa):
    from paper_1108_5673_gb300 import _abi
    with pwa.Likelihood(4, max_k=1) as L:
        with pytest.raises(_abi.PwaError) as e:
            L.nll(np.ones(4))
        assert e.value.code == _abi.PWA_ESTATE
        wl = case(4, 100, 100)
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        with pytest.raises(_abi.PwaError):
            L.nll(np.ones(4))                     # no build_norm yet
        L.build_norm()
        with pytest.raises(_abi.PwaError) as e:
            L.nll(np.ones((2, 4)))                # K > max_k
        assert e.value.code == _abi.PWA_EINVAL
        with pytest.raises(_abi.PwaError):
            L.load_events(wl.A_data, wl.A_mc, 10)  # n_gen < n_acc


def test_complex128_and_device_inputs(pwa):
    torch = pytest.importorskip("torch")
    wl = case(20, 5000, 6000, seed=3)
    V = synth.random_V(20, 4)
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    no, go, _ = oracle.nll_amp(wl.A_data, Mo, V)
    # complex128 host input is rounded to float on the device: same values as complex64
    with pwa.Likelihood(20) as L:
        L.load_events(wl.A_data.astype(np.complex128), wl.A_mc.astype(np.complex128), wl.n_gen)
        L.build_norm()
        n1, g1 = L.nll_grad(V[None])
    assert abs(n1[0] - no) <= nll_tol(5000)
    # device tensors in, device results out through the stream-ordered call
    dA = torch.from_numpy(wl.A_data).cuda()
    dM = torch.from_numpy(wl.A_mc).cuda()
    with pwa.Likelihood(20, max_k=3) as L:
        L.load_events(dA, dM, wl.n_gen)
        L.build_norm()
        dV = torch.from_numpy(np.stack([V, V, V])).cuda()
        dn = torch.empty(3, dtype=torch.float64, device="cuda")
        dg = torch.empty(3, 20, dtype=torch.complex128, device="cuda")
        L.nll_grad_async(dV, dn, dg)
        assert L.sync() == pwa.PWA_OK
        n2, g2 = dn.cpu().numpy(), dg.cpu().numpy()
    assert np.all(n2 == n1[0]) and np.all(g2 == g1[0])


@pytest.mark.slow
def test_paper_scale_one_million_events(pwa):
    """1M data events, 5M accepted MC, 20 waves: the configuration the
    benchmark times, evaluated at the scaled truth and at random V."""
    wl = synth.paper_scale()
    Vs = [scaled_truth(wl)] + list(synth.start_points(20, 3))
    check(pwa, wl, Vs)


def test_back_to_back_async_launches(pwa):
    """Hundreds of stream-ordered launches over a sample with many tiles per
    CTA (the benchmark's pattern) give bitwise-identical results."""
    torch = pytest.importorskip("torch")
    wl = case(20, 600_000, 2000, seed=9)
    V = synth.random_V(20, 77)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with pwa.Likelihood(20, max_k=1, stream=s.cuda_stream) as L:
            L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
            L.build_norm()
            n_host, g_host = L.nll_grad(V[None])
            dV = torch.from_numpy(V[None]).cuda()
            R = 300
            dn = torch.empty(R, dtype=torch.float64, device="cuda")
            dg = torch.empty(R, 20, dtype=torch.complex128, device="cuda")
            junk = torch.empty(64 << 20, dtype=torch.uint8, device="cuda")
            for r in range(R):
                if r % 3 == 0:
                    junk.fill_(r & 0xff)
                L.nll_grad_async(dV, dn[r:r + 1], dg[r:r + 1])
            assert L.sync() == pwa.PWA_OK
            n_dev, g_dev = dn.cpu().numpy(), dg.cpu().numpy()
    assert np.all(n_dev == n_host[0])
    assert np.all(g_dev == g_host[0])


@pytest.mark.parametrize("N", [3, 25, 41])
def test_async_outputs_written_exactly(pwa, N):
    """Wave counts below the kernel's padded width: the device outputs are
    written for exactly K x N gradient entries and K NLLs, nothing past them."""
    torch = pytest.importorskip("torch")
    wl = case(N, 2000, 2000, seed=N)
    K = 2
    Vs = np.stack([synth.random_V(N, 1), synth.random_V(N, 2)])
    with pwa.Likelihood(N, max_k=K) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        n_host, g_host = L.nll_grad(Vs)
        dV = torch.from_numpy(Vs).cuda()
        guard = 12345.0
        dn = torch.full((K + 8,), guard, dtype=torch.float64, device="cuda")
        dg = torch.full((K * N + 64,), guard, dtype=torch.complex128, device="cuda")
        L.nll_grad_async(dV, dn[:K], dg[:K * N])
        assert L.sync() == pwa.PWA_OK
        n_dev, g_dev = dn.cpu().numpy(), dg.cpu().numpy()
    assert np.all(n_dev[:K] == n_host) and np.all(n_dev[K:] == guard)
    assert np.all(g_dev[:K * N].reshape(K, N) == g_host) and np.all(g_dev[K * N:] == guard)


@pytest.mark.parametrize("forms", ["amp", "table", "tc"])
def test_graph_replay_matches_direct_enqueue(pwa, monkeypatch, forms):
    """Host evaluations replay a captured CUDA graph (copy in, kernels, copy
    out); results are bitwise those of enqueueing the same work directly, for
    every form, K, and with and without the gradient, across a reload."""
    N = 12
    f = {"amp": pwa.PWA_FORM_AMP, "table": pwa.PWA_FORM_TABLE, "tc": pwa.PWA_FORM_TC}[forms]
    wl = case(N, 5000, 4000, seed=3)
    Vs = synth.random_V(N, 4, k=3)
    with pwa.Likelihood(N, forms=f, max_k=3) as L:
        for rep in range(2):
            L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
            L.build_norm()
            L.set_form(f)
            monkeypatch.delenv("PWA_EVAL_GRAPHS", raising=False)
            g1 = [L.nll_grad(Vs[:k]) for k in (1, 3, 1)] + [L.nll(Vs[:2])]
            monkeypatch.setenv("PWA_EVAL_GRAPHS", "0")
            g0 = [L.nll_grad(Vs[:k]) for k in (1, 3, 1)] + [L.nll(Vs[:2])]
            for a, b in zip(g1, g0):
                if isinstance(a, tuple):
                    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
                else:
                    assert np.array_equal(a, b)
