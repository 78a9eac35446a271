"""The autotuner: timing picks a variant, the JSON cache records it and is
applied on the next call without timing, and results do not depend on the
choice beyond summation order (each variant stays within the oracle bound)."""
import json

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


def test_direct_form_tuning_and_cache(pwa, tmp_path):
    wl = synth.mixture_workload("t", synth.waves_linear(12), 200_000, 20_000)
    V = synth.random_V(12, 3)
    cache = str(tmp_path / "tune.json")
    with pwa.Likelihood(12) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        n0, g0 = L.nll_grad(V[None])
        s1 = L.autotune(cache)
        assert "timed" in s1
        n1, g1 = L.nll_grad(V[None])
        s2 = L.autotune(cache)
        assert "cached" in s2
    rows = json.load(open(cache))
    assert len(rows) == 1 and list(rows.values())[0]["choice"] in (2, 3)
    M = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    no, go, _ = oracle.nll_amp(wl.A_data, M, V)
    for n in (n0, n1):
        assert abs(n[0] - no) <= 1e-3 * (200_000 / 1e6) ** 0.5 + 2e-6


def test_resonance_tuning(pwa, tmp_path, monkeypatch):
    """The per-event free-resonance kernel has launch variants to time; the
    TMA-fed one (the default) has one launch shape."""
    wl = synth.resonance_workload("t", synth.waves_linear(8), 3, 50_000, 80_000)
    with pwa.Likelihood(8) as L:
        L.load_resonance_events(wl)
        assert "one launch shape" in L.autotune(None)
    monkeypatch.setenv("PWA_RES_KERNEL", "generic")
    V = synth.random_V(8, 4)
    cache = str(tmp_path / "tune.json")
    with pwa.Likelihood(8) as L:
        L.load_resonance_events(wl)
        r0 = L.nll_grad_res(V, wl.mass, wl.width)
        s = L.autotune(cache)
        assert "free resonances" in s and "timed" in s
        r1 = L.nll_grad_res(V, wl.mass, wl.width)
        assert "cached" in L.autotune(cache)
    assert abs(r0[0] - r1[0]) <= 1e-6 * abs(r0[0])
    assert np.allclose(r0[1], r1[1], rtol=1e-5, atol=1e-6 * np.abs(r0[1]).max())


def test_no_cache_file(pwa):
    wl = synth.mixture_workload("t", synth.waves_linear(4), 5000, 2000)
    with pwa.Likelihood(4) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        assert "timed" in L.autotune(None)


def test_tensor_core_tile_tuning(pwa, tmp_path):
    """The tensor-core form's tile parameters (sets per launch, X stages):
    timed, cached, applied; the results agree with the default shape to
    float summation order and with the oracle on the BFP16 inputs."""
    from test_gpu_batched import bfp_amplitudes, nll_tol
    wl = synth.mixture_workload("t", synth.waves_linear(16), 100_000, 20_000)
    K = 128
    Vs = synth.start_points(16, K, seed=9)
    cache = str(tmp_path / "tune.json")
    with pwa.Likelihood(16, forms=pwa.PWA_FORM_TC, max_k=K) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        L.set_form(pwa.PWA_FORM_TC)
        n0, g0 = L.nll_grad(Vs)
        s1 = L.autotune(cache)
        assert "tensor-core form" in s1 and "timed" in s1
        n1, g1 = L.nll_grad(Vs)
        assert "cached" in L.autotune(cache)
    rows = json.load(open(cache))
    (key, row), = rows.items()
    assert "tc-tiles|K128" in key and row["choice"] % 10000 in (64, 128)
    assert 2 <= row["choice"] // 10000 <= 6
    assert np.max(np.abs(n1 - n0) / np.abs(n0)) <= 1e-12
    assert np.linalg.norm(g1 - g0) <= 1e-6 * np.linalg.norm(g0)
    M = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    no, _, _ = oracle.nll_amp(bfp_amplitudes(wl.A_data, 2), M, Vs[0])
    assert abs(n1[0] - no) <= nll_tol(100_000)


def test_model_batch_tuning(pwa, tmp_path):
    """The model batch's launch shape (work items per SM, X stages): timed,
    cached and applied; results agree with the untuned batch to float
    summation order."""
    spec = [(8, 20_000), (20, 30_000), (33, 10_000)]
    wls = [synth.mixture_workload("b%d" % j, synth.waves_linear(N), n, 2 * n, seed_data=70 + j)
           for j, (N, n) in enumerate(spec)]
    K = 16
    Vs = [synth.start_points(N, K, seed=80 + j) for j, (N, _) in enumerate(spec)]
    cache = str(tmp_path / "tune.json")
    with pwa.ModelBatch([N for N, _ in spec], K) as B:
        for j, w in enumerate(wls):
            B.load_model(j, w.A_data, w.A_mc, w.n_gen)
        n0, g0 = B.nll_grad(Vs)
        s1 = B.autotune(cache)
        assert "model batch" in s1 and "timed" in s1
        n1, g1 = B.nll_grad(Vs)
        assert "cached" in B.autotune(cache)
        n2, g2 = B.nll_grad(Vs)
    (key, row), = json.load(open(cache)).items()
    assert "batch|M3" in key and row["choice"] % 100 in (4, 8, 16, 32)
    assert np.array_equal(n1, n2)
    assert np.max(np.abs(n1 - n0) / np.abs(n0)) <= 1e-12
    for a, b in zip(g0, g1):
        assert np.linalg.norm(a - b) <= 1e-6 * np.linalg.norm(a)
