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
