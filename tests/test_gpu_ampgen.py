"""GPU parity of the amplitude generator (BW x Y_l^m in FP64, rounded once to
complex64) against the FP64 oracle of the amplitude model.

Both sides evaluate the same definitions in double precision (the GPU forms
e^{i m phi} by complex powers of one sincos, the oracle calls cos and sin of
m phi), so the GPU's float is the oracle's value rounded to nearest except
where the two doubles straddle a rounding boundary: every component within
one unit in the last place of float, and almost all bitwise equal to the
rounded oracle.
"""
import math

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


def events(n, seed):
    return synth.phase_space(n, np.random.Generator(np.random.Philox(seed)))


def check_rounding(A32, ev, waves):
    Ao = oracle.amplitudes(ev["m"], ev["costh"], ev["phi"], waves)
    ref = Ao.astype(np.complex64)
    for part in (np.real, np.imag):
        g, r64 = part(A32).astype(np.float64), part(Ao)
        ulp = np.spacing(np.abs(part(ref)).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(g - r64) <= ulp), np.max(np.abs(g - r64) / np.maximum(ulp, 1e-45))
    return np.mean(A32 == ref)


@pytest.mark.parametrize("where", ["host", "device"])
def test_twenty_waves(pwa, where):
    import torch
    waves = synth.waves_linear(20)
    ev = events(20_011, 1)
    with pwa.Likelihood(20) as L:
        if where == "host":
            A = L.amplitudes(waves, ev)
        else:
            kin = torch.tensor(np.stack([ev["m"], ev["costh"], ev["phi"]], 1), device="cuda")
            out = torch.empty(20_011, 20, dtype=torch.complex64, device="cuda")
            A = L.amplitudes(waves, kin, out).cpu().numpy()
    assert check_rounding(A, ev, waves) >= 0.999


@pytest.mark.slow
def test_amplitudes_at_scale(pwa):
    """The bench configuration (5M events x 20 waves, kinematics and
    amplitudes on the device): a random sample of 200k events against the
    oracle, one by one."""
    import torch
    waves = synth.waves_linear(20)
    ev, _ = synth.mc_sample(5_000_000)
    n = ev["m"].shape[0]
    kin = torch.from_numpy(np.stack([ev["m"], ev["costh"], ev["phi"]], 1)).cuda()
    out = torch.empty(n, 20, dtype=torch.complex64, device="cuda")
    with pwa.Likelihood(20) as L:
        L.amplitudes(waves, kin, out)
    idx = np.sort(np.random.Generator(np.random.Philox(5)).choice(n, 200_000, replace=False))
    A = out[torch.from_numpy(idx).cuda()].cpu().numpy()
    sample = {k: np.ascontiguousarray(ev[k][idx]) for k in ("m", "costh", "phi")}
    assert check_rounding(A, sample, waves) >= 0.999


def test_all_l_and_m_up_to_sixteen(pwa):
    waves = [(0.9 + 0.1 * l, 0.02 + 0.03 * ((l + m) % 5), l, m)
             for l in (0, 1, 3, 7, 12, 16) for m in sorted({-l, -(l // 2), 0, l // 2, l})]
    waves = waves[:48]
    ev = events(3001, 2)
    with pwa.Likelihood(len(waves)) as L:
        A = L.amplitudes(waves, ev)
    assert check_rounding(A, ev, waves) >= 0.999


@pytest.mark.parametrize("n", [1, 31, 255, 257])
def test_ragged_counts(pwa, n):
    waves = synth.waves_small()
    ev = events(n, 3 + n)
    with pwa.Likelihood(4) as L:
        A = L.amplitudes(waves, ev)
    check_rounding(A, ev, waves)


def test_invalid_waves(pwa):
    ev = events(10, 4)
    with pwa.Likelihood(2) as L:
        for bad in ([(1.0, 0.1, 2, 3), (1.0, 0.1, 0, 0)], [(1.0, 0.1, 17, 0), (1.0, 0.1, 0, 0)],
                    [(1.0, -0.1, 1, 0), (1.0, 0.1, 0, 0)]):
            with pytest.raises(pwa.PwaError):
                L.amplitudes(bad, ev)


def test_load_generated_sample(pwa):
    """A sample loaded from kinematics evaluates like the same sample loaded
    from the oracle's amplitudes (rounded to complex64): NLL and gradient
    against the FP64 oracle on those amplitudes, direct and table forms."""
    waves = synth.waves_linear(12)
    V = synth.random_V(12, 9)
    ev_d = synth.data_sample_mixture(5000, waves, V, seed=31)
    ev_m, n_gen = synth.mc_sample(6000, seed=32)
    A_d = oracle.amplitudes(ev_d["m"], ev_d["costh"], ev_d["phi"], waves).astype(np.complex64)
    A_m = oracle.amplitudes(ev_m["m"], ev_m["costh"], ev_m["phi"], waves).astype(np.complex64)
    Mo = oracle.norm_matrix(A_m, n_gen)
    no, go, _ = oracle.nll_amp(A_d, Mo, V)
    gd = go - oracle.norm_term(Mo, V)[1]
    with pwa.Likelihood(12, forms=pwa.PWA_FORM_AMP | pwa.PWA_FORM_TABLE) as L:
        L.load_generated(waves, ev_d, ev_m, n_gen)
        M = L.build_norm()
        assert np.max(np.abs(M - Mo)) <= 1e-6 * np.abs(Mo).max()
        for form in (pwa.PWA_FORM_AMP, pwa.PWA_FORM_TABLE):
            L.set_form(form)
            nll, g = L.nll_grad(V[None, :])
            assert abs(nll[0] - no) <= 1e-3 * math.sqrt(5000 / 1e6) + 1e-4, (form, nll[0], no)
            assert np.linalg.norm(g[0] - go) <= 1e-5 * np.linalg.norm(gd) + 1e-6 * np.linalg.norm(go)
