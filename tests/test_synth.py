"""The seeded input generator against library routines and its stated recipe."""
import math

import numpy as np
import pytest
from scipy import special

import synth


@pytest.mark.parametrize("l,m", [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 1), (4, 0),
                                 (4, 3), (4, 4), (2, -1)])
def test_ylm_matches_scipy(l, m):
    rng = np.random.Generator(np.random.Philox(1))
    ev = synth.phase_space(2000, rng)
    theta = np.arccos(ev["costh"])
    want = special.sph_harm_y(l, m, theta, ev["phi"])
    got = synth.ylm(l, m, ev["costh"], ev["phi"])
    assert np.max(np.abs(got - want)) < 1e-14


def test_breit_wigner_peak_and_form():
    M, G = 1.7, 0.15
    bw = synth.breit_wigner(np.array([M]), M, G)[0]
    assert abs(bw - 1j / (M * G)) < 1e-15 * abs(bw)
    m = np.linspace(synth.M_LO, synth.M_HI, 1001)
    assert np.all(np.abs(synth.breit_wigner(m, M, G)) <= 1 / (M * G) + 1e-12)


def test_mc_acceptance_fraction_and_ngen():
    ev, n_gen = synth.mc_sample(200_000, seed=5)
    assert len(ev["m"]) == 200_000
    # E[eps] = 0.6 over uniform cos(theta)
    frac = 200_000 / n_gen
    assert abs(frac - 0.6) < 5 * math.sqrt(0.6 * 0.4 / n_gen)
    # accepted events follow eps: <cos theta> = 0.3 * (1/3) / 0.6 = 1/6
    assert abs(ev["costh"].mean() - 1 / 6) < 0.01
    assert ev["m"].min() >= synth.M_LO and ev["m"].max() <= synth.M_HI


def test_waves_linear_recipe():
    w = synth.waves_linear(20)
    assert [x.l for x in w[:6]] == [0, 2, 4, 0, 2, 4]
    assert abs(w[0].mass - 1.0) < 1e-15 and abs(w[19].mass - 2.9) < 1e-12
    assert abs(w[0].width - 0.05) < 1e-15 and abs(w[19].width - 0.4) < 1e-12
    assert all(0 <= x.m <= x.l for x in w)


def test_seeded_and_reproducible():
    a = synth.mixture_workload("t", synth.waves_linear(5), 1000, 2000)
    b = synth.mixture_workload("t", synth.waves_linear(5), 1000, 2000)
    assert np.array_equal(a.A_data, b.A_data) and np.array_equal(a.A_mc, b.A_mc)
    assert a.n_gen == b.n_gen and a.A_data.dtype == np.complex64


def test_radiative_events_physical():
    """Every radiative event lies above the K+ K- threshold, conserves the
    J/psi's momentum, and has the kaons and X on shell."""
    p3, drawn = synth.radiative_events(20_000, np.random.default_rng(3), accept=True)
    assert np.all(np.isfinite(p3)) and drawn >= 20_000
    q, k1, k2 = p3[:, 0:3], p3[:, 3:6], p3[:, 6:9]
    assert np.abs(q + k1 + k2).max() < 1e-12
    E = (np.linalg.norm(q, axis=1) + np.sqrt(synth.M_K ** 2 + np.sum(k1 ** 2, 1))
         + np.sqrt(synth.M_K ** 2 + np.sum(k2 ** 2, 1)))
    assert np.abs(E - synth.M_PSI).max() < 1e-12
    m2 = (E - np.linalg.norm(q, axis=1)) ** 2 - np.sum((k1 + k2) ** 2, 1)
    assert np.sqrt(m2).min() > 2 * synth.M_K
