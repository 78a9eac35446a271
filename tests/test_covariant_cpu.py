"""Pins of the oracle's covariant tensor amplitudes of J/psi -> gamma X,
X -> K+ K- (paper Sec. 4: amplitudes built in the covariant tensor formalism;
the conventions are stated in oracle_cov_amplitudes): checks against
physics closed forms and symmetries, each of which a plausible slip (a
metric sign, the projector orthogonal to p, the factor 1/3, the boost, a
polarization vector, the Blatt-Weisskopf factor) fails.

* Spin 0 (E1 radiation): summed over the four unobserved components,
  |A|^2 = |BW|^2 (1 + cos^2 theta_gamma), the known photon distribution.
* Spin 2: in the X rest frame the tensor reduces to r_i r_j - r^2 delta_ij/3
  of the kaons' relative momentum; averaged over the kaon direction (exact
  with the 12 vertices of an icosahedron, a spherical 5-design),
  sum_l |A_l|^2 / (|BW| B2)^2 = (r^4/15) [2 (1 + cos^2 + gamma^2 sin^2)
  + (1 + cos^2)/3] of theta_gamma, with gamma the X's Lorentz factor.
* Rotations about the beam axis multiply component l by e^{i M alpha}
  (M = +1 for l = 0, 1 and -1 for l = 2, 3), the same for every wave.
* The pole: at m = M_a the amplitude is the coupling divided by -i M G.
"""
import math

import numpy as np

import oracle
import synth

Q0 = 0.197327


def b2(m):
    Q2 = m ** 2 / 4 - synth.M_K ** 2
    return np.sqrt(13 / (Q2 ** 2 + 3 * Q2 * Q0 ** 2 + 9 * Q0 ** 4))


def bw2(m, w):
    return 1 / ((w.mass ** 2 - m ** 2) ** 2 + (w.mass * w.width) ** 2)


def test_spin0_photon_distribution():
    rng = np.random.default_rng(1)
    n = 2000
    m = rng.uniform(1.0, 3.0, n)
    cg = rng.uniform(-1, 1, n)
    p3 = synth.radiative_kinematics(m, cg, rng.uniform(0, 6.28, n), rng.uniform(-1, 1, n),
                                    rng.uniform(0, 6.28, n))
    w = synth.CovWave(1.5, 0.1, 0)
    A = oracle.covariant_amplitudes(p3, [w])[:, :, 0]
    s = np.sum(np.abs(A) ** 2, axis=1)
    assert np.allclose(s, bw2(m, w) * (1 + cg ** 2), rtol=1e-12, atol=0)


def icosahedron():
    g = (1 + math.sqrt(5)) / 2
    v = []
    for a in (-1, 1):
        for b in (-g, g):
            v += [(0, a, b), (a, b, 0), (b, 0, a)]
    v = np.array(v, dtype=np.float64)
    return v / np.linalg.norm(v, axis=1)[:, None]


def test_spin2_average_over_kaon_directions():
    V = icosahedron()
    ck = V[:, 2]
    pk = np.arctan2(V[:, 1], V[:, 0])
    w = synth.CovWave(2.0, 0.2, 2)
    for m, cg, pg in [(1.3, 0.2, 0.7), (2.1, -0.8, 3.0), (2.9, 0.95, 5.5), (1.05, 0.0, 1.1)]:
        p3 = synth.radiative_kinematics(np.full(12, m), np.full(12, cg), np.full(12, pg), ck, pk)
        A = oracle.covariant_amplitudes(p3, [w])[:, :, 0]
        avg = np.mean(np.sum(np.abs(A) ** 2, axis=1))
        Eg = (synth.M_PSI ** 2 - m ** 2) / (2 * synth.M_PSI)
        gam = (synth.M_PSI - Eg) / m
        r2 = 4 * (m ** 2 / 4 - synth.M_K ** 2)
        s2 = 1 - cg ** 2
        want = r2 ** 2 / 15 * (2 * (1 + cg ** 2 + gam ** 2 * s2) + (1 + cg ** 2) / 3)
        assert abs(avg / (bw2(m, w) * b2(m) ** 2) - want) <= 1e-12 * want, (m, cg)


def test_rotation_about_beam():
    rng = np.random.default_rng(2)
    n = 500
    m, cg, pg = rng.uniform(1, 3, n), rng.uniform(-1, 1, n), rng.uniform(0, 6.28, n)
    ck, pk = rng.uniform(-1, 1, n), rng.uniform(0, 6.28, n)
    waves = synth.cov_waves(6)
    A = oracle.covariant_amplitudes(synth.radiative_kinematics(m, cg, pg, ck, pk), waves)
    alpha = 0.83
    B = oracle.covariant_amplitudes(synth.radiative_kinematics(m, cg, pg + alpha, ck, pk + alpha),
                                    waves)
    for l, M in enumerate((1, 1, -1, -1)):
        assert np.allclose(B[:, l, :], np.exp(1j * M * alpha) * A[:, l, :], rtol=1e-11,
                           atol=1e-12 * np.abs(A).max())


def test_pole():
    w0, w2 = synth.CovWave(1.7, 0.15, 0), synth.CovWave(1.7, 0.15, 2)
    rng = np.random.default_rng(3)
    n = 50
    p3 = synth.radiative_kinematics(np.full(n, 1.7), rng.uniform(-1, 1, n), rng.uniform(0, 6, n),
                                    rng.uniform(-1, 1, n), rng.uniform(0, 6, n))
    A = oracle.covariant_amplitudes(p3, [w0, w2])
    # BW at the pole = 1 / (-i M G) = i / (M G): |A|^2 summed equals the coupling's
    s0 = np.sum(np.abs(A[:, :, 0]) ** 2, axis=1)
    cg = p3[:, 2] / np.linalg.norm(p3[:, :3], axis=1)
    assert np.allclose(s0, (1 + cg ** 2) / (1.7 * 0.15) ** 2, rtol=1e-12)


def test_bad_spin():
    import pytest
    with pytest.raises(ValueError):
        oracle.covariant_amplitudes(np.zeros((1, 9)), [(1.5, 0.1, 1)])
