"""GPU parity of the covariant tensor amplitudes of J/psi -> gamma X,
X -> K+ K- (Sec. 4) against the FP64 oracle, and of the likelihood of a
sample loaded from 3-momenta.

Both sides evaluate the same contractions in double precision, the GPU
rounding each amplitude once to float: every component within one unit in
the last place of float of the oracle's double, and almost all bitwise equal
to the rounded oracle. The likelihood of the covariant sample is the
incoherent sum over the 4 unobserved components (the J/psi helicity, the
photon polarization), compared with the oracle's Eq. 3 on the oracle's
amplitudes rounded to complex64 with the incoherent tolerances:
|dNLL| <= 1e-3 sqrt(n / 1e6) (floor 2e-6), ||dg|| / ||g_data|| <= 1e-5;
M within 1e-6 sqrt(M_aa M_bb) (a one-ulp change of a float amplitude moves a
product by at most 2^-22 of |A_a||A_b|, so |dM_ab| <= 2^-21 sqrt(M_aa M_bb)
by Cauchy-Schwarz).
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


def check_rounding(A32, p3, waves):
    Ao = oracle.covariant_amplitudes(p3, waves)
    ref = Ao.astype(np.complex64)
    for part in (np.real, np.imag):
        g, r64 = part(A32).astype(np.float64), part(Ao)
        ulp = np.spacing(np.abs(part(ref)).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(g - r64) <= ulp), np.max(np.abs(g - r64) / np.maximum(ulp, 1e-45))
    return np.mean(A32 == ref)


@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("N,n", [(12, 20_011), (1, 1), (5, 257), (48, 3001)])
def test_covariant_amplitudes(pwa, where, N, n):
    import torch
    waves = synth.cov_waves(N)
    p3, _ = synth.radiative_events(n, np.random.default_rng(100 + n))
    with pwa.Likelihood(N) as L:
        if where == "host":
            A = L.covariant_amplitudes(waves, p3)
        else:
            out = torch.empty(n, 4, N, dtype=torch.complex64, device="cuda")
            A = L.covariant_amplitudes(waves, torch.tensor(p3, device="cuda"), out).cpu().numpy()
    assert A.shape == (n, 4, N)
    assert check_rounding(A, p3, waves) >= (0.999 if n > 1000 else 0.99)


def test_covariant_edge_kinematics(pwa):
    """The photon along +z and -z (e1 falls back to the x axis), the X at the
    K+ K- threshold region and at the top of the range, kaons back to back
    with the photon."""
    waves = synth.cov_waves(6)
    m = np.array([1.0, 1.0, 2.999, 0.988, 1.5, 1.5, 2.2, 2.2])
    cg = np.array([1.0, -1.0, 0.3, -0.2, 1.0, -1.0, 0.0, 0.999999])
    pg = np.array([0.0, 1.0, 2.0, 3.0, 4.0, 5.0, 6.0, 0.5])
    ck = np.array([0.5, -0.5, 1.0, -1.0, 0.0, 1.0, -1.0, 0.2])
    pk = np.array([0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8])
    p3 = synth.radiative_kinematics(m, cg, pg, ck, pk)
    with pwa.Likelihood(6) as L:
        A = L.covariant_amplitudes(waves, p3)
    assert np.all(np.isfinite(A.view(np.float32)))
    # Event 0 sits on the pole of wave 0 (m = M_0 = 1.0): BW is i/(M G) and
    # Re A is zero up to the rounding of p.p from the momenta (~1e-14 of
    # |A| on either side), so the bound here is relative to |A|: one float
    # ulp of |A| per component, plus 1e-12 |A| for that cancellation.
    Ao = oracle.covariant_amplitudes(p3, waves)
    mag = np.abs(Ao)
    ulp = np.spacing(mag.astype(np.float32)).astype(np.float64)
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(A).astype(np.float64) - part(Ao)) <= ulp + 1e-12 * mag)


def test_covariant_invalid_waves(pwa):
    p3, _ = synth.radiative_events(10, np.random.default_rng(0))
    with pwa.Likelihood(2) as L:
        for bad in ([(1.5, 0.1, 1), (2.0, 0.2, 0)], [(1.5, 0.1, 0), (2.0, 0.0, 2)],
                    [(-1.5, 0.1, 0), (2.0, 0.2, 2)]):
            with pytest.raises(pwa.PwaError):
                L.covariant_amplitudes(bad, p3)


def covariant_case(N, n_data, n_mc, seed):
    waves = synth.cov_waves(N)
    p3d, _ = synth.radiative_events(n_data, np.random.default_rng(seed))
    p3m, drawn = synth.radiative_events(n_mc, np.random.default_rng(seed + 1), accept=True)
    return waves, p3d, p3m, drawn


@pytest.mark.parametrize("N,n_data,n_mc", [(12, 40_003, 30_001), (3, 1, 7), (8, 2049, 5000)])
def test_covariant_likelihood_against_oracle(pwa, N, n_data, n_mc):
    waves, p3d, p3m, drawn = covariant_case(N, n_data, n_mc, seed=N * 11 + n_data)
    Ad = oracle.covariant_amplitudes(p3d, waves).astype(np.complex64)
    Am = oracle.covariant_amplitudes(p3m, waves).astype(np.complex64)
    Mo = oracle.norm_matrix_incoh(Am, drawn)
    scale = 1 / np.sqrt(np.real(np.diag(Mo)))          # V_a ~ 1/sqrt(M_aa): comparable waves
    Vs = [synth.random_V(N, 41 + N) * scale, synth.random_V(N, 42 + N) * scale]
    with pwa.Likelihood(N, max_k=2) as L:
        L.load_covariant(waves, p3d, p3m, drawn)
        M = L.build_norm()
        nll, g = L.nll_grad(np.array(Vs))
        assert L.last_status == 0
    d = np.sqrt(np.real(np.diag(Mo)))
    assert np.all(np.abs(M - Mo) <= 1e-6 * np.outer(d, d) + 1e-12 * np.abs(Mo).max())
    for k, V in enumerate(Vs):
        no, go, bad = oracle.nll_incoh(Ad, Mo, V)
        assert bad == 0
        gd = go - oracle.norm_term(Mo, V)[1]
        assert abs(nll[k] - no) <= nll_tol(n_data), (k, nll[k] - no)
        assert np.linalg.norm(g[k] - go) <= 1e-5 * np.linalg.norm(gd), k
        assert np.all(np.abs(g[k] - go) <= 1e-5 * term_scale(Ad, V)), k


def test_covariant_load_equals_amplitude_load(pwa):
    """Loading from 3-momenta gives bitwise the results of loading the
    amplitudes that pwa_compute_covariant_amplitudes returns (one generator,
    two routes into the store; host and device momenta alike)."""
    import torch
    N = 10
    waves, p3d, p3m, drawn = covariant_case(N, 30_000, 20_000, seed=5)
    V = (synth.random_V(N, 9) * 30)[None, :]
    with pwa.Likelihood(N) as L:
        L.load_covariant(waves, p3d, p3m, drawn)
        M0 = L.build_norm()
        r0 = L.nll_grad(V)
        L.load_covariant(waves, torch.tensor(p3d, device="cuda"), torch.tensor(p3m, device="cuda"),
                         drawn)
        M1 = L.build_norm()
        r1 = L.nll_grad(V)
        Ad = L.covariant_amplitudes(waves, p3d)
        Am = L.covariant_amplitudes(waves, p3m)
        L.load_events(Ad, Am, drawn)
        M2 = L.build_norm()
        r2 = L.nll_grad(V)
    assert np.array_equal(M0, M1) and np.array_equal(M0, M2)
    for r in (r1, r2):
        assert np.array_equal(r0[0], r[0]) and np.array_equal(r0[1], r[1])


def test_covariant_load_limits(pwa):
    """The direct form takes up to 12 waves at 4 components; the
    tensor-core form takes coherent samples only."""
    waves, p3d, p3m, drawn = covariant_case(13, 100, 100, seed=3)
    with pwa.Likelihood(13) as L:
        with pytest.raises(pwa.PwaError):
            L.load_covariant(waves, p3d, p3m, drawn)
    with pwa.Likelihood(4, forms=pwa.PWA_FORM_TC) as L:
        with pytest.raises(pwa.PwaError):
            L.load_covariant(waves[:4], p3d, p3m, drawn)
