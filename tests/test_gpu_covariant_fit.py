"""A fit with the covariant amplitudes end to end (Sec. 4 and Eq. 3): data
events of J/psi -> gamma K+ K- drawn from the covariant intensity of four
waves (spins 0, 2, 0, 2), loaded from their 3-momenta on the device
(pwa_load_events_covariant: amplitudes generated on the GPU, incoherent sum
over the four unobserved components), fitted with L-BFGS on the GPU.

The data are drawn by accept-reject over a pool of phase-space candidates
with the oracle's FP64 amplitudes: weight eps(cos theta_gamma) I(V_true),
envelope the pool's largest weight (exact for the pool). Checks:
  * the GPU fit and the oracle's own fit (scipy L-BFGS-B with the oracle's
    gradient on the oracle's complex64-rounded amplitudes, started from the
    GPU minimum) agree: |dNLL| within the incoherent tolerance, the fitted V
    within 0.01 statistical errors (phase removed);
  * the fit recovers the generating V (yield-scaled): pulls below 5 sigma,
    and N(V) = N_data at the minimum (the extended likelihood's yield rule).
Statistical errors: the inverse of the oracle NLL's Hessian in the real
parameters (central differences of the oracle gradient, Im V_0 held).
"""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
import synth

pytestmark = pytest.mark.gpu

WAVES = [synth.CovWave(1.5, 0.15, 0), synth.CovWave(1.75, 0.12, 2),
         synth.CovWave(2.05, 0.2, 0), synth.CovWave(2.35, 0.25, 2)]
V_TRUE = np.array([1.0, 0.8 * np.exp(0.5j), 0.6 * np.exp(-1.0j), 0.5 * np.exp(2.0j)])
N = len(WAVES)
KEEP = np.array([k for k in range(2 * N) if k != N])


@pytest.fixture(scope="module")
def pwa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_5673_gb300 as pkg
    return pkg


def efficiency(p3):
    return 0.6 + 0.3 * p3[:, 2] / np.linalg.norm(p3[:, 0:3], axis=1)


@pytest.fixture(scope="module")
def sample():
    rng = np.random.default_rng(4711)
    pool, _ = synth.radiative_events(600_000, rng)
    A = oracle.covariant_amplitudes(pool, WAVES)                  # [n, 4, N]
    I = np.sum(np.abs(A @ V_TRUE) ** 2, axis=1)
    w = efficiency(pool) * I
    keep = rng.uniform(0.0, w.max(), len(w)) < w
    p3_data = pool[keep][:20_000]
    assert len(p3_data) == 20_000
    p3_mc, drawn = synth.radiative_events(60_000, np.random.default_rng(4712), accept=True)
    return p3_data, p3_mc, drawn


def pack(V):
    from paper_1108_5673_gb300 import fit
    V = fit.phase_fixed(V)
    return np.concatenate([V.real, V.imag])[KEEP]


def unpack(x):
    y = np.zeros(2 * N)
    y[KEEP] = x
    return y[:N] + 1j * y[N:]


def test_covariant_fit_against_oracle_and_truth(pwa, sample):
    from paper_1108_5673_gb300 import fit
    p3_data, p3_mc, drawn = sample
    n = len(p3_data)
    Ad = oracle.covariant_amplitudes(p3_data, WAVES).astype(np.complex64)
    Am = oracle.covariant_amplitudes(p3_mc, WAVES).astype(np.complex64)
    Mo = oracle.norm_matrix_incoh(Am, drawn)
    Vt = V_TRUE * math.sqrt(n / oracle.norm_term(Mo, V_TRUE)[0])    # yield-scaled truth
    rng = np.random.default_rng(5)
    V0 = Vt * (1 + 0.1 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)))

    with pwa.Likelihood(N) as L:
        L.load_covariant(WAVES, p3_data, p3_mc, drawn)
        L.build_norm()
        Vg, fg, info = fit.fit_lbfgs(L, V0)
    print("GPU fit:", info)

    def fgrad(x):
        nll, g, bad = oracle.nll_incoh(Ad, Mo, unpack(x))
        assert bad == 0
        return nll, np.concatenate([2 * g.real, 2 * g.imag])[KEEP]

    r = optimize.minimize(fgrad, pack(Vg), jac=True, method="L-BFGS-B",
                          options={"maxiter": 2000, "gtol": 1e-9, "ftol": 1e-15})
    Vo, fo = unpack(r.x), r.fun
    assert np.abs(r.jac).max() <= 1e-4, r
    # statistical errors from the oracle's Hessian (central differences)
    x0, h = pack(Vo), 1e-5 * np.abs(pack(Vo)).max()
    H = np.empty((len(x0), len(x0)))
    for k in range(len(x0)):
        e = np.zeros(len(x0))
        e[k] = h
        H[:, k] = (fgrad(x0 + e)[1] - fgrad(x0 - e)[1]) / (2 * h)
    sig = np.sqrt(np.diag(np.linalg.inv(0.5 * (H + H.T))))
    dv = pack(Vg) - pack(Vo)
    pull_gpu = np.max(np.abs(dv) / sig)
    pull_truth = np.max(np.abs(pack(Vo) - pack(Vt)) / sig)
    print("NLL(GPU) - NLL(oracle) = %.2e, max |dV|/sigma = %.2e, truth pulls max %.2f"
          % (fg - fo, pull_gpu, pull_truth))
    assert abs(fg - fo) <= max(1e-3 * math.sqrt(n / 1e6), 2e-6)
    assert pull_gpu <= 0.01
    assert pull_truth < 5.0
    # the extended likelihood's yield rule at the minimum: V^H M V = N_data
    assert abs(oracle.norm_term(Mo, Vo)[0] / n - 1) < 1e-6
