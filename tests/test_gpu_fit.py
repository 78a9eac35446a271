"""Fits through the autograd wrapper on the GPU against the oracle's fit."""
import math

import numpy as np
import pytest
from scipy import optimize

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pwa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_5673_gb300 as pkg
    return pkg


def accept_reject_toy(n_data=10_000, n_mc=30_000):
    """The four-wave model with data drawn from eps * I (oracle intensity)."""
    waves = synth.waves_small()
    V_true = synth.random_V(4, synth.SEED_VTRUE)
    ymax = [math.sqrt((2 * w.l + 1) / (4 * math.pi)) for w in waves]
    env = synth.EFF_MAX * sum(abs(v) / (w.mass * w.width) * y
                              for v, w, y in zip(V_true, waves, ymax)) ** 2

    def density(ev):
        A = synth.amplitudes(ev, waves, np.complex128)
        return synth.efficiency(ev["costh"]) * oracle.intensity(A, V_true)

    ev = synth.accept_reject(n_data, density, env, seed=synth.SEED_DATA)
    ev_mc, n_gen = synth.mc_sample(n_mc, seed=synth.SEED_MC)
    return (synth.amplitudes(ev, waves), synth.amplitudes(ev_mc, waves), n_gen, V_true)


def test_fit_matches_oracle_fit(pwa):
    from paper_1108_5673_gb300 import fit
    A, A_mc, n_gen, V_true = accept_reject_toy()
    M = oracle.norm_matrix(A_mc, n_gen)
    V0 = V_true * math.sqrt(len(A) / oracle.norm_term(M, V_true)[0]) * (1 + 0.2j)
    with pwa.Likelihood(4) as L:
        L.load_events(A, A_mc, n_gen)
        L.build_norm()
        Vg, fg, info = fit.fit_lbfgs(L, V0, grad_tol=1e-6, change_tol=1e-13)

    def f(x):
        n, g, _ = oracle.nll_amp(A, M, x[:4] + 1j * x[4:])
        return n, np.concatenate([2 * g.real, 2 * g.imag])
    r = optimize.minimize(f, np.concatenate([V0.real, V0.imag]), jac=True, method="L-BFGS-B",
                          options={"ftol": 1e-15, "gtol": 1e-9, "maxiter": 5000})
    Vo = r.x[:4] + 1j * r.x[4:]
    assert abs(fg - r.fun) < 1e-4
    assert np.max(np.abs(fit.phase_fixed(Vg) - fit.phase_fixed(Vo))) < 1e-4 * np.abs(Vo).max()
    assert abs(oracle.norm_term(M, Vg)[0] - len(A)) < 1e-3 * len(A)


def test_autograd_gradient_against_central_differences(pwa):
    """Central differences (h = 1e-4 relative) of the GPU NLL itself."""
    torch = pytest.importorskip("torch")
    from paper_1108_5673_gb300 import fit
    wl = synth.mixture_workload("fd", synth.waves_linear(6), 20_000, 20_000)
    V = synth.random_V(6, 5) * 3
    with pwa.Likelihood(6) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        x = torch.tensor(np.concatenate([V.real, V.imag]), requires_grad=True)
        fit.nll(x, L).backward()
        h = 1e-4 * np.abs(V).max()
        fd = np.empty(12)
        for k in range(12):
            e = np.zeros(12)
            e[k] = h
            xp, xm = x.detach().numpy() + e, x.detach().numpy() - e
            fd[k] = (float(fit.nll(torch.tensor(xp), L)) - float(fit.nll(torch.tensor(xm), L))) / (2 * h)
    g = x.grad.numpy()
    assert np.max(np.abs(fd - g)) < 1e-4 * np.max(np.abs(g))


def test_fumili_fit_matches_lbfgs(pwa):
    """FUMILI steps on the library's Hessian reach the L-BFGS minimum in the
    handful of iterations the paper reports (Sec. 5: 5-10)."""
    from paper_1108_5673_gb300 import fit
    A, A_mc, n_gen, V_true = accept_reject_toy()
    M = oracle.norm_matrix(A_mc, n_gen)
    V0 = V_true * math.sqrt(len(A) / oracle.norm_term(M, V_true)[0]) * (1 + 0.2j)
    with pwa.Likelihood(4) as L:
        L.load_events(A, A_mc, n_gen)
        L.build_norm()
        Vl, fl, _ = fit.fit_lbfgs(L, V0, grad_tol=1e-6, change_tol=1e-13)
        Vf, ff, info = fit.fit_fumili(L, V0, grad_tol=1e-6)
    assert info["iterations"] <= 12, info
    # both minima agree within the FP32 evaluation noise of the NLL: per-event
    # roundings of ~1e-7 in ln I add up as sqrt(n), the GPU tolerance
    # 1e-3 sqrt(n / 1e6) against the oracle (1e-4 at these 10k events)
    assert abs(ff - fl) < 1e-3 * math.sqrt(len(A) / 1e6), (ff, fl)
    assert np.max(np.abs(fit.phase_fixed(Vf) - fit.phase_fixed(Vl))) < 1e-4 * np.abs(Vl).max()


def test_fumili_steps_on_twenty_waves_reduce_the_nll(pwa):
    """20 waves, 200k events of the resonance-mixture sample (not drawn from
    the model's intensity, so FUMILI's dropped terms do not cancel and its
    convergence is only linear): every accepted step lowers the NLL, the
    phase stays fixed, and ten steps close a good part of the gap between a
    perturbed start and the L-BFGS minimum."""
    from paper_1108_5673_gb300 import fit
    wl = synth.mixture_workload("fu", synth.waves_linear(20), 200_000, 400_000)
    M = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    V0 = wl.V_true * math.sqrt(200_000 / oracle.norm_term(M, wl.V_true)[0]) * (1 + 0.05j)
    with pwa.Likelihood(20) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        f0 = float(L.nll(V0[None, :])[0])
        _, fl, _ = fit.fit_lbfgs(L, V0, change_tol=1e-13)
        Vf, ff, info = fit.fit_fumili(L, V0, max_iter=10)
    assert info["iterations"] == 10 and info["evaluations"] >= 11
    assert abs(Vf[0].imag) <= 1e-12 * abs(Vf[0])      # the fixed phase (V_0 real)
    assert fl <= ff < f0
    assert ff - fl <= 0.5 * (f0 - fl), (f0, ff, fl)   # measured: 0.25
