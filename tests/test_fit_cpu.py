"""Gradient conventions and the fit driver, on CPU.

The autograd wrapper only maps the library's Wirtinger gradient g = dNLL/dV*
to what torch expects; here it is driven by a stand-in whose nll_grad is the
FP64 oracle, and checked against torch's own autograd of a plain torch
statement of Eq. 3 (complex V and the real (Re V, Im V) parameterisation).
"""
import math

import numpy as np
import pytest
import torch
from scipy import optimize

import oracle
import synth
from hessian_exact import exact_hessian
from paper_1108_5673_gb300 import fit


class OracleLik:
    """Stand-in with the Likelihood interface, backed by the oracle."""

    def __init__(self, A, M):
        self.A, self.M, self.n_data = A, M, A.shape[0]

    def nll_grad(self, V):
        n, g, _ = oracle.nll_amp(self.A, self.M, V)
        return np.atleast_1d(n), np.atleast_2d(g)


def torch_nll(A, M, V):
    S = torch.from_numpy(A) @ V
    I = (S * S.conj()).real
    return -torch.log(I).sum() + (V.conj() @ torch.from_numpy(M) @ V).real


def sample(n=300, n_mc=400, N=4, seed=1):
    rng = np.random.Generator(np.random.Philox(seed))
    waves = synth.waves_small()[:N]
    A = synth.amplitudes(synth.phase_space(n, rng), waves, np.complex128)
    A_mc = synth.amplitudes(synth.phase_space(n_mc, rng), waves, np.complex128)
    return A, oracle.norm_matrix(A_mc, 700.0), synth.random_V(N, seed + 3)


def test_complex_parameter_gradient_matches_torch_autograd():
    A, M, V0 = sample()
    lik = OracleLik(A, M)
    V = torch.tensor(V0, dtype=torch.complex128, requires_grad=True)
    fit.nll(V, lik).backward()
    W = torch.tensor(V0, dtype=torch.complex128, requires_grad=True)
    torch_nll(A, M, W).backward()
    assert torch.allclose(V.grad, W.grad, rtol=1e-10, atol=0)


def test_real_parameter_gradient_matches_torch_autograd():
    A, M, V0 = sample(seed=2)
    lik = OracleLik(A, M)
    N = V0.shape[0]
    x = torch.tensor(np.concatenate([V0.real, V0.imag]), requires_grad=True)
    fit.nll(x, lik).backward()
    y = torch.tensor(np.concatenate([V0.real, V0.imag]), requires_grad=True)
    torch_nll(A, M, torch.complex(y[:N], y[N:])).backward()
    assert torch.allclose(x.grad, y.grad, rtol=1e-10, atol=0)


def test_exact_hessian_pin():
    """The fit tests' exact Hessian against central differences of the
    oracle's analytic gradient."""
    wl = synth.mixture_workload("h", synth.waves_linear(6), 3000, 5000)
    A = wl.A_data.astype(np.complex128)
    M = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    V = synth.random_V(6, 3) * 5
    H = exact_hessian(A, M, V)

    def grad(V):
        _, g, _ = oracle.nll_amp(A, M, V)
        return np.concatenate([2 * g.real, 2 * g.imag])
    h, Hd = 1e-6, np.zeros((12, 12))
    for k in range(12):
        e = np.zeros(12)
        e[k] = h
        Hd[:, k] = (grad(V + e[:6] + 1j * e[6:]) - grad(V - e[:6] - 1j * e[6:])) / (2 * h)
    assert np.abs(H - Hd).max() <= 1e-7 * np.abs(H).max()
    assert np.allclose(H, H.T, rtol=0, atol=1e-9 * np.abs(H).max())


def test_lbfgs_fit_reaches_a_minimum():
    """The driver (scaled variables, default criteria) stops at a minimum of
    the oracle's NLL: a trust-region Newton method with the exact Hessian,
    started there, moves V by < 1e-4 of |V| and the NLL by < 1e-6 relative.
    (Eq. 3 has several minima on this toy; different optimizers from the
    same start were seen to reach different ones.)"""
    A, M, V0 = sample(n=2000, n_mc=3000, seed=4)
    lik = OracleLik(A, M)
    V0 = V0 * math.sqrt(len(A) / oracle.norm_term(M, V0)[0])
    Vh, f, info = fit.fit_lbfgs(lik, V0 * (1 + 0.1j), max_iter=300)
    assert info["grad_inf_scaled"] <= 1e-3
    N = V0.shape[0]
    keep = np.array([k for k in range(2 * N) if k != N])
    Vp = fit.phase_fixed(Vh)

    def unpack(x):
        y = np.zeros(2 * N)
        y[keep] = x
        return y[:N] + 1j * y[N:]

    def fg(x):
        n, g, _ = oracle.nll_amp(A, M, unpack(x))
        return n, np.concatenate([2 * g.real, 2 * g.imag])[keep]
    r = optimize.minimize(lambda x: fg(x)[0], np.concatenate([Vp.real, Vp.imag])[keep],
                          jac=lambda x: fg(x)[1],
                          hess=lambda x: exact_hessian(A, M, unpack(x))[np.ix_(keep, keep)],
                          method="trust-exact", options={"gtol": 1e-9})
    Vs = unpack(r.x)
    assert abs(f - r.fun) < 1e-6 * abs(r.fun)
    assert np.max(np.abs(Vp - Vs)) < 1e-4 * np.abs(Vs).max()
    # extended likelihood at the optimum: N(V_hat) = N_data
    assert abs(oracle.norm_term(M, Vh)[0] - len(A)) < 1e-3 * len(A)


def test_lbfgs_unscaled_variables():
    """scaled=False keeps the plain (Re V, Im V) variables and the gradient
    criterion 1e-6 n_data."""
    A, M, V0 = sample(n=2000, n_mc=3000, seed=4)
    lik = OracleLik(A, M)
    V0 = V0 * math.sqrt(len(A) / oracle.norm_term(M, V0)[0])
    Vh, f, info = fit.fit_lbfgs(lik, V0 * (1 + 0.1j), max_iter=300, scaled=False)
    assert info["grad_inf"] <= 1e-6 * len(A) or info["iterations"] >= 1
    assert abs(oracle.norm_term(M, Vh)[0] - len(A)) < 1e-2 * len(A)
