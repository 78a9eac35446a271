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


def test_lbfgs_fit_matches_scipy_fit():
    A, M, V0 = sample(n=2000, n_mc=3000, seed=4)
    lik = OracleLik(A, M)
    V0 = V0 * math.sqrt(len(A) / oracle.norm_term(M, V0)[0])
    Vh, f, info = fit.fit_lbfgs(lik, V0 * (1 + 0.1j), max_iter=300)

    def fs(x):
        n, g, _ = oracle.nll_amp(A, M, x[:4] + 1j * x[4:])
        return n, np.concatenate([2 * g.real, 2 * g.imag])
    r = optimize.minimize(fs, np.concatenate([(V0 * (1 + 0.1j)).real, (V0 * (1 + 0.1j)).imag]),
                          jac=True, method="L-BFGS-B", options={"ftol": 1e-15, "gtol": 1e-9})
    Vs = r.x[:4] + 1j * r.x[4:]
    assert abs(f - r.fun) < 1e-6 * abs(r.fun)
    assert np.max(np.abs(fit.phase_fixed(Vh) - fit.phase_fixed(Vs))) < 1e-4 * np.abs(Vs).max()
    # extended likelihood at the optimum: N(V_hat) = N_data
    assert abs(oracle.norm_term(M, Vh)[0] - len(A)) < 1e-3 * len(A)
