"""GPU parity of the FUMILI Hessian, the MC projection weights and the fit
fractions against the FP64 oracle.

Hessian (FUMILI's sum_i grad ln I_i grad ln I_i^T): per-event gradients d_i
of ln I in FP32, so each d_i carries a few
units of 2^-24 relative to |A|/|S|; the products are summed in FP32 over runs
of a few hundred events and in float-float / FP64 beyond. The tensor-core
kernel (up to 20 waves) splits d_i into three BF16 terms (exact but for the
last bits of the third) and drops the products below 2^-23 |d_p d_q|; its
FP32 sums in tensor memory span 128 events. Bound, both kernels: max
|H - H_oracle| <= 3e-6 max |H_oracle|, and exactly symmetric. Weights: S in
FP32 by four FMA chains of ceil(N/4) waves joined pairwise, so per component
|dS| <= (gamma_k + u) sqrt(2) T with k = 2 ceil(N/4) + 2, u = 2^-24 (the +u
for V rounded to float) and T = sum_a |V_a| |A_a|; then
|d|S|^2| <= 2 |S| |dS| + |dS|^2 and four more roundings of |S|^2 / N_gen give
|w - w_exact| <= (4k + 10) u T^2 / N_gen. Fit fractions: FP64 from the same M,
to 1e-10.
"""
import math

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

H_TOL = 3e-6


@pytest.fixture(scope="module")
def pwa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_5673_gb300 as pkg
    return pkg


@pytest.fixture(params=["tc", "generic"])
def hess_kernel(request, monkeypatch):
    """Which Hessian kernel serves the sample: the tensor-core one (the
    default up to 20 waves; more waves take the other) or the CUDA-core one."""
    if request.param == "generic":
        monkeypatch.setenv("PWA_HESS_KERNEL", "generic")
    else:
        monkeypatch.delenv("PWA_HESS_KERNEL", raising=False)
    return request.param


def case(N, n_data, n_mc, seed=0):
    waves = synth.waves_linear(N)
    return synth.mixture_workload("h", waves, n_data, n_mc, seed_data=400 + seed,
                                  seed_mc=500 + seed, seed_v=600 + seed)


def real_grad(g):
    """(d/dRe V, d/dIm V) = (2 Re g, 2 Im g) from the Wirtinger gradient g."""
    return np.concatenate([2 * g.real, 2 * g.imag])


def check_hessian(L, wl, V):
    H = L.hessian(V)
    assert L.last_status == 0
    Ho, bad = oracle.hessian(wl.A_data, V)
    assert bad == 0
    assert np.array_equal(H, H.T)
    err = np.max(np.abs(H - Ho)) / np.max(np.abs(Ho))
    assert err <= H_TOL, err
    return H


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 8, 13, 20, 24, 25, 32, 40, 48])
def test_hessian_waves_sweep(pwa, hess_kernel, N):
    wl = case(N, 3000, 4000, seed=N)
    with pwa.Likelihood(N) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        for V in (wl.V_true, synth.random_V(N, 70 + N)):
            check_hessian(L, wl, V)


@pytest.mark.parametrize("n_data", [1, 7, 255, 256, 257, 2049, 10007])
def test_hessian_ragged_event_counts(pwa, hess_kernel, n_data):
    wl = case(20, n_data, 700, seed=n_data % 89)
    with pwa.Likelihood(20) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        check_hessian(L, wl, synth.random_V(20, n_data))


def test_hessian_any_form_current(pwa, hess_kernel):
    """The Hessian reads the direct-form store whichever form evaluates the NLL."""
    wl = case(12, 5000, 3000, seed=3)
    V = synth.random_V(12, 5)
    with pwa.Likelihood(12, forms=pwa.PWA_FORM_AMP | pwa.PWA_FORM_TABLE) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        H0 = L.hessian(V)
        L.set_form(pwa.PWA_FORM_TABLE)
        assert np.array_equal(L.hessian(V), H0)


def test_hessian_domain_error(pwa, hess_kernel):
    wl = case(6, 500, 500, seed=9)
    with pwa.Likelihood(6) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        H = L.hessian(np.zeros(6, complex))
        assert L.last_status == pwa.PWA_EDOMAIN
        assert not H.any()
        # the context stays usable
        check_hessian(L, wl, wl.V_true)


def test_hessian_homogeneity_at_scale(pwa, hess_kernel):
    """At a million events (the bench workload): H p = -2 grad NLL + 2 grad N
    with the GPU's own gradient (ln I_i is homogeneous of degree 2 in p, so
    H p = 2 sum_i grad ln I_i), the global phase direction (-Im V, Re V) is a
    null vector of H, and H is positive semi-definite."""
    N, n = 20, 1_000_000
    wl = case(N, n, 1_000_000, seed=1)
    V = wl.V_true * math.sqrt(n / oracle.norm_term(oracle.norm_matrix_blas(wl.A_mc, wl.n_gen),
                                                   wl.V_true)[0])
    with pwa.Likelihood(N) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        M = L.build_norm()
        H = L.hessian(V)
        _, g = L.nll_grad(V[None, :])
    p = np.concatenate([V.real, V.imag])
    gN = real_grad(M @ V)
    rhs = -2 * real_grad(g[0]) + 2 * gN
    assert np.linalg.norm(H @ p - rhs) <= 1e-5 * np.linalg.norm(gN)
    Jp = np.concatenate([-V.imag, V.real])
    assert np.linalg.norm(H @ Jp) <= 1e-5 * np.linalg.norm(H, 2) * np.linalg.norm(Jp)
    ev = np.linalg.eigvalsh(H)
    assert ev.min() >= -1e-6 * ev.max() and ev[1] > 0


@pytest.mark.slow
def test_hessian_against_oracle_at_scale(pwa, hess_kernel):
    """The bench workload (1M data events x 20 waves) against the FP64 oracle,
    at the fitted scale and at a random V."""
    N, n = 20, 1_000_000
    wl = case(N, n, 1000, seed=2)
    with pwa.Likelihood(N) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        for V in (wl.V_true, synth.random_V(N, 77)):
            check_hessian(L, wl, V)


@pytest.mark.parametrize("N", [1, 3, 8, 20, 33, 48])
@pytest.mark.parametrize("where", ["host", "device"])
@pytest.mark.parametrize("kernel", ["tma", "generic"])
def test_mc_weights(pwa, monkeypatch, N, where, kernel):
    """The TMA-fed weights mode of the direct-form kernel (S by the exact
    product split) and the per-event kernel (plain FP32 dot product) both
    meet the plain kernel's rounding bound."""
    import torch
    if kernel == "generic":
        monkeypatch.setenv("PWA_WEIGHTS_KERNEL", "generic")
    else:
        monkeypatch.delenv("PWA_WEIGHTS_KERNEL", raising=False)
    wl = case(N, 100, 5003, seed=N + 40)
    V = synth.random_V(N, N + 41)
    with pwa.Likelihood(N) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        M = L.build_norm()
        if where == "host":
            w = L.mc_weights(V)
        else:
            out = torch.empty(wl.A_mc.shape[0], dtype=torch.float32, device="cuda:0")
            w = L.mc_weights(V, out).cpu().numpy()
    wo = oracle.mc_weights(wl.A_mc, V, wl.n_gen)
    A = wl.A_mc.astype(np.complex128)
    T2 = (np.abs(A) * np.abs(V)[None, :]).sum(axis=1) ** 2 / wl.n_gen
    k = 2 * math.ceil(N / 4) + 2
    assert np.all(np.abs(w - wo) <= (4 * k + 10) * 2.0 ** -24 * T2)
    nv = oracle.norm_term(M, V)[0]
    assert abs(w.astype(np.float64).sum() - nv) <= 1e-6 * nv


@pytest.fixture(scope="module")
def paper_sample():
    """The bench workload: 1M data and 5M accepted MC events x 20 waves."""
    return synth.paper_scale()


@pytest.mark.slow
@pytest.mark.parametrize("kernel", ["tma", "generic"])
def test_mc_weights_at_scale(pwa, monkeypatch, paper_sample, kernel):
    """The bench configuration (5M accepted MC x 20 waves, weights into a
    device buffer): every weight within the bound of test_mc_weights, and
    their sum equal to V^H M V."""
    import torch
    if kernel == "generic":
        monkeypatch.setenv("PWA_WEIGHTS_KERNEL", "generic")
    else:
        monkeypatch.delenv("PWA_WEIGHTS_KERNEL", raising=False)
    wl = paper_sample
    V = synth.start_points(20, 1)[0]
    with pwa.Likelihood(20) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        M = L.build_norm()
        out = torch.empty(wl.A_mc.shape[0], dtype=torch.float32, device="cuda:0")
        w = L.mc_weights(V, out).cpu().numpy()
    wo = oracle.mc_weights(wl.A_mc, V, wl.n_gen)
    k = 2 * math.ceil(20 / 4) + 2
    for lo in range(0, wl.A_mc.shape[0], 1 << 20):
        A = wl.A_mc[lo:lo + (1 << 20)].astype(np.complex128)
        T2 = (np.abs(A) * np.abs(V)[None, :]).sum(axis=1) ** 2 / wl.n_gen
        assert np.all(np.abs(w[lo:lo + len(A)] - wo[lo:lo + len(A)]) <= (4 * k + 10) * 2.0 ** -24 * T2)
    nv = oracle.norm_term(M, V)[0]
    assert abs(w.astype(np.float64).sum() - nv) <= 1e-6 * nv


@pytest.mark.parametrize("N", [1, 2, 7, 20, 48])
def test_fit_fractions(pwa, N):
    wl = case(N, 100, 4000, seed=N + 80)
    V = synth.random_V(N, N + 81)
    with pwa.Likelihood(N) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        F = L.fit_fractions(V)
    Fo = oracle.fit_fractions(oracle.norm_matrix(wl.A_mc, wl.n_gen), V)
    assert np.max(np.abs(F - Fo)) <= 1e-10 * max(1.0, np.abs(Fo).max())
    assert abs(F.sum() - 1.0) <= 1e-12 * N * N
    assert np.all(np.diag(F) >= 0)


def test_extras_need_state(pwa):
    with pwa.Likelihood(4) as L:
        with pytest.raises(pwa.PwaError):
            L.hessian(np.ones(4, complex))
        with pytest.raises(pwa.PwaError):
            L.fit_fractions(np.ones(4, complex))


def test_hessian_async_matches_host_call(pwa, hess_kernel):
    import torch
    wl = case(9, 5000, 3000, seed=21)
    V = synth.random_V(9, 22)
    with pwa.Likelihood(9) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        H = L.hessian(V)
        dH = torch.empty(18, 18, dtype=torch.float64, device="cuda")
        L.hessian_async(torch.from_numpy(V).cuda(), dH)
        assert L.sync() == pwa.PWA_OK
        assert np.array_equal(dH.cpu().numpy(), H)
        L.hessian_async(torch.zeros(9, dtype=torch.complex128, device="cuda"), dH)
        assert L.sync() == pwa.PWA_EDOMAIN
        assert not dH.cpu().numpy().any()
