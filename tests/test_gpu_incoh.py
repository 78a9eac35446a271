"""GPU parity of the incoherent sum over unobserved components
(I = sum_l |sum_a V_a A_a^l|^2) against the FP64 oracle, in the direct form
and the table form.

Direct form: S^l by a compensated dot product (about one float rounding),
I as an FP32 sum of L squares, ln I = e ln 2 + ln f with float logf; per event
a few 1e-7 of random error in ln I, so the direct form's tolerances hold:
|dNLL| <= 1e-3 sqrt(n / 1e6) (floor 2e-6), ||dg|| / ||g_data|| <= 1e-5.
Table form: the oracle evaluates the same float32 table (its FP64 table of
the float amplitudes, each entry rounded once), with the same tolerances.
M: exact float products summed in FP64, to 1e-12 of its largest entry.
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


@pytest.fixture(params=["tma", "generic"])
def kernel(request, monkeypatch):
    """Which direct-form kernel serves the incoherent sample: the TMA-fed one
    (the default where it fits) or the one-event-per-thread one."""
    if request.param == "generic":
        monkeypatch.setenv("PWA_INCOH_KERNEL", "generic")
    else:
        monkeypatch.delenv("PWA_INCOH_KERNEL", raising=False)
    return request.param


def nll_tol(n):
    return max(1e-3 * math.sqrt(n / 1e6), 2e-6)


def case(N, L, n_data, n_mc, seed=0):
    return synth.incoherent_workload("inc", synth.waves_linear(N), n_data, n_mc, n_lambda=L,
                                     seed_data=700 + seed, seed_mc=800 + seed, seed_v=900 + seed)


def check_sets(nll, g, wl, M_ref, Vs, table=None):
    n = wl.A_data.shape[0]
    for k, V in enumerate(Vs):
        if table is None:
            no, go, bad = oracle.nll_incoh(wl.A_data, M_ref, V)
        else:
            no, go, bad = oracle.nll_table(table, M_ref, V)
        assert bad == 0
        gd = go - oracle.norm_term(M_ref, V)[1]
        assert abs(nll[k] - no) <= nll_tol(n), (k, nll[k], no, nll[k] - no)
        err = np.linalg.norm(g[k] - go) / np.linalg.norm(gd)
        assert err <= 1e-5, (k, err)
        c = term_scale(wl.A_data, V, table=table is not None)
        assert np.all(np.abs(g[k] - go) <= 1e-5 * c), (k, np.max(np.abs(g[k] - go) / c))


def run(pwa, wl, Vs, forms):
    N = wl.A_data.shape[2]
    out = {}
    with pwa.Likelihood(N, forms=forms, max_k=len(Vs)) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        out["M"] = L.build_norm()
        for form in (pwa.PWA_FORM_AMP, pwa.PWA_FORM_TABLE):
            if forms & form:
                L.set_form(form)
                out[form] = L.nll_grad(np.array(Vs))
                assert L.last_status == 0
    return out


@pytest.mark.parametrize("N,L", [(1, 2), (3, 2), (8, 2), (13, 2), (20, 2), (24, 2), (4, 3),
                                 (16, 3), (5, 4), (12, 4)])
def test_incoherent_against_oracle(pwa, kernel, N, L):
    wl = case(N, L, 3000, 2500, seed=N * 7 + L)
    Vs = [wl.V_true, synth.random_V(N, 31 + N)]
    out = run(pwa, wl, Vs, pwa.PWA_FORM_AMP | pwa.PWA_FORM_TABLE)
    Mo = oracle.norm_matrix_incoh(wl.A_mc, wl.n_gen)
    assert np.max(np.abs(out["M"] - Mo)) <= 1e-12 * np.abs(Mo).max()
    check_sets(*out[pwa.PWA_FORM_AMP], wl, Mo, Vs)
    T32 = oracle.table_incoh(wl.A_data).astype(np.float32).astype(np.float64)
    check_sets(*out[pwa.PWA_FORM_TABLE], wl, Mo, Vs, table=T32)


@pytest.mark.parametrize("n_data", [1, 7, 255, 256, 257, 2049, 10007])
def test_incoherent_ragged_event_counts(pwa, kernel, n_data):
    wl = case(20, 2, n_data, 600, seed=n_data % 83)
    Vs = [synth.random_V(20, n_data)]
    out = run(pwa, wl, Vs, pwa.PWA_FORM_AMP)
    check_sets(*out[pwa.PWA_FORM_AMP], wl, oracle.norm_matrix_incoh(wl.A_mc, wl.n_gen), Vs)


def test_one_component_equals_coherent(pwa):
    """[n, 1, N] amplitudes are the coherent sample: bitwise the same results."""
    wl = synth.mixture_workload("c", synth.waves_linear(12), 4000, 3000, seed_data=5, seed_mc=6)
    V = synth.random_V(12, 8)[None, :]
    with pwa.Likelihood(12) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        M0 = L.build_norm()
        r0 = L.nll_grad(V)
        L.load_events(wl.A_data[:, None, :], wl.A_mc[:, None, :], wl.n_gen)
        M1 = L.build_norm()
        r1 = L.nll_grad(V)
    assert np.array_equal(M0, M1)
    assert np.array_equal(r0[0], r1[0]) and np.array_equal(r0[1], r1[1])


def test_incoherent_deterministic_and_domain(pwa, kernel):
    wl = case(10, 3, 5000, 2000, seed=2)
    V = synth.random_V(10, 3)[None, :]
    with pwa.Likelihood(10) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        a = L.nll_grad(V)
        b = L.nll_grad(V)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        nll, g = L.nll_grad(np.zeros((1, 10), complex))
        assert L.last_status == pwa.PWA_EDOMAIN
        assert nll[0] == math.inf and not g.any()
        c = L.nll_grad(V)
        assert L.last_status == 0 and np.array_equal(c[0], a[0])


def test_incoherent_unsupported_paths(pwa):
    wl = case(20, 3, 100, 100, seed=4)
    with pwa.Likelihood(20) as L:   # 20 waves x 3 components exceeds the direct form
        with pytest.raises(pwa.PwaError):
            L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
    with pwa.Likelihood(20, forms=pwa.PWA_FORM_TABLE) as L:   # the table form takes it
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        L.nll_grad(synth.random_V(20, 1)[None, :])
        with pytest.raises(pwa.PwaError):
            L.hessian(synth.random_V(20, 1))
        with pytest.raises(pwa.PwaError):
            L.mc_weights(synth.random_V(20, 1))
        F = L.fit_fractions(synth.random_V(20, 1))
        assert abs(F.sum() - 1) < 1e-12
    with pwa.Likelihood(8, forms=pwa.PWA_FORM_TC) as L:
        w8 = case(8, 2, 100, 100, seed=5)
        with pytest.raises(pwa.PwaError):
            L.load_events(w8.A_data, w8.A_mc, w8.n_gen)


@pytest.mark.slow
def test_incoherent_at_scale(pwa, kernel):
    """1M events x 20 waves x 2 components (the bench workload) against the
    oracle, both forms."""
    wl = case(20, 2, 1_000_000, 1_000_000, seed=11)
    Mo = oracle.norm_matrix_incoh(wl.A_mc, wl.n_gen)
    nv = oracle.norm_term(Mo, wl.V_true)[0]
    Vs = [wl.V_true * math.sqrt(1_000_000 / nv), synth.random_V(20, 12)]
    out = run(pwa, wl, Vs, pwa.PWA_FORM_AMP | pwa.PWA_FORM_TABLE)
    assert np.max(np.abs(out["M"] - Mo)) <= 1e-12 * np.abs(Mo).max()
    check_sets(*out[pwa.PWA_FORM_AMP], wl, Mo, Vs)
    T32 = oracle.table_incoh(wl.A_data).astype(np.float32).astype(np.float64)
    check_sets(*out[pwa.PWA_FORM_TABLE], wl, Mo, Vs, table=T32)
