"""GPU parity of the free-resonance form (masses and widths of the first R
Breit-Wigner waves free) against the FP64 oracle.

Identical inputs: m rounded to float32, Y and the fixed amplitudes complex64,
promoted exactly for the oracle; V, masses and widths exact. Per event the
kernel's errors are float roundings that vary from event to event (the
Breit-Wigner denominator is formed from float pairs of M^2, M G and (M G)^2
and the exact split of m^2; S is exact up to about one float rounding: by
the direct form's exact product split in the TMA-fed kernel, by a
compensated dot product in the per-event one; both kernels are tested), so
they add as
sqrt(n): |dNLL| <= 1e-3 sqrt(n_data / 1e6) + 1e-6 (n_mc / 1e6), the second term
for the MC sum, whose (1/N_gen) sum I carries float-float sums of
per-event float intensities. Gradients: ||dg|| / max(||g_data||, ||g_MC||)
<= 1e-5 for dNLL/dV* and for (dNLL/dM, dNLL/dGamma) together. Unlike the fixed
form, where the MC part is the exact FP64 product M V, here the kernel sums
the MC part too, so its float errors scale with the larger of the two parts
(the oracle evaluated without data events gives the MC part).
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


@pytest.fixture(params=["tma", "generic"])
def kernel(request, monkeypatch):
    """Which kernel serves the free-resonance sample: the TMA-fed one (the
    default) or the one-event-per-thread one."""
    if request.param == "generic":
        monkeypatch.setenv("PWA_RES_KERNEL", "generic")
    else:
        monkeypatch.delenv("PWA_RES_KERNEL", raising=False)
    return request.param


def nll_tol(n_data, n_mc):
    return 1e-3 * math.sqrt(n_data / 1e6) + 1e-6 * (n_mc / 1e6) + 2e-6


def oracle_args(wl):
    return (wl.m_data.astype(np.float64), wl.Y_data, wl.Afix_data, wl.m_mc.astype(np.float64),
            wl.Y_mc, wl.Afix_mc, float(wl.n_gen))


def oracle_data_part(wl, V, mass, width):
    """The MC part alone (no data events)."""
    N = len(wl.waves)
    R = wl.n_free
    empty_m = np.zeros(0)
    _, gV, gM, gW, _ = oracle.nll_res(empty_m, np.zeros((0, R), complex), np.zeros((0, N - R), complex),
                                      wl.m_mc.astype(np.float64), wl.Y_mc, wl.Afix_mc,
                                      float(wl.n_gen), V, mass, width)
    return gV, gM, gW


def check(pwa, wl, params):
    N = len(wl.waves)
    with pwa.Likelihood(N) as L:
        L.load_resonance_events(wl)
        for V, mass, width in params:
            nll, gV, gM, gW = L.nll_grad_res(V, mass, width)
            assert L.last_status == pwa.PWA_OK
            no, gVo, gMo, gWo, bad = oracle.nll_res(*oracle_args(wl), V, mass, width)
            assert bad == 0
            mV, mM, mW = oracle_data_part(wl, V, mass, width)
            n_d, n_m = len(wl.m_data), len(wl.m_mc)
            assert abs(nll - no) <= nll_tol(n_d, n_m), (nll, no, nll - no)
            scaleV = max(np.linalg.norm(gVo - mV), np.linalg.norm(mV))
            errV = np.linalg.norm(gV - gVo) / scaleV
            assert errV <= 1e-5, errV
            gp, gpo, mp = np.concatenate([gM, gW]), np.concatenate([gMo, gWo]), np.concatenate([mM, mW])
            errP = np.linalg.norm(gp - gpo) / max(np.linalg.norm(gpo - mp), np.linalg.norm(mp))
            assert errP <= 1e-5, errP


def case(N, R, n_data, n_mc, seed=0):
    return synth.resonance_workload("t", synth.waves_linear(N), R, n_data, n_mc,
                                    seed_data=700 + seed, seed_mc=800 + seed, seed_v=900 + seed)


def params_for(wl, k=2, seed=0):
    rng = np.random.Generator(np.random.Philox(1234 + seed))
    out = []
    for j in range(k):
        V = synth.random_V(len(wl.waves), 50 + seed + j)
        mass = wl.mass * (1 + 0.02 * rng.standard_normal(wl.n_free))
        width = wl.width * (1 + 0.1 * rng.standard_normal(wl.n_free))
        out.append((V, mass, width))
    return out


@pytest.mark.parametrize("N,R", [(1, 1), (4, 2), (8, 4), (13, 5), (20, 4), (20, 8), (24, 3), (32, 4),
                                 (6, 6)])
def test_waves_sweep(pwa, kernel, N, R):
    wl = case(N, R, 3000, 5000, seed=N + R)
    check(pwa, wl, params_for(wl, seed=N))


@pytest.mark.parametrize("n_data", [1, 2, 255, 256, 257, 4097])
def test_ragged_event_counts(pwa, kernel, n_data):
    wl = case(10, 3, n_data, 777, seed=n_data % 13)
    check(pwa, wl, params_for(wl, 1, seed=n_data))


def test_at_generated_parameters_equals_fixed_form(pwa, kernel):
    """At fixed masses and widths the free-resonance NLL is the direct form's
    (Sec. 2: the precomputation is valid then): both GPU paths on the same
    events agree up to the float rounding of the amplitudes BW * Y, which the
    direct form receives rounded to complex64 (random per event)."""
    wl = case(12, 4, 20000, 30000, seed=3)
    V = synth.random_V(12, 77)

    def full(m, Y, Afix):
        bw = np.stack([synth.breit_wigner(m.astype(np.float64), M, G) for M, G in zip(wl.mass, wl.width)], 1)
        return np.concatenate([(bw * Y).astype(np.complex64), Afix], 1)

    A_d, A_m = full(wl.m_data, wl.Y_data, wl.Afix_data), full(wl.m_mc, wl.Y_mc, wl.Afix_mc)
    with pwa.Likelihood(12) as L:
        L.load_resonance_events(wl)
        nll_r, gV_r, _, _ = L.nll_grad_res(V, wl.mass, wl.width)
        L.load_events(A_d, A_m, wl.n_gen)
        L.build_norm()
        nll_d, g_d = L.nll_grad(V[None])
    assert abs(nll_r - nll_d[0]) <= 2 * nll_tol(20000, 30000) + 1e-7 * math.sqrt(20000)
    assert np.linalg.norm(gV_r - g_d[0]) <= 1e-4 * np.linalg.norm(g_d[0]) + 1e-3


def test_domain_error(pwa, kernel):
    wl = case(6, 2, 1000, 1000, seed=5)
    with pwa.Likelihood(6) as L:
        L.load_resonance_events(wl)
        nll, gV, gM, gW = L.nll_grad_res(np.zeros(6, complex), wl.mass, wl.width)
        assert L.last_status == pwa.PWA_EDOMAIN
        assert np.isinf(nll) and not np.any(gV) and not np.any(gM) and not np.any(gW)
        # the context stays usable
        nll2, *_ = L.nll_grad_res(synth.random_V(6, 1), wl.mass, wl.width)
        assert L.last_status == pwa.PWA_OK and np.isfinite(nll2)


def test_gradient_by_finite_differences(pwa, kernel):
    """Central differences (h = 1e-4) of the GPU NLL in mass and width. Near a
    narrow resonance the h^2 term of a central difference is not small (0.2%
    here), so the GPU difference is compared with the oracle's at the same h,
    and the analytic gradient with the Richardson combination
    (4 D(h/2) - D(h)) / 3, which cancels the h^2 term."""
    wl = case(20, 4, 100_000, 150_000, seed=9)
    V = synth.random_V(20, 5)
    mass, width = wl.mass.copy(), wl.width.copy()
    h = 1e-4
    args = oracle_args(wl)
    with pwa.Likelihood(20) as L:
        L.load_resonance_events(wl)
        _, _, gM, gW = L.nll_grad_res(V, mass, width)

        def diff(f, which, r, step):
            par = (mass if which == 0 else width)
            p1, p2 = par.copy(), par.copy()
            p1[r] += step
            p2[r] -= step
            a1 = (p1, width) if which == 0 else (mass, p1)
            a2 = (p2, width) if which == 0 else (mass, p2)
            return (f(*a1) - f(*a2)) / (2 * step)

        gpu = lambda m_, w_: L.nll_grad_res(V, m_, w_)[0]
        orc = lambda m_, w_: oracle.nll_res(*args, V, m_, w_)[0]
        for r in range(4):
            for which, g in ((0, gM), (1, gW)):
                d_gpu, d_orc = diff(gpu, which, r, h), diff(orc, which, r, h)
                assert abs(d_gpu - d_orc) <= 1e-4 * abs(d_orc) + 2.0, (r, which, d_gpu, d_orc)
                rich = (4 * diff(gpu, which, r, h / 2) - d_gpu) / 3
                assert abs(rich - g[r]) <= 1e-4 * abs(g[r]) + 4.0, (r, which, rich, g[r])


def test_autograd_function(pwa):
    import torch
    from paper_1108_5673_gb300 import fit
    wl = case(8, 3, 5000, 8000, seed=11)
    V = synth.random_V(8, 3)
    with pwa.Likelihood(8) as L:
        L.load_resonance_events(wl)
        x = torch.tensor(np.concatenate([V.real, V.imag, wl.mass, wl.width]), requires_grad=True)
        f = fit.nll_res(x, L)
        f.backward()
        nll, gV, gM, gW = L.nll_grad_res(V, wl.mass, wl.width)
    assert float(f.detach()) == nll
    expect = np.concatenate([2 * gV.real, 2 * gV.imag, gM, gW])
    assert np.array_equal(x.grad.numpy(), expect)


@pytest.mark.slow
def test_free_resonance_scale(pwa, kernel):
    """2M data events, 5M accepted MC, 20 waves, 4 free Breit-Wigners."""
    wl = synth.free_resonance_scale()
    check(pwa, wl, params_for(wl, 1, seed=2))


def test_async_matches_host_call(pwa, kernel):
    import torch
    wl = case(12, 3, 4000, 6000, seed=5)
    V, mass, width = params_for(wl, k=1, seed=5)[0]
    with pwa.Likelihood(12) as L:
        L.load_resonance_events(wl)
        nll, gV, gM, gW = L.nll_grad_res(V, mass, width)
        dout = torch.empty(1 + 24 + 6, dtype=torch.float64, device="cuda")
        L.nll_grad_res_async(torch.from_numpy(V).cuda(), torch.tensor(mass, device="cuda"),
                             torch.tensor(width, device="cuda"), dout)
        assert L.sync() == pwa.PWA_OK
    o = dout.cpu().numpy()
    assert o[0] == nll
    assert np.array_equal(o[1:25].view(np.complex128), gV)
    assert np.array_equal(o[25:28], gM) and np.array_equal(o[28:31], gW)
