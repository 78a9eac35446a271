"""Pins of the FP64 oracle to things other than itself.

Each test checks the oracle against what Eq. 1-3 and the mathematics fix:
brute force on tiny inputs, closed forms, invariants, finite differences and
truth recovery from accept-reject toys. A plausible slip in the oracle (a
dropped conjugate, a transposed M, a sign, the N_gen vs N_acc divisor, a
missing term of the table form) fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, optimize

import oracle
import synth
from oracle import brute


def small_sample(n_data=30, n_mc=40, n_waves=4, seed=3):
    waves = synth.waves_small()[:n_waves]
    rng = np.random.Generator(np.random.Philox(seed))
    ev = synth.phase_space(n_data, rng)
    ev_mc = synth.phase_space(n_mc, rng)
    A = synth.amplitudes(ev, waves, np.complex128)
    A_mc = synth.amplitudes(ev_mc, waves, np.complex128)
    V = synth.random_V(n_waves, seed + 1)
    return A, A_mc, V


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---- P1: brute force ------------------------------------------------------

@pytest.mark.parametrize("n_waves", [1, 2, 4])
def test_brute_force_nll_and_norm(n_waves):
    A, A_mc, V = small_sample(n_waves=n_waves)
    n_gen = 57.0
    M = oracle.norm_matrix(A_mc, n_gen)
    Mb = np.array(brute.norm_matrix(A_mc.tolist(), n_gen, n_waves))
    assert rel(M, Mb) < 1e-13
    nll, g, bad = oracle.nll_amp(A, M, V)
    assert bad == 0
    nb = brute.nll(A.tolist(), A_mc.tolist(), n_gen, list(V))
    assert abs(nll - nb) <= 1e-12 * abs(nb)
    gb = np.array(brute.grad_closed(A.tolist(), A_mc.tolist(), n_gen, list(V)))
    assert rel(g, gb) < 1e-12


def test_brute_force_gradient_by_differences():
    """The Wirtinger gradient against central differences of the literal
    double sum of Eq. 3."""
    A, A_mc, V = small_sample(n_waves=3, n_data=12, n_mc=15)
    n_gen = 20.0
    M = oracle.norm_matrix(A_mc, n_gen)
    _, g, _ = oracle.nll_amp(A, M, V)
    gfd = np.array(brute.wirtinger_grad(A.tolist(), A_mc.tolist(), n_gen, list(V)))
    assert rel(g, gfd) < 1e-6


# ---- P2 and the degenerate cases of C8 ---------------------------------------

def test_intensity_nonnegative_and_zero_V():
    A, A_mc, V = small_sample()
    I = oracle.intensity(A, V)
    assert np.all(I >= 0)
    M = oracle.norm_matrix(A_mc, 50.0)
    nll, g, bad = oracle.nll_amp(A, M, np.zeros_like(V))
    assert bad == 1 and math.isinf(nll) and np.all(g == 0)


def test_single_wave_closed_form():
    """N = 1: -ln L = -sum ln(|V|^2 |A_i|^2) + |V|^2 (1/N_gen) sum |A_j|^2."""
    A, A_mc, V = small_sample(n_waves=1)
    n_gen = 77.0
    M = oracle.norm_matrix(A_mc, n_gen)
    nll, g, _ = oracle.nll_amp(A, M, V)
    v2 = abs(V[0]) ** 2
    want = -np.sum(np.log(v2 * np.abs(A[:, 0]) ** 2)) + v2 * np.sum(np.abs(A_mc[:, 0]) ** 2) / n_gen
    assert abs(nll - want) < 1e-12 * abs(want)
    # dNLL/dV* = -N_d / conj(V) + V * M
    gw = -len(A) / np.conj(V[0]) + V[0] * M[0, 0]
    assert abs(g[0] - gw) < 1e-12 * abs(len(A) / V[0])


# ---- P3: table form equals amplitude form -------------------------------------

@pytest.mark.parametrize("n_waves", [1, 3, 4])
def test_table_equals_amplitude(n_waves):
    A, A_mc, V = small_sample(n_data=200, n_waves=n_waves)
    M = oracle.norm_matrix(A_mc, 80.0)
    T = oracle.table(A)
    assert T.shape == (200, n_waves * n_waves)
    # diagonal entries are |A_a|^2
    assert rel(T[:, :n_waves], np.abs(A) ** 2) < 1e-15
    na, ga, _ = oracle.nll_amp(A, M, V)
    nt, gt, _ = oracle.nll_table(T, M, V)
    assert abs(na - nt) < 1e-12 * abs(na)
    assert rel(gt, ga) < 1e-12


# ---- P4: V^H M V = (1/N_gen) sum_j I_j --------------------------------------

def test_norm_term_matches_direct_mc_sum():
    waves = synth.waves_small()
    ev, n_gen = synth.mc_sample(3000, seed=11)
    A_mc = synth.amplitudes(ev, waves, np.complex128)
    V = synth.random_V(4, 5)
    M = oracle.norm_matrix(A_mc, n_gen)
    # M is Hermitian with genuinely complex off-diagonals, so a transposed
    # convention would change V^H M V
    assert np.allclose(M, M.conj().T, rtol=0, atol=1e-15 * np.abs(M).max())
    assert np.abs(M.imag).max() > 1e-3 * np.abs(M).max()
    nv, mv = oracle.norm_term(M, V)
    direct = np.sum(oracle.intensity(A_mc, V)) / n_gen
    assert abs(nv - direct) < 1e-12 * direct
    nv_t = np.real(np.conj(V) @ M.T @ V)
    assert abs(nv_t - direct) > 1e-6 * direct


# ---- P5: global phase --------------------------------------------------------

def test_global_phase_invariance():
    A, A_mc, V = small_sample(n_data=300)
    M = oracle.norm_matrix(A_mc, 60.0)
    n0, g0, _ = oracle.nll_amp(A, M, V)
    for phi in (0.3, 2.0, -2.9):
        n1, g1, _ = oracle.nll_amp(A, M, V * np.exp(1j * phi))
        assert abs(n1 - n0) < 1e-12 * abs(n0)
        assert rel(g1, g0 * np.exp(1j * phi)) < 1e-12


# ---- P6: Euler identity and the scale profile (Eq. 2 vs Eq. 3) --------------

def test_euler_identity_and_scale_profile():
    A, A_mc, V = small_sample(n_data=400, n_mc=500)
    n_gen = 700.0
    M = oracle.norm_matrix(A_mc, n_gen)
    nll, g, _ = oracle.nll_amp(A, M, V)
    nv, _ = oracle.norm_term(M, V)
    vg = np.vdot(V, g)                      # sum_a conj(V_a) g_a
    assert abs(vg.real - (nv - len(A))) < 1e-10 * len(A)
    assert abs(vg.imag) < 1e-10 * len(A)
    # min over a real scale s of NLL(s V) = -sum ln I(V) + N ln N(V) - N ln N + N
    Nd = len(A)
    f = lambda s: oracle.nll_amp(A, M, s * V, grad=False)[0]
    s0 = math.sqrt(Nd / nv)
    res = optimize.minimize_scalar(f, bracket=(0.3 * s0, 1.1 * s0, 3.0 * s0), tol=1e-12)
    lnI = np.log(oracle.intensity(A, V)).sum()
    want = -lnI + Nd * math.log(nv) - Nd * math.log(Nd) + Nd
    assert abs(res.fun - want) < 1e-9 * abs(want)
    assert abs(res.x ** 2 - Nd / nv) < 1e-5


# ---- P8: closed-form normalisation for orthonormal toys ------------------------

def _cos_coupling(la, ma, lb, mb):
    """int cos(theta) conj(Y_la^ma) Y_lb^mb dOmega."""
    if ma != mb:
        return 0.0
    m = ma
    if lb == la + 1:
        l = la
    elif lb == la - 1:
        l = lb
    else:
        return 0.0
    return math.sqrt(((l + 1) ** 2 - m * m) / ((2 * l + 1) * (2 * l + 3)))


def _mc_closed_form_check(waves, amp_fn, n_acc, closed):
    ev, n_gen = synth.mc_sample(n_acc, seed=99)
    A = amp_fn(ev)
    M = oracle.norm_matrix(A, n_gen)
    # five standard deviations of the MC estimate: sqrt(sum_j |conj(A_a) A_b|^2) / N_gen
    A2 = np.abs(A) ** 2
    tol = 5 * np.sqrt(A2.T @ A2) / n_gen
    assert np.all(np.abs(M - closed) <= tol), (np.abs(M - closed) / tol).max()
    return M


def test_norm_closed_form_spherical_harmonics():
    """A_a = Y_a only: M = [0.6 delta + 0.3 C] / (4 pi), C the cos(theta)
    coupling of neighbouring l at equal m."""
    lm = [(0, 0), (1, 0), (1, 1), (2, 1), (2, 0), (3, 0)]
    waves = [synth.Wave(1.0, 1.0, l, m) for l, m in lm]
    closed = np.array([[0.6 * (a == b) + 0.3 * _cos_coupling(*lm[a], *lm[b])
                        for b in range(len(lm))] for a in range(len(lm))]) / (4 * math.pi)
    M = _mc_closed_form_check(waves, lambda ev: synth.angular(ev, waves, np.complex128),
                              400_000, closed)
    # the coupling term is present (it is ~0.3/(4 pi)/sqrt(3) for (0,0)-(1,0))
    assert abs(M[0, 1] - closed[0, 1]) < 0.1 * abs(closed[0, 1])


def test_norm_closed_form_breit_wigner():
    """A_a = BW_a(m) Y_a: M_ab = <conj(BW_a) BW_b>_m * <eps conj(Y_a) Y_b>_Omega.
    The imaginary part of the mass integral fixes which index carries the
    conjugate."""
    waves = [synth.Wave(1.3, 0.2, 0, 0), synth.Wave(1.5, 0.3, 1, 0), synth.Wave(2.2, 0.4, 2, 0)]
    lm = [(w.l, w.m) for w in waves]
    dm = synth.M_HI - synth.M_LO

    def mass_int(a, b):
        f = lambda m: np.conj(synth.breit_wigner(m, waves[a].mass, waves[a].width)) * \
            synth.breit_wigner(m, waves[b].mass, waves[b].width)
        re = integrate.quad(lambda m: f(m).real, synth.M_LO, synth.M_HI, limit=400)[0]
        im = integrate.quad(lambda m: f(m).imag, synth.M_LO, synth.M_HI, limit=400)[0]
        return (re + 1j * im) / dm

    closed = np.array([[mass_int(a, b) * (0.6 * (a == b) + 0.3 * _cos_coupling(*lm[a], *lm[b]))
                        / (4 * math.pi) for b in range(3)] for a in range(3)])
    assert abs(closed[0, 1].imag) > 0.2 * abs(closed[0, 1])
    _mc_closed_form_check(waves, lambda ev: synth.amplitudes(ev, waves, np.complex128),
                          400_000, closed)


# ---- P9: finite differences ----------------------------------------------------

def test_gradient_central_differences():
    A, A_mc, V = small_sample(n_data=500, n_mc=600)
    M = oracle.norm_matrix(A_mc, 900.0)
    _, g, _ = oracle.nll_amp(A, M, V)
    gdata = g - oracle.norm_term(M, V)[1]
    h = 1e-4
    gfd = np.empty_like(g)
    for a in range(len(V)):
        d = []
        for step in (h, 1j * h):
            vp, vm = V.copy(), V.copy()
            vp[a] += step
            vm[a] -= step
            d.append((oracle.nll_amp(A, M, vp, False)[0] - oracle.nll_amp(A, M, vm, False)[0]) / (2 * h))
        gfd[a] = complex(d[0], d[1]) / 2
    assert np.max(np.abs(gfd - g)) < 1e-6 * np.linalg.norm(gdata)


def _res_sample(R=2, F=2, n=300, n_mc=400, seed=8):
    waves = synth.waves_linear(R + F, 1.2, 2.4, 0.1, 0.3)
    rng = np.random.Generator(np.random.Philox(seed))
    ev, ev_mc = synth.phase_space(n, rng), synth.phase_space(n_mc, rng)
    Y = synth.angular(ev, waves[:R], np.complex128)
    Ym = synth.angular(ev_mc, waves[:R], np.complex128)
    Af = synth.amplitudes(ev, waves[R:], np.complex128)
    Afm = synth.amplitudes(ev_mc, waves[R:], np.complex128)
    mass = np.array([w.mass for w in waves[:R]])
    width = np.array([w.width for w in waves[:R]])
    V = synth.random_V(R + F, seed)
    return waves, ev, ev_mc, Y, Ym, Af, Afm, mass, width, V


def test_free_resonance_matches_fixed_form_and_differences():
    waves, ev, ev_mc, Y, Ym, Af, Afm, mass, width, V = _res_sample()
    n_gen = 650.0
    args = (ev["m"], Y, Af, ev_mc["m"], Ym, Afm, n_gen)
    nll, gV, gM, gW, bad = oracle.nll_res(*args, V, mass, width)
    assert bad == 0
    # at the same masses and widths it is the fixed-parameter NLL
    A = synth.amplitudes(ev, waves, np.complex128)
    A_mc = synth.amplitudes(ev_mc, waves, np.complex128)
    M = oracle.norm_matrix(A_mc, n_gen)
    n2, g2, _ = oracle.nll_amp(A, M, V)
    assert abs(nll - n2) < 1e-11 * abs(n2)
    assert rel(gV, g2) < 1e-10
    # dNLL/dmass, dNLL/dwidth by central differences (P12: BW derivatives)
    h = 1e-6
    for r in range(len(mass)):
        for par, gpar in ((mass, gM), (width, gW)):
            p1, p2 = par.copy(), par.copy()
            p1[r] += h
            p2[r] -= h
            if par is mass:
                fp = oracle.nll_res(*args, V, p1, width)[0]
                fm = oracle.nll_res(*args, V, p2, width)[0]
            else:
                fp = oracle.nll_res(*args, V, mass, p1)[0]
                fm = oracle.nll_res(*args, V, mass, p2)[0]
            fd = (fp - fm) / (2 * h)
            assert abs(fd - gpar[r]) < 1e-5 * max(1.0, abs(gpar[r])), (r, fd, gpar[r])


# ---- P10 / P7: truth recovery from an accept-reject toy ----------------------

def _phase_fix(V):
    return V * np.exp(-1j * np.angle(V[0]))


def _fit(A, M, V0):
    N = len(V0)

    def f(x):
        V = x[:N] + 1j * x[N:]
        nll, g, bad = oracle.nll_amp(A, M, V)
        if bad:
            return 1e300, np.zeros(2 * N)
        return nll, np.concatenate([2 * g.real, 2 * g.imag])

    x0 = np.concatenate([V0.real, V0.imag])
    r = optimize.minimize(f, x0, jac=True, method="L-BFGS-B",
                          options={"maxiter": 2000, "ftol": 1e-15, "gtol": 1e-8})
    return r.x[:N] + 1j * r.x[N:], r


@pytest.mark.slow
def test_truth_recovery_accept_reject():
    """Data drawn from eps * I with the small 4-wave model; the fit returns
    V_true within its statistical errors and N(V_hat) = N_data."""
    waves = synth.waves_small()
    V_true = synth.random_V(4, synth.SEED_VTRUE)
    ymax = [math.sqrt((2 * w.l + 1) / (4 * math.pi)) for w in waves]
    bwmax = [1.0 / (w.mass * w.width) for w in waves]
    envelope = synth.EFF_MAX * sum(abs(v) * b * y for v, b, y in zip(V_true, bwmax, ymax)) ** 2

    def density(ev):
        A = synth.amplitudes(ev, waves, np.complex128)
        return synth.efficiency(ev["costh"]) * oracle.intensity(A, V_true)

    n_data = 10_000
    ev = synth.accept_reject(n_data, density, envelope, seed=synth.SEED_DATA)
    A = synth.amplitudes(ev, waves, np.complex128)
    ev_mc, n_gen = synth.mc_sample(30_000, seed=synth.SEED_MC)   # about 50k generated
    A_mc = synth.amplitudes(ev_mc, waves, np.complex128)
    M = oracle.norm_matrix(A_mc, n_gen)
    # the truth up to the overall scale, which the extended likelihood fixes
    V0 = V_true * math.sqrt(n_data / oracle.norm_term(M, V_true)[0])
    Vh, res = _fit(A, M, V0 * (1 + 0.2j))
    nv, _ = oracle.norm_term(M, Vh)
    assert abs(nv - n_data) < 1e-3 * n_data                       # P7
    assert res.fun <= oracle.nll_amp(A, M, V0, False)[0] + 1e-9
    # pulls from the inverse Hessian of the phase-fixed real parameters
    Vf, Tf = _phase_fix(Vh), _phase_fix(V0)
    N = 4
    x = np.concatenate([Vf.real, Vf.imag[1:]])

    def grad_x(xx):
        V = xx[:N] + 1j * np.concatenate([[0.0], xx[N:]])
        _, g, _ = oracle.nll_amp(A, M, V)
        return np.concatenate([2 * g.real, 2 * g.imag[1:]])

    H = np.empty((2 * N - 1, 2 * N - 1))
    for k in range(2 * N - 1):
        e = np.zeros(2 * N - 1)
        e[k] = 1e-5
        H[:, k] = (grad_x(x + e) - grad_x(x - e)) / 2e-5
    cov = np.linalg.inv(0.5 * (H + H.T))
    t = np.concatenate([Tf.real, Tf.imag[1:]])
    pulls = (x - t) / np.sqrt(np.diag(cov))
    assert np.all(np.abs(pulls) < 5), pulls


def test_blas_norm_matrix_matches_loops():
    """The chunked library-matmul M used for large samples equals the plain loops."""
    wl = synth.mixture_workload("t", synth.waves_linear(7), 10, 50_000)
    M = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    Mb = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen, chunk=7000)
    assert rel(Mb, M) < 1e-13


# ---- FUMILI Hessian, projection weights, fit fractions -----------------------

def _real_grad(A, M, V):
    """dNLL/d(Re V, Im V) from the oracle's Wirtinger gradient g: (2 Re g, 2 Im g)."""
    _, g, _ = oracle.nll_amp(A, M, V)
    return np.concatenate([2 * g.real, 2 * g.imag])


def _hess_case(N=3, n=40, n_mc=60, seed=3):
    rng = np.random.Generator(np.random.Philox(seed))
    A = rng.standard_normal((n, N)) + 1j * rng.standard_normal((n, N))
    Am = rng.standard_normal((n_mc, N)) + 1j * rng.standard_normal((n_mc, N))
    M = oracle.norm_matrix(Am, 1.7 * n_mc)
    V = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return A, M, V


def test_hessian_brute_force():
    A, M, V = _hess_case()
    N = A.shape[1]
    H, bad = oracle.hessian(A, V)
    assert bad == 0
    Hb = np.zeros((2 * N, 2 * N))
    for i in range(A.shape[0]):
        S = sum(V[a] * A[i, a] for a in range(N))
        I = abs(S) ** 2
        d = [2 * (np.conj(A[i, a]) * S).real / I for a in range(N)] + \
            [2 * (np.conj(A[i, a]) * S).imag / I for a in range(N)]
        for x in range(2 * N):
            for y in range(2 * N):
                Hb[x, y] += d[x] * d[y]
    assert np.max(np.abs(H - Hb)) <= 1e-12 * np.max(np.abs(Hb))


def test_hessian_homogeneity_and_phase_null_vector():
    """I is homogeneous of degree 2 in p = (Re V, Im V): p . grad ln I_i = 2, so
    H p = 2 sum_i d_i = -2 grad(data NLL) = -2 grad NLL + 2 grad N. And I is
    invariant under a global phase, so grad ln I_i . (J p) = 0 with
    J p = (-Im V, Re V): the phase direction is a null vector of H."""
    A, M, V = _hess_case(N=4, seed=5)
    H, _ = oracle.hessian(A, V)
    p = np.concatenate([V.real, V.imag])
    _, mv = oracle.norm_term(M, V)
    gN = np.concatenate([2 * mv.real, 2 * mv.imag])
    rhs = -2 * _real_grad(A, M, V) + 2 * gN
    assert np.max(np.abs(H @ p - rhs)) <= 1e-10 * np.max(np.abs(rhs))
    Jp = np.concatenate([-V.imag, V.real])
    assert np.max(np.abs(H @ Jp)) <= 1e-12 * np.max(np.abs(H)) * np.max(np.abs(Jp))


def test_hessian_vs_exact_second_derivative():
    """The exact NLL Hessian (central differences of the pinned gradient) is
    H - sum_i d^2 I_i / I_i + d^2(V^H M V), with d^2 I = 2 [[Re C, -Im C],
    [Im C, Re C]] for C_ab = conj(A_a) A_b and d^2(V^H M V) the same form
    of M; checks what H drops and the parameter ordering."""
    A, M, V = _hess_case(N=3, n=30, seed=9)
    N = A.shape[1]
    H, _ = oracle.hessian(A, V)
    p0 = np.concatenate([V.real, V.imag])
    h = 1e-5
    He = np.zeros((2 * N, 2 * N))
    for k in range(2 * N):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        gp = _real_grad(A, M, pp[:N] + 1j * pp[N:])
        gm = _real_grad(A, M, pm[:N] + 1j * pm[N:])
        He[:, k] = (gp - gm) / (2 * h)
    I = oracle.intensity(A, V)
    C = np.einsum("ia,ib->ab", np.conj(A) / I[:, None], A)
    blk = lambda X: np.block([[2 * X.real, -2 * X.imag], [2 * X.imag, 2 * X.real]])
    assert np.max(np.abs(He - (H - blk(C) + blk(M)))) <= 1e-6 * np.max(np.abs(He))


def test_hessian_expectation_at_truth():
    """At the true V of a sample drawn from eps * I, the dropped terms cancel
    in expectation (E sum_i d^2 I_i / I_i = d^2 N), so H approximates the
    exact Hessian; with d^2 N kept as well it would be about twice too large.
    Four-wave accept-reject toy, 20k events: agreement to ~10%."""
    waves = synth.waves_small()
    V_true = synth.random_V(4, synth.SEED_VTRUE)
    ymax = [math.sqrt((2 * w.l + 1) / (4 * math.pi)) for w in waves]
    env = synth.EFF_MAX * sum(abs(v) / (w.mass * w.width) * y
                              for v, w, y in zip(V_true, waves, ymax)) ** 2

    def density(ev):
        return synth.efficiency(ev["costh"]) * oracle.intensity(
            synth.amplitudes(ev, waves, np.complex128), V_true)

    ev = synth.accept_reject(20_000, density, env, seed=77)
    ev_mc, n_gen = synth.mc_sample(60_000, seed=78)
    A = synth.amplitudes(ev, waves, np.complex128)
    M = oracle.norm_matrix(synth.amplitudes(ev_mc, waves, np.complex128), n_gen)
    V = V_true * math.sqrt(len(A) / oracle.norm_term(M, V_true)[0])
    H, _ = oracle.hessian(A, V)
    I = oracle.intensity(A, V)
    C = np.einsum("ia,ib->ab", np.conj(A) / I[:, None], A)
    blk = lambda X: np.block([[2 * X.real, -2 * X.imag], [2 * X.imag, 2 * X.real]])
    He = H - blk(C) + blk(M)
    assert np.linalg.norm(H - He) <= 0.1 * np.linalg.norm(He)
    assert np.linalg.norm(H + blk(M) - He) >= 0.5 * np.linalg.norm(He)


def test_mc_weights_and_fit_fractions():
    A, M, V = _hess_case(N=5, seed=11)
    rng = np.random.Generator(np.random.Philox(12))
    Am = rng.standard_normal((200, 5)) + 1j * rng.standard_normal((200, 5))
    n_gen = 333.0
    Mm = oracle.norm_matrix(Am, n_gen)
    w = oracle.mc_weights(Am, V, n_gen)
    assert np.allclose(w, np.abs(Am @ V) ** 2 / n_gen, rtol=1e-13, atol=0)
    nv, _ = oracle.norm_term(Mm, V)
    assert abs(w.sum() - nv) <= 1e-12 * nv               # sum of weights = V^H M V
    F = oracle.fit_fractions(Mm, V)
    assert abs(F.sum() - 1.0) <= 1e-12                    # fractions + interference = 1
    for a in range(5):
        assert abs(F[a, a] - abs(V[a]) ** 2 * Mm[a, a].real / nv) <= 1e-13
    # every entry from the events themselves (no M): the MC average of the
    # interference of waves a and b, Re(conj(V_a A_a) V_b A_b) / N_gen
    # (F is symmetric: F_ab + F_ba is the pair's interference fraction)
    VA = Am * V[None, :]
    for a in range(5):
        for b in range(5):
            Fb = np.sum((np.conj(VA[:, a]) * VA[:, b]).real) / n_gen / nv
            assert abs(F[a, b] - Fb) <= 1e-12, (a, b)


# ---- incoherent sums over unobserved components --------------------------------

def incoh_sample(n_data=20, n_mc=30, n_waves=3, L=2, seed=5):
    waves = synth.waves_small()[:n_waves]
    rng = np.random.Generator(np.random.Philox(seed))
    A = synth.helicity_amplitudes(synth.phase_space(n_data, rng), waves, L, np.complex128)
    A_mc = synth.helicity_amplitudes(synth.phase_space(n_mc, rng), waves, L, np.complex128)
    return A, A_mc, synth.random_V(n_waves, seed + 1)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_incoherent_brute_force(L):
    """NLL and gradient against the literal double sums with the products
    summed over components, and the gradient against their differences."""
    A, A_mc, V = incoh_sample(L=L)
    n_gen = 47.0
    M = oracle.norm_matrix_incoh(A_mc, n_gen)
    nll, g, bad = oracle.nll_incoh(A, M, V)
    assert bad == 0
    nb = brute.nll_incoh(A.tolist(), A_mc.tolist(), n_gen, list(V))
    assert abs(nll - nb) <= 1e-12 * abs(nb)
    gfd = np.array(brute.wirtinger_grad_incoh(A.tolist(), A_mc.tolist(), n_gen, list(V)))
    assert rel(g, gfd) < 1e-6


def test_incoherent_one_component_is_coherent():
    A, A_mc, V = incoh_sample(n_data=50, n_mc=60, n_waves=4, L=1)
    M = oracle.norm_matrix_incoh(A_mc, 90.0)
    assert rel(M, oracle.norm_matrix(A_mc[:, 0, :], 90.0)) < 1e-15
    n1, g1, _ = oracle.nll_incoh(A, M, V)
    n0, g0, _ = oracle.nll_amp(A[:, 0, :], M, V)
    assert abs(n1 - n0) <= 1e-14 * abs(n0) and rel(g1, g0) < 1e-14


def test_incoherent_scaled_copies_closed_form():
    """Components that are copies A^l = c_l A of one amplitude set give
    I = (sum_l |c_l|^2) |S|^2 and M = (sum_l |c_l|^2) M_coherent, so
    NLL = NLL_coherent(A, c2 M) - n ln c2 with c2 = sum_l |c_l|^2."""
    A, A_mc, V = incoh_sample(n_data=40, n_mc=50, n_waves=4, L=1)
    c = np.array([0.7 + 0.2j, -0.3 + 1.1j, 0.5j])
    c2 = float(np.sum(np.abs(c) ** 2))
    Ai = A[:, 0, None, :] * c[None, :, None]
    Ai_mc = A_mc[:, 0, None, :] * c[None, :, None]
    M = oracle.norm_matrix_incoh(Ai_mc, 80.0)
    M0 = oracle.norm_matrix(A_mc[:, 0, :], 80.0)
    assert rel(M, c2 * M0) < 1e-14
    n, g, _ = oracle.nll_incoh(Ai, M, V)
    n0, g0, _ = oracle.nll_amp(A[:, 0, :], c2 * M0, V)
    assert abs(n - (n0 - len(A) * math.log(c2))) <= 1e-13 * abs(n)
    # the data gradient is unchanged by the common factor, the MC part scales with it
    assert rel(g, g0) < 1e-13


def test_incoherent_component_phases_and_table_form():
    """A phase per component leaves the incoherent sum unchanged (a coherent
    sum over components would not be), and the table form with the products
    summed over components gives the same NLL and gradient."""
    A, A_mc, V = incoh_sample(n_data=60, n_mc=70, n_waves=4, L=3)
    M = oracle.norm_matrix_incoh(A_mc, 100.0)
    n, g, _ = oracle.nll_incoh(A, M, V)
    ph = np.exp(1j * np.array([0.4, -2.1, 1.3]))
    n2, g2, _ = oracle.nll_incoh(A * ph[None, :, None], oracle.norm_matrix_incoh(
        A_mc * ph[None, :, None], 100.0), V)
    assert abs(n2 - n) <= 1e-13 * abs(n) and rel(g2, g) < 1e-12
    coh = lambda X: oracle.intensity(X.sum(axis=1), V)
    assert rel(coh(A * ph[None, :, None]), coh(A)) > 1e-3
    nt, gt, _ = oracle.nll_table(oracle.table_incoh(A), M, V)
    assert abs(nt - n) <= 1e-13 * abs(n) and rel(gt, g) < 1e-12


def test_incoherent_euler_identity_and_phase():
    A, A_mc, V = incoh_sample(n_data=200, n_mc=300, n_waves=4, L=2)
    M = oracle.norm_matrix_incoh(A_mc, 400.0)
    n, g, _ = oracle.nll_incoh(A, M, V)
    nv, _ = oracle.norm_term(M, V)
    vg = np.vdot(V, g)
    assert abs(vg.real - (nv - len(A))) < 1e-10 * len(A) and abs(vg.imag) < 1e-10 * len(A)
    n2, g2, _ = oracle.nll_incoh(A, M, V * np.exp(0.8j))
    assert abs(n2 - n) < 1e-12 * abs(n) and rel(g2, g * np.exp(0.8j)) < 1e-12


# ---- the amplitude model: Breit-Wigner x spherical harmonic ---------------------

def _grid(n=200, seed=21):
    rng = np.random.Generator(np.random.Philox(seed))
    return (rng.uniform(0.98, 3.0, n), rng.uniform(-1.0, 1.0, n), rng.uniform(0.0, 2 * math.pi, n))


def test_amplitude_closed_forms():
    """Y_0^0, Y_1^{0,1,-1}, Y_2^{0,1,2} and Y_3^3 written out, times the
    Breit-Wigner 1 / (M^2 - m^2 - i M G)."""
    m, c, p = _grid()
    s = np.sqrt(1 - c * c)
    e = np.exp(1j * p)
    pi = math.pi
    closed = {
        (0, 0): np.full_like(c, 1 / math.sqrt(4 * pi)) + 0j,
        (1, 0): math.sqrt(3 / (4 * pi)) * c + 0j,
        (1, 1): -math.sqrt(3 / (8 * pi)) * s * e,
        (1, -1): math.sqrt(3 / (8 * pi)) * s / e,
        (2, 0): math.sqrt(5 / (16 * pi)) * (3 * c * c - 1) + 0j,
        (2, 1): -math.sqrt(15 / (8 * pi)) * s * c * e,
        (2, 2): math.sqrt(15 / (32 * pi)) * s * s * e ** 2,
        (3, 3): -math.sqrt(35 / (64 * pi)) * s ** 3 * e ** 3,
    }
    waves = [(1.3, 0.2, l, mm) for (l, mm) in closed]
    A = oracle.amplitudes(m, c, p, waves)
    bw = 1.0 / (1.3 ** 2 - m ** 2 - 1j * 1.3 * 0.2)
    for k, key in enumerate(closed):
        assert np.max(np.abs(A[:, k] - bw * closed[key])) <= 1e-13 * np.max(np.abs(A[:, k])), key


def test_amplitude_library_and_identities():
    """Against scipy's spherical harmonics (Condon-Shortley phase) up to l = 6,
    the conjugation rule Y_l^{-m} = (-1)^m conj(Y_l^m), the addition theorem
    sum_m |Y_l^m|^2 = (2l + 1)/(4 pi), and |BW|^2 = 1/(M G)^2 at m = M."""
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    m, c, p = _grid(100, seed=22)
    theta = np.arccos(c)
    for l in range(7):
        waves = [(2.0, 0.3, l, mm) for mm in range(-l, l + 1)]
        A = oracle.amplitudes(np.full_like(m, 2.0), c, p, waves)
        Y = A * (-1j * 2.0 * 0.3)       # BW(M; M, G) = 1 / (-i M G) = i / (M G)
        for k, mm in enumerate(range(-l, l + 1)):
            ref = special.sph_harm_y(l, mm, theta, p)
            assert np.max(np.abs(Y[:, k] - ref)) <= 1e-12, (l, mm)
            assert np.max(np.abs(Y[:, l - mm] - (-1) ** mm * np.conj(Y[:, k]))) <= 1e-14
        assert np.max(np.abs((np.abs(Y) ** 2).sum(axis=1) - (2 * l + 1) / (4 * math.pi))) <= 1e-12
    A = oracle.amplitudes([1.7], [0.3], [0.4], [(1.7, 0.11, 0, 0)])
    assert abs(abs(A[0, 0]) ** 2 * 4 * math.pi - 1 / (1.7 * 0.11) ** 2) <= 1e-12 / (1.7 * 0.11) ** 2


def test_amplitude_orthonormality_by_quadrature():
    """int conj(Y_l^m) Y_l'^m' dOmega = delta_ll' delta_mm' (Gauss-Legendre in
    cos theta, uniform in phi; exact for these degrees)."""
    x, wx = np.polynomial.legendre.leggauss(12)
    nphi = 16
    ph = 2 * math.pi * np.arange(nphi) / nphi
    C, P = np.meshgrid(x, ph, indexing="ij")
    W = (wx[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).ravel()
    keys = [(l, mm) for l in range(5) for mm in range(-l, l + 1)]
    waves = [(2.0, 0.3, l, mm) for (l, mm) in keys]
    Y = oracle.amplitudes(np.full(C.size, 2.0), C.ravel(), P.ravel(), waves) * (1j * 0.6)
    G = (np.conj(Y) * W[:, None]).T @ Y
    assert np.max(np.abs(G - np.eye(len(keys)))) <= 1e-12


def test_amplitudes_match_the_sample_generator():
    """The oracle's model and the seeded sample generator agree in FP64 (the
    generator is what every other test feeds both sides)."""
    m, c, p = _grid(300, seed=23)
    waves = synth.waves_linear(13)
    A = oracle.amplitudes(m, c, p, waves)
    As = synth.amplitudes({"m": m, "costh": c, "phi": p}, waves, np.complex128)
    assert np.max(np.abs(A - As)) <= 1e-13 * np.max(np.abs(As))
