"""Seeded synthetic inputs for the partial wave analysis likelihood.

This module only draws events and evaluates the physics amplitude model
(Breit-Wigner line shape x spherical harmonic) that both the oracle and the
CUDA path consume. It holds none of the likelihood's arithmetic: it never
forms a coherent sum over waves, an intensity, a logarithm or a normalisation
integral.

Phase space follows the radiative decay J/psi -> gamma X, X -> K+ K- used as
the example of Sec. 2: each event is (m_KK, cos theta, phi) with m_KK uniform
in [0.98, 3.0] GeV, cos theta uniform in [-1, 1] and phi uniform in [0, 2 pi).
The detector efficiency is eps = 0.6 + 0.3 cos theta; accepted Monte Carlo is
drawn by keeping a uniformly generated candidate with probability eps, and the
number of candidates drawn is N_MC^Gen (Sec. 2, the text after Eq. 2).

Amplitudes: A_alpha(Omega) = BW(m; M_alpha, Gamma_alpha) * Y_{l_alpha}^{m_alpha}
(cos theta, phi) with the fixed-width Breit-Wigner 1 / (M^2 - m^2 - i M Gamma)
and orthonormal spherical harmonics carrying the Condon-Shortley phase.

Incoherent components (an unobserved helicity, e.g. of the radiated photon):
component l of wave alpha uses the magnetic number
mu = clip(m_alpha + h_l, -l_alpha, l_alpha) with h = (+1, -1, 0, +2, -2)[l],
A_alpha^l(Omega) = BW(m; M_alpha, Gamma_alpha) * Y_{l_alpha}^{mu}(cos theta, phi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

M_LO, M_HI = 0.98, 3.0
EFF_MAX = 0.9

SEED_DATA = 1108
SEED_MC = 5673
SEED_VTRUE = 42
SEED_STARTS = 7


@dataclass(frozen=True)
class Wave:
    mass: float
    width: float
    l: int
    m: int


def efficiency(costh):
    """Detector efficiency eps(Omega) = 0.6 + 0.3 cos theta (always in [0.3, 0.9])."""
    return 0.6 + 0.3 * np.asarray(costh)


def waves_small():
    """Four waves: (M, Gamma) = (1.5, 0.1), (1.7, 0.15), (2.0, 0.2), (2.3, 0.25) GeV,
    (l, m) = (0,0), (2,0), (2,1), (4,0)."""
    return [Wave(1.5, 0.10, 0, 0), Wave(1.7, 0.15, 2, 0),
            Wave(2.0, 0.20, 2, 1), Wave(2.3, 0.25, 4, 0)]


def waves_linear(n, m_lo=1.0, m_hi=2.9, w_lo=0.05, w_hi=0.4):
    """n waves with masses and widths linearly spaced over the given ranges,
    l = (0, 2, 4)[alpha mod 3] and m = 0 for l = 0, else floor(alpha/3) mod (l+1)."""
    if n == 1:
        return [Wave(m_lo, w_lo, 0, 0)]
    out = []
    for a in range(n):
        l = (0, 2, 4)[a % 3]
        mm = 0 if l == 0 else (a // 3) % (l + 1)
        t = a / (n - 1)
        out.append(Wave(m_lo + (m_hi - m_lo) * t, w_lo + (w_hi - w_lo) * t, l, mm))
    return out


def breit_wigner(m, mass, width):
    """Fixed-width Breit-Wigner 1 / (M^2 - m^2 - i M Gamma), complex128."""
    m = np.asarray(m, dtype=np.float64)
    return 1.0 / (mass * mass - m * m - 1j * mass * width)


def _assoc_legendre(l, mm, x):
    """P_l^m(x) for m >= 0 including the Condon-Shortley phase (-1)^m,
    by the standard upward recurrence in l."""
    x = np.asarray(x, dtype=np.float64)
    s = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    fact = 1.0
    for _ in range(mm):
        pmm = -pmm * fact * s
        fact += 2.0
    if l == mm:
        return pmm
    pm1 = x * (2 * mm + 1) * pmm
    if l == mm + 1:
        return pm1
    p2, p1 = pmm, pm1
    for ll in range(mm + 2, l + 1):
        p = ((2 * ll - 1) * x * p1 - (ll + mm - 1) * p2) / (ll - mm)
        p2, p1 = p1, p
    return p1


def ylm(l, mm, costh, phi):
    """Orthonormal spherical harmonic Y_l^m(theta, phi), Condon-Shortley phase."""
    if mm < 0:
        return (-1) ** (-mm) * np.conj(ylm(l, -mm, costh, phi))
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - mm) / math.factorial(l + mm))
    return norm * _assoc_legendre(l, mm, costh) * np.exp(1j * mm * np.asarray(phi, dtype=np.float64))


def phase_space(n, rng):
    """n events uniform in (m_KK, cos theta, phi)."""
    m = rng.uniform(M_LO, M_HI, n)
    c = rng.uniform(-1.0, 1.0, n)
    p = rng.uniform(0.0, 2.0 * math.pi, n)
    return {"m": m, "costh": c, "phi": p}


def _concat(parts, n):
    return {k: np.concatenate([p[k] for p in parts])[:n] for k in parts[0]}


def mc_sample(n_acc, seed=SEED_MC, batch=1 << 20):
    """Accepted Monte Carlo: uniform candidates kept with probability eps.
    Returns (events, n_gen) where n_gen counts every candidate drawn up to and
    including the n_acc-th accepted one."""
    rng = np.random.Generator(np.random.Philox(seed))
    parts, got, n_gen = [], 0, 0
    while got < n_acc:
        ev = phase_space(batch, rng)
        keep = rng.uniform(0.0, 1.0, batch) < efficiency(ev["costh"])
        idx = np.nonzero(keep)[0]
        need = n_acc - got
        if len(idx) >= need:
            n_gen += int(idx[need - 1]) + 1
            idx = idx[:need]
        else:
            n_gen += batch
        parts.append({k: v[idx] for k, v in ev.items()})
        got += len(idx)
    return _concat(parts, n_acc), n_gen


def data_sample_mixture(n, waves, V, seed=SEED_DATA, batch=1 << 20):
    """Data-like events concentrated on the resonances without evaluating the
    likelihood's intensity: pick wave alpha with probability proportional to
    |V_alpha|^2, draw m_KK from a Cauchy of location M_alpha and half-width
    Gamma_alpha/2 truncated to [0.98, 3.0] GeV, cos theta from the efficiency
    shape (accept with eps/0.9) and phi uniform."""
    rng = np.random.Generator(np.random.Philox(seed))
    w = np.abs(np.asarray(V)) ** 2
    w = w / w.sum()
    M = np.array([wv.mass for wv in waves])
    G = np.array([wv.width for wv in waves])
    parts, got = [], 0
    while got < n:
        a = rng.choice(len(waves), size=batch, p=w)
        lo = np.arctan((M_LO - M[a]) / (G[a] / 2)) / math.pi + 0.5
        hi = np.arctan((M_HI - M[a]) / (G[a] / 2)) / math.pi + 0.5
        u = lo + (hi - lo) * rng.uniform(0.0, 1.0, batch)
        m = M[a] + (G[a] / 2) * np.tan(math.pi * (u - 0.5))
        m = np.clip(m, M_LO, M_HI)
        c = rng.uniform(-1.0, 1.0, batch)
        keep = rng.uniform(0.0, 1.0, batch) < efficiency(c) / EFF_MAX
        p = rng.uniform(0.0, 2.0 * math.pi, batch)
        parts.append({"m": m[keep], "costh": c[keep], "phi": p[keep]})
        got += int(keep.sum())
    return _concat(parts, n)


def accept_reject(n, density, envelope, seed, batch=1 << 16):
    """Events drawn from a caller-supplied density over phase space by
    accept-reject against a constant envelope. `density(events)` returns
    non-negative weights; every weight must stay below `envelope` (a weight
    above it raises, since the sample would then be biased)."""
    rng = np.random.Generator(np.random.Philox(seed))
    parts, got = [], 0
    while got < n:
        ev = phase_space(batch, rng)
        d = np.asarray(density(ev), dtype=np.float64)
        if np.any(d > envelope):
            raise ValueError("accept-reject envelope violated: max %g > %g" % (d.max(), envelope))
        keep = rng.uniform(0.0, envelope, batch) < d
        parts.append({k: v[keep] for k, v in ev.items()})
        got += int(keep.sum())
    return _concat(parts, n)


def amplitudes(events, waves, dtype=np.complex64, chunk=1 << 20):
    """Event-major amplitude matrix A[i, alpha] = BW_alpha(m_i) Y_alpha(Omega_i),
    evaluated in float64 and rounded once to `dtype`."""
    n = len(events["m"])
    out = np.empty((n, len(waves)), dtype=dtype)
    for s in range(0, n, chunk):
        e = slice(s, min(n, s + chunk))
        m, c, p = events["m"][e], events["costh"][e], events["phi"][e]
        for a, wv in enumerate(waves):
            out[e, a] = breit_wigner(m, wv.mass, wv.width) * ylm(wv.l, wv.m, c, p)
    return out


def angular(events, waves, dtype=np.complex64):
    """Angular factors Y_alpha(Omega_i) alone, [n, len(waves)]."""
    n = len(events["m"])
    out = np.empty((n, len(waves)), dtype=dtype)
    for a, wv in enumerate(waves):
        out[:, a] = ylm(wv.l, wv.m, events["costh"], events["phi"])
    return out


HELICITIES = (1, -1, 0, 2, -2)


def helicity_amplitudes(events, waves, n_lambda, dtype=np.complex64, chunk=1 << 20):
    """Event-major [n, n_lambda, N] amplitudes of the incoherent components:
    A[i, l, alpha] = BW_alpha(m_i) Y_{l_alpha}^{mu}(Omega_i) with
    mu = clip(m_alpha + h_l, -l_alpha, l_alpha), h = HELICITIES[l]."""
    if not 1 <= n_lambda <= len(HELICITIES):
        raise ValueError("n_lambda must be in [1, %d]" % len(HELICITIES))
    n = len(events["m"])
    out = np.empty((n, n_lambda, len(waves)), dtype=dtype)
    for s in range(0, n, chunk):
        e = slice(s, min(n, s + chunk))
        m, c, p = events["m"][e], events["costh"][e], events["phi"][e]
        for a, wv in enumerate(waves):
            bw = breit_wigner(m, wv.mass, wv.width)
            for lam in range(n_lambda):
                mu = max(-wv.l, min(wv.l, wv.m + HELICITIES[lam]))
                out[e, lam, a] = bw * ylm(wv.l, mu, c, p)
    return out


def random_V(n_waves, seed=SEED_VTRUE, k=None):
    """Production amplitudes with Re and Im drawn N(0, 1): shape [n_waves] or [k, n_waves]."""
    rng = np.random.Generator(np.random.Philox(seed))
    shape = (n_waves,) if k is None else (k, n_waves)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@dataclass
class Workload:
    name: str
    waves: list
    A_data: np.ndarray   # [n_data, N] complex64, event-major
    A_mc: np.ndarray     # [n_mc_acc, N] complex64, event-major
    n_gen: int
    V_true: np.ndarray   # [N] complex128


def mixture_workload(name, waves, n_data, n_mc_acc, seed_data=SEED_DATA, seed_mc=SEED_MC,
                     seed_v=SEED_VTRUE, dtype=np.complex64):
    """A sample of the given sizes: data-like events from `data_sample_mixture`
    with V_true ~ N(0,1) and accepted MC from `mc_sample`."""
    V = random_V(len(waves), seed_v)
    ev_d = data_sample_mixture(n_data, waves, V, seed_data)
    ev_m, n_gen = mc_sample(n_mc_acc, seed_mc)
    return Workload(name, waves, amplitudes(ev_d, waves, dtype), amplitudes(ev_m, waves, dtype),
                    n_gen, V)


def incoherent_workload(name, waves, n_data, n_mc_acc, n_lambda=2, seed_data=SEED_DATA,
                        seed_mc=SEED_MC, seed_v=SEED_VTRUE, dtype=np.complex64):
    """As mixture_workload, with [n, n_lambda, N] amplitudes of incoherent
    components (helicity_amplitudes) for the data and the accepted MC."""
    V = random_V(len(waves), seed_v)
    ev_d = data_sample_mixture(n_data, waves, V, seed_data)
    ev_m, n_gen = mc_sample(n_mc_acc, seed_mc)
    return Workload(name, waves, helicity_amplitudes(ev_d, waves, n_lambda, dtype),
                    helicity_amplitudes(ev_m, waves, n_lambda, dtype), n_gen, V)


def paper_scale(n_data=1_000_000, n_mc_acc=5_000_000, n_waves=20, **kw):
    """The paper-scale single fit: 20 waves, 1M data events, 5M accepted MC."""
    return mixture_workload("pwa_1M_events_20_waves", waves_linear(n_waves), n_data, n_mc_acc, **kw)


def multistart_scale(n_data=4_000_000, n_mc_acc=10_000_000, n_waves=32, **kw):
    """The batched multistart sample: 32 waves, 4M data events, 10M accepted MC."""
    return mixture_workload("pwa_4M_events_32_waves", waves_linear(n_waves), n_data, n_mc_acc, **kw)


def start_points(n_waves, k, seed=SEED_STARTS):
    """K starting parameter sets, Re/Im ~ N(0,1): [k, n_waves] complex128."""
    return random_V(n_waves, seed, k)


@dataclass
class ResonanceWorkload:
    """Samples for fits with free masses and widths of the first n_free waves:
    the mass variable m, the angular factors Y of the free waves and the full
    amplitudes of the fixed ones (float32 / complex64, event-major)."""
    name: str
    waves: list
    n_free: int
    m_data: np.ndarray     # [n_data] float32
    Y_data: np.ndarray     # [n_data, n_free] complex64
    Afix_data: np.ndarray  # [n_data, N - n_free] complex64
    m_mc: np.ndarray
    Y_mc: np.ndarray
    Afix_mc: np.ndarray
    n_gen: int
    V_true: np.ndarray
    mass: np.ndarray       # [n_free] the generated masses
    width: np.ndarray      # [n_free] the generated widths


def resonance_workload(name, waves, n_free, n_data, n_mc_acc, seed_data=SEED_DATA, seed_mc=SEED_MC,
                       seed_v=SEED_VTRUE):
    """Data-like events from `data_sample_mixture` and accepted MC from
    `mc_sample`, split into (m, Y of the free waves, amplitudes of the fixed
    waves); m is rounded to float32."""
    V = random_V(len(waves), seed_v)
    ev_d = data_sample_mixture(n_data, waves, V, seed_data)
    ev_m, n_gen = mc_sample(n_mc_acc, seed_mc)
    free, fixed = waves[:n_free], waves[n_free:]
    return ResonanceWorkload(
        name, waves, n_free,
        ev_d["m"].astype(np.float32), angular(ev_d, free), amplitudes(ev_d, fixed),
        ev_m["m"].astype(np.float32), angular(ev_m, free), amplitudes(ev_m, fixed),
        n_gen, V, np.array([w.mass for w in free]), np.array([w.width for w in free]))


def free_resonance_scale(n_data=2_000_000, n_mc_acc=5_000_000, n_waves=20, n_free=4, **kw):
    """Free masses and widths: 20 waves of which 4 Breit-Wigners are free,
    2M data events, 5M accepted MC."""
    return resonance_workload("pwa_2M_events_20_waves_4_free", waves_linear(n_waves), n_free,
                              n_data, n_mc_acc, **kw)


# ---- the same model, drawn on a GPU (for samples too large for the host) ----
# Distributions, amplitude model and seeding scheme are those above; the
# random streams are torch's (Philox on the device), so a given seed gives a
# different sample from the numpy functions. Used where only the shape and
# value distribution matter (throughput of the largest workloads).

def _torch_legendre(l, mm, x):
    import torch
    s = torch.sqrt(torch.clamp(1.0 - x * x, min=0.0))
    pmm = torch.ones_like(x)
    fact = 1.0
    for _ in range(mm):
        pmm = -pmm * fact * s
        fact += 2.0
    if l == mm:
        return pmm
    pm1 = x * (2 * mm + 1) * pmm
    if l == mm + 1:
        return pm1
    p2, p1 = pmm, pm1
    for ll in range(mm + 2, l + 1):
        p = ((2 * ll - 1) * x * p1 - (ll + mm - 1) * p2) / (ll - mm)
        p2, p1 = p1, p
    return p1


def torch_amplitudes(ev, waves):
    """Event-major complex64 [n, len(waves)] on the events' device, evaluated
    in float64 like `amplitudes`."""
    import torch
    m, c, p = ev["m"], ev["costh"], ev["phi"]
    out = torch.empty((m.shape[0], len(waves)), dtype=torch.complex64, device=m.device)
    for a, wv in enumerate(waves):
        bw = 1.0 / torch.complex(wv.mass * wv.mass - m * m, torch.full_like(m, -wv.mass * wv.width))
        norm = math.sqrt((2 * wv.l + 1) / (4 * math.pi) * math.factorial(wv.l - wv.m)
                         / math.factorial(wv.l + wv.m))
        y = norm * _torch_legendre(wv.l, wv.m, c) * torch.exp(torch.complex(torch.zeros_like(p), wv.m * p))
        out[:, a] = (bw * y).to(torch.complex64)
    return out


def torch_mixture_workload(waves, n_data, n_mc_acc, seed, device="cuda", batch=1 << 22):
    """(A_data, A_mc, n_gen): data from the resonance mixture of
    `data_sample_mixture` (V_true from `random_V(len(waves), seed)`), accepted
    MC as in `mc_sample`; complex64 tensors on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = lambda k: torch.rand(k, generator=g, device=device, dtype=torch.float64)
    V = random_V(len(waves), seed)
    w = torch.tensor(np.abs(V) ** 2, device=device)
    M = torch.tensor([wv.mass for wv in waves], device=device, dtype=torch.float64)
    G = torch.tensor([wv.width for wv in waves], device=device, dtype=torch.float64)
    parts, got = [], 0
    while got < n_data:
        a = torch.multinomial(w, batch, replacement=True, generator=g)
        lo = torch.atan((M_LO - M[a]) / (G[a] / 2)) / math.pi + 0.5
        hi = torch.atan((M_HI - M[a]) / (G[a] / 2)) / math.pi + 0.5
        t = lo + (hi - lo) * u(batch)
        m = torch.clamp(M[a] + (G[a] / 2) * torch.tan(math.pi * (t - 0.5)), M_LO, M_HI)
        c = 2.0 * u(batch) - 1.0
        keep = u(batch) < (0.6 + 0.3 * c) / EFF_MAX
        p = 2.0 * math.pi * u(batch)
        parts.append((m[keep], c[keep], p[keep]))
        got += int(keep.sum())
    ev = {k: torch.cat([q[i] for q in parts])[:n_data] for i, k in enumerate(("m", "costh", "phi"))}
    A_data = torch_amplitudes(ev, waves)
    parts, got, n_gen = [], 0, 0
    while got < n_mc_acc:
        m = M_LO + (M_HI - M_LO) * u(batch)
        c = 2.0 * u(batch) - 1.0
        p = 2.0 * math.pi * u(batch)
        keep = u(batch) < 0.6 + 0.3 * c
        idx = torch.nonzero(keep).squeeze(1)
        need = n_mc_acc - got
        if idx.numel() >= need:
            n_gen += int(idx[need - 1]) + 1
            idx = idx[:need]
        else:
            n_gen += batch
        parts.append((m[idx], c[idx], p[idx]))
        got += idx.numel()
    ev = {k: torch.cat([q[i] for q in parts]) for i, k in enumerate(("m", "costh", "phi"))}
    return A_data, torch_amplitudes(ev, waves), n_gen


def model_batch_spec(n_models=64, n_lo=8, n_hi=48, d_lo=100_000, d_hi=2_000_000, seed=SEED_DATA):
    """The uneven trial-model batch: per model (n_waves ~ U{n_lo..n_hi},
    n_data ~ U[d_lo, d_hi], seed); its MC sample has 2 n_data accepted events."""
    rng = np.random.Generator(np.random.Philox(seed))
    nw = rng.integers(n_lo, n_hi + 1, n_models)
    nd = rng.integers(d_lo, d_hi + 1, n_models)
    return [(int(a), int(b), seed + 1000 * (j + 1)) for j, (a, b) in enumerate(zip(nw, nd))]


# ---- radiative decay kinematics for the covariant tensor amplitudes --------
M_PSI = 3.0969    # J/psi mass (GeV)
M_K = 0.493677    # charged kaon mass (GeV)


@dataclass(frozen=True)
class CovWave:
    """A wave of J/psi -> gamma X, X -> K+ K-: X's Breit-Wigner and spin (0, 2)."""
    mass: float
    width: float
    spin: int


def cov_waves(n):
    """n waves, spins alternating 0, 2, masses and widths as waves_linear."""
    base = waves_linear(n)
    return [CovWave(w.mass, w.width, 2 * (a % 2)) for a, w in enumerate(base)]


def radiative_kinematics(m, cos_g, phi_g, cos_k, phi_k):
    """3-momenta (photon, K+, K-) in the J/psi rest frame, [n, 9] float64:
    the photon at polar angles (cos_g, phi_g) about the beam (z) axis, X of
    mass m recoiling against it, K+ at (cos_k, phi_k) in the X rest frame
    (axes parallel to the J/psi frame's)."""
    m, cos_g, phi_g, cos_k, phi_k = (np.asarray(x, dtype=np.float64) for x in
                                     (m, cos_g, phi_g, cos_k, phi_k))
    sg, sk = np.sqrt(1 - cos_g ** 2), np.sqrt(1 - cos_k ** 2)
    qhat = np.stack([sg * np.cos(phi_g), sg * np.sin(phi_g), cos_g], axis=1)
    Eg = (M_PSI ** 2 - m ** 2) / (2 * M_PSI)
    q = Eg[:, None] * qhat
    EX = M_PSI - Eg
    beta = -q / EX[:, None]                       # X's velocity
    gam = EX / m
    kstar = np.sqrt(m ** 2 / 4 - M_K ** 2)
    ks = kstar[:, None] * np.stack([sk * np.cos(phi_k), sk * np.sin(phi_k), cos_k], axis=1)
    b2 = np.sum(beta ** 2, axis=1)

    def boost(k3, E):
        bk = np.sum(beta * k3, axis=1)
        coef = np.where(b2 > 0, (gam - 1) * bk / np.where(b2 > 0, b2, 1), 0.0)
        return k3 + coef[:, None] * beta + (gam * E)[:, None] * beta

    k1 = boost(ks, m / 2)
    k2 = boost(-ks, m / 2)
    return np.concatenate([q, k1, k2], axis=1)


# K+ K- mass range of the radiative samples: from just above the threshold
# 2 mK = 0.98735 GeV to 3.0 GeV (below M_PSI)
M_KK_LO, M_KK_HI = 0.99, 3.0


def radiative_events(n, rng, accept=False):
    """n radiative events uniform in (m, cos_g, phi_g, cos_k, phi_k), m in
    [M_KK_LO, M_KK_HI]; with
    accept, kept with probability 0.6 + 0.3 cos_g (returns the candidates
    drawn as well)."""
    out, drawn, got = [], 0, 0
    while got < n:
        k = max(1024, 2 * (n - got))
        m = rng.uniform(M_KK_LO, M_KK_HI, k)
        cg = rng.uniform(-1.0, 1.0, k)
        pg = rng.uniform(0.0, 2 * math.pi, k)
        ck = rng.uniform(-1.0, 1.0, k)
        pk = rng.uniform(0.0, 2 * math.pi, k)
        if accept:
            keep = rng.uniform(0.0, 1.0, k) < 0.6 + 0.3 * cg
            idx = np.nonzero(keep)[0]
            if idx.size > n - got:
                drawn += int(idx[n - got - 1]) + 1
                idx = idx[:n - got]
            else:
                drawn += k
        else:
            idx = np.arange(min(k, n - got))
            drawn += idx.size
        out.append(radiative_kinematics(m[idx], cg[idx], pg[idx], ck[idx], pk[idx]))
        got += idx.size
    return np.concatenate(out)[:n], drawn
