"""FP64 CPU oracle for the partial wave analysis likelihood (Eq. 1 and Eq. 3).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the CPU-baseline
leg of bench.py may import this package. The library itself never does; it
shares no code with the CUDA path.

The arithmetic lives in pwa_oracle.c (plain double-precision loops with
Neumaier sums); this module compiles it with gcc on first use and wraps it with
ctypes. All inputs are promoted to complex128 first, so the oracle sees exactly
the values the GPU path consumes when it is handed the same (rounded) arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pwa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile pwa_oracle.c into liboracle.so (single-threaded, no fast-math,
    no floating-point contraction so x86 and Arm give the same bits)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                           "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.oracle_intensity.argtypes = [P, I64, I, P, P]
        lib.oracle_norm_matrix.argtypes = [P, I64, I, D, P]
        lib.oracle_norm_matrix.restype = I
        lib.oracle_norm_term.argtypes = [P, I, P, P, P]
        lib.oracle_nll_amp.argtypes = [P, I64, I, P, P, I, P, P]
        lib.oracle_nll_amp.restype = I
        lib.oracle_table.argtypes = [P, I64, I, P]
        lib.oracle_nll_table.argtypes = [P, I64, I, P, P, I, P, P]
        lib.oracle_nll_table.restype = I
        lib.oracle_nll_res.argtypes = [I, I, P, P, P, I64, P, P, P, I64, D, P, P, P, P, P, P, P]
        lib.oracle_hessian.argtypes = [P, I64, I, P, P]
        lib.oracle_hessian.restype = I
        lib.oracle_mc_weights.argtypes = [P, I64, I, P, D, P]
        lib.oracle_fit_fractions.argtypes = [P, I, P, P]
        lib.oracle_nll_res.restype = I
        lib.oracle_amplitudes.argtypes = [P, I64, I, P, P, P, P, P]
        lib.oracle_amplitudes.restype = I
        lib.oracle_norm_incoh.argtypes = [P, I64, I, I, D, P]
        lib.oracle_norm_incoh.restype = I
        lib.oracle_table_incoh.argtypes = [P, I64, I, I, P]
        lib.oracle_nll_incoh.argtypes = [P, I64, I, I, P, P, I, P, P]
        lib.oracle_nll_incoh.restype = I
        lib.oracle_cov_amplitudes.argtypes = [P, I64, I, P, P, P, P]
        lib.oracle_cov_amplitudes.restype = I
        _lib = lib
    return _lib


def _c128(x):
    return np.ascontiguousarray(np.asarray(x), dtype=np.complex128)


def _f64(x):
    return np.ascontiguousarray(np.asarray(x), dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def intensity(A, V):
    """Eq. 1 per event: I_i = |sum_a V_a A_ia|^2. A: [n, N], V: [N]."""
    A, V = _c128(A), _c128(V)
    n, N = A.shape
    out = np.empty(n)
    _load().oracle_intensity(_p(A), n, N, _p(V), _p(out))
    return out


def norm_matrix(A_mc, n_gen):
    """M[a, b] = (1/N_gen) sum_j conj(A_ja) A_jb over the accepted MC events."""
    A = _c128(A_mc)
    n, N = A.shape
    M = np.empty((N, N), dtype=np.complex128)
    if _load().oracle_norm_matrix(_p(A), n, N, float(n_gen), _p(M)) != 0:
        raise ValueError("bad arguments")
    return M


def norm_matrix_blas(A_mc, n_gen, chunk=1 << 20):
    """The same M as norm_matrix, with the sum over events done by a library
    complex128 matrix product (conj(A)^T A) in chunks; for samples where the
    plain loops take minutes. Pinned against norm_matrix in the tests."""
    A = np.asarray(A_mc)
    N = A.shape[1]
    M = np.zeros((N, N), dtype=np.complex128)
    for s in range(0, A.shape[0], chunk):
        a = A[s:s + chunk].astype(np.complex128)
        M += a.conj().T @ a
    return M / float(n_gen)


def norm_term(M, V):
    """(V^H M V, M V)."""
    M, V = _c128(M), _c128(V)
    N = M.shape[0]
    nv = ctypes.c_double()
    mv = np.empty(N, dtype=np.complex128)
    _load().oracle_norm_term(_p(M), N, _p(V), ctypes.byref(nv), _p(mv))
    return nv.value, mv


def nll_amp(A, M, V, grad=True):
    """Eq. 3 on the amplitudes. V: [N] or [K, N]. Returns (nll, grad, n_bad)
    with nll of shape [K] (or scalar) and grad dNLL/dV* of V's shape."""
    A, M, V = _c128(A), _c128(M), _c128(V)
    single = V.ndim == 1
    V2 = V.reshape(-1, A.shape[1])
    K = V2.shape[0]
    nll = np.empty(K)
    g = np.empty_like(V2) if grad else None
    bad = _load().oracle_nll_amp(_p(A), A.shape[0], A.shape[1], _p(M), _p(V2), K, _p(nll),
                                 _p(g) if grad else None)
    if single:
        return nll[0], (g[0] if grad else None), bad
    return nll, g, bad


def table(A):
    """Per-event Hermitian table, [n, N*N] float64 (diagonal, then Re/Im pairs a < b)."""
    A = _c128(A)
    n, N = A.shape
    T = np.empty((n, N * N))
    _load().oracle_table(_p(A), n, N, _p(T))
    return T


def nll_table(T, M, V, grad=True):
    """Eq. 3 on the precomputed table. Same returns as nll_amp."""
    T, M, V = _f64(T), _c128(M), _c128(V)
    N = M.shape[0]
    single = V.ndim == 1
    V2 = V.reshape(-1, N)
    K = V2.shape[0]
    nll = np.empty(K)
    g = np.empty_like(V2) if grad else None
    bad = _load().oracle_nll_table(_p(T), T.shape[0], N, _p(M), _p(V2), K, _p(nll),
                                   _p(g) if grad else None)
    if single:
        return nll[0], (g[0] if grad else None), bad
    return nll, g, bad


def nll_res(m_d, Y_d, Afix_d, m_mc, Y_mc, Afix_mc, n_gen, V, mass, width):
    """NLL with free Breit-Wigner masses and widths for the first R waves.
    Returns (nll, gV [N] complex = dNLL/dV*, gM [R], gW [R], bad)."""
    Y_d, Afix_d, Y_mc, Afix_mc = map(_c128, (Y_d, Afix_d, Y_mc, Afix_mc))
    m_d, m_mc, mass, width = map(_f64, (m_d, m_mc, mass, width))
    V = _c128(V)
    R = Y_d.shape[1]
    N = R + Afix_d.shape[1]
    nll = ctypes.c_double()
    gV = np.empty(N, dtype=np.complex128)
    gM, gW = np.empty(R), np.empty(R)
    bad = _load().oracle_nll_res(N, R, _p(m_d), _p(Y_d), _p(Afix_d), len(m_d),
                                 _p(m_mc), _p(Y_mc), _p(Afix_mc), len(m_mc), float(n_gen),
                                 _p(V), _p(mass), _p(width), ctypes.byref(nll),
                                 _p(gV), _p(gM), _p(gW))
    return nll.value, gV, gM, gW, bad


def hessian(A, V):
    """FUMILI's approximation of the NLL Hessian in p = (Re V, Im V):
    sum_i grad ln I_i grad ln I_i^T, [2N, 2N] float64; and n_bad."""
    A, V = _c128(A), _c128(V)
    n, N = A.shape
    H = np.empty((2 * N, 2 * N))
    bad = _load().oracle_hessian(_p(A), n, N, _p(V), _p(H))
    return H, bad


def mc_weights(A_mc, V, n_gen):
    """Per accepted MC event I(Omega_j) / N_gen."""
    A, V = _c128(A_mc), _c128(V)
    w = np.empty(A.shape[0])
    _load().oracle_mc_weights(_p(A), A.shape[0], A.shape[1], _p(V), float(n_gen), _p(w))
    return w


def fit_fractions(M, V):
    """F[a, b] = Re(conj(V_a) M_ab V_b) / V^H M V."""
    M, V = _c128(M), _c128(V)
    N = M.shape[0]
    F = np.empty((N, N))
    _load().oracle_fit_fractions(_p(M), N, _p(V), _p(F))
    return F


def norm_matrix_incoh(A_mc, n_gen):
    """M[a, b] = (1/N_gen) sum_j sum_l conj(A_a^l(j)) A_b^l(j) for A_mc [n, L, N]."""
    A = _c128(A_mc)
    n, L, N = A.shape
    M = np.empty((N, N), dtype=np.complex128)
    _load().oracle_norm_incoh(_p(A), n, L, N, float(n_gen), _p(M))
    return M


def table_incoh(A):
    """Per-event table of the incoherent sum, [n, N*N] float64, for A [n, L, N]."""
    A = _c128(A)
    n, L, N = A.shape
    T = np.empty((n, N * N))
    _load().oracle_table_incoh(_p(A), n, L, N, _p(T))
    return T


def nll_incoh(A, M, V, grad=True):
    """Eq. 3 with I = sum_l |sum_a V_a A_a^l|^2, A [n, L, N]. Returns as nll_amp."""
    A, M, V = _c128(A), _c128(M), _c128(V)
    n, L, N = A.shape
    single = V.ndim == 1
    V2 = V.reshape(-1, N)
    K = V2.shape[0]
    nll = np.empty(K)
    g = np.empty_like(V2) if grad else None
    bad = _load().oracle_nll_incoh(_p(A), n, L, N, _p(M), _p(V2), K, _p(nll),
                                   _p(g) if grad else None)
    if single:
        return nll[0], (g[0] if grad else None), bad
    return nll, g, bad


def amplitudes(m, costh, phi, waves):
    """A[i, a] = BW(m_i; M_a, G_a) Y_{l_a}^{m_a}(costh_i, phi_i), complex128
    [n, N]; `waves` holds objects with mass, width, l, m (or 4-tuples)."""
    kin = np.ascontiguousarray(np.stack([_f64(m), _f64(costh), _f64(phi)], axis=1))
    w = [(x.mass, x.width, x.l, x.m) if hasattr(x, "mass") else tuple(x) for x in waves]
    mass = _f64([x[0] for x in w])
    width = _f64([x[1] for x in w])
    ls = np.ascontiguousarray([x[2] for x in w], dtype=np.int32)
    ms = np.ascontiguousarray([x[3] for x in w], dtype=np.int32)
    A = np.empty((kin.shape[0], len(w)), dtype=np.complex128)
    rc = _load().oracle_amplitudes(_p(kin), kin.shape[0], len(w), _p(mass), _p(width), _p(ls),
                                   _p(ms), _p(A))
    if rc:
        raise ValueError("a wave has |m| > l or l < 0")
    return A


def covariant_amplitudes(p3, waves):
    """Covariant tensor amplitudes of J/psi -> gamma X, X -> K+ K- (see
    oracle_cov_amplitudes in pwa_oracle.c): p3 [n, 9] = 3-momenta (GeV) of the
    photon, K+ and K- in the J/psi rest frame; `waves` holds (mass, width,
    spin) with spin 0 or 2. Returns [n, 4, N] complex128: component l = 2 m +
    p for J/psi helicity (+1, -1)[m] and photon polarization p."""
    p3 = np.ascontiguousarray(p3, dtype=np.float64)
    w = [(x.mass, x.width, x.spin) if hasattr(x, "spin") else tuple(x) for x in waves]
    mass = _f64([x[0] for x in w])
    width = _f64([x[1] for x in w])
    spin = np.ascontiguousarray([x[2] for x in w], dtype=np.int32)
    out = np.empty((p3.shape[0], 4, len(w)), dtype=np.complex128)
    if _load().oracle_cov_amplitudes(_p(p3), p3.shape[0], len(w), _p(mass), _p(width), _p(spin),
                                     _p(out)):
        raise ValueError("a wave's spin is not 0 or 2")
    return out
