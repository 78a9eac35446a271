"""ctypes binding of libpwa (include/pwa.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the likelihood; all computation runs in the library's CUDA
kernels. Arrays may be numpy arrays (host memory) or CUDA tensors of any
library exposing `data_ptr()` and `is_cuda` (device memory).

Importing this module loads the compiled library and fails loudly if it is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libpwa.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "pwa.h")

PWA_OK = 0
PWA_EINVAL = -1
PWA_ENOMEM = -2
PWA_ECUDA = -3
PWA_ESTATE = -4
PWA_EDOMAIN = -5
PWA_ETIMEOUT = -6
PWA_ENOTSUP = -7
PWA_FORM_AMP = 1
PWA_FORM_TABLE = 2
PWA_FORM_TC = 4
PWA_C64 = 1
PWA_C128 = 2
PWA_PREC_DEFAULT = 0
PWA_PREC_BFP16 = 1
PWA_PREC_BFP8 = 2

ERROR_NAMES = {PWA_EINVAL: "PWA_EINVAL", PWA_ENOMEM: "PWA_ENOMEM", PWA_ECUDA: "PWA_ECUDA",
               PWA_ESTATE: "PWA_ESTATE", PWA_EDOMAIN: "PWA_EDOMAIN",
               PWA_ETIMEOUT: "PWA_ETIMEOUT", PWA_ENOTSUP: "PWA_ENOTSUP"}


class PwaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERROR_NAMES.get(code, str(code)), msg))
        self.code = code


class pwa_config(ctypes.Structure):
    _fields_ = [("n_waves", ctypes.c_int), ("forms", ctypes.c_int), ("precision", ctypes.c_int),
                ("max_k", ctypes.c_int), ("stream", ctypes.c_void_p)]


_lib = None


def load(path=LIB_PATH):
    """Load libpwa.so (built by paper_1108_5673_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libpwa.so not found at %s: run paper_1108_5673_gb300.build.build() "
                          "(nvcc, sm_103a); there is no CPU fallback" % path)
    lib = ctypes.CDLL(path)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "pwa_create": ([ctypes.POINTER(ctypes.c_void_p), I, ctypes.POINTER(pwa_config)], I),
        "pwa_destroy": ([P], I),
        "pwa_load_events": ([P, P, I64, P, I64, D, I], I),
        "pwa_build_norm": ([P, P], I),
        "pwa_set_form": ([P, I], I),
        "pwa_nll": ([P, P, I, P], I),
        "pwa_nll_grad": ([P, P, I, P, P], I),
        "pwa_nll_grad_async": ([P, P, I, P, P], I),
        "pwa_sync": ([P], I),
        "pwa_last_error": ([P], ctypes.c_char_p),
        "pwa_table_bytes": ([I, I64, ctypes.POINTER(ctypes.c_int64)], I),
        "pwa_version": ([], I),
        "pwa_nll_grad_noalloc": ([P, I64, I64, I, P, P, P, P, P, P, P], I),
        "pwa_load_resonance_events": ([P, I, P, P, P, I64, P, P, P, I64, D, I], I),
        "pwa_nll_grad_res": ([P, P, P, P, P, P, P, P], I),
        "pwa_batch_create": ([ctypes.POINTER(ctypes.c_void_p), I, I, P, I, I, P], I),
        "pwa_batch_destroy": ([P], I),
        "pwa_batch_load_model": ([P, I, P, I64, P, I64, D, I], I),
        "pwa_batch_nll_grad": ([P, P, I, P, P], I),
        "pwa_batch_last_error": ([P], ctypes.c_char_p),
        "pwa_autotune": ([P, ctypes.c_char_p, ctypes.c_char_p, I], I),
        "pwa_batch_autotune": ([P, ctypes.c_char_p, ctypes.c_char_p, I], I),
        "pwa_hessian": ([P, P, P], I),
        "pwa_hessian_async": ([P, P, P], I),
        "pwa_nll_grad_res_async": ([P, P, P, P, P], I),
        "pwa_load_events_incoherent": ([P, I, P, I64, P, I64, D, I], I),
        "pwa_compute_amplitudes": ([P, P, P, I64, P], I),
        "pwa_load_events_generated": ([P, P, P, I64, P, I64, D], I),
        "pwa_compute_covariant_amplitudes": ([P, P, P, I64, P], I),
        "pwa_load_events_covariant": ([P, P, P, I64, P, I64, D], I),
        "pwa_mc_weights": ([P, P, P], I),
        "pwa_fit_fractions": ([P, P, P], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def header_symbols(header=HEADER):
    """Names of the functions declared in include/pwa.h."""
    text = open(header).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(pwa_\w+)\s*\(", text, re.M)))


def _ptr(x, dtype=None):
    """(pointer, keepalive) for a numpy array or a CUDA tensor."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr") and getattr(x, "is_cuda", False):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x
    a = np.ascontiguousarray(x, dtype=dtype) if dtype is not None else np.ascontiguousarray(x)
    return a.ctypes.data_as(ctypes.c_void_p), a


def _check(ctx, rc, allow=()):
    if rc != PWA_OK and rc not in allow:
        msg = load().pwa_last_error(ctx)
        raise PwaError(rc, msg.decode() if msg else "")
    return rc


def pwa_version():
    return load().pwa_version()


def pwa_table_bytes(n_waves, n_events):
    out = ctypes.c_int64()
    _check(None, load().pwa_table_bytes(n_waves, n_events, ctypes.byref(out)))
    return out.value


def pwa_create(device, n_waves, forms=PWA_FORM_AMP, precision=0, max_k=1, stream=None):
    cfg = pwa_config(n_waves, forms, precision, max_k,
                     ctypes.c_void_p(stream) if stream else None)
    h = ctypes.c_void_p()
    _check(None, load().pwa_create(ctypes.byref(h), device, ctypes.byref(cfg)))
    return h


def pwa_destroy(ctx):
    return load().pwa_destroy(ctx)


def pwa_load_events(ctx, data_amp, mc_amp, n_mc_gen):
    """data_amp / mc_amp: [n, n_waves] complex64 or complex128 (numpy or CUDA tensor)."""
    def kind(x):
        dt = str(getattr(x, "dtype", ""))
        if "complex64" in dt:
            return PWA_C64
        if "complex128" in dt:
            return PWA_C128
        raise ValueError("amplitudes must be complex64 or complex128, got %s" % dt)
    kd, km = kind(data_amp), kind(mc_amp)
    if kd != km:
        raise ValueError("data and MC amplitudes must share one dtype")
    pd, kd_ = _ptr(data_amp)
    pm, km_ = _ptr(mc_amp)
    return _check(ctx, load().pwa_load_events(ctx, pd, int(data_amp.shape[0]), pm,
                                              int(mc_amp.shape[0]), float(n_mc_gen), kd))


def pwa_load_events_incoherent(ctx, data_amp, mc_amp, n_mc_gen):
    """data_amp / mc_amp: [n, n_lambda, n_waves] complex64 or complex128 (numpy
    or CUDA tensor, contiguous): n_lambda incoherent components per event."""
    def kind(x):
        dt = str(getattr(x, "dtype", ""))
        if "complex64" in dt:
            return PWA_C64
        if "complex128" in dt:
            return PWA_C128
        raise ValueError("amplitudes must be complex64 or complex128, got %s" % dt)
    kd, km = kind(data_amp), kind(mc_amp)
    if kd != km:
        raise ValueError("data and MC amplitudes must share one dtype")
    if len(data_amp.shape) != 3 or tuple(data_amp.shape[1:]) != tuple(mc_amp.shape[1:]):
        raise ValueError("amplitudes must be [n, n_lambda, n_waves] with matching trailing shapes")
    pd, kd_ = _ptr(data_amp)
    pm, km_ = _ptr(mc_amp)
    return _check(ctx, load().pwa_load_events_incoherent(
        ctx, int(data_amp.shape[1]), pd, int(data_amp.shape[0]), pm, int(mc_amp.shape[0]),
        float(n_mc_gen), kd))


class pwa_wave(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("width", ctypes.c_double), ("l", ctypes.c_int),
                ("m", ctypes.c_int)]


def _waves(waves):
    """A ctypes array of pwa_wave from objects with mass, width, l, m (or 4-tuples)."""
    arr = (pwa_wave * len(waves))()
    for k, w in enumerate(waves):
        t = (w.mass, w.width, w.l, w.m) if hasattr(w, "mass") else tuple(w)
        arr[k] = pwa_wave(float(t[0]), float(t[1]), int(t[2]), int(t[3]))
    return arr


def _kin(kin):
    """(pointer, keepalive, n) for kinematics: a dict with m, costh, phi, an
    [n, 3] float64 array, or an [n, 3] float64 CUDA tensor."""
    if isinstance(kin, dict):
        kin = np.stack([np.asarray(kin["m"], np.float64), np.asarray(kin["costh"], np.float64),
                        np.asarray(kin["phi"], np.float64)], axis=1)
    if getattr(kin, "is_cuda", False):
        if "float64" not in str(kin.dtype) or tuple(kin.shape[1:]) != (3,):
            raise ValueError("device kinematics must be [n, 3] float64")
    else:
        kin = np.ascontiguousarray(kin, dtype=np.float64)
        if kin.ndim != 2 or kin.shape[1] != 3:
            raise ValueError("kinematics must be [n, 3] (m, cos theta, phi)")
    p, keep = _ptr(kin)
    return p, keep, int(kin.shape[0])


def pwa_compute_amplitudes(ctx, waves, kin, out=None):
    """[n, n_waves] complex64 amplitudes BW x Y_l^m of the given events
    (numpy, or into `out`: a numpy array or a CUDA tensor of that shape)."""
    pk, keep, n = _kin(kin)
    if out is None:
        out = np.empty((n, len(waves)), dtype=np.complex64)
    elif not getattr(out, "is_cuda", False) and not (
            isinstance(out, np.ndarray) and out.dtype == np.complex64 and out.flags.c_contiguous):
        raise ValueError("host output must be a contiguous complex64 numpy array")
    po, keep_o = _ptr(out)
    _check(ctx, load().pwa_compute_amplitudes(ctx, _waves(waves), pk, n, po))
    return out


def pwa_load_events_generated(ctx, waves, data_kin, mc_kin, n_mc_gen):
    pd, kd, nd = _kin(data_kin)
    pm, km, nm = _kin(mc_kin)
    return _check(ctx, load().pwa_load_events_generated(ctx, _waves(waves), pd, nd, pm, nm,
                                                        float(n_mc_gen)))


class pwa_cov_wave(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("width", ctypes.c_double), ("spin", ctypes.c_int)]


def _cov_waves(waves):
    """A ctypes array of pwa_cov_wave from objects with mass, width, spin (or 3-tuples)."""
    arr = (pwa_cov_wave * len(waves))()
    for k, w in enumerate(waves):
        t = (w.mass, w.width, w.spin) if hasattr(w, "mass") else tuple(w)
        arr[k] = pwa_cov_wave(float(t[0]), float(t[1]), int(t[2]))
    return arr


def _p3(p3):
    """(pointer, keepalive, n) for [n, 9] float64 momenta (photon, K+, K-),
    a numpy array or a CUDA tensor."""
    if getattr(p3, "is_cuda", False):
        if "float64" not in str(p3.dtype) or tuple(p3.shape[1:]) != (9,) or not p3.is_contiguous():
            raise ValueError("device momenta must be a contiguous [n, 9] float64 tensor")
    else:
        p3 = np.ascontiguousarray(p3, dtype=np.float64)
        if p3.ndim != 2 or p3.shape[1] != 9:
            raise ValueError("momenta must be [n, 9] (photon, K+, K- 3-momenta)")
    p, keep = _ptr(p3)
    return p, keep, int(p3.shape[0])


def pwa_compute_covariant_amplitudes(ctx, waves, p3, out=None):
    """[n, 4, n_waves] complex64 covariant amplitudes of J/psi -> gamma X,
    X -> K+ K- (numpy, or into `out`: a numpy array or a CUDA tensor of that
    shape)."""
    pk, keep, n = _p3(p3)
    if out is None:
        out = np.empty((n, 4, len(waves)), dtype=np.complex64)
    elif not getattr(out, "is_cuda", False) and not (
            isinstance(out, np.ndarray) and out.dtype == np.complex64 and out.flags.c_contiguous):
        raise ValueError("host output must be a contiguous complex64 numpy array")
    po, keep_o = _ptr(out)
    _check(ctx, load().pwa_compute_covariant_amplitudes(ctx, _cov_waves(waves), pk, n, po))
    return out


def pwa_load_events_covariant(ctx, waves, data_p3, mc_p3, n_mc_gen):
    pd, kd, nd = _p3(data_p3)
    pm, km, nm = _p3(mc_p3)
    return _check(ctx, load().pwa_load_events_covariant(ctx, _cov_waves(waves), pd, nd, pm, nm,
                                                        float(n_mc_gen)))


def pwa_build_norm(ctx, n_waves):
    M = np.empty((n_waves, n_waves), dtype=np.complex128)
    _check(ctx, load().pwa_build_norm(ctx, M.ctypes.data_as(ctypes.c_void_p)))
    return M


def pwa_set_form(ctx, form):
    return _check(ctx, load().pwa_set_form(ctx, form))


def pwa_nll(ctx, V):
    """V: [K, n_waves] complex128 (host). Returns (nll [K], status)."""
    V = np.ascontiguousarray(np.atleast_2d(V), dtype=np.complex128)
    nll = np.empty(V.shape[0])
    rc = _check(ctx, load().pwa_nll(ctx, V.ctypes.data_as(ctypes.c_void_p), V.shape[0],
                                    nll.ctypes.data_as(ctypes.c_void_p)), allow=(PWA_EDOMAIN,))
    return nll, rc


def pwa_nll_grad(ctx, V):
    """V: [K, n_waves] complex128 (host). Returns (nll [K], grad [K, n_waves], status)."""
    V = np.ascontiguousarray(np.atleast_2d(V), dtype=np.complex128)
    nll = np.empty(V.shape[0])
    g = np.empty_like(V)
    # integer addresses: the per-call marshalling is a measurable part of a
    # ~40 us evaluation
    rc = (_lib or load()).pwa_nll_grad(ctx, V.ctypes.data, V.shape[0], nll.ctypes.data,
                                       g.ctypes.data)
    if rc != PWA_OK and rc != PWA_EDOMAIN:
        _check(ctx, rc)
    return nll, g, rc


def pwa_nll_grad_raw(ctx, V_addr, K, nll_addr, grad_addr):
    """pwa_nll_grad on host addresses the caller keeps valid (the Likelihood
    object's buffers); returns the status (PWA_OK or PWA_EDOMAIN), raises on
    other errors."""
    rc = (_lib or load()).pwa_nll_grad(ctx, V_addr, K, nll_addr, grad_addr)
    if rc != PWA_OK and rc != PWA_EDOMAIN:
        _check(ctx, rc)
    return rc


def pwa_nll_grad_async(ctx, d_V, K, d_nll, d_grad=None):
    """Device pointers (CUDA tensors): d_V [K, n_waves] complex128, d_nll [K]
    float64, d_grad [K, n_waves] complex128 or None."""
    pv, _a = _ptr(d_V)
    pn, _b = _ptr(d_nll)
    pg, _c = _ptr(d_grad)
    return _check(ctx, load().pwa_nll_grad_async(ctx, pv, K, pn, pg))


def pwa_sync(ctx):
    return _check(ctx, load().pwa_sync(ctx), allow=(PWA_EDOMAIN,))


def pwa_nll_grad_noalloc(d_planes, plane_pitch, n_events, n_waves, d_amax, d_M, d_V, d_nll,
                         d_grad=None, d_status=None, stream=None):
    """Context-free, allocation-free evaluation (see include/pwa.h): every
    argument is a CUDA tensor already on the current device."""
    ptrs = [_ptr(x) for x in (d_planes, d_amax, d_M, d_V, d_nll, d_grad, d_status)]
    rc = load().pwa_nll_grad_noalloc(ptrs[0][0], plane_pitch, n_events, n_waves, ptrs[1][0],
                                     ptrs[2][0], ptrs[3][0], ptrs[4][0], ptrs[5][0], ptrs[6][0],
                                     ctypes.c_void_p(stream) if stream else None)
    if rc != PWA_OK:
        raise PwaError(rc, "pwa_nll_grad_noalloc failed")
    return rc


def pwa_load_resonance_events(ctx, n_free, m_data, Y_data, Afix_data, m_mc, Y_mc, Afix_mc,
                              n_mc_gen):
    """m_*: [n] masses (any float type, passed as float64); Y_*: [n, n_free]
    and Afix_*: [n, n_waves - n_free] complex64 or complex128 (Afix may be None
    when every wave is free)."""
    def kind(x):
        dt = str(getattr(x, "dtype", ""))
        if "complex64" in dt:
            return PWA_C64
        if "complex128" in dt:
            return PWA_C128
        raise ValueError("amplitudes must be complex64 or complex128, got %s" % dt)
    k = kind(Y_data)
    for x in (Y_mc, Afix_data, Afix_mc):
        if x is not None and kind(x) != k:
            raise ValueError("Y and Afix of both samples must share one dtype")
    for x in (m_data, m_mc):
        if getattr(x, "is_cuda", False) and "float64" not in str(x.dtype):
            raise ValueError("device mass arrays must be float64")
    md, a1 = _ptr(m_data, np.float64)
    mm, a2 = _ptr(m_mc, np.float64)
    yd, a3 = _ptr(Y_data)
    ym, a4 = _ptr(Y_mc)
    fd, a5 = _ptr(Afix_data)
    fm, a6 = _ptr(Afix_mc)
    return _check(ctx, load().pwa_load_resonance_events(
        ctx, int(n_free), md, yd, fd, int(len(m_data)), mm, ym, fm, int(len(m_mc)),
        float(n_mc_gen), k))


def pwa_nll_grad_res(ctx, V, mass, width):
    """Host V [n_waves] complex128, mass/width [n_free]. Returns
    (nll, gV [n_waves] complex128 = dNLL/dV*, gM, gW, status)."""
    V = np.ascontiguousarray(V, dtype=np.complex128)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    width = np.ascontiguousarray(width, dtype=np.float64)
    nll = np.empty(1)
    gV = np.empty_like(V)
    gM, gW = np.empty_like(mass), np.empty_like(width)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = _check(ctx, load().pwa_nll_grad_res(ctx, p(V), p(mass), p(width), p(nll), p(gV), p(gM),
                                             p(gW)), allow=(PWA_EDOMAIN,))
    return float(nll[0]), gV, gM, gW, rc


def pwa_hessian(ctx, V, n_waves):
    """FUMILI Hessian over (Re V, Im V), sum_i grad ln I_i grad ln I_i^T:
    ([2N, 2N] float64, status); an all-zero H with PWA_EDOMAIN when a data
    intensity was not positive."""
    V = np.ascontiguousarray(V, dtype=np.complex128)
    H = np.empty((2 * n_waves, 2 * n_waves))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = _check(ctx, load().pwa_hessian(ctx, p(V), p(H)), allow=(PWA_EDOMAIN,))
    return H, rc


def pwa_hessian_async(ctx, d_V, d_H):
    """Device tensors: d_V [n_waves] complex128, d_H [2N, 2N] float64."""
    pv, _a = _ptr(d_V)
    ph, _b = _ptr(d_H)
    return _check(ctx, load().pwa_hessian_async(ctx, pv, ph))


def pwa_nll_grad_res_async(ctx, d_V, d_mass, d_width, d_out):
    """Device tensors: d_V [N] complex128, d_mass/d_width [R] float64, d_out
    [1 + 2N + 2R] float64 (nll, dNLL/dV* as (re, im) pairs, dNLL/dM, dNLL/dG)."""
    ptrs = [_ptr(x) for x in (d_V, d_mass, d_width, d_out)]
    return _check(ctx, load().pwa_nll_grad_res_async(ctx, *[p for p, _ in ptrs]))


def pwa_mc_weights(ctx, V, w):
    """Fill w ([n_mc_acc] float32: a numpy array or a CUDA tensor) with
    I(Omega_j) / n_mc_gen of each accepted MC event; returns w."""
    V = np.ascontiguousarray(V, dtype=np.complex128)
    if not getattr(w, "is_cuda", False):
        if not (isinstance(w, np.ndarray) and w.dtype == np.float32 and w.flags.c_contiguous):
            raise ValueError("host weights must be a contiguous float32 numpy array")
    elif "float32" not in str(w.dtype):
        raise ValueError("device weights must be float32")
    pw, _k = _ptr(w)
    _check(ctx, load().pwa_mc_weights(ctx, V.ctypes.data_as(ctypes.c_void_p), pw))
    return w


def pwa_fit_fractions(ctx, V, n_waves):
    """[N, N] float64: Re(conj(V_a) M_ab V_b) / V^H M V."""
    V = np.ascontiguousarray(V, dtype=np.complex128)
    F = np.empty((n_waves, n_waves))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    _check(ctx, load().pwa_fit_fractions(ctx, p(V), p(F)))
    return F


def _bcheck(b, rc, allow=()):
    if rc != PWA_OK and rc not in allow:
        msg = load().pwa_batch_last_error(b)
        raise PwaError(rc, msg.decode() if msg else "")
    return rc


def pwa_batch_create(device, n_waves, max_k, precision=0, stream=None):
    nw = np.ascontiguousarray(n_waves, dtype=np.int32)
    h = ctypes.c_void_p()
    _bcheck(None, load().pwa_batch_create(ctypes.byref(h), device, len(nw),
                                          nw.ctypes.data_as(ctypes.c_void_p), max_k, precision,
                                          ctypes.c_void_p(stream) if stream else None))
    return h


def pwa_batch_destroy(b):
    return load().pwa_batch_destroy(b)


def pwa_batch_load_model(b, model, data_amp, mc_amp, n_mc_gen):
    kinds = {"complex64": PWA_C64, "complex128": PWA_C128}
    kd = kinds.get(str(data_amp.dtype).replace("torch.", ""))
    if kd is None or str(mc_amp.dtype) != str(data_amp.dtype):
        raise ValueError("amplitudes must be complex64 or complex128, both alike")
    pd, a = _ptr(data_amp)
    pm, c = _ptr(mc_amp)
    return _bcheck(b, load().pwa_batch_load_model(b, model, pd, int(data_amp.shape[0]), pm,
                                                  int(mc_amp.shape[0]), float(n_mc_gen), kd))


def pwa_batch_nll_grad(b, V_all, K, n_models, grad=True):
    """V_all: host complex128, the models' [K][n_waves[m]] blocks concatenated.
    Returns (nll [n_models][K], grad like V_all or None, status)."""
    V_all = np.ascontiguousarray(V_all, dtype=np.complex128)
    nll = np.empty((n_models, K))
    g = np.empty_like(V_all) if grad else None
    rc = _bcheck(b, load().pwa_batch_nll_grad(b, V_all.ctypes.data_as(ctypes.c_void_p), K,
                                              nll.ctypes.data_as(ctypes.c_void_p),
                                              g.ctypes.data_as(ctypes.c_void_p) if grad else None),
                 allow=(PWA_EDOMAIN,))
    return nll, g, rc


def pwa_autotune(ctx, cache_path=None):
    """Returns the one-line summary of the choices applied."""
    buf = ctypes.create_string_buffer(512)
    _check(ctx, load().pwa_autotune(ctx, cache_path.encode() if cache_path else None, buf, 512))
    return buf.value.decode()


def pwa_batch_autotune(b, cache_path=None):
    """Returns the one-line summary of the choice applied to the model batch."""
    buf = ctypes.create_string_buffer(512)
    _bcheck(b, load().pwa_batch_autotune(b, cache_path.encode() if cache_path else None, buf, 512))
    return buf.value.decode()


def pwa_last_error(ctx):
    m = load().pwa_last_error(ctx)
    return m.decode() if m else ""
