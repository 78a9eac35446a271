"""GB300-native partial wave analysis likelihood (Berger, arXiv:1108.5673).

The hot path, the extended negative log-likelihood of Eq. 3 and its gradient
with respect to the production amplitudes V, runs in hand-written CUDA
kernels for sm_103a behind the C ABI of include/pwa.h. This package is the
thin Python binding of that ABI (`_abi`, same function names) plus a small
object wrapper; PyTorch is only used by callers for device memory and
streams.

The compiled library is built by `paper_1108_5673_gb300.build.build()`.
"""
import numpy as np

from ._abi import (PWA_C64, PWA_C128, PWA_EDOMAIN, PWA_FORM_AMP, PWA_FORM_TABLE, PWA_FORM_TC,
                   PWA_OK, PWA_PREC_BFP8, PWA_PREC_BFP16, PWA_PREC_DEFAULT, PwaError)

__all__ = ["Likelihood", "ModelBatch", "PwaError", "PWA_FORM_AMP", "PWA_FORM_TABLE", "PWA_FORM_TC", "PWA_OK",
           "PWA_EDOMAIN", "PWA_C64", "PWA_C128", "PWA_PREC_DEFAULT", "PWA_PREC_BFP16",
           "PWA_PREC_BFP8"]


class Likelihood:
    """One library context: a loaded sample, its normalisation matrix, and
    evaluations of NLL(V) and dNLL/dV* (Wirtinger) for K parameter sets."""

    def __init__(self, n_waves, device=0, forms=PWA_FORM_AMP, max_k=1, stream=None,
                 precision=PWA_PREC_DEFAULT):
        from . import _abi
        self._abi = _abi
        self.n_waves = n_waves
        self.max_k = max_k
        self.ctx = _abi.pwa_create(device, n_waves, forms, precision, max_k, stream)
        self.last_status = PWA_OK
        self.M = None
        self._bufs = {}

    def load_events(self, data_amp, mc_amp, n_mc_gen):
        """[n, N] amplitudes (coherent sum, Eq. 1), or [n, n_lambda, N] for an
        incoherent sum over n_lambda unobserved components per event."""
        if len(data_amp.shape) == 3:
            self._abi.pwa_load_events_incoherent(self.ctx, data_amp, mc_amp, n_mc_gen)
        else:
            self._abi.pwa_load_events(self.ctx, data_amp, mc_amp, n_mc_gen)
        self.M = None
        self.n_data = int(data_amp.shape[0])
        self.n_mc = int(mc_amp.shape[0])
        return self

    def load_generated(self, waves, data_kin, mc_kin, n_mc_gen):
        """Load samples given by kinematics (m, cos theta, phi): the amplitudes
        BW x Y_l^m of `waves` are computed on the device."""
        self._abi.pwa_load_events_generated(self.ctx, waves, data_kin, mc_kin, n_mc_gen)
        self.M = None
        self.n_data = int(len(data_kin["m"]) if isinstance(data_kin, dict) else data_kin.shape[0])
        self.n_mc = int(len(mc_kin["m"]) if isinstance(mc_kin, dict) else mc_kin.shape[0])
        return self

    def load_covariant(self, waves, data_p3, mc_p3, n_mc_gen):
        """Load J/psi -> gamma K+ K- samples given by their 3-momenta ([n, 9]:
        photon, K+, K-): the covariant amplitudes of `waves` (mass, width,
        spin 0 or 2) are computed on the device and loaded as an incoherent
        sample over the 4 unobserved components."""
        self._abi.pwa_load_events_covariant(self.ctx, waves, data_p3, mc_p3, n_mc_gen)
        self.M = None
        self.n_data = int(data_p3.shape[0])
        self.n_mc = int(mc_p3.shape[0])
        return self

    def covariant_amplitudes(self, waves, p3, out=None):
        """[n, 4, N] complex64 covariant amplitudes of `waves` at the events
        `p3`, on the device."""
        return self._abi.pwa_compute_covariant_amplitudes(self.ctx, waves, p3, out)

    def amplitudes(self, waves, kin, out=None):
        """[n, N] complex64 amplitudes of `waves` at the events `kin`, on the device."""
        return self._abi.pwa_compute_amplitudes(self.ctx, waves, kin, out)

    def build_norm(self):
        """Build M on the device; returns a host copy ([N, N] complex128),
        also kept as self.M (the fit drivers scale their variables by it)."""
        self.M = self._abi.pwa_build_norm(self.ctx, self.n_waves)
        return self.M

    def set_form(self, form):
        self._abi.pwa_set_form(self.ctx, form)

    def nll(self, V):
        nll, self.last_status = self._abi.pwa_nll(self.ctx, V)
        return nll

    def nll_grad(self, V):
        """NLL and Wirtinger gradient for V ([K, N] or [N] complex, host):
        (nll [K], grad [K, N]). The call goes through buffers kept per K, whose
        addresses are computed once (taking an array's address costs about
        1 us in Python, against a ~40 us evaluation)."""
        V = np.asarray(V)
        K = V.shape[0] if V.ndim == 2 else 1
        buf = self._bufs.get(K)
        if buf is None:
            Vb = np.empty((K, self.n_waves), dtype=np.complex128)
            nb = np.empty(K)
            gb = np.empty((K, self.n_waves), dtype=np.complex128)
            buf = self._bufs[K] = (Vb, nb, gb, Vb.ctypes.data, nb.ctypes.data, gb.ctypes.data)
        Vb, nb, gb, aV, an, ag = buf
        np.copyto(Vb, V.reshape(K, -1))
        self.last_status = self._abi.pwa_nll_grad_raw(self.ctx, aV, K, an, ag)
        return nb.copy(), gb.copy()

    def hessian(self, V):
        """FUMILI's approximation of the NLL Hessian over p = (Re V, Im V),
        sum_i grad ln I_i grad ln I_i^T: [2N, 2N] float64 (singular along the
        global phase direction)."""
        H, self.last_status = self._abi.pwa_hessian(self.ctx, V, self.n_waves)
        return H

    def hessian_async(self, d_V, d_H):
        """Enqueue the Hessian with device tensors (see pwa_hessian_async)."""
        self._abi.pwa_hessian_async(self.ctx, d_V, d_H)

    def mc_weights(self, V, out=None):
        """I(Omega_j) / n_mc_gen per accepted MC event, float32 (into `out`, a
        numpy array or CUDA tensor, when given)."""
        if out is None:
            out = np.empty(self.n_mc, dtype=np.float32)
        return self._abi.pwa_mc_weights(self.ctx, V, out)

    def fit_fractions(self, V):
        """[N, N]: Re(conj(V_a) M_ab V_b) / V^H M V (diagonal: wave fractions)."""
        return self._abi.pwa_fit_fractions(self.ctx, V, self.n_waves)

    def load_resonance_events(self, wl):
        """Samples for free masses and widths (a synth.ResonanceWorkload or any
        object with the same fields: n_free, m_data, Y_data, Afix_data, m_mc,
        Y_mc, Afix_mc, n_gen)."""
        afd = wl.Afix_data if wl.Afix_data.shape[1] else None
        afm = wl.Afix_mc if wl.Afix_mc.shape[1] else None
        self._abi.pwa_load_resonance_events(self.ctx, wl.n_free, wl.m_data, wl.Y_data, afd,
                                            wl.m_mc, wl.Y_mc, afm, wl.n_gen)
        self.n_free = wl.n_free
        self.n_data_res = len(wl.m_data)
        return self

    def nll_grad_res(self, V, mass, width):
        """(nll, dNLL/dV* [N] complex, dNLL/dM [R], dNLL/dGamma [R])."""
        nll, gV, gM, gW, self.last_status = self._abi.pwa_nll_grad_res(self.ctx, V, mass, width)
        return nll, gV, gM, gW

    def nll_grad_res_async(self, d_V, d_mass, d_width, d_out):
        """Enqueue the free-resonance evaluation with device tensors (see
        pwa_nll_grad_res_async); results in d_out after sync()."""
        self._abi.pwa_nll_grad_res_async(self.ctx, d_V, d_mass, d_width, d_out)

    def autotune(self, cache_path=None):
        """Pick the fastest launch variants on the loaded sample (see
        pwa_autotune); returns a one-line summary of the choices."""
        return self._abi.pwa_autotune(self.ctx, cache_path)

    def nll_grad_async(self, d_V, d_nll, d_grad=None):
        self._abi.pwa_nll_grad_async(self.ctx, d_V, d_V.shape[0], d_nll, d_grad)

    def sync(self):
        self.last_status = self._abi.pwa_sync(self.ctx)
        return self.last_status

    def close(self):
        if self.ctx is not None:
            self._abi.pwa_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ModelBatch:
    """Several trial models, each with its own waves and samples, evaluated
    for K parameter sets per model in one graph launch (tensor-core form)."""

    def __init__(self, n_waves, max_k, device=0, precision=PWA_PREC_DEFAULT, stream=None):
        from . import _abi
        self._abi = _abi
        self.n_waves = list(n_waves)
        self.max_k = max_k
        self.b = _abi.pwa_batch_create(device, self.n_waves, max_k, precision, stream)
        self.last_status = PWA_OK

    def load_model(self, m, data_amp, mc_amp, n_mc_gen):
        self._abi.pwa_batch_load_model(self.b, m, data_amp, mc_amp, n_mc_gen)

    def autotune(self, cache_path=None):
        """Time the batch's launch shapes (work items per SM, X stages) and
        apply the fastest (pwa_batch_autotune); returns a one-line summary."""
        return self._abi.pwa_batch_autotune(self.b, cache_path)

    def nll_grad(self, Vs):
        """Vs: list over models of [K, n_waves[m]] complex arrays. Returns
        (nll [n_models, K], list of [K, n_waves[m]] gradients)."""
        K = Vs[0].shape[0]
        flat = np.concatenate([np.asarray(V, dtype=np.complex128).reshape(-1) for V in Vs])
        nll, g, self.last_status = self._abi.pwa_batch_nll_grad(self.b, flat, K, len(self.n_waves))
        out, o = [], 0
        for n in self.n_waves:
            out.append(g[o:o + K * n].reshape(K, n))
            o += K * n
        return nll, out

    def close(self):
        if self.b is not None:
            self._abi.pwa_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
