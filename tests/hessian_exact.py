"""Exact Hessian of Eq. 3 in the real parameters, for the fit tests (FP64).

NLL(V) = -sum_i ln I_i + V^H M V with I_i = |S_i|^2, S_i = sum_a V_a A_a(i).
Over p = (Re V, Im V), dS_i/dRe V_a = A_a(i) and dS_i/dIm V_a = i A_a(i), so
  d2NLL/dp dq = sum_i J_ip J_iq - sum_i 2 Re(conj(dS_i/dp) dS_i/dq) / I_i
                + 2 Re(conj(u_p)^T M u_q),
with J_ip = d ln I_i / dp = 2 Re(conj(S_i) dS_i/dp) / I_i and u_p = dV/dp:
FUMILI's sum of J J^T (the library's Hessian) less the intensity's second
derivatives plus those of the normalisation term. Pinned in test_fit_cpu.py
by central differences of the oracle's gradient.
"""
import numpy as np


def exact_hessian(A, M, V):
    S = A @ V
    I = (S.conj() * S).real
    w = (S.conj()[:, None] * A) / I[:, None]
    J = np.concatenate([2 * w.real, -2 * w.imag], axis=1)
    C = A.conj().T @ (A / I[:, None])            # sum_i conj(A_a) A_b / I_i
    H2 = np.block([[C.real, -C.imag], [C.imag, C.real]])
    HM = np.block([[M.real, -M.imag], [M.imag, M.real]])
    return J.T @ J - 2 * H2 + 2 * HM
