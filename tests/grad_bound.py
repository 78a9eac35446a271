"""Per-component scale of the data gradient, for bounds beside the norm
checks: c_a = sum_i sum_l |A_a^l(i)| |S_i^l| / I_i, the sum of the absolute
values of the terms of g_a = -sum_i sum_l conj(A_a^l(i)) S_i^l / I_i + (M V)_a.

A rounding of relative size r per term (S, I, S / I, the product with
conj(A), each summation step) moves g_a by at most r c_a, whatever the other
components do, so |dg_a| <= r c_a checks every component on its own scale
(a norm over all components can hide one bad one).
  * FP32 forms: S correctly rounded or nearly (exact product split), S / I
    within a few units of 2^-24, then FP32 sums of up to ~60 terms per thread
    and warp before float-float: r = 60 * 2^-24 = 3.6e-6 in the worst case;
    the tests take 1e-5.
  * Table form (scale with table=True): the table entries rounded once to
    float, the FP32 sums as above: 1e-5.
  * Tensor-core form: R' = S / I rounded once to BF16 per event (both parts,
    2^-9 relative each, so |dR'| <= sqrt2 2^-9 |R'|), the sums exact:
    r = 2.8e-3; the tests take 3e-3.
"""
import numpy as np


def term_scale(A, V, table=False, chunk=1 << 18):
    """c_a for amplitudes A [n, N] (coherent) or [n, L, N] (incoherent), V [N].

    table: the table form's scale. It sums G^[b][a] = sum_i t_i[b][a] / I_i
    over the events and only then contracts with V (in FP64), so its terms
    are |V_b| |A_b| |A_a| / I_i: c_a = sum_i sum_l |A_a^l| (sum_b |V_b|
    |A_b^l|) / I_i, which is c_a with |S_i^l| replaced by its triangle bound."""
    A = np.asarray(A)
    if A.ndim == 2:
        A = A[:, None, :]
    V = np.asarray(V, dtype=np.complex128)
    c = np.zeros(A.shape[2])
    for s in range(0, A.shape[0], chunk):
        a = A[s:s + chunk].astype(np.complex128)
        S = a @ V                                  # [n, L]
        I = np.sum(np.abs(S) ** 2, axis=1)         # [n]
        T = np.abs(a) @ np.abs(V) if table else np.abs(S)
        w = T / I[:, None]                         # [n, L]
        c += np.einsum("nl,nla->a", w, np.abs(a))
    return c
