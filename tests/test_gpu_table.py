"""GPU parity of the precomputed-table form (Sec. 2, after Eq. 3).

The table is stored in single precision, each entry the float nearest to its
exact value. The oracle builds the same table (exact products of the float
amplitudes in FP64, each entry rounded once to float32) and evaluates Eq. 3
on it in FP64: identical inputs. Tolerances as for the direct form. The
table's own rounding moves the NLL away from the amplitude form by an amount
of the same order as the tolerance; that difference is a property of storing
the table in floats, reported but not a kernel error.
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


def nll_tol(n):
    return max(1e-3 * math.sqrt(n / 1e6), 2e-6)


def float_table(A):
    """The oracle's table of the float amplitudes, each entry rounded to float32."""
    return oracle.table(A).astype(np.float32).astype(np.float64)


def run_both(pwa, wl, Vs):
    N = wl.A_data.shape[1]
    out = {}
    with pwa.Likelihood(N, forms=pwa.PWA_FORM_AMP | pwa.PWA_FORM_TABLE, max_k=len(Vs)) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        M = L.build_norm()
        out["amp"] = L.nll_grad(np.array(Vs))
        L.set_form(pwa.PWA_FORM_TABLE)
        out["table"] = L.nll_grad(np.array(Vs))
        L.set_form(pwa.PWA_FORM_AMP)
        out["amp2"] = L.nll_grad(np.array(Vs))
    return M, out


@pytest.mark.parametrize("N", [1, 3, 4, 8, 13, 17, 20, 24])
def test_table_form_against_oracle(pwa, N):
    wl = synth.mixture_workload("t", synth.waves_linear(N), 5000, 4000, seed_data=N, seed_mc=N + 1)
    Vs = [synth.random_V(N, 3 + N), synth.random_V(N, 4 + N) * 10]
    M, out = run_both(pwa, wl, Vs)
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    T32 = float_table(wl.A_data)
    nt, gt = out["table"]
    for k, V in enumerate(Vs):
        no, go, _ = oracle.nll_table(T32, Mo, V)
        gd = go - oracle.norm_term(Mo, V)[1]
        assert abs(nt[k] - no) <= nll_tol(len(wl.A_data)), (k, nt[k] - no)
        assert np.linalg.norm(gt[k] - go) <= 1e-5 * np.linalg.norm(gd)
        assert np.all(np.abs(gt[k] - go) <= 1e-5 * term_scale(wl.A_data, V, table=True))
    # switching forms back and forth leaves the direct form unchanged
    assert np.array_equal(out["amp"][0], out["amp2"][0])


@pytest.mark.parametrize("n_data", [1, 31, 33, 1000, 100_003])
def test_table_form_ragged_counts(pwa, n_data):
    N = 20
    wl = synth.mixture_workload("t", synth.waves_linear(N), n_data, 700, seed_data=n_data)
    V = synth.random_V(N, 9)
    M, out = run_both(pwa, wl, [V])
    Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    no, go, _ = oracle.nll_table(float_table(wl.A_data), Mo, V)
    assert abs(out["table"][0][0] - no) <= nll_tol(n_data)


@pytest.mark.slow
def test_table_form_one_million_events(pwa):
    wl = synth.paper_scale(n_mc_acc=1_000_000)
    V = synth.start_points(20, 2)
    M, out = run_both(pwa, wl, list(V))
    Mo = oracle.norm_matrix_blas(wl.A_mc, wl.n_gen)
    T32 = float_table(wl.A_data)
    for k in range(2):
        no, go, _ = oracle.nll_table(T32, Mo, V[k])
        gd = go - oracle.norm_term(Mo, V[k])[1]
        assert abs(out["table"][0][k] - no) <= 1e-3
        assert np.linalg.norm(out["table"][1][k] - go) <= 1e-5 * np.linalg.norm(gd)
        assert np.all(np.abs(out["table"][1][k] - go) <= 1e-5 * term_scale(wl.A_data, V[k], table=True))


def test_table_form_limits(pwa):
    from paper_1108_5673_gb300 import _abi
    with pytest.raises(_abi.PwaError) as e:
        pwa.Likelihood(25, forms=pwa.PWA_FORM_TABLE)
    assert e.value.code == _abi.PWA_ENOTSUP
    with pwa.Likelihood(4) as L:                      # table not requested
        with pytest.raises(_abi.PwaError):
            L.set_form(pwa.PWA_FORM_TABLE)
