"""The per-component gradient scale of grad_bound against the oracle: c_a
bounds |g_data,a| (triangle inequality), equals it for one event, and the
table scale bounds c_a."""
import numpy as np

import oracle
import synth
from grad_bound import term_scale


def test_term_scale_bounds_the_data_gradient():
    wl = synth.mixture_workload("g", synth.waves_linear(6), 500, 800, seed_data=1, seed_mc=2)
    V = synth.random_V(6, 3)
    M = oracle.norm_matrix(wl.A_mc, wl.n_gen)
    _, g, _ = oracle.nll_amp(wl.A_data, M, V)
    gd = g - oracle.norm_term(M, V)[1]
    c, ct = term_scale(wl.A_data, V), term_scale(wl.A_data, V, table=True)
    assert np.all(np.abs(gd) <= c * (1 + 1e-12))
    assert np.all(c <= ct * (1 + 1e-12))
    _, g1, _ = oracle.nll_amp(wl.A_data[:1], M, V)
    assert np.allclose(np.abs(g1 - oracle.norm_term(M, V)[1]), term_scale(wl.A_data[:1], V),
                       rtol=1e-12, atol=0)


def test_term_scale_incoherent():
    wl = synth.incoherent_workload("g", synth.waves_linear(5), 300, 400, n_lambda=3)
    V = synth.random_V(5, 4)
    M = oracle.norm_matrix_incoh(wl.A_mc, wl.n_gen)
    _, g, _ = oracle.nll_incoh(wl.A_data, M, V)
    gd = g - oracle.norm_term(M, V)[1]
    assert np.all(np.abs(gd) <= term_scale(wl.A_data, V) * (1 + 1e-12))
