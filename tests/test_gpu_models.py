"""GPU parity of the uneven model batch (several trial models, each with its
own waves and samples, K parameter sets each, one graph launch).

Every model's results must be bit-identical to the same model evaluated alone
in a tensor-core context (the graph replays the same kernels on the same
inputs), and agree with the FP64 oracle on the block-floating-point inputs the
tensor-core form consumes, within that form's bound (see test_gpu_batched).
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_batched import GRAD_TOL, bfp_amplitudes, nll_tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pwa():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1108_5673_gb300 as pkg
    return pkg


def models(spec, seed=0):
    out = []
    for j, (N, n) in enumerate(spec):
        out.append(synth.mixture_workload("m%d" % j, synth.waves_linear(N), n, 2 * n,
                                          seed_data=1000 + seed + j, seed_mc=2000 + seed + j,
                                          seed_v=3000 + seed + j))
    return out


SPEC = [(8, 3000), (13, 1500), (20, 5000), (32, 2500), (48, 2000), (5, 700)]


def test_batch_matches_single_and_oracle(pwa):
    wls = models(SPEC)
    K = 16
    Vs = [synth.start_points(len(w.waves), K, seed=40 + j) for j, w in enumerate(wls)]
    with pwa.ModelBatch([len(w.waves) for w in wls], K) as B:
        for j, w in enumerate(wls):
            B.load_model(j, w.A_data, w.A_mc, w.n_gen)
        nll, g = B.nll_grad(Vs)
        assert B.last_status == pwa.PWA_OK
        nll2, g2 = B.nll_grad(Vs)           # graph replay
    assert np.array_equal(nll, nll2) and all(np.array_equal(a, b) for a, b in zip(g, g2))
    for j, w in enumerate(wls):
        N = len(w.waves)
        with pwa.Likelihood(N, forms=pwa.PWA_FORM_TC, max_k=K) as L:
            L.load_events(w.A_data, w.A_mc, w.n_gen)
            L.build_norm()
            L.set_form(pwa.PWA_FORM_TC)
            n1, g1 = L.nll_grad(Vs[j])
        assert np.array_equal(n1, nll[j]), j
        assert np.array_equal(g1, g[j]), j
        Ap = bfp_amplitudes(w.A_data, 2)
        Mo = oracle.norm_matrix(w.A_mc, w.n_gen)
        for k in (0, K - 1):
            no, go, bad = oracle.nll_amp(Ap, Mo, Vs[j][k])
            gd = go - oracle.norm_term(Mo, Vs[j][k])[1]
            assert abs(nll[j][k] - no) <= nll_tol(len(w.A_data)), (j, k, nll[j][k] - no)
            assert np.linalg.norm(g[j][k] - go) / np.linalg.norm(gd) <= GRAD_TOL


def test_batch_k_change_and_domain(pwa):
    """A different K rebuilds the graph; a zero parameter set in one model is
    flagged (EDOMAIN, nll = +inf) without touching the others."""
    wls = models([(10, 1000), (16, 1200)], seed=7)
    with pwa.ModelBatch([10, 16], 32) as B:
        for j, w in enumerate(wls):
            B.load_model(j, w.A_data, w.A_mc, w.n_gen)
        for K in (4, 32, 4):
            Vs = [synth.start_points(10, K, seed=1), synth.start_points(16, K, seed=2)]
            Vs[1][K - 1] = 0
            nll, g = B.nll_grad(Vs)
            assert B.last_status == pwa.PWA_EDOMAIN
            assert np.isinf(nll[1][K - 1]) and not np.any(g[1][K - 1])
            assert np.all(np.isfinite(nll[0])) and np.all(np.isfinite(nll[1][:K - 1]))


def test_batch_errors(pwa):
    from paper_1108_5673_gb300._abi import PwaError
    with pytest.raises(PwaError):
        pwa.ModelBatch([8, 49], 16)        # too many waves
    with pytest.raises(PwaError):
        pwa.ModelBatch([48], 1000)          # K beyond the tensor-core limit
    with pwa.ModelBatch([8, 8], 16) as B:
        w = models([(8, 500)])[0]
        B.load_model(0, w.A_data, w.A_mc, w.n_gen)
        with pytest.raises(PwaError):       # model 1 not loaded
            B.nll_grad([synth.start_points(8, 16), synth.start_points(8, 16)])
