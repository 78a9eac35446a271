"""GPU parity of the uneven model batch (several trial models, each with its
own waves and samples, K parameter sets each).

Two forms of the batch: one launch over work items of every model (the
default; each item a contiguous range of one model's tiles) and, with
PWA_BATCH_MODE=graph, a graph of per-model launches. Every model's results
agree with the FP64 oracle on the block-floating-point inputs the tensor-
core form consumes, within that form's bound (see test_gpu_batched), and with
the same model evaluated alone in a tensor-core context: bit for bit in the
graph form (the same kernels on the same inputs), and in the one-launch form
up to the order of the FP32 sums of G over tiles (the log sums are exact
integer sums in both): NLL to 1e-12 relative, gradient to 1e-6 of its norm.
Each form is bitwise reproducible from call to call.
"""
import os

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


def batch(pwa, n_waves, K, mode):
    old = os.environ.pop("PWA_BATCH_MODE", None)
    if mode == "graph":
        os.environ["PWA_BATCH_MODE"] = "graph"
    try:
        return pwa.ModelBatch(n_waves, K)
    finally:
        os.environ.pop("PWA_BATCH_MODE", None)
        if old is not None:
            os.environ["PWA_BATCH_MODE"] = old


@pytest.mark.parametrize("mode", ["items", "graph"])
def test_batch_matches_single_and_oracle(pwa, mode):
    wls = models(SPEC)
    K = 16
    Vs = [synth.start_points(len(w.waves), K, seed=40 + j) for j, w in enumerate(wls)]
    with batch(pwa, [len(w.waves) for w in wls], K, mode) as B:
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
        if mode == "graph":
            assert np.array_equal(n1, nll[j]), j
            assert np.array_equal(g1, g[j]), j
        else:
            assert np.max(np.abs(n1 - nll[j]) / np.abs(n1)) <= 1e-12, j
            assert np.linalg.norm(g1 - g[j]) <= 1e-6 * np.linalg.norm(g1), j
        Ap = bfp_amplitudes(w.A_data, 2)
        Mo = oracle.norm_matrix(w.A_mc, w.n_gen)
        for k in (0, K - 1):
            no, go, bad = oracle.nll_amp(Ap, Mo, Vs[j][k])
            gd = go - oracle.norm_term(Mo, Vs[j][k])[1]
            assert abs(nll[j][k] - no) <= nll_tol(len(w.A_data)), (j, k, nll[j][k] - no)
            assert np.linalg.norm(g[j][k] - go) / np.linalg.norm(gd) <= GRAD_TOL


@pytest.mark.parametrize("mode", ["items", "graph"])
def test_batch_k_change_and_domain(pwa, mode):
    """A different K rebuilds the graph; a zero parameter set in one model is
    flagged (EDOMAIN, nll = +inf) without touching the others."""
    wls = models([(10, 1000), (16, 1200)], seed=7)
    with batch(pwa, [10, 16], 32, mode) as B:
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


@pytest.mark.slow
def test_batch_bench_configuration(pwa):
    """The model batch as the bench runs it: 64 models (8..48 waves,
    100k..2M events each, MC twice the data, 63.4M data events in all, the
    device generator), 16 sets per model, one launch over work items. Three
    models checked against the oracle on their BFP16 inputs (the one with
    the most waves, the one with the most events, the first), two sets
    each: NLL within the tensor-core form's tolerance, the gradient by norm
    and per component."""
    import torch
    from grad_bound import term_scale
    spec = synth.model_batch_spec()
    K = 16
    pick = sorted({int(np.argmax([s[0] for s in spec])), int(np.argmax([s[1] for s in spec])), 0})
    kept = {}
    with pwa.ModelBatch([s[0] for s in spec], K) as B:
        for j, (nw, nd, seed) in enumerate(spec):
            A_d, A_m, n_gen = synth.torch_mixture_workload(synth.waves_linear(nw), nd, 2 * nd, seed)
            B.load_model(j, A_d, A_m, n_gen)
            if j in pick:
                kept[j] = (A_d.cpu().numpy(), A_m.cpu().numpy(), n_gen)
            del A_d, A_m
        torch.cuda.empty_cache()
        Vs = [synth.start_points(s[0], K, seed=s[2] + 7) * 2.0 for s in spec]
        nll, g = B.nll_grad(Vs)
        assert B.last_status == pwa.PWA_OK
    for j in pick:
        A_d, A_m, n_gen = kept[j]
        Ap = bfp_amplitudes(A_d, 2)
        Mo = oracle.norm_matrix_blas(A_m, n_gen)
        for k in (0, K - 1):
            no, go, bad = oracle.nll_amp(Ap, Mo, Vs[j][k])
            assert bad == 0
            gd = go - oracle.norm_term(Mo, Vs[j][k])[1]
            assert abs(nll[j][k] - no) <= nll_tol(len(A_d)), (j, k, nll[j][k] - no)
            assert np.linalg.norm(g[j][k] - go) <= GRAD_TOL * np.linalg.norm(gd), (j, k)
            assert np.all(np.abs(g[j][k] - go) <= 3e-3 * term_scale(Ap, Vs[j][k])), (j, k)
