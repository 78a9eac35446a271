"""The direct-form kernel's shared-memory ring under reuse: every stage
filled and released many times, in each of its shapes.

With one CTA per SM, the parity tests' samples give a CTA one tile or a few,
so a stage is used once and its barriers never change phase. Here a child
process forces a grid of three CTAs (PWA_AMP_GRID, read once per process)
and the consumer groups per CTA (PWA_AMP_GROUPS), so that each CTA streams
26 to 35 tiles through its ring (256-event tiles below 40 waves, 192-event
ones from 40 waves on and for several components). The cases cover the
ring's shapes:
  * owned stages (two or more per consumer group; tile j to group j % G and
    its stage (j / G) % SPG): 4, 12, 13, 20 and 24 waves with two groups,
    4 and 12 waves with three, incoherent 5 waves x 4 components;
  * shared stages with as many stages as groups: 48 waves with two groups,
    20 and 32 waves with three, incoherent 16 x 3 and 12 x 4;
  * shared stages with more stages than groups (a stage used by different
    groups in turn, two full barriers per stage): 32 and 40 waves with two
    groups, incoherent 20 x 2 and 12 x 3 (three stages each).
Each result against the FP64 oracle with the direct form's tolerances:
|dNLL| <= 1e-3 sqrt(n / 1e6) (floor 2e-6), ||dg|| / ||g_data|| <= 1e-5, and
|dg_a| <= 1e-5 c_a per component (grad_bound.py). The event counts leave a
ragged last tile.
"""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from grad_bound import term_scale

pytestmark = pytest.mark.gpu

GRID = 3
N_DATA, N_MC = 20_011, 3_000
# (waves, components, consumer groups)
CASES = [(4, 1, 2), (12, 1, 2), (13, 1, 2), (20, 1, 2), (24, 1, 2), (32, 1, 2), (40, 1, 2), (48, 1, 2),
         (4, 1, 3), (12, 1, 3), (20, 1, 3), (32, 1, 3),
         (20, 2, 2), (12, 3, 2), (16, 3, 2), (5, 4, 2), (12, 4, 2)]
HERE = os.path.dirname(os.path.abspath(__file__))


def workload(N, L):
    seed = 31 * N + L
    if L == 1:
        return synth.mixture_workload("ring", synth.waves_linear(N), N_DATA, N_MC,
                                      seed_data=100 + seed, seed_mc=200 + seed, seed_v=300 + seed)
    return synth.incoherent_workload("ring", synth.waves_linear(N), N_DATA, N_MC, n_lambda=L,
                                     seed_data=700 + seed, seed_mc=800 + seed, seed_v=900 + seed)


def parameter_sets(wl, N):
    return np.array([wl.V_true, synth.random_V(N, 17 + N)])


def key(N, L, G):
    return "n%d_l%d_g%d" % (N, L, G)


def child(path, groups):
    """Runs in the child process: evaluates the cases of this group count."""
    import paper_1108_5673_gb300 as pwa
    out = {}
    for N, L, G in CASES:
        if G != groups:
            continue
        wl = workload(N, L)
        Vs = parameter_sets(wl, N)
        with pwa.Likelihood(N, max_k=len(Vs)) as lk:
            lk.load_events(wl.A_data, wl.A_mc, wl.n_gen)
            out[key(N, L, G) + "_M"] = lk.build_norm()
            nll, g = lk.nll_grad(Vs)
            out[key(N, L, G) + "_status"] = np.array(lk.last_status)
        out[key(N, L, G) + "_nll"] = nll
        out[key(N, L, G) + "_g"] = g
    np.savez(path, **out)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("groups", [2, 3])
def test_ring_reuse_against_oracle(built, tmp_path, groups):
    path = str(tmp_path / "ring.npz")
    env = dict(os.environ, PWA_AMP_GRID=str(GRID), PWA_AMP_GROUPS=str(groups),
               PYTHONPATH=os.pathsep.join([os.path.dirname(HERE), HERE,
                                           os.environ.get("PYTHONPATH", "")]))
    env.pop("PWA_INCOH_KERNEL", None)
    r = subprocess.run([sys.executable, "-c",
                        "import test_gpu_ring as t; t.child(%r, %d)" % (path, groups)],
                       env=env, cwd=HERE, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    res = np.load(path)
    n = N_DATA
    tol = max(1e-3 * math.sqrt(n / 1e6), 2e-6)
    checked = 0
    for N, L, G in CASES:
        if G != groups:
            continue
        k = key(N, L, G)
        wl = workload(N, L)
        Vs = parameter_sets(wl, N)
        assert int(res[k + "_status"]) == 0, k
        if L == 1:
            Mo = oracle.norm_matrix(wl.A_mc, wl.n_gen)
        else:
            Mo = oracle.norm_matrix_incoh(wl.A_mc, wl.n_gen)
        assert np.max(np.abs(res[k + "_M"] - Mo)) <= 1e-12 * np.abs(Mo).max(), k
        for s, V in enumerate(Vs):
            if L == 1:
                no, go, bad = oracle.nll_amp(wl.A_data, Mo, V)
            else:
                no, go, bad = oracle.nll_incoh(wl.A_data, Mo, V)
            assert bad == 0
            gd = go - oracle.norm_term(Mo, V)[1]
            nll, g = res[k + "_nll"][s], res[k + "_g"][s]
            assert abs(nll - no) <= tol, (k, s, nll - no)
            assert np.linalg.norm(g - go) / np.linalg.norm(gd) <= 1e-5, (k, s)
            c = term_scale(wl.A_data, V)
            assert np.all(np.abs(g - go) <= 1e-5 * c), (k, s, np.max(np.abs(g - go) / c))
        checked += 1
    assert checked == sum(1 for c in CASES if c[2] == groups)
