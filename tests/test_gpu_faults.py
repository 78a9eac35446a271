"""Error paths under host-side fault injection: PWA_FAULT=alloc:n makes the
n-th device allocation of the process fail (the failure is injected before
the allocation, so no GPU state is touched by it). For every n up to the
number of allocations a short session makes (create, load, M, NLL and
gradient, Hessian), the call that allocates reports PWA_ENOMEM with a
message, nothing crashes, and repeating the session in the same process
(the counter has passed n) gives the same results as a run without faults.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SESSION = r'''
import json, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_1108_5673_gb300 as pwa
import synth

wl = synth.mixture_workload("f", synth.waves_linear(8), 3000, 2000, seed_data=1, seed_mc=2,
                            seed_v=3)
V = synth.random_V(8, 4)


def session():
    with pwa.Likelihood(8) as L:
        L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
        L.build_norm()
        nll, g = L.nll_grad(V[None, :])
        H = L.hessian(V)
    return [float(nll[0])] + [float(x) for x in g[0].view(np.float64)] + [float(H[0, 0])]


out = {"errors": []}
for attempt in range(2):
    try:
        out["values"] = session()
        break
    except pwa.PwaError as e:
        out["errors"].append([e.code, str(e)])
print(json.dumps(out))
'''


def run(fault):
    env = dict(os.environ)
    env.pop("PWA_FAULT", None)
    if fault:
        env["PWA_FAULT"] = fault
    r = subprocess.run([sys.executable, "-c", SESSION, ROOT], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, (fault, r.stderr[-3000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    __graft_entry__.build()


def test_allocation_failures_reported_and_recoverable(built):
    from paper_1108_5673_gb300 import _abi
    clean = run(None)
    assert not clean["errors"] and len(clean["values"]) == 1 + 16 + 1
    failed = 0
    for n in range(1, 25):
        out = run("alloc:%d" % n)
        assert out.get("values") == clean["values"], (n, out)
        if not out["errors"]:
            break   # past the session's allocations
        assert len(out["errors"]) == 1, (n, out)
        code, msg = out["errors"][0]
        assert code == _abi.PWA_ENOMEM and "ENOMEM" in msg, (n, out)
        failed += 1
    assert failed >= 3


def test_bounded_wait_runs_out_and_context_recovers(built):
    """The device-side waits are bounded: with PWA_TEST_TIMEOUT_NS the
    direct-form producer issues no copies, so every consumer's wait for its
    first tile runs out (after 1 ms) with nothing in flight. The call reports
    PWA_ETIMEOUT (host call and async call with pwa_sync), the NLL is NaN and
    the gradient zero; the next normal call on the same context gives the
    results of a call made before."""
    import numpy as np
    import torch
    import paper_1108_5673_gb300 as pwa
    import synth
    from paper_1108_5673_gb300 import _abi

    wl = synth.mixture_workload("t", synth.waves_linear(12), 50_000, 20_000, seed_data=8,
                                seed_mc=9, seed_v=10)
    V = synth.random_V(12, 11)
    old = os.environ.pop("PWA_TEST_TIMEOUT_NS", None)
    try:
        with pwa.Likelihood(12) as L:
            L.load_events(wl.A_data, wl.A_mc, wl.n_gen)
            L.build_norm()
            n0, g0 = L.nll_grad(V[None, :])
            dV = torch.from_numpy(V[None, :].copy()).cuda()
            dn = torch.zeros(1, dtype=torch.float64, device="cuda")
            dg = torch.ones(1, 12, dtype=torch.complex128, device="cuda")
            os.environ["PWA_TEST_TIMEOUT_NS"] = "1000000"
            with pytest.raises(pwa.PwaError) as e:
                L.nll_grad(V[None, :])
            assert e.value.code == _abi.PWA_ETIMEOUT
            L.nll_grad_async(dV, dn, dg)
            with pytest.raises(pwa.PwaError) as e:
                L.sync()
            assert e.value.code == _abi.PWA_ETIMEOUT
            assert np.isnan(float(dn.item())) and bool((dg == 0).all())
            del os.environ["PWA_TEST_TIMEOUT_NS"]
            n1, g1 = L.nll_grad(V[None, :])
            assert n1[0] == n0[0] and np.array_equal(g1, g0)
            L.nll_grad_async(dV, dn, dg)
            assert L.sync() == _abi.PWA_OK
            assert float(dn.item()) == n0[0]
    finally:
        os.environ.pop("PWA_TEST_TIMEOUT_NS", None)
        if old is not None:
            os.environ["PWA_TEST_TIMEOUT_NS"] = old
