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
