"""A model of the tensor-core form's barrier protocol (k_batched.cu), run
under random schedules on the CPU.

Actors: the TMA producer (x_full / x_empty per stage), the MMA thread
(GEMM 1 per half step into the one S accumulator; GEMM 2 per chunk step from
R', issued as soon as r_full completes while it waits for its other
barriers, and never more than one chunk step late: GEMM 1 of the first half
of chunk step cq waits until the GEMM 2 of cq - 2 is issued), and 16 epilogue
warps (read S, free it, compute, wait r_free before writing the first half of
a chunk step's R', arrive r_full after the last half). Tensor operations
complete in issue order; a commit arrives when every earlier operation of
the thread has completed. Barriers follow the mbarrier parity rule: a wait
for parity P passes when the current phase's parity is not P.

The model asserts the data hazards themselves, not the barriers: S is read
before GEMM 1 overwrites it, R' is complete when GEMM 2 reads it and not
overwritten before GEMM 2 has finished, an X stage is not refilled before the
GEMM 2 that reads it has finished, and every run ends (no deadlock).
"""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count, self.arr, self.C = count, 0, 0

    def arrive(self, n=1):
        self.arr += n
        assert self.arr <= self.count, "more arrivals than the phase expects"
        if self.arr == self.count:
            self.arr, self.C = 0, self.C + 1

    def passes(self, parity):
        return parity != (self.C & 1)


def simulate(HPT, NCH, n_tiles, NXS, seed, lag_rule=True, epilogue_waits_r_free=True):
    rnd = random.Random(seed)
    x_full = [Bar(1) for _ in range(NXS)]
    x_empty = [Bar(1) for _ in range(NXS)]
    s_full, s_free, r_full, r_free, g_done = Bar(1), Bar(16), Bar(16), Bar(1), Bar(1)
    steps = n_tiles * HPT
    ops = []                                   # in-flight tensor operations, in order
    st = {"S": None, "read": {}, "g2_done": set(), "r_rows": {}, "x": {}}

    def retire():
        kind, arg = ops.pop(0)
        if kind == "g1":
            assert st["read"].get(arg - 1, 0) == 16 or arg == 0, "S overwritten before it was read"
            st["S"] = arg
        elif kind == "g2":
            j = arg // NCH
            assert st["x"].get(j % NXS) == j, "X stage refilled before GEMM 2 read it"
            st["g2_done"].add(arg)
        else:
            arg.arrive()

    def producer():
        for j in range(n_tiles):
            s, u = j % NXS, j // NXS
            while u > 0 and not x_empty[s].passes((u & 1) ^ 1):
                yield
            st["x"][s] = j
            x_full[s].arrive()
            yield

    def mma():
        g2, ready = [0], [0]

        def gemm2(cq):
            c = cq % NCH
            halves = 2 if 2 * c + 1 < HPT else 1
            assert st["r_rows"].get(cq, 0) == 16 * halves, "GEMM 2 on an incomplete R'"
            ops.extend([("g2", cq), ("commit", r_free)])
            if c == NCH - 1:
                ops.append(("commit", x_empty[(cq // NCH) % NXS]))

        def serve(bar, parity, need):
            while True:
                if g2[0] < ready[0] and r_full.passes(g2[0] & 1):
                    gemm2(g2[0])
                    g2[0] += 1
                    yield
                    continue
                if g2[0] >= need and (bar is None or bar.passes(parity)):
                    return
                yield

        for q in range(steps):
            j, ch = divmod(q, HPT)
            c, h = ch >> 1, ch & 1
            need = j * NCH + c - 1 if (h == 0 and lag_rule) else 0
            if ch == 0:
                yield from serve(x_full[j % NXS], (j // NXS) & 1, need)
            if q >= 1:
                yield from serve(s_free, (q - 1) & 1, need)
            assert st["x"].get(j % NXS) == j
            ops.extend([("g1", q), ("commit", s_full)])
            if h == 1 or ch == HPT - 1:
                ready[0] = j * NCH + c + 1
            yield
        yield from serve(None, 0, ready[0])
        ops.append(("commit", g_done))

    def warp():
        for q in range(steps):
            j, ch = divmod(q, HPT)
            h, cq = ch & 1, j * NCH + (ch >> 1)
            while not s_full.passes(q & 1):
                yield
            assert st["S"] == q, "S does not hold this step"
            yield
            st["read"][q] = st["read"].get(q, 0) + 1
            s_free.arrive()
            for _ in range(rnd.randint(0, 6)):
                yield
            if epilogue_waits_r_free and h == 0 and cq >= 1:
                while not r_free.passes((cq - 1) & 1):
                    yield
            assert cq == 0 or (cq - 1) in st["g2_done"], "R' overwritten before GEMM 2 finished"
            st["r_rows"][cq] = st["r_rows"].get(cq, 0) + 1
            if h == 1 or ch == HPT - 1:
                r_full.arrive()
            yield

    alive = [producer(), mma()] + [warp() for _ in range(16)]
    for _ in range(3_000_000):
        if not alive and not ops:
            break
        if ops and (not alive or rnd.random() < 0.3):
            retire()
            continue
        a = rnd.choice(alive)
        try:
            next(a)
        except StopIteration:
            alive.remove(a)
    else:
        raise RuntimeError("deadlock")
    assert g_done.C == 1


def configs(n, seed0=0):
    for seed in range(seed0, seed0 + n):
        r = random.Random(seed)
        HPT = r.choice([1, 2, 3, 4, 5, 6, 7, 8])
        yield HPT, (HPT + 1) // 2, r.choice([0, 1, 2, 3, 5, 9, 17]), r.choice([2, 3, 4, 6]), seed


@pytest.mark.parametrize("lag_rule", [True, False])
def test_protocol_has_no_hazard(lag_rule):
    for HPT, NCH, n_tiles, NXS, seed in configs(150):
        simulate(HPT, NCH, n_tiles, NXS, seed, lag_rule=lag_rule)


def test_model_catches_a_missing_wait():
    """Planted mistake: without the epilogue's r_free wait, R' is overwritten
    while GEMM 2 still needs it, in some schedule."""
    caught = 0
    for HPT, NCH, n_tiles, NXS, seed in configs(150, seed0=1000):
        try:
            simulate(HPT, NCH, n_tiles, NXS, seed, epilogue_waits_r_free=False)
        except AssertionError:
            caught += 1
    assert caught > 0
