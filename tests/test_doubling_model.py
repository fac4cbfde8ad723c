"""Reading R11 pinned on the CPU: on a graph whose rows hold one entry at most, exact pointer
doubling reaches the least fix-point of Section 2's propagation.

Written from the recurrence, not from any kernel: with src(v) the one entry of row v,
Q_0 = src and B_0 the dense round's values (the offer of src(v): its id if accepting),
    B_{k+1}(v) = max(B_k(v), B_k(Q_k(v))),   Q_{k+1}(v) = Q_k(Q_k(v)),
stopping after the first pass that changes no B.  The outer loop around it is Section 2's
(self-map test, then elimination of every map value).  Checked against the oracle (every outer
iteration's map, verdict, witness, outer count) and, on small graphs, against brute force: the
round count (the dense round plus the passes) is 2 + ceil(log2 D) for D = max_v d+(v, map(v)) >= 1
(1 with no value at all), never above the synchronous schedule's 1 + D.
"""
import math

import numpy as np
import pytest

import mapgen
import oracle
from tests import _brute

NONE = 0xFFFFFFFF


def functional(n, seed, acc_p, none_p):
    rng = np.random.default_rng(seed)
    succ = rng.integers(0, n, size=n)
    keep = rng.random(n) >= none_p
    rowptr = np.zeros(n + 1, np.uint32)
    np.cumsum(keep, out=rowptr[1:])
    acc = (rng.random(n) < acc_p).astype(np.uint8)
    return mapgen.Graph(n, rowptr, succ[keep].astype(np.uint32), acc)


def successors(g):
    """src(v), or -1 for an empty row."""
    lens = np.diff(g.rowptr.astype(np.int64))
    assert lens.max(initial=0) <= 1
    src = np.full(g.n, -1, np.int64)
    src[lens == 1] = g.colidx.astype(np.int64)
    return src


def doubling_fixpoint(src, accepting):
    """One outer iteration: values encoded u + 1 (0 = none); returns (values, rounds)."""
    n = src.size
    offer = np.where(accepting, np.arange(1, n + 1, dtype=np.int64), 0)
    has = src >= 0
    b = np.zeros(n, np.int64)
    b[has] = offer[src[has]]  # the dense round
    rounds = 1
    if not b.any():
        return b, rounds
    q = src.copy()
    while True:
        rounds += 1
        live = q >= 0
        nb = b.copy()
        nb[live] = np.maximum(b[live], b[q[live]])
        nq = np.full(n, -1, np.int64)
        nq[live] = q[q[live]]
        changed = bool((nb != b).any())
        b, q = nb, nq
        if not changed:
            return b, rounds


def doubling_run(g):
    """Section 2's outer loop with doubling as the fix-point: (verdict, witness, outer, maps, rounds)."""
    src = successors(g)
    accepting = g.acc.astype(bool).copy()
    maps, rounds, outer = [], [], 0
    while accepting.any():
        outer += 1
        b, k = doubling_fixpoint(src, accepting)
        m = np.where(b > 0, b - 1, NONE).astype(np.uint32)
        maps.append(m)
        rounds.append(k)
        self_mapped = np.nonzero(b == np.arange(1, g.n + 1))[0]
        if self_mapped.size:
            return 1, int(self_mapped.min()), outer, maps, rounds
        e = np.unique(b[b > 0] - 1)
        if e.size == 0:
            return 0, NONE, outer, maps, rounds
        accepting[e] = False
    return 0, NONE, outer, maps, rounds


def closed_form_rounds(g, acc_bits):
    """2 + ceil(log2 D) with D = max d+(v, map(v)) over the vertices with a value (1 if none)."""
    dp = _brute.dist_plus(g.n, g.rowptr, g.colidx)
    mp = _brute.map_at_round(dp, acc_bits)
    d = max((int(dp[v, mp[v]]) for v in range(g.n) if mp[v] != NONE), default=0)
    return 1 if d == 0 else 2 + math.ceil(math.log2(d))


@pytest.mark.parametrize("seed", range(40))
def test_doubling_equals_the_oracle(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.choice([1, 2, 3, 17, 200, 3000]))
    g = functional(n, 7000 + seed, acc_p=float(rng.choice([0.02, 0.1, 0.5, 1.0])),
                   none_p=float(rng.choice([0.0, 0.05, 0.4])))
    want = oracle.run_graph(g, keep_trace=True)
    verdict, witness, outer, maps, rounds = doubling_run(g)
    assert (verdict, witness, outer) == (want.verdict, want.witness, want.outer)
    assert len(maps) == len(want.trace)
    for m, (_, wm, wk), k in zip(maps, want.trace, rounds):
        assert np.array_equal(m, wm)
        assert k <= wk  # never above the synchronous rounds


@pytest.mark.parametrize("seed", range(30))
def test_doubling_rounds_closed_form(seed):
    """The first outer iteration's round count from brute-force distances."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 120))
    g = functional(n, 8000 + seed, acc_p=float(rng.choice([0.05, 0.2, 0.6])), none_p=float(rng.choice([0.0, 0.1])))
    src = successors(g)
    _, k = doubling_fixpoint(src, g.acc.astype(bool))
    assert k == closed_form_rounds(g, g.acc.astype(bool))


def test_long_chain_rounds():
    """Row v holds v - 1 and vertex 0 is accepting: D = n - 1, so 2 + ceil(log2(n - 1)) rounds
    against the n synchronous ones."""
    for n in (2, 3, 5, 9, 1000, 4097):
        rows = [[]] + [[u] for u in range(n - 1)]
        acc = np.zeros(n, np.uint8)
        acc[0] = 1
        g = mapgen.from_lists(rows, acc)
        _, k = doubling_fixpoint(successors(g), acc.astype(bool))
        assert k == 2 + math.ceil(math.log2(n - 1))
        assert oracle.run_graph(g).rounds[0] == n
