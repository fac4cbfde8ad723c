"""Pins for the CPU oracle of MAP (Section 2 of the paper), independent of the oracle itself.

* hand-derived cases (tests/golden/hand_cases.json), each worked out from the definition;
* brute force on small random graphs: every map from explicit reachability, the round count
  and the relaxation count from their closed forms over shortest-path distances, the outer
  loop replayed from those maps;
* the verdict against strongly connected components (scipy);
* invariants: eliminated vertices never lie on an accepting cycle, a witness lies on one;
* the known answers of the planted workloads.
"""
import json
import os

import numpy as np
import pytest

import mapgen
import oracle
from tests import _brute as bf

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = json.load(open(os.path.join(HERE, "golden", "hand_cases.json")))["cases"]


def _u32(vals):
    return np.array([oracle.NONE if x is None else x for x in vals], dtype=np.uint32)


@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_cases(case):
    g = mapgen.from_lists(case["rows"], case["acc"])
    r = oracle.run_graph(g, keep_trace=True)
    assert r.status == oracle.OK
    assert r.verdict == case["verdict"]
    assert r.witness == (oracle.NONE if case["witness"] is None else case["witness"])
    assert r.outer == case["outer"]
    assert r.rounds == case["rounds"]
    assert np.array_equal(r.map, _u32(case["final_map"]))
    assert len(r.trace) == len(case["maps"])
    for (outer, mp, k), want, kk in zip(r.trace, case["maps"], case["rounds"]):
        assert np.array_equal(mp, _u32(want))
        assert k == kk


def _check_against_brute(g):
    r = oracle.run_graph(g, keep_trace=True)
    assert r.status == oracle.OK
    verdict, witness, outer, rounds, maps, relax = bf.brute_map_run(g.n, g.rowptr, g.colidx, g.acc)
    assert r.verdict == verdict
    assert r.witness == (oracle.NONE if witness is None else witness)
    assert r.outer == outer
    assert r.rounds == rounds
    assert r.relaxations == relax
    assert r.inner_total == sum(rounds)
    assert len(r.trace) == len(maps)
    for (_, mp, _), want in zip(r.trace, maps):
        assert np.array_equal(mp, want)
    has_cycle, on_cycle = bf.tarjan_verdict(g.n, g.rowptr, g.colidx, g.acc)
    assert (r.verdict == oracle.CYCLE) == has_cycle
    if r.verdict == oracle.CYCLE:
        assert g.acc[r.witness] and on_cycle[r.witness]
    # eliminated vertices (map values of non-final iterations) never lie on an accepting cycle
    for _, mp, _ in r.trace[:-1] if r.verdict == oracle.CYCLE else r.trace:
        E = np.unique(mp[mp != oracle.NONE])
        assert not np.any(on_cycle[E])
    return r


@pytest.mark.parametrize("seed", range(160))
def test_random_small_vs_brute_force(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 40))
    g = mapgen.tiny_graph(seed, n, max_deg=int(rng.integers(0, 5)), acc_p=float(rng.choice([0.0, 0.1, 0.3, 0.7, 1.0])))
    _check_against_brute(g)


@pytest.mark.parametrize("seed", range(12))
def test_acyclic_many_outer_vs_brute_force(seed):
    """DAG-shaped graphs (edges only to larger ids... and smaller): many outer iterations."""
    rng = np.random.default_rng(seed)
    n = 60
    rows = [sorted(set(int(x) for x in rng.integers(v + 1, n, size=int(rng.integers(0, 4))))) if v + 1 < n else []
            for v in range(n)]
    acc = (rng.random(n) < 0.6).astype(np.uint8)
    r = _check_against_brute(mapgen.from_lists(rows, acc))
    assert r.verdict == oracle.NO_CYCLE


def test_outer_bound_and_monotone_accepting_set():
    """outer <= |A0| + 1 and the accepting set only shrinks (each non-final iteration eliminates >= 1)."""
    for seed in range(30):
        g = mapgen.tiny_graph(500 + seed, 30, max_deg=2, acc_p=0.5, self_loops=False)
        r = oracle.run_graph(g, keep_trace=True)
        assert r.outer <= int(g.acc.sum()) + 1
        A = g.acc.astype(bool).copy()
        for outer, mp, _ in r.trace:
            vals = mp[mp != oracle.NONE]
            assert np.all(A[vals])  # every map value is a currently accepting vertex
            A[np.unique(vals)] = False


def test_random_16k_planted_cycle():
    g = mapgen.random_16k("cycle")
    r = oracle.run_graph(g)
    assert r.verdict == oracle.CYCLE
    assert r.witness == g.meta["planted"]
    assert r.outer == 1


def test_random_16k_no_cycle_matches_scc():
    g = mapgen.random_16k("nocycle")
    r = oracle.run_graph(g)
    has_cycle, _ = bf.tarjan_verdict(g.n, g.rowptr, g.colidx, g.acc)
    assert not has_cycle
    assert r.verdict == oracle.NO_CYCLE
    assert r.outer >= 1


def test_layered_small_no_cycle_and_planted():
    g = mapgen.layered_graph(20000, 200, seed=7, D=8)
    r = oracle.run_graph(g)
    assert not bf.tarjan_verdict(g.n, g.rowptr, g.colidx, g.acc)[0]
    assert r.verdict == oracle.NO_CYCLE and r.outer > 3
    gp = mapgen.layered_graph(20000, 200, seed=7, D=8, plant=True)
    rp = oracle.run_graph(gp)
    assert bf.tarjan_verdict(gp.n, gp.rowptr, gp.colidx, gp.acc)[0]
    assert rp.verdict == oracle.CYCLE
    assert gp.acc[rp.witness]


def test_product_small_matches_scc():
    for interleave in (False, True):
        g = mapgen.product_graph(4, 5, interleave)
        r = oracle.run_graph(g)
        assert (r.verdict == oracle.CYCLE) == bf.tarjan_verdict(g.n, g.rowptr, g.colidx, g.acc)[0]


def test_invalid_inputs_rejected():
    ok = mapgen.from_lists([[1], [0]], [1, 0])
    assert oracle.run_graph(ok).status == oracle.OK
    bad_col = np.array([0, 1, 2], np.uint32), np.array([1, 2], np.uint32)
    assert oracle.run(2, bad_col[0], bad_col[1], [1, 0]).status == oracle.ERR_ARG
    bad_rp = np.array([0, 2, 1], np.uint32), np.array([1, 0], np.uint32)
    assert oracle.run(2, bad_rp[0], bad_rp[1], [1, 0]).status == oracle.ERR_ARG
    bad_start = np.array([1, 1, 2], np.uint32), np.array([1, 0], np.uint32)
    assert oracle.run(2, bad_start[0], bad_start[1], [1, 0]).status == oracle.ERR_ARG


def test_outer_limit():
    g = mapgen.from_lists([[1], [2], []], [1, 1, 1])
    r = oracle.run_graph(g, max_outer=2)
    assert r.status == oracle.LIMIT and r.outer == 2


def test_discovery_order_is_a_bfs_numbering():
    """Input plumbing for the on-the-fly tests: a renumbering of the reachable part in which
    breadth-first distance never decreases and every vertex is known before its row is expanded."""
    g = mapgen.random_graph(3000, 1, 4, 0.05, seed=11)
    d, known = mapgen.discovery_order(g, start=5)
    dist = oracle.bfs_dist(g.n, g.rowptr, g.colidx, 5)
    assert d.n == int(np.count_nonzero(dist >= 0))
    dd = oracle.bfs_dist(d.n, d.rowptr, d.colidx, 0)
    assert np.all(np.diff(dd) >= 0) and np.all(dd >= 0)
    assert sorted(np.diff(d.rowptr.astype(np.int64))) == sorted(
        np.diff(g.rowptr.astype(np.int64))[dist >= 0])
    for R in range(d.n + 1):
        top = int(d.colidx[:d.rowptr[R]].max()) + 1 if d.rowptr[R] else 1
        assert known[R] == max(R, 1, top)
    assert known[-1] == d.n
