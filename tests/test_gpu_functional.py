"""Pointer doubling: on a graph whose every row holds at most one entry (the state graph of a
deterministic system, each state with one successor), an asynchronous single-graph run with the
dense start propagates by doubling each vertex's jump pointer along its chain instead of pushing
round after round.  The values are the least fix-point's, so verdict, witness, outer count and the map of
every outer iteration are the oracle's; the pass count per outer iteration is at most the
synchronous schedule's rounds, and on long chains it is about log2 of them.  MAP_FLAG_PUSH keeps
the push rounds, which must agree."""
import numpy as np
import pytest

import mapgen
import oracle
from tests.test_doubling_model import doubling_run

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0912_2555_gb300 as p

    return p


def functional_graph(n, seed, acc_p, none_p=0.0):
    """Each vertex v gets one successor succ(v) (uniform, self-loops allowed), or none with
    probability none_p: every row of the CSR holds at most one entry."""
    rng = np.random.default_rng(seed)
    succ = rng.integers(0, n, size=n)
    keep = rng.random(n) >= none_p
    rowptr = np.zeros(n + 1, np.uint32)
    np.cumsum(keep, out=rowptr[1:])
    colidx = succ[keep].astype(np.uint32)
    acc = (rng.random(n) < acc_p).astype(np.uint8)
    return mapgen.Graph(n, rowptr, colidx, acc, (0,) * 8, f"functional-{n}-{seed}", {})


def chain_graph(n, acc_at):
    """Row v holds v - 1 (v >= 1): a value travels one vertex further per synchronous round;
    the accepting vertices acc_at."""
    rows = [[]] + [[u] for u in range(n - 1)]
    acc = np.zeros(n, np.uint8)
    acc[list(acc_at)] = 1
    return mapgen.from_lists(rows, acc, f"chain-{n}")


def run(pkg, g, sched=1, flags=0, **kw):
    rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
    ci = torch.from_numpy(g.colidx.view(np.int32) if g.m else np.zeros(1, np.int32)).cuda()
    ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
    h = pkg.map_create(g.n, rp, ci, ab, torch.cuda.current_stream())
    try:
        out = np.empty(g.n, np.uint32)
        r = pkg.map_run(h, sched=sched, flags=flags, map_out=out, **kw)
        return r, out
    finally:
        pkg.map_destroy(h)


def same_as_oracle(pkg, r, out, want):
    assert (r.status, r.verdict, r.witness, r.outer) == (pkg.MAP_OK, want.verdict, want.witness, want.outer)
    assert np.array_equal(out, want.map)
    assert all(a <= b for a, b in zip(r.rounds, want.rounds))


@pytest.mark.parametrize("seed", range(12))
def test_random_functional_graphs(pkg, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.choice([1, 2, 7, 300, 5000, 120000]))
    g = functional_graph(n, 500 + seed, acc_p=float(rng.choice([0.0, 0.002, 0.05, 0.5])),
                         none_p=float(rng.choice([0.0, 0.01, 0.3])))
    want = oracle.run_graph(g, keep_trace=True)
    r, out = run(pkg, g)
    same_as_oracle(pkg, r, out, want)
    # the passes are exact doubling steps: the same round count per outer iteration as the
    # recurrence stepped on the CPU (tests/test_doubling_model.py, pinned to brute force)
    if g.acc.any():
        assert list(r.rounds) == doubling_run(g)[4]
    # every outer iteration's map (host-stepped: the same kernels, one launch per step)
    h = pkg.map_create(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc))
    try:
        t = pkg.map_run(h, sched=1, keep_trace=True)
        assert len(t.trace) == want.outer
        for (o1, m1, k1), (o2, m2, k2) in zip(t.trace, want.trace):
            assert np.array_equal(m1, m2), f"map differs at outer iteration {o1}"
            assert k1 <= k2
    finally:
        pkg.map_destroy(h)
    # the push rounds agree
    rp, outp = run(pkg, g, flags=pkg.MAP_FLAG_PUSH)
    same_as_oracle(pkg, rp, outp, want)


def test_long_chain_takes_about_log_passes(pkg):
    """20,000 vertices in a chain with the first one accepting: the synchronous schedule needs
    20,000 rounds; pointer doubling about log2(20,000) + 2 passes."""
    g = chain_graph(20000, [0])
    want = oracle.run_graph(g)
    r, out = run(pkg, g)
    same_as_oracle(pkg, r, out, want)
    assert want.rounds[0] >= 20000
    assert r.rounds[0] <= 20
    rp, outp = run(pkg, g, flags=pkg.MAP_FLAG_PUSH)
    same_as_oracle(pkg, rp, outp, want)
    assert rp.rounds[0] > 100 * r.rounds[0]


def test_chain_with_accepting_vertices_along_it(pkg):
    """Several outer iterations: each eliminates the accepting vertices that are some vertex's
    value; the ones further up the chain win first."""
    g = chain_graph(3000, [5, 700, 701, 2999, 1500])
    want = oracle.run_graph(g, keep_trace=True)
    assert want.outer > 1
    r, out = run(pkg, g)
    same_as_oracle(pkg, r, out, want)


@pytest.mark.parametrize("k,s", [(4, 5), (5, 6), (6, 7)])
def test_deterministic_products(pkg, k, s):
    g = mapgen.product_graph(k, s, interleave=False)
    want = oracle.run_graph(g)
    r, out = run(pkg, g)
    same_as_oracle(pkg, r, out, want)


def test_product_8x7(pkg):
    """The 5.8 M-state synchronous product (11.5 M vertices with the automaton), 930 synchronous
    rounds: the doubling passes are a small fraction of the push sweeps, with the same result."""
    g = mapgen.product_8x7()
    want = oracle.run_graph(g)
    r, out = run(pkg, g)
    same_as_oracle(pkg, r, out, want)
    assert list(r.rounds) == doubling_run(g)[4]
    rp, outp = run(pkg, g, flags=pkg.MAP_FLAG_PUSH)
    same_as_oracle(pkg, rp, outp, want)
    assert r.inner_iters * 5 < rp.inner_iters


def _on_cycle(g, v):
    seen, todo = set(), [int(u) for u in g.colidx[g.rowptr[v]:g.rowptr[v + 1]]]
    while todo:
        u = todo.pop()
        if u == v:
            return True
        if u in seen:
            continue
        seen.add(u)
        todo.extend(int(w) for w in g.colidx[g.rowptr[u]:g.rowptr[u + 1]])
    return False


@pytest.mark.parametrize("seed", range(6))
def test_early_exit_and_limits(pkg, seed):
    g = functional_graph(4000, 900 + seed, acc_p=0.01, none_p=0.05)
    want = oracle.run_graph(g, keep_trace=True)
    r, _ = run(pkg, g, flags=pkg.MAP_FLAG_EARLY_EXIT)
    assert r.verdict == want.verdict
    if r.verdict:
        assert g.acc[r.witness] and _on_cycle(g, r.witness)
    if want.outer >= 1 and max(want.rounds) >= 3:
        r2, _ = run(pkg, g, max_inner=2, allow_limit=True)
        assert r2.status == pkg.MAP_ERR_LIMIT
    r1, out1 = run(pkg, g, max_outer=1, allow_limit=True)
    if want.outer > 1:
        assert r1.status == pkg.MAP_ERR_LIMIT and r1.outer == 1
        assert np.array_equal(out1, want.trace[0][1])


@pytest.mark.parametrize("n,seed", [(5000, 31), (300_001, 32)])
def test_other_schedules_after_doubling_on_one_handle(pkg, n, seed):
    """Pointer doubling keeps its (value, pointer) pairs in the change-list and frontier-list
    spaces; the runs that follow on the same handle (synchronous rounds with their canonical
    counts, forced push rounds, the frontier start, doubling again) must still equal the oracle."""
    g = functional_graph(n, seed, acc_p=0.01, none_p=0.02)
    want = oracle.run_graph(g)
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        plan = [(1, 0), (0, 0), (1, pkg.MAP_FLAG_PUSH), (1, 0), (1, pkg.MAP_FLAG_FRONTIER_START),
                (0, pkg.MAP_FLAG_FRONTIER_START), (1, 0)]
        for sched, flags in plan:
            out = np.empty(g.n, np.uint32)
            r = pkg.map_run(h, sched=sched, flags=flags, map_out=out)
            same_as_oracle(pkg, r, out, want)
            if sched == 0:
                assert (r.rounds, r.relaxations) == (want.rounds, want.relaxations)
    finally:
        pkg.map_destroy(h)
