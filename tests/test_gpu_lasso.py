"""Counterexamples on the GPU (map_lasso) against the oracle's shortest lasso lengths.

Shortest paths are not unique, so the lengths are compared with the oracle and the paths
themselves are checked to be lassos of the graph: every step an edge, the prefix from the
initial vertex into the witness, the cycle from the witness back to it."""
import numpy as np
import pytest

import mapgen
import oracle

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


def is_edge(g, a, b):
    row = g.colidx[g.rowptr[a]:g.rowptr[a + 1]]
    return bool((row == b).any())


def check_lasso(g, prefix, cycle, witness, init):
    assert cycle[0] == cycle[-1] == witness and len(cycle) >= 2
    assert all(is_edge(g, a, b) for a, b in zip(cycle, cycle[1:]))
    if init is None or init == witness:
        assert prefix == []
    else:
        assert prefix[0] == init and witness not in prefix
        path = prefix + [witness]
        assert all(is_edge(g, a, b) for a, b in zip(path, path[1:]))


def ancestor(g, v, steps):
    """A vertex that reaches v: walk back along edges (the first edge into the current vertex)."""
    for _ in range(steps):
        j = np.flatnonzero(g.colidx == v)
        if j.size == 0:
            break
        v = int(np.searchsorted(g.rowptr, j[0], side="right")) - 1
    return v


def lasso_case(pkg, g, init=0, lengths=True, back=None):
    with pkg.Graph(g.n, g.rowptr, g.colidx, g.acc) as h:
        r = h.run()
        assert r.verdict == 1 and g.acc[r.witness]
        if back is not None:  # the initial vertex: `back` steps up the witness's ancestry
            init = ancestor(g, r.witness, back)
        prefix, cycle = h.lasso(r.witness, init=pkg.MAP_NONE if init is None else init)
        check_lasso(g, prefix, cycle, r.witness, init)
        if lengths:
            want = oracle.lasso_lengths(g.n, g.rowptr, g.colidx, r.witness, init)
            assert (len(prefix), len(cycle) - 1) == want
        # the work space is shared with runs: a run after the lasso is unchanged
        out = np.empty(g.n, np.uint32)
        r2 = h.run(map_out=out)
        assert (r2.verdict, r2.witness, r2.rounds) == (r.verdict, r.witness, r.rounds)
    return prefix, cycle


def test_small_cycles(pkg):
    n_cases = 0
    for seed in range(120):
        rng = np.random.default_rng(900 + seed)
        g = mapgen.tiny_graph(seed, int(rng.integers(1, 200)), max_deg=int(rng.integers(1, 4)), acc_p=0.2)
        want = oracle.run_graph(g)
        if want.verdict != 1:
            continue
        n_cases += 1
        lasso_case(pkg, g, init=None)
        init = int(rng.integers(0, g.n))
        if oracle.bfs_dist(g.n, g.rowptr, g.colidx, init)[want.witness] >= 0:
            lasso_case(pkg, g, init=init)
    assert n_cases > 30


def test_self_loop_and_ring(pkg):
    k = 1000
    g = mapgen.from_lists([[(i + 1) % k] for i in range(k)] + [[0]], [0] * (k - 1) + [1, 0])
    prefix, cycle = lasso_case(pkg, g, init=k)
    assert prefix == [k] + list(range(k - 1)) and cycle == [k - 1] + list(range(k))
    g1 = mapgen.from_lists([[1], [1]], [0, 1])
    prefix, cycle = lasso_case(pkg, g1, init=0)
    assert prefix == [0] and cycle == [1, 1]


@pytest.mark.parametrize("name", ["random_16k", "product_8x7", "layered_4m"])
def test_workloads(pkg, name):
    g = {"random_16k": lambda: mapgen.random_16k("cycle"),
         "product_8x7": mapgen.product_8x7,
         "layered_4m": lambda: mapgen.layered_graph(1 << 22, 250, seed=3, plant=True)}[name]()
    lasso_case(pkg, g, back=25)
    lasso_case(pkg, g, init=None)


def test_unreachable_initial_vertex(pkg):
    """product 8x7 is deterministic (out-degree 1): vertex 0 does not reach the witness."""
    g = mapgen.product_8x7()
    with pkg.Graph(g.n, g.rowptr, g.colidx, g.acc) as h:
        r = h.run()
        assert oracle.bfs_dist(g.n, g.rowptr, g.colidx, 0)[r.witness] < 0
        with pytest.raises(pkg.MapError) as e:
            h.lasso(r.witness, init=0)
        assert e.value.code == pkg.MAP_ERR_ARG


def test_layered_64m_planted_lasso_is_valid(pkg):
    """Full size: 2^26 vertices, 4,000 layers, one planted back edge; the lasso is checked for
    validity (the oracle's BFS at this size is left to the 4M-vertex case)."""
    g = mapgen.layered_graph(1 << 26, 4000, seed=3, plant=True)
    lasso_case(pkg, g, lengths=False, back=10)


def test_errors(pkg):
    g = mapgen.from_lists([[1], [2], [1], []], [0, 1, 0, 1])
    with pkg.Graph(g.n, g.rowptr, g.colidx, g.acc) as h:
        with pytest.raises(pkg.MapError) as e:  # 3 has no cycle
            h.lasso(3)
        assert e.value.code == pkg.MAP_ERR_ARG
        with pytest.raises(pkg.MapError) as e:  # 3 is not reachable from 0
            h.lasso(1, init=3)
        assert e.value.code == pkg.MAP_ERR_ARG
        with pytest.raises(pkg.MapError) as e:
            h.lasso(4)
        assert e.value.code == pkg.MAP_ERR_ARG
        with pytest.raises(pkg.MapError) as e:  # prefix 0 and cycle 1 2 1 need 4 entries
            h.lasso(1, init=0, cap=3)
        assert e.value.code == pkg.MAP_ERR_LIMIT
        assert h.lasso(1, init=0, cap=4) == ([0], [1, 2, 1])
    hb = pkg.map_batch_create([(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))])
    try:
        with pytest.raises(pkg.MapError) as e:
            pkg.map_lasso(hb, 1)
        assert e.value.code == pkg.MAP_ERR_ARG
    finally:
        pkg.map_destroy(hb)
