"""Pins of the oracle's accepting-part reduction against things other than itself: brute-force
transitive closure on tiny graphs (with and without component labels), the verdict of the
whole graph from its strongly connected components, and the layered graphs' construction."""
import numpy as np
import pytest

import mapgen
import oracle


def closure(n, edges):
    """Reflexive-transitive closure as a boolean matrix (Warshall)."""
    R = np.eye(n, dtype=bool)
    for u, v in edges:
        R[u, v] = True
    for k in range(n):
        R |= R[:, [k]] & R[[k], :]
    return R


def brute_reduce(g, part=None):
    rows = [[int(v) for v in g.colidx[g.rowptr[u]:g.rowptr[u + 1]]] for u in range(g.n)]
    ok = lambda u, v: part is None or part[u] == part[v]
    R = closure(g.n, [(u, v) for u in range(g.n) for v in rows[u] if ok(u, v)])
    A = [a for a in range(g.n) if g.acc[a]]
    kept = [v for v in range(g.n) if any(R[a, v] for a in A) and any(R[v, a] for a in A)]
    new = {v: i for i, v in enumerate(kept)}
    rowptr, colidx = [0], []
    for u in kept:
        colidx += [new[v] for v in rows[u] if v in new and ok(u, v)]
        rowptr.append(len(colidx))
    return kept, rowptr, colidx, [int(g.acc[v]) for v in kept]


def has_accepting_cycle(g):
    """An accepting vertex in a strongly connected component with a cycle (scipy SCCs)."""
    sp = pytest.importorskip("scipy.sparse")
    from scipy.sparse.csgraph import connected_components
    A = sp.csr_matrix((np.ones(len(g.colidx)), g.colidx.astype(np.int64), g.rowptr.astype(np.int64)),
                      shape=(g.n, g.n))
    _, lab = connected_components(A, directed=True, connection="strong")
    size = np.bincount(lab)
    loop = np.zeros(g.n, bool)
    for u in range(g.n):
        if u in g.colidx[g.rowptr[u]:g.rowptr[u + 1]]:
            loop[u] = True
    return bool(np.any(g.acc.astype(bool) & ((size[lab] > 1) | loop))), lab


def as_lists(r):
    ids, rp, ci, acc = r
    return [int(x) for x in ids], [int(x) for x in rp], [int(x) for x in ci], [int(x) for x in acc]


@pytest.mark.parametrize("seed", range(60))
def test_reduce_brute_force(seed):
    rng = np.random.default_rng(seed)
    g = mapgen.tiny_graph(seed, int(rng.integers(1, 24)), max_deg=3, acc_p=float(rng.choice([0.0, 0.1, 0.3])))
    got = as_lists(oracle.reduce_graph(g.n, g.rowptr, g.colidx, g.acc))
    assert got == brute_reduce(g)


@pytest.mark.parametrize("seed", range(30))
def test_reduce_with_labels_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    g = mapgen.tiny_graph(seed, int(rng.integers(2, 24)), max_deg=4, acc_p=0.25)
    part = rng.integers(0, 3, size=g.n).astype(np.uint32)
    got = as_lists(oracle.reduce_graph(g.n, g.rowptr, g.colidx, g.acc, part))
    kept, rp, ci, acc = brute_reduce(g, part)
    assert got == (kept, rp, ci, acc)


@pytest.mark.parametrize("seed", range(40))
def test_reduce_keeps_the_verdict(seed):
    rng = np.random.default_rng(200 + seed)
    g = mapgen.tiny_graph(seed, int(rng.integers(2, 150)), max_deg=3, acc_p=0.1)
    want, lab = has_accepting_cycle(g)
    size = np.bincount(lab)
    # no labels, and labels constant on every strongly connected component (cycles stay inside one)
    for part in (None, (lab % 3).astype(np.uint32)):
        ids, rp, ci, acc = oracle.reduce_graph(g.n, g.rowptr, g.colidx, g.acc, part)
        if len(ids) == 0:
            assert not want
            continue
        r = oracle.run(len(ids), rp, ci, acc)
        assert r.verdict == int(want)
        if want:  # the witness, mapped back, is accepting and on a cycle of the whole graph
            w = int(ids[r.witness])
            assert g.acc[w] and (size[lab[w]] > 1 or w in g.colidx[g.rowptr[w]:g.rowptr[w + 1]])


def test_layered_graph_keeps_exactly_the_accepting_vertices():
    """By construction no non-accepting vertex of a layered graph reaches an accepting one, and
    every accepting vertex is kept: the reduced graph is the accepting DAG."""
    g = mapgen.layered_graph(200_000, 12, seed=9)
    ids, rp, ci, acc = oracle.reduce_graph(g.n, g.rowptr, g.colidx, g.acc)
    A = np.flatnonzero(g.acc)
    assert np.array_equal(ids, A) and acc.all()
    src = np.repeat(np.arange(g.n), np.diff(g.rowptr.astype(np.int64)))
    assert len(ci) == int(np.sum(g.acc[src].astype(bool) & g.acc[g.colidx].astype(bool)))


def test_no_accepting_vertex():
    g = mapgen.from_lists([[1], [0]], [0, 0])
    ids, rp, ci, acc = oracle.reduce_graph(g.n, g.rowptr, g.colidx, g.acc)
    assert len(ids) == 0 and list(rp) == [0] and len(ci) == 0
