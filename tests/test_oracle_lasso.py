"""Pins of the oracle's counterexample lengths (plain BFS) against things other than itself:
scipy's unweighted shortest paths, and brute-force enumeration of simple paths on tiny graphs."""
import itertools

import numpy as np
import pytest

import mapgen
import oracle


def _edges(g):
    return {(u, int(v)) for u in range(g.n) for v in g.colidx[g.rowptr[u]:g.rowptr[u + 1]]}


def _brute_lengths(g, w, init):
    """Shortest lasso lengths by enumerating every vertex sequence of up to n + 1 vertices."""
    E = _edges(g)

    def shortest(a, b, min_edges):
        for k in range(min_edges, g.n + 1):  # k edges, k - 1 inner vertices
            for inner in itertools.product(range(g.n), repeat=k - 1):
                seq = (a,) + inner + (b,)
                if all((seq[i], seq[i + 1]) in E for i in range(k)):
                    return k
        return None

    pre = 0 if init is None or init == w else shortest(init, w, 1)
    return pre, shortest(w, w, 1)


@pytest.mark.parametrize("seed", range(40))
def test_lasso_lengths_brute_force(seed):
    g = mapgen.tiny_graph(seed, n=1 + seed % 5, max_deg=3, acc_p=0.5, self_loops=True, dups=True)
    for w in range(g.n):
        for init in [None] + list(range(g.n)):
            assert oracle.lasso_lengths(g.n, g.rowptr, g.colidx, w, init) == _brute_lengths(g, w, init)


@pytest.mark.parametrize("seed", range(6))
def test_bfs_dist_matches_scipy(seed):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    g = mapgen.random_graph(300, deg_lo=1, deg_hi=2 + seed % 3, seed=seed + 1)
    A = sp.csr_matrix((np.ones(len(g.colidx)), g.colidx.astype(np.int64), g.rowptr.astype(np.int64)),
                      shape=(g.n, g.n))
    for src in (0, g.n // 2, g.n - 1):
        ref = csgraph.shortest_path(A, unweighted=True, indices=src)
        got = oracle.bfs_dist(g.n, g.rowptr, g.colidx, src).astype(float)
        got[got < 0] = np.inf
        assert np.array_equal(got, ref)


def test_lasso_lengths_closed_forms():
    # a directed ring 0 -> 1 -> ... -> k-1 -> 0 with a tail t -> 0: the cycle has k edges and the
    # prefix from the tail one; a self-loop is a cycle of one edge
    k = 7
    lists = [[(i + 1) % k] for i in range(k)] + [[0]]
    g = mapgen.from_lists(lists, acc=[True] * (k + 1))
    for w in range(k):
        assert oracle.lasso_lengths(g.n, g.rowptr, g.colidx, w, k) == (1 + w, k)
    assert oracle.lasso_lengths(g.n, g.rowptr, g.colidx, k, 0) == (None, None)
    g1 = mapgen.from_lists([[0]], acc=[True])
    assert oracle.lasso_lengths(g1.n, g1.rowptr, g1.colidx, 0) == (0, 1)
