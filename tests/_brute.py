"""Brute-force statements of MAP's quantities, used to pin the oracle.

Nothing here iterates MAP's propagation.  Each quantity is computed from its
closed form over explicit shortest-path distances (scipy's BFS shortest paths)
or from strongly connected components (scipy's Tarjan-style SCC routine):

* map(v) = max{u in A : v reaches u by a path of >= 1 edge}         (Section 2)
* the synchronous round-k value m_k(v) = max{u in A : 1 <= d+(v,u) <= k},
  where d+ is the shortest path length using at least one edge;
* rounds per outer iteration = 1 + max_v d+(v, map(v)) (0 where map undefined);
* an accepting cycle exists iff some accepting vertex lies in a strongly
  connected component with an internal edge (size >= 2, or a self-loop).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, shortest_path

NONE = 0xFFFFFFFF
INF = np.inf


def adjacency(n, rowptr, colidx):
    rowptr = np.asarray(rowptr, dtype=np.int64)
    colidx = np.asarray(colidx, dtype=np.int64)
    data = np.ones(colidx.size, dtype=np.float64)
    a = sp.csr_matrix((data, colidx, rowptr), shape=(n, n))
    a.sum_duplicates()
    a.data[:] = 1.0
    return a


def dist_plus(n, rowptr, colidx):
    """d+[v, u]: length of the shortest path v -> u with at least one edge (inf if none)."""
    a = adjacency(n, rowptr, colidx)
    d0 = shortest_path(a, method="D", directed=True, unweighted=True)  # d0[v, v] = 0
    dp = np.full((n, n), INF)
    rp = np.asarray(rowptr, dtype=np.int64)
    ci = np.asarray(colidx, dtype=np.int64)
    for v in range(n):
        succ = ci[rp[v]:rp[v + 1]]
        if succ.size:
            dp[v] = 1.0 + d0[succ].min(axis=0)
    return dp


def map_at_round(dp, A, k=None):
    """m_k(v) (k=None: the fix-point map) as uint32 with NONE for undefined."""
    n = dp.shape[0]
    out = np.full(n, NONE, dtype=np.uint32)
    reach = dp <= (k if k is not None else n + 1)
    reach &= np.asarray(A, dtype=bool)[None, :]
    for v in range(n):
        us = np.nonzero(reach[v])[0]
        if us.size:
            out[v] = us.max()
    return out


def rounds_closed_form(dp, mp):
    """1 + max over v of d+(v, map(v)), with 0 where map(v) is undefined."""
    best = 0
    for v in range(dp.shape[0]):
        if mp[v] != NONE:
            best = max(best, int(dp[v, mp[v]]))
    return 1 + best


def relaxations_closed_form(n, rowptr, colidx, dp, A):
    """Edges relaxed by the synchronous schedule (round 1: every row; round k+1: the rows
    reading a vertex whose value changed in round k), with every m_k from its closed form."""
    rp = np.asarray(rowptr, dtype=np.int64)
    ci = np.asarray(colidx, dtype=np.int64)
    deg = np.diff(rp)
    readers = [set() for _ in range(n)]
    for w in range(n):
        for u in ci[rp[w]:rp[w + 1]]:
            readers[int(u)].add(w)
    total = int(deg.sum())
    prev = np.full(n, NONE, dtype=np.uint32)
    k = 1
    while True:
        cur = map_at_round(dp, A, k)
        changed = np.nonzero(cur != prev)[0]
        if changed.size == 0:
            return total, k
        front = set()
        for u in changed:
            front |= readers[int(u)]
        total += int(sum(deg[w] for w in front))
        prev = cur
        k += 1


def brute_map_run(n, rowptr, colidx, acc):
    """Replay the outer loop of Section 2 with every map from reachability.
    Returns (verdict, witness, outer, rounds list, maps list, relaxations)."""
    dp = dist_plus(n, rowptr, colidx)
    A = np.asarray(acc, dtype=bool).copy()
    outer, rounds, maps, relax = 0, [], [], 0
    while A.any():
        outer += 1
        mp = map_at_round(dp, A)
        maps.append(mp)
        r, k = relaxations_closed_form(n, rowptr, colidx, dp, A)
        assert k == rounds_closed_form(dp, mp)
        rounds.append(k)
        relax += r
        selfmap = np.nonzero(mp == np.arange(n, dtype=np.uint32))[0]
        if selfmap.size:
            return 1, int(selfmap.min()), outer, rounds, maps, relax
        E = np.unique(mp[mp != NONE])
        if E.size == 0:
            break
        A[E] = False
    return 0, None, outer, rounds, maps, relax


def tarjan_verdict(n, rowptr, colidx, acc):
    """True iff an accepting vertex lies on a cycle (SCC with an internal edge)."""
    a = adjacency(n, rowptr, colidx)
    ncomp, lab = connected_components(a, directed=True, connection="strong")
    size = np.bincount(lab, minlength=ncomp)
    rp = np.asarray(rowptr, dtype=np.int64)
    ci = np.asarray(colidx, dtype=np.int64)
    selfloop = np.zeros(n, dtype=bool)
    for v in range(n):
        if np.any(ci[rp[v]:rp[v + 1]] == v):
            selfloop[v] = True
    on_cycle = (size[lab] >= 2) | selfloop
    return bool(np.any(on_cycle & np.asarray(acc, dtype=bool))), on_cycle
