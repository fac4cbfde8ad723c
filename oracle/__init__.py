"""TEST INFRASTRUCTURE ONLY: ctypes loader for the CPU oracle of MAP.

The oracle (``map_oracle.c``) is a plain single-threaded C statement of the
MAP accepting-cycle detection loop of Section 2 of the DiVinE-CUDA paper
(Barnat, Brim, Ceska, PDMC 2009).  Only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the GPU
library never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "map_oracle.c")
_HDR = os.path.join(_HERE, "map_oracle.h")
_LIB = os.path.join(_HERE, "libmaporacle.so")

NONE = 0xFFFFFFFF
CYCLE, NO_CYCLE = 1, 0
OK, ERR_ARG, ERR_OOM, LIMIT = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile libmaporacle.so with gcc (plain -O2, portable to x86_64 and aarch64)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(_HDR)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


class _Result(ctypes.Structure):
    _fields_ = [
        ("verdict", ctypes.c_uint32),
        ("witness", ctypes.c_uint32),
        ("outer", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
        ("inner_total", ctypes.c_uint64),
        ("relaxations", ctypes.c_uint64),
    ]


_TRACE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                          ctypes.c_uint32, ctypes.c_uint32)
_lib = None


def load_library(path: str):
    """Load a compiled oracle library from ``path`` (the default build, or a test's variant)."""
    lib = ctypes.CDLL(path)
    lib.oracle_map.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_uint32, _TRACE, ctypes.c_void_p, ctypes.POINTER(_Result),
                                   ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
    lib.oracle_map.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


@dataclass
class OracleResult:
    status: int
    verdict: int
    witness: int
    outer: int
    rounds: list
    inner_total: int
    relaxations: int
    map: np.ndarray  # uint32[n], NONE where undefined: the last outer iteration's map
    trace: list = field(default_factory=list)  # [(outer, map copy, rounds)] when requested


def run(n: int, rowptr, colidx, acc, max_outer: int = 0, keep_trace: bool = False, hash_trace=None,
        lib=None) -> OracleResult:
    """Run the oracle on a CSR of successor lists and accepting flags (one byte per vertex).

    keep_trace: keep a copy of the map vector of every outer iteration.
    hash_trace: optional callable(map ndarray) -> object stored instead of the full vector.
    """
    lib = lib or _load()
    rowptr = np.ascontiguousarray(rowptr, dtype=np.uint32)
    colidx = np.ascontiguousarray(colidx, dtype=np.uint32)
    acc = np.ascontiguousarray(acc, dtype=np.uint8)
    if colidx.size == 0:
        colidx = np.zeros(1, dtype=np.uint32)
    cap = 1 << 20
    rounds = np.zeros(cap, dtype=np.uint32)
    mp = np.zeros(max(n, 1), dtype=np.uint32)
    res = _Result()
    tr = []

    def _cb(_user, outer, mptr, nn, k):
        if keep_trace or hash_trace is not None:
            vec = np.ctypeslib.as_array(mptr, shape=(nn,))
            tr.append((int(outer), hash_trace(vec) if hash_trace else vec.copy(), int(k)))

    cb = _TRACE(_cb) if (keep_trace or hash_trace is not None) else _TRACE()
    st = lib.oracle_map(n, rowptr.ctypes.data, colidx.ctypes.data, acc.ctypes.data, max_outer, cb, None,
                        ctypes.byref(res), rounds.ctypes.data, cap, mp.ctypes.data)
    return OracleResult(st, res.verdict, res.witness, res.outer, [int(x) for x in rounds[:min(res.outer, cap)]],
                        res.inner_total, res.relaxations, mp[:n], tr)


def run_graph(g, **kw) -> OracleResult:
    """Run the oracle on a ``mapgen.Graph``."""
    return run(g.n, g.rowptr, g.colidx, g.acc, **kw)


# ---------------------------------------------------------------------------
# Counterexamples (the lasso behind a cycle verdict).  Section 5 of the paper
# names counterexample generation as missing; a lasso is the standard form
# of an LTL counterexample: a path from the initial vertex to an accepting
# vertex, then a cycle through that vertex.  Shortest paths are not unique, so
# the oracle fixes what is: the lengths.  Plain breadth-first search.
# ---------------------------------------------------------------------------

def _levels(n, rowptr, colidx, sources):
    """Edge count of a shortest path from the nearest source to every v along rows (-1 if none).
    Level by level: the unseen successors of level d form level d + 1."""
    rowptr = np.asarray(rowptr, np.int64)
    colidx = np.asarray(colidx, np.int64)
    dist = np.full(n, -1, np.int64)
    front = np.unique(np.asarray(sources, np.int64))
    dist[front] = 0
    level = 0
    while front.size:
        level += 1
        b, e = rowptr[front], rowptr[front + 1]
        cnt = e - b
        first = np.cumsum(cnt) - cnt  # where each frontier row's successors start in succ
        succ = colidx[np.repeat(b - first, cnt) + np.arange(int(cnt.sum()))]
        new = np.unique(succ[dist[succ] < 0])
        dist[new] = level
        front = new
    return dist


def bfs_dist(n, rowptr, colidx, source):
    """Edge count of a shortest path source -> v along rows (successors) for every v (an int64
    array); -1 if none."""
    return _levels(n, rowptr, colidx, [source])


def lasso_lengths(n, rowptr, colidx, witness, init=None):
    """(prefix edges, cycle edges) of a shortest lasso: dist(init, witness) (0 without init or when
    init is the witness) and the shortest cycle through the witness, 1 + min dist(witness, u) over
    the edges u -> witness; None for a part that does not exist."""
    rowptr = np.asarray(rowptr, np.int64)
    colidx = np.asarray(colidx, np.int64)
    d = bfs_dist(n, rowptr, colidx, witness)
    cyc = None
    for j in np.nonzero(colidx == witness)[0]:  # the edges u -> witness
        u = int(np.searchsorted(rowptr, j, side="right")) - 1  # the row holding position j
        if d[u] >= 0:
            cyc = int(d[u]) + 1 if cyc is None else min(cyc, int(d[u]) + 1)
    if init is None or init == witness:
        pre = 0
    else:
        pre = int(bfs_dist(n, rowptr, colidx, init)[witness])
        pre = None if pre < 0 else pre
    return pre, cyc


# ---------------------------------------------------------------------------
# Accepting-part reduction.  Section 2 of the paper: the matrix lists only the
# states of components that contain accepting states (components of the
# property automaton, after Lafuente).  Stated on the graph: with optional
# component labels part[v] (edges between different labels dropped), keep the
# vertices reachable from an accepting vertex and reaching an accepting vertex
# (paths of zero or more edges); the result is the subgraph they induce, its
# vertices renumbered in increasing order of their original ids.
# ---------------------------------------------------------------------------

def _csr_from_edges(n, src, dst):
    """CSR with rows by src; a row keeps the edges in their given order (stable sort)."""
    order = np.argsort(src, kind="stable")
    rowptr = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=n))]).astype(np.int64)
    return rowptr, dst[order]


def reduce_graph(n, rowptr, colidx, acc, part=None):
    """(ids, rowptr', colidx', acc') of the reduced graph: ids[i] = original id of vertex i."""
    rowptr = np.asarray(rowptr, np.int64)
    colidx = np.asarray(colidx, np.int64)
    acc = np.asarray(acc).astype(bool)
    src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr))  # the row of every edge
    ok = np.ones(len(colidx), bool) if part is None else (np.asarray(part)[src] == np.asarray(part)[colidx])
    seeds = np.flatnonzero(acc)
    fwd = _levels(n, *_csr_from_edges(n, src[ok], colidx[ok]), seeds) >= 0  # reached from A
    bwd = _levels(n, *_csr_from_edges(n, colidx[ok], src[ok]), seeds) >= 0  # reaching A
    keep = fwd & bwd
    ids = np.flatnonzero(keep)
    new = np.cumsum(keep) - 1  # new id of each kept vertex
    e = ok & keep[src] & keep[colidx]  # edges of the induced subgraph, in CSR order
    rowptr2 = np.concatenate([[0], np.cumsum(np.bincount(new[src[e]], minlength=len(ids)))]).astype(np.uint32)
    return ids.astype(np.uint32), rowptr2, new[colidx[e]].astype(np.uint32), acc[ids].astype(np.uint8)
