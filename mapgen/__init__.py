"""Seeded synthetic workloads for MAP accepting-cycle detection.

Inputs only: graphs as CSR successor lists of the state graph G plus
accepting flags, batch plans and arrival schedules.  Nothing here computes
any part of MAP, so the CPU oracle and the GPU path can both consume it.

The recipes stand in for the DiVinE models of the paper's experiments
(Section 4, Tables 1-2), which are not available:

* ``random_16k``  uniform random digraph, 16,384 vertices, out-degree
  U{1..6}, 3 % accepting, seed 1; ``variant='nocycle'`` moves every accepting
  flag onto a vertex that no cycle reaches, ``variant='cycle'`` then plants a
  20-vertex cycle through the largest accepting id.
* ``product_8x7``  synchronous product of 8 cyclic 7-state processes with a
  2-state Buchi automaton (2 * 7**8 = 11,529,602 vertices).
* ``layered_64m``  layered graph: 2**26 vertices in 4,000 layers, geometric
  out-degree with mean 4, 92 % forward edges, back edges over 50 layers,
  1 % accepting, accepting vertices on no cycle (D = 16 layer segments).
* ``batch_plan`` / ``arrivals``  batch (256 graphs) and serving (Poisson) schedules.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mapgen.c")
_LIB = os.path.join(_HERE, "libmapgen.so")


def build(force: bool = False) -> str:
    """Compile libmapgen.so with gcc (portable flags: x86_64 and aarch64)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mapgen.h"))
    ):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(
        ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
         "-o", tmp, _SRC, "-lm"]
    )
    os.replace(tmp, _LIB)
    return _LIB


class _MgGraph(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32),
        ("m", ctypes.c_uint64),
        ("rowptr", ctypes.POINTER(ctypes.c_uint32)),
        ("colidx", ctypes.POINTER(ctypes.c_uint32)),
        ("acc", ctypes.POINTER(ctypes.c_uint8)),
        ("info", ctypes.c_uint32 * 8),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        u32, u64, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int
        pg = ctypes.POINTER(_MgGraph)
        lib.mg_free.argtypes = [pg]
        lib.mg_random.argtypes = [u32, u32, u32, u32, u64, i32, u32, pg]
        lib.mg_product.argtypes = [u32, u32, i32, pg]
        lib.mg_layered.argtypes = [u32, u32, u32, u32, u32, u32, u32, u64, i32, pg]
        lib.mg_batch_plan.argtypes = [u32, u32, u32, u32, u64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.mg_arrivals.argtypes = [u32, ctypes.c_double, ctypes.c_double, ctypes.c_double, u32, u32, u64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]
        lib.mg_peel.argtypes = [u32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.mg_peel.restype = u32
        for f in ("mg_random", "mg_product", "mg_layered", "mg_batch_plan", "mg_arrivals"):
            getattr(lib, f).restype = i32
        _lib = lib
    return _lib


@dataclass
class Graph:
    """CSR successor lists of G (row v = targets of v's out-edges) + flags."""

    n: int
    rowptr: np.ndarray  # uint32[n + 1]
    colidx: np.ndarray  # uint32[m]
    acc: np.ndarray  # uint8[n]
    info: tuple = ()
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.rowptr[-1])

    def acc_bits(self) -> np.ndarray:
        """Accepting set as an LSB-first uint32 bitmap (bit v of word v>>5)."""
        return pack_bits(self.acc)


def pack_bits(flags: np.ndarray) -> np.ndarray:
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    n = flags.shape[0]
    words = (n + 31) // 32
    padded = np.zeros(words * 32, dtype=np.uint8)
    padded[:n] = flags != 0
    return np.packbits(padded, bitorder="little").view("<u4").astype(np.uint32)


def from_lists(rows, acc, name: str = "") -> Graph:
    """Build a Graph from Python successor lists and a flag sequence."""
    n = len(rows)
    rowptr = np.zeros(n + 1, dtype=np.uint32)
    rowptr[1:] = np.cumsum([len(r) for r in rows], dtype=np.uint64).astype(np.uint32)
    colidx = np.array([u for r in rows for u in r], dtype=np.uint32)
    return Graph(n, rowptr, colidx, np.asarray(acc, dtype=np.uint8).copy(), (), name)


def _take(g: _MgGraph, name: str, meta: dict) -> Graph:
    lib = _load()
    n, m = int(g.n), int(g.m)
    rowptr = np.ctypeslib.as_array(g.rowptr, shape=(n + 1,)).copy()
    colidx = np.ctypeslib.as_array(g.colidx, shape=(max(m, 1),))[:m].copy()
    acc = np.ctypeslib.as_array(g.acc, shape=(n,)).copy()
    info = tuple(int(x) for x in g.info)
    lib.mg_free(ctypes.byref(g))
    return Graph(n, rowptr, colidx, acc, info, name, meta)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"{what} failed with code {rc}")


def random_graph(n: int, deg_lo: int = 1, deg_hi: int = 6, acc_p: float = 0.03, seed: int = 1,
                 variant: str = "plain", cycle_len: int = 20) -> Graph:
    v = {"plain": 0, "nocycle": 1, "cycle": 2}[variant]
    g = _MgGraph()
    _check(_load().mg_random(n, deg_lo, deg_hi, int(round(acc_p * 1e6)), seed, v, cycle_len, ctypes.byref(g)),
           "mg_random")
    meta = dict(kind="random", n=n, deg=(deg_lo, deg_hi), acc_p=acc_p, seed=seed, variant=variant)
    out = _take(g, f"random-{variant}-{n}", meta)
    if v >= 1:
        out.meta.update(acc_drawn=out.info[0], acc_placed=out.info[1])
    if v == 2:
        out.meta.update(planted=out.info[2], cycle_len=cycle_len)
    return out


def product_graph(k: int = 8, s: int = 7, interleave: bool = False) -> Graph:
    g = _MgGraph()
    _check(_load().mg_product(k, s, 1 if interleave else 0, ctypes.byref(g)), "mg_product")
    meta = dict(kind="product", k=k, s=s, interleave=bool(interleave))
    return _take(g, f"product-{'i' if interleave else 's'}-{k}x{s}", meta)


def layered_graph(n: int, layers: int, seed: int, D: int = 16, window: int = 50, acc_p: float = 0.01,
                  fwd_p: float = 0.92, accfwd_p: float = 0.5, plant: bool = False) -> Graph:
    g = _MgGraph()
    _check(_load().mg_layered(n, layers, D, window, int(round(acc_p * 1e6)), int(round(fwd_p * 1e6)),
                              int(round(accfwd_p * 1e6)), seed, 1 if plant else 0, ctypes.byref(g)),
           "mg_layered")
    meta = dict(kind="layered", n=n, layers=layers, D=D, window=window, acc_p=acc_p, fwd_p=fwd_p,
                accfwd_p=accfwd_p, seed=seed, plant=bool(plant))
    out = _take(g, f"layered-{n}-{layers}{'-cycle' if plant else ''}", meta)
    if plant:
        out.meta.update(planted=out.info[0], planted_from=out.info[1])
    return out


# ------------------------------------------------------- named workloads --

def random_16k(variant: str = "cycle") -> Graph:
    """16,384 vertices, degree U{1..6}, 3 % accepting, seed 1."""
    return random_graph(16384, 1, 6, 0.03, 1, variant, 20)


def product_8x7(interleave: bool = False) -> Graph:
    """8 cyclic 7-state processes x 2-state Buchi automaton."""
    return product_graph(8, 7, interleave)


def layered_64m(n: int = 1 << 26, layers: int = 4000, seed: int = 3, D: int = 16) -> Graph:
    """Large layered no-cycle graph (default 2**26 vertices, 4,000 layers)."""
    return layered_graph(n, layers, seed, D=D)


def layers_for(n: int) -> int:
    """Layer count of a batch/serving layered graph: about 16,777 vertices per layer, at least 8."""
    return max(8, int(round(n / 16777)))


def batch_plan(count: int = 256, lo: int = 1000, hi: int = 2_000_000, frac_cycle: float = 0.4, seed: int = 4):
    sizes = np.zeros(count, dtype=np.uint32)
    planted = np.zeros(count, dtype=np.uint8)
    seeds = np.zeros(count, dtype=np.uint64)
    ncyc = int(round(frac_cycle * count))
    _check(_load().mg_batch_plan(count, lo, hi, ncyc, seed, sizes.ctypes.data, planted.ctypes.data,
                                 seeds.ctypes.data), "mg_batch_plan")
    return sizes, planted.astype(bool), seeds


def batch_graph(size: int, planted: bool, seed: int) -> Graph:
    return layered_graph(int(size), layers_for(int(size)), int(seed), plant=bool(planted))


def arrivals(count: int, rate: float, seed: int = 5, median: float = 1e5, sigma: float = 1.5,
                     lo: int = 1000, hi: int = 10_000_000):
    t = np.zeros(count, dtype=np.float64)
    sizes = np.zeros(count, dtype=np.uint32)
    kind = np.zeros(count, dtype=np.uint8)
    pk = np.zeros(count, dtype=np.uint8)
    ps = np.zeros(count, dtype=np.uint8)
    seeds = np.zeros(count, dtype=np.uint64)
    _check(_load().mg_arrivals(count, rate, median, sigma, lo, hi, seed, t.ctypes.data, sizes.ctypes.data,
                               kind.ctypes.data, pk.ctypes.data, ps.ctypes.data, seeds.ctypes.data),
           "mg_arrivals")
    return dict(t=t, sizes=sizes, kind=kind, k=pk, s=ps, seeds=seeds)


def arrival_graph(arr: dict, i: int) -> Graph:
    if int(arr["kind"][i]) == 1:
        return product_graph(int(arr["k"][i]), int(arr["s"][i]), False)
    n = int(arr["sizes"][i])
    return layered_graph(n, layers_for(n), int(arr["seeds"][i]))


def peel(g: Graph) -> np.ndarray:
    """Vertices that no cycle reaches (Kahn peeling), as a bool array."""
    out = np.zeros(g.n, dtype=np.uint8)
    _load().mg_peel(g.n, g.rowptr.ctypes.data, g.colidx.ctypes.data, out.ctypes.data)
    return out.astype(bool)


def tiny_graph(seed: int, n: int, max_deg: int = 4, acc_p: float = 0.3, self_loops: bool = True,
               dups: bool = True) -> Graph:
    """Small random digraph for property tests: out-degree uniform in [0, max_deg], targets
    uniform over all vertices (self-loops and duplicate targets allowed unless switched off),
    each vertex accepting with probability acc_p.  numpy PCG64 seeded by ``seed``."""
    rng = np.random.default_rng(seed)
    rows = []
    for v in range(n):
        d = int(rng.integers(0, max_deg + 1))
        r = [int(x) for x in rng.integers(0, n, size=d)]
        if not self_loops:
            r = [u for u in r if u != v]
        if not dups:
            r = sorted(set(r))
        rows.append(r)
    acc = (rng.random(n) < acc_p).astype(np.uint8)
    return from_lists(rows, acc, f"tiny-{seed}-{n}")


# ------------------------------------------------------ on-the-fly streams --

def discovery_order(g: Graph, start: int = 0):
    """The part of g reachable from `start`, renumbered in breadth-first discovery order (the order
    an explicit-state generator numbers states in), and known[R] = the vertices known once rows
    0 .. R-1 are expanded (R = 0 .. n).  Returns (graph, known)."""
    rowptr = g.rowptr.astype(np.int64)
    colidx = g.colidx.astype(np.int64)
    newid = np.full(g.n, -1, np.int64)
    newid[start] = 0
    order = [np.array([start], np.int64)]
    count, front = 1, order[0]
    while front.size:
        b, e = rowptr[front], rowptr[front + 1]
        cnt = e - b
        succ = colidx[np.repeat(b - (np.cumsum(cnt) - cnt), cnt) + np.arange(int(cnt.sum()))]
        cand = succ[newid[succ] < 0]
        _, first = np.unique(cand, return_index=True)
        fresh = cand[np.sort(first)]  # first occurrences, in queue order
        newid[fresh] = count + np.arange(fresh.size)
        count += fresh.size
        order.append(fresh)
        front = fresh
    order = np.concatenate(order)
    deg = (rowptr[order + 1] - rowptr[order])
    rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.uint32)
    src_pos = np.repeat(rowptr[order] - (np.cumsum(deg) - deg), deg) + np.arange(int(deg.sum()))
    ci = newid[colidx[src_pos]].astype(np.uint32)
    out = Graph(n=len(order), rowptr=rp, colidx=ci, acc=g.acc[order].astype(np.uint8),
                name=f"{g.name}-discovery", meta=dict(g.meta, start=start, order="bfs-discovery"))
    # known after R rows: the start, the expanded rows and every target seen so far
    known = np.maximum(np.arange(out.n + 1, dtype=np.int64), 1)
    if len(ci):
        seen = np.maximum.accumulate(ci.astype(np.int64)) + 1  # after each edge
        R = np.flatnonzero(rp > 0)
        known[R] = np.maximum(known[R], seen[rp[R].astype(np.int64) - 1])
    return out, known
