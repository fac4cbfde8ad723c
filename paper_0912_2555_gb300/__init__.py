"""Python binding of libmapgpu.so, the GB300 MAP accepting-cycle detection library.

Argument marshalling only: every step of MAP (Section 2 of the DiVinE-CUDA paper)
runs in the library's CUDA kernels.  The names follow the C ABI of
``include/map.h``: ``map_create``, ``map_run``, ``map_destroy``.  Inputs may be
numpy arrays (host memory) or CUDA torch tensors (device memory); PyTorch is
used only for device memory and streams.

There is no CPU fallback: importing works without a GPU, but every call that
reaches the library fails loudly if the compiled library is missing.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmapgpu.so")

MAP_NONE = 0xFFFFFFFF
MAP_OK, MAP_ERR_ARG, MAP_ERR_CSR, MAP_ERR_OOM, MAP_ERR_CUDA, MAP_ERR_TIMEOUT, MAP_ERR_LIMIT, \
    MAP_ERR_NOT_READY, MAP_ERR_BUSY = range(9)
MAP_NO_CYCLE, MAP_CYCLE = 0, 1
MAP_SCHED_SYNC, MAP_SCHED_ASYNC = 0, 1
MAP_FLAG_PROFILE = 1
MAP_FLAG_EARLY_EXIT = 2
MAP_FLAG_FRONTIER_START = 4
MAP_FLAG_DENSE_START = 8
MAP_FLAG_PUSH = 64
MAP_FLAG_PULL = 128
STATUS_NAMES = ["MAP_OK", "MAP_ERR_ARG", "MAP_ERR_CSR", "MAP_ERR_OOM", "MAP_ERR_CUDA", "MAP_ERR_TIMEOUT",
                "MAP_ERR_LIMIT", "MAP_ERR_NOT_READY", "MAP_ERR_BUSY"]

# exported symbols of include/map.h (checked by the tests)
EXPORTS = ["map_create", "map_run", "map_destroy", "map_graph_info", "map_last_error", "map_run_static",
           "map_batch_create", "map_batch_run", "map_server_create", "map_submit", "map_poll", "map_server_destroy",
           "map_server_batch_limit",
           "map_autotune", "map_lasso", "map_create_reduced", "map_graph_vertex_ids", "map_graph_csr",
           "map_grow_create", "map_append"]
MAP_STATIC_MAX_N = 65536
MAP_STATIC_MAX_M = 524288

TRACE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32),
                            ctypes.c_uint32, ctypes.c_uint32)


class MapOpts(ctypes.Structure):
    _fields_ = [
        ("sched", ctypes.c_uint32),
        ("max_outer", ctypes.c_uint32),
        ("max_inner", ctypes.c_uint32),
        ("flags", ctypes.c_uint32),
        ("trace", TRACE_FN),
        ("user", ctypes.c_void_p),
        ("rounds_out", ctypes.POINTER(ctypes.c_uint32)),
        ("rounds_cap", ctypes.c_uint32),
        ("timeout_ms", ctypes.c_uint32),
        ("repeat", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 2),
    ]


class MapResult(ctypes.Structure):
    _fields_ = [
        ("verdict", ctypes.c_uint32),
        ("witness", ctypes.c_uint32),
        ("outer_iters", ctypes.c_uint32),
        ("inner_canonical", ctypes.c_uint32),
        ("inner_iters", ctypes.c_uint64),
        ("relaxations", ctypes.c_uint64),
        ("edges_total", ctypes.c_uint64),
        ("device_ms", ctypes.c_double),
        ("dense_ms", ctypes.c_double),
        ("dense_launches", ctypes.c_uint32),
        ("accepting_left", ctypes.c_uint32),
        ("launches", ctypes.c_uint64),
        ("round_ms", ctypes.c_double),
        ("check_ms", ctypes.c_double),
        ("frontier_rows", ctypes.c_uint64),
        ("status", ctypes.c_uint32),
        ("batch_jobs", ctypes.c_uint32),
        ("queue_ms", ctypes.c_double),
        ("setup_ms", ctypes.c_double),
        ("run_ms", ctypes.c_double),
    ]


class TuneResult(ctypes.Structure):
    _fields_ = [
        ("dense_blocks_per_sm", ctypes.c_uint32),
        ("rounds_blocks_per_sm", ctypes.c_uint32),
        ("dense_ms", ctypes.c_double),
        ("rounds_ms", ctypes.c_double),
        ("trials", ctypes.c_uint32),
        ("frontier_start", ctypes.c_uint32),
        ("dense_start_ms", ctypes.c_double),
        ("frontier_start_ms", ctypes.c_double),
        ("pull_share", ctypes.c_double),
        ("pull_ms", ctypes.c_double),
        ("push_only_ms", ctypes.c_double),
        ("solo_max", ctypes.c_uint32),
        ("dense_unroll", ctypes.c_uint32),
        ("solo_ms", ctypes.c_double),
        ("local_passes", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]


def map_autotune(handle, sched: int = MAP_SCHED_SYNC) -> dict:
    """Pick the handle's launch shapes by measurement (see include/map.h)."""
    lib = load()
    t = TuneResult()
    rc = lib.map_autotune(handle, sched, ctypes.byref(t))
    if rc != MAP_OK:
        raise MapError(rc, "map_autotune", last_error())
    return {"dense_blocks_per_sm": t.dense_blocks_per_sm, "rounds_blocks_per_sm": t.rounds_blocks_per_sm,
            "dense_ms": t.dense_ms, "rounds_ms": t.rounds_ms, "trials": t.trials,
            "frontier_start": bool(t.frontier_start), "dense_start_ms": t.dense_start_ms,
            "frontier_start_ms": t.frontier_start_ms, "pull_share": t.pull_share, "pull_ms": t.pull_ms,
            "push_only_ms": t.push_only_ms, "solo_max": t.solo_max, "solo_ms": t.solo_ms,
            "dense_unroll": t.dense_unroll, "local_passes": t.local_passes}


def map_lasso(handle, witness: int, init: int = MAP_NONE, cap: int = 1 << 20):
    """Counterexample for a cycle verdict: (prefix list, cycle list) -- see include/map.h."""
    lib = load()
    path = np.zeros(cap, np.uint32)
    pl, cl = ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib.map_lasso(handle, init, witness, path.ctypes.data, cap, ctypes.byref(pl), ctypes.byref(cl))
    if rc != MAP_OK:
        raise MapError(rc, "map_lasso", last_error())
    return [int(x) for x in path[:pl.value]], [int(x) for x in path[pl.value:pl.value + cl.value]]


class MapError(RuntimeError):
    def __init__(self, code: int, what: str, msg: str):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else code}: {msg}")


_lib = None


def load(path: str = LIB_PATH):
    """Load the compiled library; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libmapgpu.so not found at {path}: build it with "
                           f"`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    vp, u32 = ctypes.c_void_p, ctypes.c_uint32
    lib.map_create.argtypes = [u32, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.map_run.argtypes = [vp, ctypes.POINTER(MapOpts), ctypes.POINTER(MapResult), vp]
    lib.map_destroy.argtypes = [vp]
    lib.map_graph_info.argtypes = [vp, ctypes.POINTER(u32), ctypes.POINTER(ctypes.c_uint64)]
    lib.map_last_error.restype = ctypes.c_char_p
    lib.map_run_static.argtypes = [u32, vp, vp, vp, ctypes.POINTER(MapOpts), ctypes.POINTER(MapResult), vp, vp]
    lib.map_batch_create.argtypes = [u32, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.map_batch_run.argtypes = [vp, ctypes.POINTER(MapOpts), ctypes.POINTER(MapResult), vp, vp, u32]
    lib.map_server_create.argtypes = [ctypes.c_size_t, u32, ctypes.POINTER(vp)]
    lib.map_submit.argtypes = [vp, u32, vp, vp, vp, ctypes.POINTER(MapOpts), ctypes.POINTER(ctypes.c_uint64)]
    lib.map_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(MapResult), vp]
    lib.map_server_destroy.argtypes = [vp]
    lib.map_server_batch_limit.argtypes = [vp, u32]
    lib.map_autotune.argtypes = [vp, u32, ctypes.POINTER(TuneResult)]
    lib.map_lasso.argtypes = [vp, u32, u32, vp, u32, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.map_create_reduced.argtypes = [u32, vp, vp, vp, vp, vp, ctypes.POINTER(vp)]
    lib.map_graph_vertex_ids.argtypes = [vp, vp]
    lib.map_graph_csr.argtypes = [vp, vp, vp, vp]
    lib.map_grow_create.argtypes = [u32, vp, vp, ctypes.POINTER(vp)]
    lib.map_append.argtypes = [vp, u32, vp, u32, vp, vp]
    for f in ("map_create", "map_run", "map_destroy", "map_graph_info", "map_run_static", "map_batch_create",
              "map_batch_run", "map_server_create", "map_submit", "map_poll", "map_server_destroy", "map_autotune",
              "map_lasso", "map_create_reduced", "map_graph_vertex_ids", "map_graph_csr", "map_grow_create",
              "map_append"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def last_error() -> str:
    return load().map_last_error().decode()


def _ptr(x):
    """(address, keep-alive) of a numpy array or torch tensor (host or device)."""
    if x is None:
        return None, None
    if hasattr(x, "data_ptr"):  # torch tensor
        return x.data_ptr(), x
    a = np.ascontiguousarray(x, dtype=np.uint32)
    return a.ctypes.data, a


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def map_create(n: int, rowptr, colidx, acc_bits, stream=None):
    """Create a device-resident graph (see include/map.h).  Returns an opaque handle."""
    lib = load()
    rp, k1 = _ptr(rowptr)
    ci, k2 = _ptr(colidx)
    ab, k3 = _ptr(acc_bits)
    h = ctypes.c_void_p()
    rc = lib.map_create(n, rp, ci, ab, _stream_handle(stream), ctypes.byref(h))
    if rc != MAP_OK:
        raise MapError(rc, "map_create", last_error())
    return h


def map_create_reduced(n: int, rowptr, colidx, acc_bits, part=None, stream=None):
    """Create the graph restricted to the vertices that can lie on an accepting cycle (see
    include/map.h); results use the reduced numbering, map_graph_vertex_ids maps it back."""
    lib = load()
    rp, k1 = _ptr(rowptr)
    ci, k2 = _ptr(colidx)
    ab, k3 = _ptr(acc_bits)
    pt, k4 = _ptr(part)
    h = ctypes.c_void_p()
    rc = lib.map_create_reduced(n, rp, ci, ab, pt, _stream_handle(stream), ctypes.byref(h))
    if rc != MAP_OK:
        raise MapError(rc, "map_create_reduced", last_error())
    return h


def map_grow_create(n: int, acc_bits, stream=None):
    """A growing graph of n known vertices, none expanded (see include/map.h)."""
    ab, k = _ptr(acc_bits)
    h = ctypes.c_void_p()
    rc = load().map_grow_create(n, ab, _stream_handle(stream), ctypes.byref(h))
    if rc != MAP_OK:
        raise MapError(rc, "map_grow_create", last_error())
    return h


def map_append(handle, n_add: int, acc_bits_add, rowptr_add=None, colidx_add=None):
    """Add n_add known vertices and the rows of the next len(rowptr_add) - 1 unexpanded ones."""
    k = 0 if rowptr_add is None else len(rowptr_add) - 1
    ab, k1 = _ptr(acc_bits_add)
    rp, k2 = _ptr(rowptr_add)
    ci, k3 = _ptr(colidx_add)
    rc = load().map_append(handle, n_add, ab, k, rp, ci)
    if rc != MAP_OK:
        raise MapError(rc, "map_append", last_error())


def map_graph_info(handle):
    """(n, m) of a handle."""
    n, m = ctypes.c_uint32(), ctypes.c_uint64()
    rc = load().map_graph_info(handle, ctypes.byref(n), ctypes.byref(m))
    if rc != MAP_OK:
        raise MapError(rc, "map_graph_info", last_error())
    return n.value, m.value


def map_graph_vertex_ids(handle) -> np.ndarray:
    """Original id of each vertex of the handle (identity unless it was reduced)."""
    n, _ = map_graph_info(handle)
    ids = np.empty(n, np.uint32)
    rc = load().map_graph_vertex_ids(handle, ids.ctypes.data)
    if rc != MAP_OK:
        raise MapError(rc, "map_graph_vertex_ids", last_error())
    return ids


def map_graph_csr(handle):
    """(rowptr, colidx, acc_bits) as the handle holds them, as host arrays."""
    n, m = map_graph_info(handle)
    rp = np.empty(n + 1, np.uint32)
    ci = np.empty(max(m, 1), np.uint32)
    ab = np.empty((n + 31) // 32, np.uint32)
    rc = load().map_graph_csr(handle, rp.ctypes.data, ci.ctypes.data, ab.ctypes.data)
    if rc != MAP_OK:
        raise MapError(rc, "map_graph_csr", last_error())
    return rp, ci[:m], ab


def map_destroy(handle) -> None:
    if handle is not None and handle.value:
        load().map_destroy(handle)
        handle.value = None


@dataclass
class RunResult:
    status: int
    verdict: int
    witness: int
    outer: int
    rounds: list
    inner_iters: int
    inner_canonical: bool
    relaxations: int
    edges_total: int
    device_ms: float
    dense_ms: float
    dense_launches: int
    accepting_left: int
    launches: int
    round_ms: float
    check_ms: float
    frontier_rows: int
    trace: list
    queue_ms: float = 0.0  # served jobs: waiting for a worker
    setup_ms: float = 0.0  # served jobs: map_create
    run_ms: float = 0.0  # served jobs: run and map back to host memory
    batch_jobs: int = 0  # served jobs: how many jobs shared the job's run (1: alone)


def map_run(handle, sched: int = MAP_SCHED_SYNC, max_outer: int = 0, max_inner: int = 0, flags: int = 0,
            map_out=None, keep_trace: bool = False, hash_trace=None, rounds_cap: int = 1 << 16,
            allow_limit: bool = False, timeout_ms: int = 0, repeat: int = 0) -> RunResult:
    """Run MAP on a created graph.  map_out: optional uint32 numpy array or CUDA tensor of n entries.
    repeat > 1: the same run that many times back to back (see map_opts.repeat)."""
    lib = load()
    opts = MapOpts()
    opts.sched, opts.max_outer, opts.max_inner, opts.flags = sched, max_outer, max_inner, flags
    opts.repeat = repeat
    rounds = np.zeros(max(rounds_cap, 1), dtype=np.uint32)
    opts.rounds_out = rounds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    opts.rounds_cap = rounds_cap
    opts.timeout_ms = timeout_ms
    tr = []
    if keep_trace or hash_trace is not None:
        def _cb(_user, outer, mptr, nn, k):
            vec = np.ctypeslib.as_array(mptr, shape=(nn,))
            tr.append((int(outer), hash_trace(vec) if hash_trace else vec.copy(), int(k)))
        cb = TRACE_FN(_cb)
        opts.trace = cb
    res = MapResult()
    out_ptr, keep = (None, None)
    if map_out is not None:
        if hasattr(map_out, "data_ptr"):
            out_ptr = map_out.data_ptr()
        else:
            assert isinstance(map_out, np.ndarray) and map_out.dtype == np.uint32 and map_out.flags.c_contiguous
            out_ptr = map_out.ctypes.data
    rc = lib.map_run(handle, ctypes.byref(opts), ctypes.byref(res), out_ptr)
    if rc != MAP_OK and not (allow_limit and rc == MAP_ERR_LIMIT):
        raise MapError(rc, "map_run", last_error())
    return RunResult(rc, res.verdict, res.witness, res.outer_iters,
                     [int(x) for x in rounds[:min(res.outer_iters, rounds_cap)]], res.inner_iters,
                     bool(res.inner_canonical), res.relaxations, res.edges_total, res.device_ms, res.dense_ms,
                     res.dense_launches, res.accepting_left, res.launches, res.round_ms, res.check_ms,
                     res.frontier_rows, tr)


def map_run_static(n: int, rowptr, colidx, acc_bits, sched: int = MAP_SCHED_SYNC, max_outer: int = 0,
                   max_inner: int = 0, flags: int = 0, map_out=None, stream=None, rounds_cap: int = 1 << 16,
                   allow_limit: bool = False, timeout_ms: int = 0) -> RunResult:
    """One MAP run without any allocation (small graphs only; see include/map.h).

    For callers that cannot allocate device memory at run time; the library's work space is
    one fixed device array shared by every call on a device, so calls must not overlap.  The
    call blocks and must not be issued on a stream that is being captured."""
    lib = load()
    rp, k1 = _ptr(rowptr)
    ci, k2 = _ptr(colidx)
    ab, k3 = _ptr(acc_bits)
    opts = MapOpts()
    opts.sched, opts.max_outer, opts.max_inner, opts.flags = sched, max_outer, max_inner, flags
    opts.timeout_ms = timeout_ms
    rounds = np.zeros(max(rounds_cap, 1), dtype=np.uint32)
    opts.rounds_out = rounds.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    opts.rounds_cap = rounds_cap
    res = MapResult()
    out_ptr = None
    if map_out is not None:
        out_ptr = map_out.data_ptr() if hasattr(map_out, "data_ptr") else map_out.ctypes.data
    rc = lib.map_run_static(n, rp, ci, ab, ctypes.byref(opts), ctypes.byref(res), out_ptr, _stream_handle(stream))
    if rc != MAP_OK and not (allow_limit and rc == MAP_ERR_LIMIT):
        raise MapError(rc, "map_run_static", last_error())
    return RunResult(rc, res.verdict, res.witness, res.outer_iters,
                     [int(x) for x in rounds[:min(res.outer_iters, rounds_cap)]], res.inner_iters,
                     bool(res.inner_canonical), res.relaxations, res.edges_total, res.device_ms, res.dense_ms,
                     res.dense_launches, res.accepting_left, res.launches, res.round_ms, res.check_ms,
                     res.frontier_rows, [])


def map_batch_create(graphs, stream=None):
    """A batch handle for many graphs: ``graphs`` is a sequence of (n, rowptr, colidx, acc_bits)
    with numpy arrays or CUDA tensors (see map_batch_create in include/map.h)."""
    lib = load()
    count = len(graphs)
    keep = []
    ns = np.array([int(gr[0]) for gr in graphs], dtype=np.uint32)
    arrs = []
    for col in (1, 2, 3):
        ptrs = np.zeros(count, dtype=np.uint64)
        for i, gr in enumerate(graphs):
            p, k = _ptr(gr[col])
            keep.append(k)
            ptrs[i] = p or 0
        arrs.append(ptrs)
    h = ctypes.c_void_p()
    rc = lib.map_batch_create(count, ns.ctypes.data, arrs[0].ctypes.data, arrs[1].ctypes.data, arrs[2].ctypes.data,
                              _stream_handle(stream), ctypes.byref(h))
    if rc != MAP_OK:
        raise MapError(rc, "map_batch_create", last_error())
    h.count = count
    h.total_n = int(ns.sum(dtype=np.uint64))
    return h


def map_batch_run(handle, count: int, sched: int = MAP_SCHED_SYNC, max_outer: int = 0, max_inner: int = 0,
                  flags: int = 0, map_out=None, rounds_cap: int = 256, allow_limit: bool = False):
    """Run a batch; returns a list of RunResult (one per graph, ``rounds`` filled)."""
    lib = load()
    opts = MapOpts()
    opts.sched, opts.max_outer, opts.max_inner, opts.flags = sched, max_outer, max_inner, flags
    res = (MapResult * count)()
    rounds = np.zeros(count * max(rounds_cap, 1), dtype=np.uint32)
    out_ptr = None
    if map_out is not None:
        out_ptr = map_out.data_ptr() if hasattr(map_out, "data_ptr") else map_out.ctypes.data
    rc = lib.map_batch_run(handle, ctypes.byref(opts), res, out_ptr, rounds.ctypes.data, rounds_cap)
    if rc != MAP_OK and not (allow_limit and rc in (MAP_ERR_LIMIT, MAP_ERR_TIMEOUT)):
        raise MapError(rc, "map_batch_run", last_error())
    out = []
    for c in range(count):
        r = res[c]
        rl = [int(x) for x in rounds[c * rounds_cap: c * rounds_cap + min(r.outer_iters, rounds_cap)]]
        out.append(RunResult(r.status, r.verdict, r.witness, r.outer_iters, rl, r.inner_iters,
                             bool(r.inner_canonical), r.relaxations, r.edges_total, r.device_ms, r.dense_ms,
                             r.dense_launches, r.accepting_left, r.launches, r.round_ms, r.check_ms,
                             r.frontier_rows, []))
    return out


def _result(r, trace=()):
    return RunResult(r.status, r.verdict, r.witness, r.outer_iters, [], r.inner_iters, bool(r.inner_canonical),
                     r.relaxations, r.edges_total, r.device_ms, r.dense_ms, r.dense_launches, r.accepting_left,
                     r.launches, r.round_ms, r.check_ms, r.frontier_rows, list(trace), r.queue_ms, r.setup_ms,
                     r.run_ms, r.batch_jobs)


class Server:
    """Continuous-admission serving (map_server_* in include/map.h)."""

    def __init__(self, hbm_budget_bytes: int = 0, slots: int = 4, max_batch: int = 0):
        """max_batch: jobs per run at most (0: the library's default; 1: every job alone)."""
        lib = load()
        self.handle = ctypes.c_void_p()
        rc = lib.map_server_create(hbm_budget_bytes, slots, ctypes.byref(self.handle))
        if rc != MAP_OK:
            raise MapError(rc, "map_server_create", last_error())
        self.sizes = {}
        if max_batch:
            rc = lib.map_server_batch_limit(self.handle, max_batch)
            if rc != MAP_OK:
                self.close()
                raise MapError(rc, "map_server_batch_limit", last_error())

    def submit(self, n, rowptr, colidx, acc_bits, sched: int = MAP_SCHED_SYNC, max_outer: int = 0,
               flags: int = 0) -> int:
        lib = load()
        rp = np.ascontiguousarray(rowptr, dtype=np.uint32)
        ci = np.ascontiguousarray(colidx, dtype=np.uint32) if colidx is not None else None
        ab = np.ascontiguousarray(acc_bits, dtype=np.uint32)
        opts = MapOpts()
        opts.sched, opts.max_outer, opts.flags = sched, max_outer, flags
        jid = ctypes.c_uint64()
        rc = lib.map_submit(self.handle, n, rp.ctypes.data, ci.ctypes.data if ci is not None and ci.size else None,
                            ab.ctypes.data, ctypes.byref(opts), ctypes.byref(jid))
        if rc != MAP_OK:
            raise MapError(rc, "map_submit", last_error())
        self.sizes[jid.value] = n
        return jid.value

    def poll(self, job_id: int, want_map: bool = True):
        """None while the job is queued or running; else (RunResult, map vector or None)."""
        lib = load()
        res = MapResult()
        n = self.sizes.get(job_id)
        out = np.empty(n, np.uint32) if (want_map and n) else None
        rc = lib.map_poll(self.handle, job_id, ctypes.byref(res), out.ctypes.data if out is not None else None)
        if rc == MAP_ERR_NOT_READY:
            return None
        self.sizes.pop(job_id, None)
        if rc != MAP_OK:
            raise MapError(rc, "map_poll", last_error())
        return _result(res), out

    def close(self):
        if self.handle is not None and self.handle.value:
            load().map_server_destroy(self.handle)
            self.handle.value = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def pack_bits(flags) -> np.ndarray:
    """Accepting flags (one byte per vertex) -> LSB-first uint32 bitmap, the layout map_create takes."""
    flags = np.ascontiguousarray(flags, dtype=np.uint8)
    n = flags.shape[0]
    padded = np.zeros(((n + 31) // 32) * 32, dtype=np.uint8)
    padded[:n] = flags != 0
    return np.packbits(padded, bitorder="little").view("<u4").astype(np.uint32)


class Graph:
    """Owning wrapper: ``with Graph(n, rowptr, colidx, acc_flags) as g: g.run()``."""

    def __init__(self, n, rowptr, colidx, acc_flags=None, acc_bits=None, stream=None):
        if acc_bits is None:
            acc_bits = pack_bits(acc_flags)
        self.n = int(n)
        self.handle = map_create(self.n, rowptr, colidx, acc_bits, stream)

    def run(self, **kw) -> RunResult:
        return map_run(self.handle, **kw)

    def lasso(self, witness: int, init: int = MAP_NONE, cap: int = 1 << 20):
        return map_lasso(self.handle, witness, init, cap)

    def close(self):
        map_destroy(self.handle)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
