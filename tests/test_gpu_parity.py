"""GPU <-> oracle parity through the C ABI (bit-exact: MAP is integer work).

Compared element by element: verdict, witness, outer count, round count of every outer
iteration, relaxation count, the map vector of every outer iteration (full vectors for the
small graphs, a blake2b digest per iteration for the large ones) and the final map vector.
Under the asynchronous schedule everything but the round and relaxation counts must match,
and the sweep count never exceeds the synchronous round count.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import mapgen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CASES = json.load(open(os.path.join(HERE, "golden", "hand_cases.json")))["cases"]


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__

    __graft_entry__.build()
    import paper_0912_2555_gb300 as p

    return p


def digest(vec):
    return hashlib.blake2b(np.ascontiguousarray(vec).tobytes(), digest_size=16).hexdigest()


def gpu_run(pkg, g, sched=0, on_device=False, keep_trace=True, hash_trace=None, **kw):
    """One map_run through the C ABI.  With a trace the library steps the loop from the host
    (same kernels); without one the whole run is a single CUDA-graph launch."""
    if on_device:
        rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
        ci = torch.from_numpy(g.colidx.view(np.int32) if g.m else np.zeros(1, np.int32)).cuda()
        ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
        out = torch.empty(g.n, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
    else:
        rp, ci, ab = g.rowptr, (g.colidx if g.m else None), pkg.pack_bits(g.acc)
        out = np.empty(g.n, np.uint32)
        stream = None
    h = pkg.map_create(g.n, rp, ci, ab, stream)
    try:
        r = pkg.map_run(h, sched=sched, map_out=out, keep_trace=keep_trace and hash_trace is None,
                        hash_trace=hash_trace, **kw)
    finally:
        pkg.map_destroy(h)
    final = out.cpu().numpy().view(np.uint32) if on_device else out
    return r, final


def assert_graph_path(pkg, g, want, sched, on_device, per_outer, flags=0):
    """The CUDA-graph driver (no trace): same verdict, counts and final map; with per_outer,
    the map of every outer iteration k from a run stopped by max_outer = k."""
    got, final = gpu_run(pkg, g, sched, on_device, keep_trace=False, flags=flags)
    assert got.status == pkg.MAP_OK
    assert (got.verdict, got.witness, got.outer) == (want.verdict, want.witness, want.outer)
    assert np.array_equal(final, want.map)
    if sched == pkg.MAP_SCHED_SYNC:
        assert (got.rounds, got.relaxations, got.inner_iters) == (want.rounds, want.relaxations, want.inner_total)
    if per_outer:
        for k in range(1, want.outer):
            r, fk = gpu_run(pkg, g, sched, on_device, keep_trace=False, max_outer=k, allow_limit=True, flags=flags)
            assert r.status == pkg.MAP_ERR_LIMIT and r.outer == k
            tr = want.trace[k - 1][1]
            assert (fk == tr).all() if not isinstance(tr, str) else digest(fk) == tr


def assert_parity(pkg, g, sched=0, on_device=False, hashed=False, per_outer=None, want=None, flags=0):
    if want is None:
        want = oracle.run_graph(g, keep_trace=not hashed, hash_trace=digest if hashed else None)
    if per_outer is None:
        per_outer = g.n <= 5000 and want.outer <= 20
    assert_graph_path(pkg, g, want, sched, on_device, per_outer, flags)
    got, final = gpu_run(pkg, g, sched, on_device, keep_trace=not hashed, hash_trace=digest if hashed else None,
                         flags=flags)
    assert got.status == pkg.MAP_OK
    assert (got.verdict, got.witness, got.outer) == (want.verdict, want.witness, want.outer)
    assert np.array_equal(final, want.map)
    assert len(got.trace) == len(want.trace) == want.outer
    for (o1, m1, k1), (o2, m2, k2) in zip(got.trace, want.trace):
        assert o1 == o2
        if hashed:
            assert m1 == m2, f"map differs at outer iteration {o1}"
        else:
            assert np.array_equal(m1, m2), f"map differs at outer iteration {o1}"
    if sched == pkg.MAP_SCHED_SYNC:
        assert got.rounds == want.rounds
        assert got.relaxations == want.relaxations
        assert got.inner_iters == want.inner_total and got.inner_canonical
    else:
        assert all(a <= b for a, b in zip(got.rounds, want.rounds))
        assert not got.inner_canonical
    assert got.edges_total == g.m * want.outer
    return got, want


@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c["name"] for c in CASES])
def test_hand_cases(pkg, case, sched):
    g = mapgen.from_lists(case["rows"], case["acc"])
    assert_parity(pkg, g, sched)


@pytest.mark.parametrize("sched", [0, 1])
def test_random_small(pkg, sched):
    for seed in range(150):
        rng = np.random.default_rng(7000 + seed)
        n = int(rng.integers(1, 300))
        g = mapgen.tiny_graph(seed, n, max_deg=int(rng.integers(0, 9)),
                              acc_p=float(rng.choice([0.0, 0.02, 0.1, 0.3, 1.0])))
        assert_parity(pkg, g, sched)


@pytest.mark.parametrize("variant", ["cycle", "nocycle"])
@pytest.mark.parametrize("on_device", [False, True])
def test_random_16k(pkg, variant, on_device):
    g = mapgen.random_16k(variant)
    got, want = assert_parity(pkg, g, 0, on_device)
    if variant == "cycle":
        assert got.verdict == 1 and got.witness == g.meta["planted"] and got.outer == 1
    assert_parity(pkg, g, 1, on_device)


@pytest.mark.parametrize("G_deg", [(1, 1), (2, 3), (5, 9), (10, 20), (20, 40), (40, 80)])
def test_degree_ranges_select_every_group_size(pkg, G_deg):
    lo, hi = G_deg
    g = mapgen.random_graph(3001, lo, hi, 0.05, seed=lo * 100 + hi, variant="plain")
    assert_parity(pkg, g, 0)
    assert_parity(pkg, g, 1)


def test_ragged_and_degenerate(pkg):
    # n not a multiple of 32, empty rows, a 60k-edge row, self-loops, duplicates
    rng = np.random.default_rng(3)
    n = 1000 + 17
    rows = [[] if v % 7 == 0 else [int(x) for x in rng.integers(0, n, size=int(rng.integers(1, 5)))] for v in range(n)]
    rows[5] = [int(x) for x in rng.integers(0, n, size=60000)]
    rows[9] = [9, 9, 9]
    acc = (rng.random(n) < 0.05).astype(np.uint8)
    acc[9] = 0
    for a in (acc, np.ones(n, np.uint8), np.zeros(n, np.uint8)):
        g = mapgen.from_lists(rows, a)
        assert_parity(pkg, g, 0)
        assert_parity(pkg, g, 1)
    # single vertex, no edges
    assert_parity(pkg, mapgen.from_lists([[]], [1]), 0)
    # graph without any edge at all
    assert_parity(pkg, mapgen.from_lists([[] for _ in range(100)], np.ones(100, np.uint8)), 0)


def test_long_rows_among_short_ones(pkg):
    """Rows of 254-257 and 510 entries next to short and empty ones, in full and ragged
    128-row tiles of the dense round, with and without accepting targets in them."""
    rng = np.random.default_rng(11)
    for n in (300, 128 * 5 + 3):
        lens = rng.integers(0, 6, size=n)
        for v, L in zip(rng.choice(n, size=8, replace=False), (254, 255, 256, 257, 510, 255, 0, 1)):
            lens[v] = L
        rows = [[int(x) for x in rng.integers(0, n, size=int(L))] for L in lens]
        acc = (rng.random(n) < 0.04).astype(np.uint8)
        g = mapgen.from_lists(rows, acc)
        assert_parity(pkg, g, 0)
        assert_parity(pkg, g, 1)


def test_layered_medium(pkg):
    g = mapgen.layered_graph(1 << 20, 62, seed=3)
    assert_parity(pkg, g, 0, on_device=True)
    assert_parity(pkg, g, 1, on_device=True)
    gp = mapgen.layered_graph(1 << 20, 62, seed=3, plant=True)
    got, _ = assert_parity(pkg, gp, 0, on_device=True)
    assert got.verdict == 1


def test_product_8x7_full(pkg):
    g = mapgen.product_8x7()
    got, want = assert_parity(pkg, g, 0, on_device=True, hashed=True)
    assert_parity(pkg, g, 1, on_device=True, hashed=True)


def test_product_interleaved_small(pkg):
    g = mapgen.product_graph(6, 6, interleave=True)
    assert_parity(pkg, g, 0)
    assert_parity(pkg, g, 1)


def test_runs_repeat_exactly(pkg):
    g = mapgen.layered_graph(200000, 12, seed=9)
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        outs = []
        for _ in range(3):
            out = np.empty(g.n, np.uint32)
            r = pkg.map_run(h, map_out=out)
            outs.append((r.verdict, r.witness, r.outer, tuple(r.rounds), r.relaxations, digest(out)))
        assert outs[0] == outs[1] == outs[2]
    finally:
        pkg.map_destroy(h)


def test_invalid_csr_and_limits(pkg):
    with pytest.raises(pkg.MapError) as e:
        pkg.map_create(2, np.array([0, 1, 2], np.uint32), np.array([1, 2], np.uint32), np.array([1], np.uint32))
    assert e.value.code == pkg.MAP_ERR_CSR
    with pytest.raises(pkg.MapError) as e:
        pkg.map_create(2, np.array([0, 2, 1], np.uint32), np.array([1, 0], np.uint32), np.array([1], np.uint32))
    assert e.value.code == pkg.MAP_ERR_CSR
    with pytest.raises(pkg.MapError) as e:
        pkg.map_create(2, np.array([1, 1, 2], np.uint32), np.array([1, 0], np.uint32), np.array([1], np.uint32))
    assert e.value.code == pkg.MAP_ERR_CSR
    g = mapgen.from_lists([[1], [2], []], [1, 1, 1])
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        r = pkg.map_run(h, max_outer=2, allow_limit=True)
        assert r.status == pkg.MAP_ERR_LIMIT and r.outer == 2
        r = pkg.map_run(h, max_inner=2, allow_limit=True)
        assert r.status == pkg.MAP_ERR_LIMIT
        r = pkg.map_run(h)
        assert r.status == pkg.MAP_OK and r.outer == 3 and r.rounds == [3, 2, 1]
    finally:
        pkg.map_destroy(h)


def test_layered_64m_full_size(pkg):
    """The 2^26-vertex layered no-cycle graph, 4,000 layers: full parity, map digests per outer
    iteration, under both schedules."""
    g = mapgen.layered_64m()
    got, want = assert_parity(pkg, g, 0, on_device=True, hashed=True)
    assert got.verdict == 0 and got.outer > 10
    # the asynchronous schedule (the benchmark's): same maps at every outer iteration, fewer sweeps
    assert_parity(pkg, g, 1, on_device=True, hashed=True, per_outer=False, want=want)
    # round 1 pushed from the accepting vertices instead of the dense round, both schedules
    for sched in (0, 1):
        assert_parity(pkg, g, sched, on_device=True, hashed=True, per_outer=False, want=want,
                      flags=pkg.MAP_FLAG_FRONTIER_START)


@pytest.mark.parametrize("sched", [0, 1])
def test_early_exit_mode(pkg, sched):
    """MAP_FLAG_EARLY_EXIT: same verdict; a cycle's witness is accepting and lies on a cycle;
    the outer count never exceeds the full algorithm's; no-cycle graphs are unaffected."""
    from tests import _brute as bf

    gs = [mapgen.random_16k("cycle"), mapgen.random_16k("nocycle"), mapgen.layered_graph(1 << 20, 62, seed=3),
          mapgen.layered_graph(1 << 20, 62, seed=3, plant=True)]
    for seed in range(40):
        rng = np.random.default_rng(300 + seed)
        gs.append(mapgen.tiny_graph(seed, int(rng.integers(2, 120)), max_deg=3, acc_p=0.3))
    for g in gs:
        want = oracle.run_graph(g)
        h = pkg.map_create(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc))
        try:
            final = np.empty(g.n, np.uint32)
            got = pkg.map_run(h, sched=sched, flags=pkg.MAP_FLAG_EARLY_EXIT, map_out=final)
            again = pkg.map_run(h, sched=sched)  # a normal run on the same handle after an early one
        finally:
            pkg.map_destroy(h)
        assert got.verdict == want.verdict, g.name
        assert got.outer <= want.outer
        assert (again.verdict, again.witness, again.outer) == (want.verdict, want.witness, want.outer)
        if sched == 0:
            assert (again.rounds, again.relaxations) == (want.rounds, want.relaxations)
        if got.verdict == 1:
            _, on_cycle = bf.tarjan_verdict(g.n, g.rowptr, g.colidx, g.acc)
            assert g.acc[got.witness] and on_cycle[got.witness]
        else:
            assert (got.outer, got.witness) == (want.outer, want.witness)
            assert np.array_equal(final, want.map)
