"""MAP_FLAG_FRONTIER_START: round 1 of every outer iteration pushed from the accepting
vertices instead of the dense round.

Round 1 relaxes every row from "no value" everywhere (Section 2), so a row gets the largest
accepting vertex it holds and no other row gets anything.  The flag computes exactly those
values from the accepting set, so everything the oracle fixes must match bit for bit: the map
vector of every outer iteration, the verdict, the witness, the outer count and, on the
synchronous schedule, the round and relaxation counts (relaxations stay the canonical counts
of the pull schedule).  The full-size layered graph is checked in test_gpu_parity.py, batches
in test_gpu_batch.py.
"""
import numpy as np
import pytest

import mapgen
import oracle
from tests.test_gpu_parity import CASES, assert_parity, digest, pkg  # noqa: F401  (fixture)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fs(pkg):
    return pkg.MAP_FLAG_FRONTIER_START


@pytest.mark.parametrize("sched", [0, 1])
def test_hand_cases(pkg, sched):
    for case in CASES:
        g = mapgen.from_lists(case["rows"], case["acc"])
        assert_parity(pkg, g, sched, flags=_fs(pkg))


@pytest.mark.parametrize("sched", [0, 1])
def test_random_small(pkg, sched):
    for seed in range(100):
        rng = np.random.default_rng(9100 + seed)
        n = int(rng.integers(1, 300))
        g = mapgen.tiny_graph(seed + 500, n, max_deg=int(rng.integers(0, 9)),
                              acc_p=float(rng.choice([0.0, 0.02, 0.1, 0.3, 1.0])))
        assert_parity(pkg, g, sched, flags=_fs(pkg))


@pytest.mark.parametrize("sched", [0, 1])
def test_workloads(pkg, sched):
    for g in (mapgen.random_16k("cycle"), mapgen.random_16k("nocycle"),
              mapgen.random_graph(3001, 20, 40, 0.05, seed=2040, variant="plain"),
              mapgen.product_graph(6, 6, interleave=True)):
        assert_parity(pkg, g, sched, flags=_fs(pkg))


def test_ragged_and_degenerate(pkg):
    rng = np.random.default_rng(5)
    n = 1000 + 17
    rows = [[] if v % 7 == 0 else [int(x) for x in rng.integers(0, n, size=int(rng.integers(1, 5)))] for v in range(n)]
    rows[5] = [int(x) for x in rng.integers(0, n, size=60000)]  # one accepting target read by a huge row
    rows[9] = [9, 9, 9]
    acc = (rng.random(n) < 0.05).astype(np.uint8)
    acc[9] = 0
    hub = [[0] for _ in range(n)]  # every row reads vertex 0: one accepting vertex with n readers
    for r, a in ((rows, acc), (rows, np.ones(n, np.uint8)), (rows, np.zeros(n, np.uint8)),
                 (hub, np.eye(1, n, 0, dtype=np.uint8)[0])):
        g = mapgen.from_lists(r, a)
        for sched in (0, 1):
            assert_parity(pkg, g, sched, flags=_fs(pkg))
    assert_parity(pkg, mapgen.from_lists([[]], [1]), 0, flags=_fs(pkg))
    assert_parity(pkg, mapgen.from_lists([[0]], [1]), 1, flags=_fs(pkg))


def test_layered_medium_device_inputs(pkg):
    g = mapgen.layered_graph(1 << 20, 62, seed=3)
    want = oracle.run_graph(g, keep_trace=False, hash_trace=digest)
    for sched in (0, 1):
        assert_parity(pkg, g, sched, on_device=True, hashed=True, want=want, flags=_fs(pkg))
    gp = mapgen.layered_graph(1 << 20, 62, seed=3, plant=True)
    got, _ = assert_parity(pkg, gp, 1, on_device=True, flags=_fs(pkg))
    assert got.verdict == 1


def test_product_8x7_full(pkg):
    g = mapgen.product_8x7()
    want = oracle.run_graph(g, keep_trace=False, hash_trace=digest)
    for sched in (0, 1):
        assert_parity(pkg, g, sched, on_device=True, hashed=True, want=want, flags=_fs(pkg))


def test_alternating_starts_on_one_handle(pkg):
    """Runs with and without the flag, early exit mixed in, on one handle: each equals the
    oracle (the two starts leave the values and matrix flags in a state the other accepts)."""
    gs = [mapgen.layered_graph(200000, 12, seed=9), mapgen.layered_graph(200000, 12, seed=9, plant=True)]
    for g in gs:
        want = oracle.run_graph(g)
        h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
        try:
            seq = [(0, 0), (0, _fs(pkg)), (1, _fs(pkg)), (0, 0), (1, _fs(pkg) | pkg.MAP_FLAG_EARLY_EXIT),
                   (0, _fs(pkg)), (1, 0), (0, _fs(pkg) | pkg.MAP_FLAG_PROFILE), (0, 0)]
            for sched, flags in seq:
                out = np.empty(g.n, np.uint32)
                r = pkg.map_run(h, sched=sched, flags=flags, map_out=out)
                assert r.verdict == want.verdict, (sched, flags)
                if flags & pkg.MAP_FLAG_EARLY_EXIT:
                    continue
                assert (r.witness, r.outer) == (want.witness, want.outer), (sched, flags)
                assert np.array_equal(out, want.map), (sched, flags)
                if sched == 0:
                    assert (r.rounds, r.relaxations) == (want.rounds, want.relaxations), (sched, flags)
                if flags & pkg.MAP_FLAG_PROFILE:
                    assert r.dense_launches == 0
        finally:
            pkg.map_destroy(h)


def test_refused_for_static_runs(pkg):
    g = mapgen.from_lists([[1], [0]], [1, 0])
    lib = pkg.load()
    import ctypes
    opts = pkg.MapOpts()
    opts.flags = _fs(pkg)
    res = pkg.MapResult()
    rc = lib.map_run_static(g.n, g.rowptr.ctypes.data, g.colidx.ctypes.data, pkg.pack_bits(g.acc).ctypes.data,
                            ctypes.byref(opts), ctypes.byref(res), None, None)
    assert rc == pkg.MAP_ERR_ARG


@pytest.mark.parametrize("sched", [0, 1])
def test_autotune_chooses_a_start(pkg, sched):
    """map_autotune also times both starts and keeps the faster; every later run (the chosen
    start, each start forced) still equals the oracle, and both start flags together are refused."""
    for g in (mapgen.layered_graph(1 << 20, 62, seed=3), mapgen.random_graph(3001, 2, 6, 1.0, seed=77,
                                                                              variant="plain")):
        want = oracle.run_graph(g)
        h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
        try:
            tune = pkg.map_autotune(h, sched)
            assert tune["dense_start_ms"] > 0 and tune["frontier_start_ms"] > 0
            assert tune["frontier_start"] == (tune["frontier_start_ms"] < tune["dense_start_ms"])
            for flags in (0, pkg.MAP_FLAG_DENSE_START, _fs(pkg)):
                out = np.empty(g.n, np.uint32)
                r = pkg.map_run(h, sched=sched, flags=flags, map_out=out)
                assert (r.verdict, r.witness, r.outer) == (want.verdict, want.witness, want.outer), flags
                assert np.array_equal(out, want.map), flags
                if sched == 0:
                    assert (r.rounds, r.relaxations) == (want.rounds, want.relaxations), flags
            p = pkg.map_run(h, sched=sched, flags=pkg.MAP_FLAG_PROFILE)
            assert (p.dense_launches == 0) == tune["frontier_start"]
            p = pkg.map_run(h, sched=sched, flags=pkg.MAP_FLAG_PROFILE | pkg.MAP_FLAG_DENSE_START)
            assert p.dense_launches == p.outer
            with pytest.raises(pkg.MapError) as e:
                pkg.map_run(h, flags=_fs(pkg) | pkg.MAP_FLAG_DENSE_START)
            assert e.value.code == pkg.MAP_ERR_ARG
        finally:
            pkg.map_destroy(h)
