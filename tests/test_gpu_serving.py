"""Serving with continuous admission: jobs submitted over time while others run, admitted as
workers and the memory budget free up; every job's result must be exactly its result alone
(checked against the oracle), whatever else is in flight.  With several workers each job's
cooperative fix-point kernel runs on a share of the device, so these cases also cover the
smaller launch shapes (4, 3 and 8 workers)."""
import threading
import time

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


def _jobs():
    gs = []
    for seed in range(20):
        rng = np.random.default_rng(4000 + seed)
        gs.append(mapgen.tiny_graph(seed, int(rng.integers(1, 300)), max_deg=int(rng.integers(0, 6)),
                                    acc_p=float(rng.choice([0.0, 0.1, 0.5]))))
    gs += [mapgen.random_16k("cycle"), mapgen.random_16k("nocycle"), mapgen.layered_graph(80000, 10, seed=2),
           mapgen.layered_graph(80000, 10, seed=2, plant=True), mapgen.product_graph(5, 6, interleave=False)]
    return gs


@pytest.mark.parametrize("slots,budget,sched", [(4, 0, 0), (3, 8 << 20, 0), (8, 0, 1)])
def test_jobs_in_flight_get_their_own_results(pkg, slots, budget, sched):
    gs = _jobs()
    want = [oracle.run_graph(g) for g in gs]
    ids = [None] * len(gs)
    with pkg.Server(hbm_budget_bytes=budget, slots=slots) as sv:
        def submitter():
            rng = np.random.default_rng(1)
            for i in rng.permutation(len(gs)):
                g = gs[i]
                ids[i] = sv.submit(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc), sched=sched)
                time.sleep(float(rng.exponential(0.002)))
        th = threading.Thread(target=submitter)
        th.start()
        th.join()
        results = [None] * len(gs)
        deadline = time.time() + 120
        while any(r is None for r in results) and time.time() < deadline:
            for i, jid in enumerate(ids):
                if results[i] is None:
                    results[i] = sv.poll(jid)
            time.sleep(0.001)
    assert all(r is not None for r in results)
    for g, w, (r, mp) in zip(gs, want, results):
        assert (r.verdict, r.witness, r.outer) == (w.verdict, w.witness, w.outer), g.name
        if sched == 0:  # canonical counts; asynchronous sweeps are at most the rounds
            assert (r.relaxations, r.inner_iters) == (w.relaxations, w.inner_total), g.name
        else:
            assert r.inner_iters <= w.inner_total, g.name
        assert np.array_equal(mp, w.map), g.name


def test_poll_before_ready_and_unknown_job(pkg):
    g = mapgen.layered_graph(200000, 12, seed=3)
    with pkg.Server(slots=1) as sv:
        jid = sv.submit(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
        first = sv.poll(jid)  # most likely still running
        while first is None:
            time.sleep(0.001)
            first = sv.poll(jid)
        assert first[0].verdict == oracle.run_graph(g).verdict
        with pytest.raises(pkg.MapError) as e:
            sv.poll(jid)  # released after the first successful poll
        assert e.value.code == pkg.MAP_ERR_ARG


def test_submit_refuses_device_inputs(pkg):
    g = mapgen.from_lists([[1], [0]], [1, 0])
    lib = pkg.load()
    import ctypes
    with pkg.Server(slots=1) as sv:
        d = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
        jid = ctypes.c_uint64()
        rc = lib.map_submit(sv.handle, g.n, d.data_ptr(), g.colidx.ctypes.data, pkg.pack_bits(g.acc).ctypes.data,
                            None, ctypes.byref(jid))
        assert rc == pkg.MAP_ERR_ARG


def test_injected_allocation_failure_fails_only_that_job(pkg, monkeypatch):
    """Host-side fault injection (MAPGPU_INJECT_OOM): the 3rd device allocation of job 4's set-up
    fails.  That job reports MAP_ERR_OOM at map_poll; the jobs before, beside and after it still get
    the oracle's results, and the server keeps serving (its memory accounting is intact)."""
    monkeypatch.setenv("MAPGPU_INJECT_OOM", "4:3,9:1")
    gs = _jobs()[18:]  # two tiny graphs, both 16k workloads, the layered graphs, the product
    want = [oracle.run_graph(g) for g in gs]
    with pkg.Server(slots=3) as sv:
        ids = [sv.submit(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc), sched=s)
               for s in (0, 1) for g in gs]
        assert ids == list(range(1, len(ids) + 1))
        done = {}
        deadline = time.time() + 120
        while len(done) < len(ids) and time.time() < deadline:
            for k, jid in enumerate(ids):
                if jid in done:
                    continue
                try:
                    got = sv.poll(jid)
                except pkg.MapError as e:
                    done[jid] = e
                    continue
                if got is not None:
                    done[jid] = got
            time.sleep(0.001)
        assert len(done) == len(ids)
        for k, jid in enumerate(ids):
            g, w = gs[k % len(gs)], want[k % len(gs)]
            if jid in (4, 9):
                assert isinstance(done[jid], pkg.MapError) and done[jid].code == pkg.MAP_ERR_OOM
                assert "injected" in str(done[jid])
                continue
            r, mp = done[jid]
            assert (r.verdict, r.witness, r.outer) == (w.verdict, w.witness, w.outer), g.name
            assert np.array_equal(mp, w.map), g.name
            assert r.queue_ms >= 0 and r.setup_ms > 0 and r.run_ms > 0
        # still serving after the failures
        g = gs[2]
        jid = sv.submit(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
        got = None
        while got is None:
            got = sv.poll(jid)
            time.sleep(0.001)
        assert np.array_equal(got[1], want[2].map)


def test_queued_jobs_share_batched_runs(pkg):
    """Continuous batching: with one worker busy on a larger job, the jobs queued behind it are
    joined into batched runs (jobs with the same schedule and start only; early exit keeps a job
    to itself).  Every job still gets exactly its own result, and a job with an invalid graph
    fails alone: its batch falls back to single runs."""
    big = mapgen.layered_graph(4_000_000, 240, seed=8)
    gs, scheds, flags = [], [], []
    for seed in range(48):
        rng = np.random.default_rng(7000 + seed)
        if seed % 6 == 5:
            g = mapgen.layered_graph(int(rng.integers(2000, 30000)), 6, seed=seed, plant=bool(seed % 2))
        else:
            g = mapgen.tiny_graph(seed + 300, int(rng.integers(1, 400)), max_deg=int(rng.integers(0, 6)),
                                  acc_p=float(rng.choice([0.0, 0.1, 0.5])))
        gs.append(g)
        scheds.append(0 if (seed // 12) % 2 == 0 else 1)  # runs of 12 sync jobs, then 12 async ones
        flags.append(pkg.MAP_FLAG_EARLY_EXIT if seed == 30 else (pkg.MAP_FLAG_FRONTIER_START if seed % 7 == 3 else 0))
    want = [oracle.run_graph(g) for g in gs]
    bad_at = 20  # an entry >= n: the graph is refused
    bad_rowptr = np.array([0, 1, 2], np.uint32)
    bad_colidx = np.array([1, 5], np.uint32)
    with pkg.Server(slots=1) as sv:
        first = sv.submit(big.n, big.rowptr, big.colidx, pkg.pack_bits(big.acc))
        ids = []
        for i, g in enumerate(gs):
            if i == bad_at:
                ids.append(sv.submit(2, bad_rowptr, bad_colidx, np.array([3], np.uint32), sched=scheds[i]))
            ids.append(sv.submit(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc), sched=scheds[i],
                                 flags=flags[i]))
        deadline = time.time() + 120
        done = {}
        while len(done) < len(ids) + 1 and time.time() < deadline:
            for jid in [first] + ids:
                if jid in done:
                    continue
                try:
                    got = sv.poll(jid)
                except pkg.MapError as e:
                    got = e
                if got is not None:
                    done[jid] = got
            time.sleep(0.001)
    assert len(done) == len(ids) + 1
    bad_id = ids.pop(bad_at)
    assert isinstance(done[bad_id], pkg.MapError) and done[bad_id].code == pkg.MAP_ERR_CSR
    batched = 0
    for i, (g, w, jid) in enumerate(zip(gs, want, ids)):
        r, mp = done[jid]
        assert r.status == pkg.MAP_OK, g.name
        assert r.verdict == w.verdict, g.name
        if flags[i] == pkg.MAP_FLAG_EARLY_EXIT:
            assert r.batch_jobs == 1
            continue
        assert (r.witness, r.outer) == (w.witness, w.outer), g.name
        assert np.array_equal(mp, w.map), g.name
        if scheds[i] == 0:
            assert (r.relaxations, r.inner_iters) == (w.relaxations, w.inner_total), g.name
        else:
            assert r.inner_iters <= w.inner_total, g.name
        batched += r.batch_jobs > 1
    assert batched >= len(ids) // 2  # most of the queued jobs shared a run


def test_many_workers_many_small_jobs(pkg):
    """Eight workers, one job each (no batching), hundreds of small jobs submitted at once: the
    device is shared by up to eight cooperative fix-point launches plus the others' set-up and
    dense rounds, so a launch's blocks may start well apart.  Rounds over few vertices run in
    block 0 alone while the other blocks wait for its hand-back; every job must finish with
    exactly its own result (a late-starting block must not miss or mistake a hand-back)."""
    gs, scheds = [], []
    for seed in range(320):
        rng = np.random.default_rng(9100 + seed)
        kind = seed % 4
        if kind == 0:
            g = mapgen.tiny_graph(seed + 5000, int(rng.integers(20, 400)), max_deg=int(rng.integers(1, 5)),
                                  acc_p=float(rng.choice([0.02, 0.1, 0.3])))
        elif kind in (1, 2):
            g = mapgen.layered_graph(int(rng.integers(2000, 40000)), int(rng.integers(6, 30)), seed=seed,
                                     plant=bool(seed % 3 == 0))
        else:
            g = mapgen.product_graph(4, int(rng.integers(4, 6)), interleave=bool(seed % 2))
        gs.append(g)
        scheds.append(int(seed % 2))
    want = [oracle.run_graph(g) for g in gs]
    with pkg.Server(slots=8, max_batch=1) as sv:
        ids = [sv.submit(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc), sched=sc)
               for g, sc in zip(gs, scheds)]
        results = [None] * len(ids)
        deadline = time.time() + 180
        while any(r is None for r in results) and time.time() < deadline:
            for i, jid in enumerate(ids):
                if results[i] is None:
                    results[i] = sv.poll(jid)
            time.sleep(0.001)
    assert all(r is not None for r in results)
    for g, w, sc, (r, mp) in zip(gs, want, scheds, results):
        assert r.batch_jobs == 1
        assert (r.status, r.verdict, r.witness, r.outer) == (pkg.MAP_OK, w.verdict, w.witness, w.outer), g.name
        assert np.array_equal(mp, w.map), g.name
        if sc == 0:
            assert (r.relaxations, r.inner_iters) == (w.relaxations, w.inner_total), g.name
