"""The device-side time limit (map_opts.timeout_ms): the kernels compare %globaltimer against
the run's start at every outer iteration and every fix-point round, and stop the run with
MAP_ERR_TIMEOUT -- no fault, no hang, the context stays usable.  The next plain run on the same
handle must give the oracle's result exactly (the round state a stopped run leaves behind is
cleared, and the eliminated vertices' flags are restored).  Checked with the loop as one CUDA
graph and stepped from the host, for both schedules and with pull rounds."""
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


def handle(pkg, g):
    rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
    ci = torch.from_numpy(g.colidx.view(np.int32)).cuda()
    ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
    return pkg.map_create(g.n, rp, ci, ab, torch.cuda.current_stream())


@pytest.fixture(scope="module")
def layered24():
    g = mapgen.layered_graph(1 << 24, 1000, seed=3)
    return g, oracle.run_graph(g)


MODES = ["sync-graph", "sync-stepped", "async-graph", "async-stepped", "sync-pull-graph", "frontier-async-graph"]


@pytest.mark.parametrize("mode", MODES)
def test_time_limit_then_exact_run(pkg, layered24, mode):
    """timeout_ms = 1 on a run of several milliseconds (40 outer iterations on 2^24 vertices)."""
    g, want = layered24
    sched = pkg.MAP_SCHED_SYNC if mode.startswith("sync") else pkg.MAP_SCHED_ASYNC
    flags = 0
    if "stepped" in mode:
        flags |= pkg.MAP_FLAG_PROFILE
    if "pull" in mode:
        flags |= pkg.MAP_FLAG_PULL
    if mode.startswith("frontier"):
        flags |= pkg.MAP_FLAG_FRONTIER_START
    h = handle(pkg, g)
    try:
        with pytest.raises(pkg.MapError) as e:
            pkg.map_run(h, sched=sched, flags=flags, timeout_ms=1)
        assert e.value.code == pkg.MAP_ERR_TIMEOUT
        for _ in range(2):
            out = np.empty(g.n, np.uint32)
            r = pkg.map_run(h, sched=sched, flags=flags & ~pkg.MAP_FLAG_PROFILE, map_out=out)
            assert (r.status, r.verdict, r.witness, r.outer) == (pkg.MAP_OK, want.verdict, want.witness, want.outer)
            assert np.array_equal(out, want.map)
            if sched == pkg.MAP_SCHED_SYNC:
                assert (r.rounds, r.relaxations) == (want.rounds, want.relaxations)
            else:
                assert all(a <= b for a, b in zip(r.rounds, want.rounds))
    finally:
        pkg.map_destroy(h)


def test_time_limit_inside_the_rounds(pkg):
    """The product graph has one outer iteration whose 930 synchronous rounds take milliseconds:
    the limit is reached inside the fix-point loop, whose blocks all stop after the same barrier;
    the next run is the oracle's, canonical counts included."""
    g = mapgen.product_8x7()
    want = oracle.run_graph(g)
    h = handle(pkg, g)
    try:
        with pytest.raises(pkg.MapError) as e:
            pkg.map_run(h, sched=pkg.MAP_SCHED_SYNC, timeout_ms=1)
        assert e.value.code == pkg.MAP_ERR_TIMEOUT
        out = np.empty(g.n, np.uint32)
        r = pkg.map_run(h, sched=pkg.MAP_SCHED_SYNC, map_out=out)
        assert (r.verdict, r.witness, r.outer, r.rounds, r.relaxations) == (
            want.verdict, want.witness, want.outer, want.rounds, want.relaxations)
        assert np.array_equal(out, want.map)
    finally:
        pkg.map_destroy(h)
