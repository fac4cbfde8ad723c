"""map_opts.repeat: the same MAP run several times back to back from one map_run call (queued on
the stream with no host step between the runs, as a throughput measurement issues them).  Every
run must give what one run gives -- verdict, witness, outer count, canonical counts under the
synchronous schedule, the map vector (the oracle's) -- and the options that leave round state
behind for the host to clear are refused."""
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


@pytest.mark.parametrize("make", [lambda: mapgen.random_16k("cycle"), lambda: mapgen.layered_graph(1 << 20, 64, seed=23),
                                  lambda: mapgen.product_graph(6, 6, interleave=False)],
                         ids=["16k-cycle", "layered-2^20", "product-6x6"])
def test_repeat_gives_one_runs_result(pkg, make):
    g = make()
    want = oracle.run_graph(g)
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        for sched in (0, 1):
            for flags in (pkg.MAP_FLAG_DENSE_START, pkg.MAP_FLAG_FRONTIER_START):
                out = np.full(g.n, 7, np.uint32)
                r = pkg.map_run(h, sched=sched, flags=flags, map_out=out, repeat=4)
                assert (r.status, r.verdict, r.witness, r.outer) == (pkg.MAP_OK, want.verdict, want.witness, want.outer)
                assert np.array_equal(out, want.map)
                if sched == 0:
                    assert (r.rounds, r.relaxations) == (want.rounds, want.relaxations)
        # and a plain run after them still gives the oracle's result
        out = np.empty(g.n, np.uint32)
        r = pkg.map_run(h, sched=0, map_out=out)
        assert (r.verdict, r.witness, r.outer, r.rounds) == (want.verdict, want.witness, want.outer, want.rounds)
        assert np.array_equal(out, want.map)
    finally:
        pkg.map_destroy(h)


def test_repeat_refused_where_a_run_may_stop_early(pkg):
    g = mapgen.random_16k("nocycle")
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        for kw in (dict(flags=pkg.MAP_FLAG_EARLY_EXIT), dict(max_outer=2), dict(max_inner=3),
                   dict(flags=pkg.MAP_FLAG_PROFILE), dict(keep_trace=True)):
            with pytest.raises(pkg.MapError) as e:
                pkg.map_run(h, repeat=2, **kw)
            assert e.value.code == pkg.MAP_ERR_ARG
    finally:
        pkg.map_destroy(h)
