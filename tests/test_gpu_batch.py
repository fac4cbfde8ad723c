"""Batched runs (many graphs in one launch): every graph must get exactly what it gets alone --
verdict, witness (in its own ids), outer count, rounds of every outer iteration, relaxation
count and final map vector -- checked against separate map_run calls and against the oracle,
with the dense start and with the frontier start (MAP_FLAG_FRONTIER_START)."""
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


def _mixed_graphs():
    gs = []
    for seed in range(24):
        rng = np.random.default_rng(9000 + seed)
        gs.append(mapgen.tiny_graph(seed, int(rng.integers(1, 200)), max_deg=int(rng.integers(0, 6)),
                                    acc_p=float(rng.choice([0.0, 0.05, 0.3, 1.0]))))
    gs.append(mapgen.random_16k("cycle"))
    gs.append(mapgen.random_16k("nocycle"))
    gs.append(mapgen.layered_graph(50000, 8, seed=4))
    gs.append(mapgen.layered_graph(50000, 8, seed=4, plant=True))
    gs.append(mapgen.product_graph(5, 5, interleave=True))
    gs.append(mapgen.from_lists([[]], [1]))
    gs.append(mapgen.from_lists([[0]], [1]))
    gs.append(mapgen.from_lists([[1], [2], []], [1, 1, 1]))
    return gs


@pytest.mark.parametrize("start", ["dense", "frontier"])
@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("on_device", [False, True])
def test_batch_equals_separate_runs_and_oracle(pkg, sched, on_device, start):
    flags = pkg.MAP_FLAG_FRONTIER_START if start == "frontier" else 0
    gs = _mixed_graphs()
    dev = (lambda a: torch.from_numpy(a.view(np.int32)).cuda()) if on_device else (lambda a: a)
    items = [(g.n, dev(g.rowptr), dev(g.colidx if g.m else np.zeros(1, np.uint32)), dev(pkg.pack_bits(g.acc)))
             for g in gs]
    total = sum(g.n for g in gs)
    h = pkg.map_batch_create(items)
    try:
        out = np.empty(total, np.uint32)
        res = pkg.map_batch_run(h, len(gs), sched=sched, map_out=out, flags=flags)
        res2 = pkg.map_batch_run(h, len(gs), sched=sched, flags=flags)  # runs repeat exactly
    finally:
        pkg.map_destroy(h)
    off = 0
    for g, r, r2 in zip(gs, res, res2):
        want = oracle.run_graph(g)
        assert r.status == pkg.MAP_OK
        assert (r.verdict, r.witness, r.outer) == (want.verdict, want.witness, want.outer), g.name
        assert np.array_equal(out[off:off + g.n], want.map), g.name
        if sched == 0:
            assert r.rounds == want.rounds, g.name
            assert r.relaxations == want.relaxations, g.name
            assert r.inner_iters == want.inner_total
        assert (r2.verdict, r2.witness, r2.outer) == (r.verdict, r.witness, r.outer)
        if sched == 0:  # asynchronous sweep and relaxation counts depend on the schedule
            assert (r2.rounds, r2.relaxations) == (r.rounds, r.relaxations)
        else:
            assert all(a <= b for a, b in zip(r.rounds, want.rounds))
        off += g.n


def test_batch_of_layered_graphs_with_planted_cycles(pkg):
    sizes, planted, seeds = mapgen.batch_plan(count=24, lo=1000, hi=100000, frac_cycle=0.4, seed=4)
    gs = [mapgen.batch_graph(int(s), bool(p), int(sd)) for s, p, sd in zip(sizes, planted, seeds)]
    h = pkg.map_batch_create([(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc)) for g in gs])
    try:
        res = pkg.map_batch_run(h, len(gs))
        resf = pkg.map_batch_run(h, len(gs), flags=pkg.MAP_FLAG_FRONTIER_START)
    finally:
        pkg.map_destroy(h)
    for g, p, r, rf in zip(gs, planted, res, resf):
        want = oracle.run_graph(g)
        for x in (r, rf):
            assert (x.verdict, x.witness, x.outer, x.rounds, x.relaxations) == (
                want.verdict, want.witness, want.outer, want.rounds, want.relaxations)
        assert r.verdict == int(p)


def test_batch_handle_refused_by_map_run(pkg):
    g = mapgen.from_lists([[1], [0]], [1, 0])
    h = pkg.map_batch_create([(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))])
    try:
        with pytest.raises(pkg.MapError) as e:
            pkg.map_run(h)
        assert e.value.code == pkg.MAP_ERR_ARG
    finally:
        pkg.map_destroy(h)
    with pytest.raises(pkg.MapError) as e:  # an edge leaving its graph is rejected
        pkg.map_batch_create([(2, np.array([0, 1, 1], np.uint32), np.array([2], np.uint32), np.array([1], np.uint32)),
                              (1, np.array([0, 0], np.uint32), None, np.array([1], np.uint32))])
    assert e.value.code == pkg.MAP_ERR_CSR


def test_autotune_keeps_results(pkg):
    """map_autotune only changes launch shapes: results before and after are identical."""
    gs = _mixed_graphs()[-8:]
    h = pkg.map_batch_create([(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc)) for g in gs])
    try:
        before = pkg.map_batch_run(h, len(gs))
        tune = pkg.map_autotune(h)
        after = pkg.map_batch_run(h, len(gs))
    finally:
        pkg.map_destroy(h)
    assert tune["trials"] >= 2 and tune["dense_blocks_per_sm"] >= 1 and tune["rounds_blocks_per_sm"] >= 1
    for a, b in zip(before, after):
        assert (a.verdict, a.witness, a.outer, a.rounds, a.relaxations) == (
            b.verdict, b.witness, b.outer, b.rounds, b.relaxations)
    g = mapgen.random_16k("nocycle")
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        want = oracle.run_graph(g)
        pkg.map_autotune(h)
        r = pkg.map_run(h)
        assert (r.verdict, r.outer, r.rounds, r.relaxations) == (want.verdict, want.outer, want.rounds,
                                                                 want.relaxations)
    finally:
        pkg.map_destroy(h)


def test_full_256_graph_batch_sampled_against_oracle(pkg):
    """The batch the benchmark times (256 layered graphs, n log-uniform in [1e3, 2e6], 40 % planted
    cycles, seed 4), run as one batch; a sample of graphs across the size range is checked one by
    one against the oracle, and every graph's verdict against its planted cycle."""
    sizes, planted, seeds = mapgen.batch_plan(count=256, lo=1000, hi=2_000_000, frac_cycle=0.4, seed=4)
    gs = [mapgen.batch_graph(int(s), bool(p), int(sd)) for s, p, sd in zip(sizes, planted, seeds)]
    h = pkg.map_batch_create([(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc)) for g in gs])
    try:
        total = sum(g.n for g in gs)
        out = torch.empty(total, dtype=torch.int32, device="cuda")
        res = pkg.map_batch_run(h, len(gs), map_out=out)
        out = out.cpu().numpy().view(np.uint32)
    finally:
        pkg.map_destroy(h)
    assert [r.verdict for r in res] == [int(p) for p in planted]
    offs = np.concatenate([[0], np.cumsum([g.n for g in gs])])
    order = np.argsort(sizes)
    sample = sorted(set(int(order[i]) for i in np.linspace(0, len(gs) - 1, 10).astype(int)))
    for i in sample:
        want = oracle.run_graph(gs[i])
        r = res[i]
        assert (r.verdict, r.witness, r.outer, r.rounds, r.relaxations) == (
            want.verdict, want.witness, want.outer, want.rounds, want.relaxations), i
        assert np.array_equal(out[offs[i]:offs[i + 1]], want.map), i
