"""map_run_static: the entry point that allocates nothing.

Some callers cannot allocate device memory while they run: plug-ins whose host application
owns the whole device budget and hands none of it out, and real-time loops that must never
enter an allocator.  map_run_static serves them from one fixed device array.

It must give exactly what map_create + map_run give on the same graph -- verdict, witness,
outer count, per-iteration round counts, relaxation count, status and final map vector
(integer work: the tolerance is zero) -- on two calls in a row, since every call reuses the
same device array and must clear what the previous call left in it.  Each result is also
checked against the CPU oracle, and the options the call accepts besides the defaults
(early exit, the outer-iteration limit, the dense start) are compared with map_run too.
This file is collected last and is self-contained, so it passes alone in a fresh process
as well."""
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


def _reference(pkg, g, sched, **kw):
    out = np.empty(g.n, np.uint32)
    h = pkg.map_create(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc))
    try:
        r = pkg.map_run(h, sched=sched, map_out=out, **kw)
    finally:
        pkg.map_destroy(h)
    return r, out


def _static(pkg, g, sched, on_device, **kw):
    if on_device:
        rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
        ci = torch.from_numpy(g.colidx.view(np.int32) if g.m else np.zeros(1, np.int32)).cuda()
        ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        r = pkg.map_run_static(g.n, rp, ci, ab, sched=sched, map_out=out, stream=torch.cuda.current_stream(), **kw)
        return r, out.cpu().numpy().view(np.uint32)
    out = np.full(g.n, 7, np.uint32)
    r = pkg.map_run_static(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc), sched=sched, map_out=out,
                           **kw)
    return r, out


def _same(a, b, sched=0):
    ra, ma = a
    rb, mb = b
    assert (ra.status, ra.verdict, ra.witness, ra.outer, ra.edges_total, ra.inner_canonical) == \
        (rb.status, rb.verdict, rb.witness, rb.outer, rb.edges_total, rb.inner_canonical)
    if sched == 0:  # the asynchronous schedule's sweep and relaxation counts depend on timing
        assert (ra.rounds, ra.inner_iters, ra.relaxations) == (rb.rounds, rb.inner_iters, rb.relaxations)
    assert np.array_equal(ma, mb)


def _matches_oracle(got, want, sched):
    r, final = got
    assert r.status == 0
    assert (r.verdict, r.witness, r.outer) == (want.verdict, want.witness, want.outer)
    assert np.array_equal(final, want.map)
    if sched == 0:
        assert (r.rounds, r.relaxations, r.inner_iters) == (want.rounds, want.relaxations, want.inner_total)
    else:
        assert all(a <= b for a, b in zip(r.rounds, want.rounds))


GRAPHS = [
    ("random-cycle", lambda: mapgen.random_16k("cycle")),
    ("random-nocycle", lambda: mapgen.random_16k("nocycle")),
    ("layered-60k", lambda: mapgen.layered_graph(60000, 8, seed=5)),
    ("product-4x6", lambda: mapgen.product_graph(4, 6, interleave=True)),
    ("tiny", lambda: mapgen.tiny_graph(3, 40, max_deg=3, acc_p=0.4)),
    ("no-accepting", lambda: mapgen.from_lists([[1], [0], []], [0, 0, 0])),
]


@pytest.mark.parametrize("sched", [0, 1])
@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_matches_map_run_on_two_calls_in_a_row(pkg, name, make, sched):
    g = make()
    want = _reference(pkg, g, sched)
    truth = oracle.run_graph(g)
    for on_device in (False, True):
        first = _static(pkg, g, sched, on_device)
        second = _static(pkg, g, sched, on_device)
        _same(first, want, sched)
        _same(second, want, sched)
        _matches_oracle(first, truth, sched)
        _matches_oracle(second, truth, sched)


def test_a_larger_then_a_smaller_graph(pkg):
    """The second call must not see the first call's leftovers."""
    big = mapgen.layered_graph(60000, 8, seed=9)
    small = mapgen.tiny_graph(11, 50, max_deg=4, acc_p=0.5)
    want_small = _reference(pkg, small, 0)
    _static(pkg, big, 0, True)
    got = _static(pkg, small, 0, True)
    _same(got, want_small)
    _matches_oracle(got, oracle.run_graph(small), 0)


def _on_cycle(g, v):
    """v reaches itself along rows by at least one edge (plain BFS over the successor lists)."""
    seen = np.zeros(g.n, bool)
    todo = [int(u) for u in g.colidx[g.rowptr[v]:g.rowptr[v + 1]]]
    while todo:
        u = todo.pop()
        if u == v:
            return True
        if seen[u]:
            continue
        seen[u] = True
        todo.extend(int(w) for w in g.colidx[g.rowptr[u]:g.rowptr[u + 1]])
    return False


@pytest.mark.parametrize("name,make", GRAPHS[:4], ids=[g[0] for g in GRAPHS[:4]])
def test_early_exit_as_map_run(pkg, name, make):
    """MAP_FLAG_EARLY_EXIT is honoured: under the synchronous schedule the run stops after the
    same round as map_run's (same witness, outer count and round counts, no longer canonical
    once it stopped early); the verdict is the oracle's and a witness is accepting and on a cycle."""
    g = make()
    fl = pkg.MAP_FLAG_EARLY_EXIT
    truth = oracle.run_graph(g)
    want = _reference(pkg, g, 0, flags=fl)
    for _ in range(2):
        got = _static(pkg, g, 0, False, flags=fl)
        ra, _ = got
        rb, _ = want
        assert (ra.status, ra.verdict, ra.witness, ra.outer, ra.rounds, ra.inner_canonical) == \
            (rb.status, rb.verdict, rb.witness, rb.outer, rb.rounds, rb.inner_canonical)
        assert ra.verdict == truth.verdict
        if ra.verdict:
            assert g.acc[ra.witness] and _on_cycle(g, ra.witness)
        else:  # no cycle: the full fix-point every time, the oracle's result
            _matches_oracle(got, truth, 0)
    r_async, _ = _static(pkg, g, 1, True, flags=fl)
    assert r_async.verdict == truth.verdict
    if r_async.verdict:
        assert g.acc[r_async.witness] and _on_cycle(g, r_async.witness)


@pytest.mark.parametrize("sched", [0, 1])
def test_outer_limit_and_dense_start_as_map_run(pkg, sched):
    """max_outer = 1 stops with MAP_ERR_LIMIT after the first outer iteration (status set in the
    result, the map of that iteration out) exactly as map_run does; MAP_FLAG_DENSE_START is the
    default start and changes nothing."""
    g = mapgen.layered_graph(60000, 8, seed=5)
    truth = oracle.run_graph(g, keep_trace=True)
    assert truth.outer > 1
    want = _reference(pkg, g, sched, max_outer=1, allow_limit=True)
    got = _static(pkg, g, sched, False, max_outer=1, allow_limit=True)
    _same(got, want, sched)
    assert got[0].status == pkg.MAP_ERR_LIMIT and got[0].outer == 1
    assert np.array_equal(got[1], truth.trace[0][1])
    if sched == 0:
        assert got[0].rounds == truth.rounds[:1]
    dense = _static(pkg, g, sched, True, flags=pkg.MAP_FLAG_DENSE_START)
    _same(dense, _reference(pkg, g, sched), sched)
    _matches_oracle(dense, truth, sched)


def test_rejects_sizes_beyond_the_limit(pkg):
    n = pkg.MAP_STATIC_MAX_N + 1
    rp = np.zeros(n + 1, np.uint32)
    with pytest.raises(pkg.MapError) as e:
        pkg.map_run_static(n, rp, None, np.zeros((n + 31) // 32, np.uint32))
    assert e.value.code == pkg.MAP_ERR_ARG and "MAP_STATIC_MAX_N" in str(e.value)
    n = 1000
    m = pkg.MAP_STATIC_MAX_M + 1
    rp = np.zeros(n + 1, np.uint32)
    rp[1:] = m
    with pytest.raises(pkg.MapError) as e:
        pkg.map_run_static(n, rp, np.zeros(m, np.uint32), np.zeros((n + 31) // 32, np.uint32))
    assert e.value.code == pkg.MAP_ERR_ARG and "MAP_STATIC_MAX_M" in str(e.value)
