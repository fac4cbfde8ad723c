"""map_run_static: the entry point that allocates nothing (for callers that cannot allocate
device memory while they run, e.g. while their stream is captured into a CUDA graph).

It must give exactly what map_create + map_run give on the same graph -- verdict, witness,
outer count, per-iteration round counts, relaxation count and final map vector (integer
work: the tolerance is zero) -- on two calls in a row, since every call reuses the same
device array and must clear what the previous call left in it.  This file is collected
last and is self-contained, so it passes alone in a fresh process as well."""
import numpy as np
import pytest

import mapgen

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


def _reference(pkg, g, sched):
    out = np.empty(g.n, np.uint32)
    h = pkg.map_create(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc))
    try:
        r = pkg.map_run(h, sched=sched, map_out=out)
    finally:
        pkg.map_destroy(h)
    return r, out


def _static(pkg, g, sched, on_device):
    if on_device:
        rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
        ci = torch.from_numpy(g.colidx.view(np.int32) if g.m else np.zeros(1, np.int32)).cuda()
        ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
        out = torch.full((g.n,), 7, dtype=torch.int32, device="cuda")
        r = pkg.map_run_static(g.n, rp, ci, ab, sched=sched, map_out=out, stream=torch.cuda.current_stream())
        return r, out.cpu().numpy().view(np.uint32)
    out = np.full(g.n, 7, np.uint32)
    r = pkg.map_run_static(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc), sched=sched, map_out=out)
    return r, out


def _same(a, b, sched=0):
    ra, ma = a
    rb, mb = b
    assert (ra.verdict, ra.witness, ra.outer, ra.edges_total) == (rb.verdict, rb.witness, rb.outer, rb.edges_total)
    if sched == 0:  # the asynchronous schedule's sweep and relaxation counts depend on timing
        assert (ra.rounds, ra.inner_iters, ra.relaxations) == (rb.rounds, rb.inner_iters, rb.relaxations)
    assert np.array_equal(ma, mb)


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
    for on_device in (False, True):
        first = _static(pkg, g, sched, on_device)
        second = _static(pkg, g, sched, on_device)
        _same(first, want, sched)
        _same(second, want, sched)


def test_a_larger_then_a_smaller_graph(pkg):
    """The second call must not see the first call's leftovers."""
    big = mapgen.layered_graph(60000, 8, seed=9)
    small = mapgen.tiny_graph(11, 50, max_deg=4, acc_p=0.5)
    want_small = _reference(pkg, small, 0)
    _static(pkg, big, 0, True)
    _same(_static(pkg, small, 0, True), want_small)


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
