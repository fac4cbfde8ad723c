"""map_create from every kind of source array.

Device arrays and page-locked host arrays are read by the set-up pass itself, which copies them
into the graph while it validates, counts in-degrees and packs the accepting flags (one pass over
HBM or the host link instead of a copy and then a pass).  Pageable host arrays, and a colidx that
is not 16-byte aligned, are copied first and then ingested in place.  Every route must build the
same graph: the run gives the oracle's verdict, witness, outer count, canonical counts and final
map, and an invalid CSR is refused from each route."""
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


def _arrays(kind, rowptr, colidx):
    """rowptr / colidx as the source kind asks; 'misaligned' variants start 4 bytes past a
    16-byte boundary (a view one element into a larger buffer)."""
    rp = np.ascontiguousarray(rowptr, np.uint32).view(np.int32)
    ci = np.ascontiguousarray(colidx if len(colidx) else np.zeros(1, np.uint32), np.uint32).view(np.int32)
    if kind == "pageable":
        return rowptr, colidx if len(colidx) else None
    if kind in ("pinned", "pinned-misaligned"):
        trp = torch.from_numpy(rp).pin_memory()
        if kind == "pinned":
            return trp, torch.from_numpy(ci).pin_memory()
        big = torch.from_numpy(np.concatenate([np.zeros(1, np.int32), ci])).pin_memory()
        view = big[1:]
        assert view.data_ptr() % 16 == 4
        return trp, view
    trp = torch.from_numpy(rp).cuda()
    if kind == "device":
        return trp, torch.from_numpy(ci).cuda()
    big = torch.from_numpy(np.concatenate([np.zeros(1, np.int32), ci])).cuda()
    view = big[1:]
    assert view.data_ptr() % 16 == 4
    return trp, view


KINDS = ["pageable", "pinned", "device", "pinned-misaligned", "device-misaligned"]

GRAPHS = [
    ("layered-60k", lambda: mapgen.layered_graph(60000, 8, seed=5)),
    ("layered-60k-cycle", lambda: mapgen.layered_graph(60000, 8, seed=6, plant=True)),
    ("random-16k-cycle", lambda: mapgen.random_16k("cycle")),
    ("product-4x6", lambda: mapgen.product_graph(4, 6, interleave=True)),
    ("tiny-odd-m", lambda: mapgen.from_lists([[1, 2], [2], [0], [], [4]], [1, 0, 1, 0, 1])),
    ("no-edges", lambda: mapgen.from_lists([[], [], []], [1, 0, 1])),
]


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("name,make", GRAPHS, ids=[g[0] for g in GRAPHS])
def test_every_source_builds_the_same_graph(pkg, name, make, kind):
    g = make()
    want = oracle.run_graph(g)
    rp, ci = _arrays(kind, g.rowptr, g.colidx)
    h = pkg.map_create(g.n, rp, ci if g.m else None, pkg.pack_bits(g.acc), torch.cuda.current_stream())
    try:
        for sched in (0, 1):
            out = np.empty(g.n, np.uint32)
            r = pkg.map_run(h, sched=sched, map_out=out)
            assert (r.status, r.verdict, r.witness, r.outer) == (pkg.MAP_OK, want.verdict, want.witness, want.outer)
            assert np.array_equal(out, want.map)
            if sched == 0:
                assert (r.rounds, r.relaxations) == (want.rounds, want.relaxations)
    finally:
        pkg.map_destroy(h)
    # the caller's arrays are read, never written
    back_rp = rp.cpu().numpy().view(np.uint32) if hasattr(rp, "cpu") else rp
    assert np.array_equal(back_rp, g.rowptr)
    if g.m:
        back_ci = ci.cpu().numpy().view(np.uint32) if hasattr(ci, "cpu") else ci
        assert np.array_equal(back_ci, g.colidx)


@pytest.mark.parametrize("kind", KINDS)
def test_invalid_csr_refused_from_every_source(pkg, kind):
    acc = np.array([1], np.uint32)
    cases = [
        ([0, 1, 2, 4, 5], [1, 2, 3, 9, 0]),  # an entry >= n
        ([0, 2, 1, 4, 5], [1, 0, 2, 3, 0]),  # rowptr decreasing
        ([0, 1, 2, 3, 7], [1, 2, 3, 0, 1, 2, 4]),  # the last entry >= n (in the scalar tail)
    ]
    for rowptr, colidx in cases:
        rp, ci = _arrays(kind, np.array(rowptr, np.uint32), np.array(colidx, np.uint32))
        with pytest.raises(pkg.MapError) as e:
            pkg.map_create(4, rp, ci, acc, torch.cuda.current_stream())
        assert e.value.code == pkg.MAP_ERR_CSR, (kind, rowptr, colidx)
