"""Accepting-part reduction on the GPU (map_create_reduced) against the oracle's reduction:
the reduced graph (ids, CSR, accepting set) bit for bit, then MAP on it against the oracle's MAP
on the oracle's reduced graph, and the verdict against the whole graph's."""
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


def unpack(bits, n):
    return ((bits[np.arange(n) >> 5] >> (np.arange(n) & 31)) & 1).astype(np.uint8)


def reduce_case(pkg, g, part=None, on_device=False, run=True):
    want = oracle.reduce_graph(g.n, g.rowptr, g.colidx, g.acc, part)
    if on_device:
        args = [torch.from_numpy(a.view(np.int32)).cuda() for a in
                (g.rowptr, g.colidx if g.m else np.zeros(1, np.uint32), pkg.pack_bits(g.acc))]
        pt = None if part is None else torch.from_numpy(np.asarray(part, np.uint32).view(np.int32)).cuda()
    else:
        args = [g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc)]
        pt = part
    h = pkg.map_create_reduced(g.n, *args, part=pt)
    try:
        ids = pkg.map_graph_vertex_ids(h)
        rp, ci, ab = pkg.map_graph_csr(h)
        n2 = len(ids)
        if len(want[0]) == 0:  # nothing kept: one isolated non-accepting stand-in vertex
            assert list(ids) == [pkg.MAP_NONE] and list(rp) == [0, 0] and len(ci) == 0 and ab[0] == 0
            r = pkg.map_run(h)
            assert r.verdict == 0 and r.outer == 0
            return want
        assert np.array_equal(ids, want[0])
        assert np.array_equal(rp, want[1]) and np.array_equal(ci, want[2])
        assert np.array_equal(unpack(ab, n2), want[3])
        if run:
            out = np.empty(n2, np.uint32)
            r = pkg.map_run(h, map_out=out)
            o = oracle.run(n2, want[1], want[2], want[3])
            assert (r.verdict, r.witness, r.outer, r.rounds, r.relaxations) == (
                o.verdict, o.witness, o.outer, o.rounds, o.relaxations)
            assert np.array_equal(out, o.map)
    finally:
        pkg.map_destroy(h)
    return want


def test_small_graphs(pkg):
    for seed in range(120):
        rng = np.random.default_rng(4000 + seed)
        g = mapgen.tiny_graph(seed, int(rng.integers(1, 300)), max_deg=int(rng.integers(0, 6)),
                              acc_p=float(rng.choice([0.0, 0.02, 0.1, 0.5])))
        part = rng.integers(0, 3, size=g.n).astype(np.uint32) if seed % 3 == 0 else None
        reduce_case(pkg, g, part, on_device=seed % 2 == 1)


@pytest.mark.parametrize("variant", ["cycle", "nocycle"])
def test_random_16k(pkg, variant):
    g = mapgen.random_16k(variant)
    reduce_case(pkg, g)
    reduce_case(pkg, g, on_device=True)


def test_product_8x7_with_automaton_labels(pkg):
    """Labels = the component of the 2-state property automaton each state projects to (one
    component: both automaton states reach each other), and a split labelling by the automaton
    state, which drops the automaton's edges between its two states."""
    g = mapgen.product_8x7()
    reduce_case(pkg, g, on_device=True, run=False)
    b = (np.arange(g.n) >= g.n // 2).astype(np.uint32)  # id = b * 7^8 + ...
    reduce_case(pkg, g, part=b, on_device=True, run=False)


def test_layered_medium(pkg):
    for plant in (False, True):
        g = mapgen.layered_graph(1 << 20, 62, seed=3, plant=plant)
        reduce_case(pkg, g, on_device=True)


def test_layered_64m_full_size(pkg):
    """The 2^26-vertex bench graph: by construction the reduced graph is the accepting DAG (every
    accepting vertex, the edges between accepting vertices); its MAP has the whole graph's
    verdict and elimination sequence (non-accepting vertices never have a value there)."""
    g = mapgen.layered_64m()
    h = pkg.map_create_reduced(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        ids = pkg.map_graph_vertex_ids(h)
        rp, ci, ab = pkg.map_graph_csr(h)
        A = np.flatnonzero(g.acc)
        assert np.array_equal(ids, A)
        acc_rows = np.repeat(g.acc.astype(bool), np.diff(g.rowptr.astype(np.int64)))
        assert len(ci) == int(np.count_nonzero(acc_rows & g.acc.astype(bool)[g.colidx]))
        r = pkg.map_run(h)
    finally:
        pkg.map_destroy(h)
    hf = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        rf = pkg.map_run(hf)
    finally:
        pkg.map_destroy(hf)
    assert (r.verdict, r.outer) == (rf.verdict, rf.outer) == (0, rf.outer)


def test_plain_handle_exports(pkg):
    g = mapgen.random_16k("cycle")
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        rp, ci, ab = pkg.map_graph_csr(h)
        assert np.array_equal(rp, g.rowptr) and np.array_equal(ci, g.colidx)
        assert np.array_equal(unpack(ab, g.n), g.acc.astype(np.uint8))
        assert np.array_equal(pkg.map_graph_vertex_ids(h), np.arange(g.n, dtype=np.uint32))
        ids = torch.empty(g.n, dtype=torch.int32, device="cuda")
        assert pkg.load().map_graph_vertex_ids(h, ids.data_ptr()) == pkg.MAP_OK
        assert np.array_equal(ids.cpu().numpy(), np.arange(g.n, dtype=np.int32))
    finally:
        pkg.map_destroy(h)


def test_no_accepting_vertex(pkg):
    reduce_case(pkg, mapgen.from_lists([[1], [0], []], [0, 0, 0]))
