"""On-the-fly detection over a growing graph (map_grow_create / map_append): after every append
the handle holds exactly the part expanded so far (unexpanded vertices have empty rows) and a
run on it matches the oracle's MAP on that partial graph bit for bit."""
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


def partial(g, R, K):
    """The graph once rows 0..R-1 are expanded and K vertices are known."""
    rp = np.concatenate([g.rowptr[:R + 1], np.full(K - R, g.rowptr[R], np.uint32)]).astype(np.uint32)
    return mapgen.Graph(n=K, rowptr=rp, colidx=g.colidx[:g.rowptr[R]].copy(), acc=g.acc[:K].copy())


def stream(pkg, g, known, cuts, on_device=False, check=True):
    """Grow g along `cuts` (row counts); returns the runs after each append."""
    dev = (lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()) if on_device else (lambda a: a)
    K = int(known[0])
    h = pkg.map_grow_create(K, dev(pkg.pack_bits(g.acc[:K])))
    runs = []
    try:
        R = 0
        for R2 in cuts:
            K2 = int(known[R2])
            rp = (g.rowptr[R:R2 + 1] - g.rowptr[R]).astype(np.uint32)
            ci = g.colidx[g.rowptr[R]:g.rowptr[R2]]
            pkg.map_append(h, K2 - K, dev(pkg.pack_bits(g.acc[K:K2])) if K2 > K else None, dev(rp),
                           dev(ci) if len(ci) else None)
            R, K = R2, K2
            out = np.empty(K, np.uint32)
            r = pkg.map_run(h, map_out=out)
            runs.append(r)
            if check:
                p = partial(g, R, K)
                rph, cih, abh = pkg.map_graph_csr(h)
                assert np.array_equal(rph, p.rowptr) and np.array_equal(cih, p.colidx)
                want = oracle.run_graph(p)
                assert (r.verdict, r.witness, r.outer, r.rounds, r.relaxations) == (
                    want.verdict, want.witness, want.outer, want.rounds, want.relaxations), R
                assert np.array_equal(out, want.map), R
    finally:
        pkg.map_destroy(h)
    return runs


def test_small_streams(pkg):
    for seed in range(30):
        rng = np.random.default_rng(600 + seed)
        g0 = mapgen.tiny_graph(seed, int(rng.integers(2, 250)), max_deg=int(rng.integers(1, 5)), acc_p=0.1)
        g, known = mapgen.discovery_order(g0, start=0)
        cuts = sorted(set(int(x) for x in rng.integers(1, g.n + 1, size=4)) | {g.n})
        stream(pkg, g, known, cuts, on_device=seed % 2 == 1)


def test_cycle_found_before_the_graph_is_complete(pkg):
    """random 16k with its planted cycle, streamed in 16 chunks: the verdict turns to a cycle
    before the last chunk, and stays; the final run equals a run on the whole graph."""
    g, known = mapgen.discovery_order(mapgen.random_16k("cycle"), start=0)
    cuts = [int(x) for x in np.linspace(0, g.n, 17)[1:]]
    runs = stream(pkg, g, known, cuts)
    v = [r.verdict for r in runs]
    assert v[-1] == 1 and v.index(1) < len(v) - 1 and all(v[v.index(1):])
    with pkg.Graph(g.n, g.rowptr, g.colidx, g.acc) as h:
        whole = h.run()
    assert (runs[-1].verdict, runs[-1].witness, runs[-1].rounds) == (whole.verdict, whole.witness, whole.rounds)


def test_interleaved_product_streamed(pkg):
    """The interleaving product of 6 processes with 6 states in discovery order from its initial
    state (45,927 states): partial graphs with tens to over a hundred outer iterations."""
    g, known = mapgen.discovery_order(mapgen.product_graph(6, 6, interleave=True), start=0)
    cuts = [g.n // 8, g.n // 3, (2 * g.n) // 3, g.n]
    stream(pkg, g, known, cuts)
    stream(pkg, g, known, cuts, on_device=True)


def test_layered_1m_streamed(pkg):
    """A planted layered graph of 2^20 vertices in discovery order, in five chunks."""
    g, known = mapgen.discovery_order(mapgen.layered_graph(1 << 20, 62, seed=3, plant=True), start=0)
    runs = stream(pkg, g, known, [int(x) for x in np.linspace(0, g.n, 6)[1:]], on_device=True)
    assert runs[-1].verdict == 1


def test_append_to_a_created_graph_and_errors(pkg):
    g = mapgen.from_lists([[1], [0]], [1, 0])
    h = pkg.map_create(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))
    try:
        assert pkg.map_run(h).verdict == 1
        # two new vertices; the row of vertex 2 (-> 3) and of vertex 3 (-> 2)
        pkg.map_append(h, 2, pkg.pack_bits([0, 1]), np.array([0, 1, 2], np.uint32), np.array([3, 2], np.uint32))
        rp, ci, ab = pkg.map_graph_csr(h)
        assert list(rp) == [0, 1, 2, 3, 4] and list(ci) == [1, 0, 3, 2] and ab[0] == 0b1001
        out = np.empty(4, np.uint32)
        r = pkg.map_run(h, map_out=out)
        want = oracle.run(4, rp, ci, [1, 0, 0, 1])  # 0 and 3 are self-mapped: the smaller is the witness
        assert (r.verdict, r.witness, want.witness) == (1, 0, 0) and np.array_equal(out, want.map)
        for args, code in [((1, pkg.pack_bits([0]), np.array([1, 1], np.uint32), np.array([0], np.uint32)),
                            pkg.MAP_ERR_CSR),
                           ((1, pkg.pack_bits([0]), np.array([0, 1], np.uint32), np.array([9], np.uint32)),
                            pkg.MAP_ERR_CSR),
                           ((0, None, np.array([0, 1], np.uint32), np.array([0], np.uint32)), pkg.MAP_ERR_ARG)]:
            with pytest.raises(pkg.MapError) as e:
                pkg.map_append(h, *args)
            assert e.value.code == code
        # the handle is unchanged by the failed appends
        rp2, ci2, _ = pkg.map_graph_csr(h)
        assert np.array_equal(rp, rp2) and np.array_equal(ci, ci2)
        assert pkg.map_run(h).witness == 0
    finally:
        pkg.map_destroy(h)
    hb = pkg.map_batch_create([(g.n, g.rowptr, g.colidx, pkg.pack_bits(g.acc))])
    try:
        with pytest.raises(pkg.MapError) as e:
            pkg.map_append(hb, 1, pkg.pack_bits([0]))
        assert e.value.code == pkg.MAP_ERR_ARG
    finally:
        pkg.map_destroy(hb)
