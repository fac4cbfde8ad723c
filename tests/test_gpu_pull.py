"""Pull rounds: a round whose list is a large share of the graph streams the whole matrix and
lets every row take the largest offer of its changed entries, instead of pushing from the
list through the reverse CSR.  Under the synchronous schedule it is the same Jacobi step, so
everything stays bit-exact with the oracle -- verdict, witness, outer count, the map of every
outer iteration, and the canonical round and relaxation counts -- whether every round pulls
(MAP_FLAG_PULL), none does (MAP_FLAG_PUSH) or the handle's threshold decides, in single graphs
and in batches, under the asynchronous schedule's sweeps as well."""
import hashlib

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


def digest(vec):
    return hashlib.blake2b(np.ascontiguousarray(vec).tobytes(), digest_size=16).hexdigest()


def handle(pkg, g):
    rp = torch.from_numpy(g.rowptr.view(np.int32)).cuda()
    ci = torch.from_numpy(g.colidx.view(np.int32) if g.m else np.zeros(1, np.int32)).cuda()
    ab = torch.from_numpy(pkg.pack_bits(g.acc).view(np.int32)).cuda()
    return pkg.map_create(g.n, rp, ci, ab, torch.cuda.current_stream())


def check(pkg, h, g, want, sched, flags, hashed=False, per_outer=True):
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    r = pkg.map_run(h, sched=sched, flags=flags, map_out=out)
    assert r.status == pkg.MAP_OK
    assert (r.verdict, r.witness, r.outer) == (want.verdict, want.witness, want.outer)
    assert np.array_equal(out.cpu().numpy().view(np.uint32), want.map)
    if sched == pkg.MAP_SCHED_SYNC:
        assert (r.rounds, r.relaxations, r.inner_iters) == (want.rounds, want.relaxations, want.inner_total)
        assert r.inner_canonical
    else:
        assert all(a <= b for a, b in zip(r.rounds, want.rounds))
    if per_outer:
        t = pkg.map_run(h, sched=sched, flags=flags, keep_trace=not hashed, hash_trace=digest if hashed else None)
        assert len(t.trace) == want.outer
        for (o1, m1, k1), (o2, m2, k2) in zip(t.trace, want.trace):
            assert (m1 == m2) if hashed else np.array_equal(m1, m2), f"map differs at outer iteration {o1}"
            assert (k1 == k2) if sched == pkg.MAP_SCHED_SYNC else (k1 <= k2)
        if sched == pkg.MAP_SCHED_SYNC:
            assert (t.rounds, t.relaxations) == (want.rounds, want.relaxations)
    return r


MODES = [("sync-pull", 0, 128), ("sync-default", 0, 0), ("async-pull", 1, 128)]
STARTS = [("dense", 8), ("frontier", 4)]


@pytest.mark.parametrize("start,sflag", STARTS, ids=[s[0] for s in STARTS])
@pytest.mark.parametrize("mode,sched,mflag", MODES, ids=[m[0] for m in MODES])
def test_random_small(pkg, mode, sched, mflag, start, sflag):
    for seed in range(100):
        rng = np.random.default_rng(9700 + seed)
        n = int(rng.integers(1, 300))
        g = mapgen.tiny_graph(seed + 900, n, max_deg=int(rng.integers(0, 9)),
                              acc_p=float(rng.choice([0.0, 0.02, 0.1, 0.3, 1.0])))
        want = oracle.run_graph(g, keep_trace=True)
        h = handle(pkg, g)
        try:
            check(pkg, h, g, want, sched, mflag | sflag)
        finally:
            pkg.map_destroy(h)


@pytest.mark.parametrize("make", [lambda: mapgen.random_16k("cycle"), lambda: mapgen.random_16k("nocycle"),
                                  lambda: mapgen.layered_graph(1 << 20, 64, seed=21),
                                  lambda: mapgen.layered_graph(1 << 20, 64, seed=22, plant=True),
                                  lambda: mapgen.product_graph(5, 6, interleave=True),
                                  lambda: mapgen.product_graph(6, 6, interleave=False)],
                         ids=["16k-cycle", "16k-nocycle", "layered-2^20", "layered-2^20-cycle", "interleaved-5x6",
                              "product-6x6"])
def test_workloads(pkg, make):
    g = make()
    want = oracle.run_graph(g, hash_trace=digest)
    h = handle(pkg, g)
    try:
        for _, sched, mflag in MODES + [("sync-push", 0, 64)]:
            for _, sflag in STARTS:
                check(pkg, h, g, want, sched, mflag | sflag, hashed=True)
    finally:
        pkg.map_destroy(h)


def test_product_8x7_sync_pull_canonical(pkg):
    """930 synchronous rounds, the first ones over 1.5 million changed vertices: pulled or pushed,
    the canonical counts are the oracle's."""
    g = mapgen.product_8x7()
    want = oracle.run_graph(g)
    h = handle(pkg, g)
    try:
        for fl in (128, 0, 64):
            check(pkg, h, g, want, 0, fl, per_outer=False)
    finally:
        pkg.map_destroy(h)


def test_batch_pull(pkg):
    """Batched runs pull over the union (finished graphs' tiles skipped) with each graph's own
    counts: every graph gets exactly its result alone, canonical counts included."""
    gs = []
    for seed in range(14):
        rng = np.random.default_rng(300 + seed)
        gs.append(mapgen.tiny_graph(seed + 40, int(rng.integers(1, 200)), max_deg=int(rng.integers(0, 6)),
                                    acc_p=float(rng.choice([0.0, 0.1, 0.4]))))
    gs += [mapgen.random_16k("cycle"), mapgen.random_16k("nocycle"), mapgen.layered_graph(120000, 12, seed=6),
           mapgen.layered_graph(120000, 12, seed=7, plant=True), mapgen.product_graph(5, 6, interleave=False)]
    want = [oracle.run_graph(g) for g in gs]
    items = [(g.n, g.rowptr, g.colidx if g.m else None, pkg.pack_bits(g.acc)) for g in gs]
    hb = pkg.map_batch_create(items)
    try:
        for sched, fl in ((0, 128), (0, 0), (1, 128), (0, 64)):
            out = np.empty(sum(g.n for g in gs), np.uint32)
            res = pkg.map_batch_run(hb, len(gs), sched=sched, flags=fl, map_out=out)
            off = 0
            for g, w, r in zip(gs, want, res):
                assert (r.verdict, r.witness, r.outer) == (w.verdict, w.witness, w.outer), g.name
                assert np.array_equal(out[off:off + g.n], w.map), g.name
                if sched == 0:
                    assert (r.rounds, r.relaxations) == (w.rounds, w.relaxations), g.name
                else:
                    assert all(a <= b for a, b in zip(r.rounds, w.rounds)), g.name
                off += g.n
    finally:
        pkg.map_destroy(hb)


def test_push_and_pull_flags_refused_together(pkg):
    g = mapgen.random_16k("nocycle")
    h = handle(pkg, g)
    try:
        with pytest.raises(pkg.MapError) as e:
            pkg.map_run(h, flags=pkg.MAP_FLAG_PUSH | pkg.MAP_FLAG_PULL)
        assert e.value.code == pkg.MAP_ERR_ARG
    finally:
        pkg.map_destroy(h)
