"""The oracle's pins catch plausible mistakes.

Each case copies the oracle's C source, plants one mistake (a dropped term, a wrong
comparison, a wrong schedule or tie-break), builds the copy in a temporary directory
and checks that the hand-derived cases or the brute-force comparison reject it.
The oracle in the repository is never modified.
"""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

import mapgen
import oracle
from tests import _brute as bf

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "map_oracle.c")
HDR = os.path.join(os.path.dirname(HERE), "oracle", "map_oracle.h")
CASES = json.load(open(os.path.join(HERE, "golden", "hand_cases.json")))["cases"]

MUTANTS = {
    # a non-accepting vertex offers its own id
    "offer_non_accepting": ("if (A[u] && (int64_t)u > offered)", "if ((int64_t)u > offered)"),
    # reflexive map: a vertex offers itself to itself
    "reflexive": ("int64_t best = map[v];", "int64_t best = (A[v] && (int64_t)v > map[v]) ? (int64_t)v : map[v];"),
    # witness = largest self-mapped vertex instead of the smallest
    "witness_max": ("                witness = v;\n                break;", "                witness = v;"),
    # map not reset when the procedure restarts
    "no_reset": ("for (uint32_t v = 0; v < n; ++v) map[v] = NONE;\n        uint32_t nf", "uint32_t nf"),
    # new values applied during the round (Gauss-Seidel instead of synchronous)
    "in_place": ("                    chg_val[nc] = best;\n", "                    chg_val[nc] = best;\n                    map[v] = best;\n"),
    # the final no-change round not counted
    "rounds_minus_one": ("rounds[outer - 1] = k;", "rounds[outer - 1] = k - 1;"),
    # next round relaxes the successors of changed vertices instead of their readers
    "wrong_frontier": ("for (uint32_t e = rdeg[u]; e < rdeg[u + 1]; ++e) {\n                    uint32_t w = readers[e];",
                       "for (uint32_t e = rowptr[u]; e < rowptr[u + 1]; ++e) {\n                    uint32_t w = colidx[e];"),
    # elimination only of the map values of accepting vertices
    "elim_from_accepting_only": ("if (map[v] != NONE && !elim[map[v]])", "if (map[v] != NONE && A[v] && !elim[map[v]])"),
    # loop ends while one accepting vertex is left
    "stop_when_one_left": ("while (nacc > 0) {", "while (nacc > 1) {"),
    # the propagated term dropped: only direct successors offer values
    "no_propagation": ("int64_t offered = map[u];", "int64_t offered = NONE;"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    d = tmp_path / name
    d.mkdir()
    (d / "map_oracle.c").write_text(src.replace(old, new))
    shutil.copy(HDR, d / "map_oracle.h")
    lib = d / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(lib), str(d / "map_oracle.c")])
    return oracle.load_library(str(lib))


def _pins_pass(lib):
    """True if every pin accepts this oracle build."""
    for c in CASES:
        g = mapgen.from_lists(c["rows"], c["acc"])
        r = oracle.run_graph(g, keep_trace=True, lib=lib, max_outer=g.n + 2)
        want_w = oracle.NONE if c["witness"] is None else c["witness"]
        if (r.verdict, r.witness, r.outer, r.rounds) != (c["verdict"], want_w, c["outer"], c["rounds"]):
            return False
        for (_, mp, _), want in zip(r.trace, c["maps"]):
            if not np.array_equal(mp, np.array([oracle.NONE if x is None else x for x in want], np.uint32)):
                return False
    for seed in range(60):
        rng = np.random.default_rng(1000 + seed)
        n = int(rng.integers(1, 30))
        g = mapgen.tiny_graph(seed, n, max_deg=int(rng.integers(0, 5)), acc_p=float(rng.choice([0.1, 0.3, 0.7])))
        r = oracle.run_graph(g, keep_trace=True, lib=lib, max_outer=g.n + 2)
        verdict, witness, outer, rounds, maps, relax = bf.brute_map_run(g.n, g.rowptr, g.colidx, g.acc)
        if (r.verdict, r.witness, r.outer, r.rounds, r.relaxations) != (
                verdict, oracle.NONE if witness is None else witness, outer, rounds, relax):
            return False
        if any(not np.array_equal(mp, want) for (_, mp, _), want in zip(r.trace, maps)):
            return False
    return True


def test_unmodified_copy_passes(tmp_path):
    lib = _build_mutant(tmp_path, "identity", "int oracle_map(", "int oracle_map(")
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    lib = _build_mutant(tmp_path, name, old, new)
    assert not _pins_pass(lib), f"mutant {name} passed every pin"
