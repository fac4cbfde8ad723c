"""Property tests of the CPU oracle (Hypothesis): on generated graphs of up to 40 vertices --
self-loops, duplicate entries, empty rows and any density of accepting vertices allowed --
the oracle must equal the brute-force statement of Section 2 (every map from explicit
reachability, round and relaxation counts from their closed forms, the outer loop replayed
from those maps) and the verdict from strongly connected components.  Hypothesis shrinks a
failing graph to a small one.  (Not on hosts without Hypothesis: the test is skipped.)"""
import numpy as np
import pytest

import mapgen
from tests.test_oracle import _check_against_brute

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies


@st.composite
def graphs(draw):
    n = draw(st.integers(min_value=1, max_value=40))
    rows = draw(st.lists(st.lists(st.integers(min_value=0, max_value=n - 1), max_size=6), min_size=n, max_size=n))
    density = draw(st.sampled_from([0.0, 0.1, 0.3, 0.6, 1.0]))
    u = draw(st.lists(st.floats(min_value=0.0, max_value=1.0, exclude_max=True), min_size=n, max_size=n))
    return mapgen.from_lists(rows, (np.asarray(u) < density).astype(np.uint8))


@hypothesis.settings(max_examples=200, deadline=None, database=None,
                     suppress_health_check=[hypothesis.HealthCheck.too_slow])
@hypothesis.given(graphs())
def test_oracle_equals_brute_force(g):
    _check_against_brute(g)


@hypothesis.settings(max_examples=60, deadline=None, database=None)
@hypothesis.given(st.integers(min_value=2, max_value=30), st.data())
def test_cycle_through_an_accepting_vertex_is_found(n, data):
    """Any graph plus a cycle through an accepting vertex has the verdict 'cycle', with a
    witness that is accepting and lies on a cycle (checked inside _check_against_brute)."""
    rows = data.draw(st.lists(st.lists(st.integers(0, n - 1), max_size=3), min_size=n, max_size=n))
    ring = data.draw(st.lists(st.integers(0, n - 1), min_size=1, max_size=n, unique=True))
    for a, b in zip(ring, ring[1:] + ring[:1]):
        rows[a] = rows[a] + [b]
    acc = np.zeros(n, np.uint8)
    acc[data.draw(st.sampled_from(ring))] = 1
    r = _check_against_brute(mapgen.from_lists(rows, acc))
    assert r.verdict == 1
