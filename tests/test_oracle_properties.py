"""Property tests of the CPU oracle on generated multigraphs (hypothesis).

Each example is a small list of pairs with self-loops, repeats and both
directions mixed in.  The oracle must agree with the all-triples count and
with trace(A^3)/6, and its results must not depend on the presentation of
the input: the order of the pairs, their directions, added repeats and
loops, a relabelling of the vertices, or isolated vertices appended at the
end.  CPU only; skipped where hypothesis is not installed."""
import numpy as np
import pytest

import oracle
from tests import helpers

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings


@st.composite
def multigraphs(draw, max_n=24, max_m=160):
    n = draw(st.integers(1, max_n))
    m = draw(st.integers(0, max_m))
    ids = st.integers(0, n - 1)
    pairs = draw(st.lists(st.tuples(ids, ids), min_size=m, max_size=m))
    s = np.array([p[0] for p in pairs], np.int32)
    d = np.array([p[1] for p in pairs], np.int32)
    return s, d, n


SETTINGS = dict(max_examples=150, deadline=None, derandomize=True)


@settings(**SETTINGS)
@given(multigraphs())
def test_matches_brute_force_and_trace(g):
    s, d, n = g
    r = oracle.forward(s, d, n)
    T, t = helpers.brute_force(s, d, n)
    assert r["T"] == T and np.array_equal(r["t"], t)
    T3, t3 = helpers.trace_cubed(s, d, n)
    assert r["T"] == T3 and np.array_equal(r["t"], t3)
    assert np.array_equal(r["deg"], helpers.simple_degrees(s, d, n))
    assert int(r["t"].sum()) == 3 * r["T"]


@settings(**SETTINGS)
@given(multigraphs(), st.integers(0, 2 ** 32 - 1))
def test_presentation_does_not_matter(g, seed):
    s, d, n = g
    r = oracle.forward(s, d, n)
    rng = np.random.default_rng(seed)
    # shuffled order, random directions, every pair repeated up to twice, loops added
    flip = rng.random(len(s)) < 0.5
    s2 = np.where(flip, d, s)
    d2 = np.where(flip, s, d)
    rep = rng.integers(1, 3, len(s))
    s2, d2 = np.repeat(s2, rep), np.repeat(d2, rep)
    loops = rng.integers(0, n, 5).astype(np.int32)
    s2 = np.concatenate([s2, loops]).astype(np.int32)
    d2 = np.concatenate([d2, loops]).astype(np.int32)
    order = rng.permutation(len(s2))
    r2 = oracle.forward(s2[order], d2[order], n)
    assert r2["T"] == r["T"] and np.array_equal(r2["t"], r["t"])
    assert np.array_equal(r2["deg"], r["deg"])
    # relabelled ids, and isolated vertices appended
    perm = rng.permutation(n).astype(np.int32)
    r3 = oracle.forward(perm[s], perm[d], n + 7)
    assert r3["T"] == r["T"]
    assert np.array_equal(r3["t"][perm], r["t"]) and not r3["t"][n:].any()
    assert np.array_equal(r3["deg"][perm], r["deg"])


@settings(**SETTINGS)
@given(multigraphs())
def test_forward_lists_obey_the_bound(g):
    """Every forward list is at most sqrt(2m) long (Sec. II-B), and the
    forward lists hold every distinct edge once."""
    s, d, n = g
    r = oracle.forward(s, d, n)
    assert r["max_out_degree"] ** 2 <= 2 * r["m"]
    assert r["m"] == int(helpers.simple_degrees(s, d, n).sum()) // 2
