"""Comparison rules shared by the GPU parity tests.

Integer-valued inputs are exact in float32 on both sides, so there the GPU must
equal the oracle bit for bit (ids, counts) and distances to float32 rounding.

Float inputs: the GPU ranks in float32, the oracle in float64, so a decision
between two values closer than the float32 rounding error may go either way.
  - Distances are compared with a tolerance of 1e-5 relative.
  - A GPU squared distance passes through at most 39 roundings (one per
    coordinate difference and square, at most 32 sequential sums per lane at
    d <= 1024, five reduction levels), so its relative error is below
    39 * 2^-24 = 2.3e-6 and a distance's below 1.2e-6.  Two such values, or a
    value and the bound r(1+eps) (computed in double from a float32 r^2), can
    therefore be ordered differently only if they are within 2.4e-6 relative:
    DECIDE = 3e-6 is the threshold of a near-tied decision.
  - kNN lists: an id may differ only where the competing float64 distances are
    within 1e-5 relative (the multiset of distances agrees within 1e-5).
  - search (Algorithm 1): a near-tie may change which node is expanded next,
    and from there the whole run.  The oracle reports per query the smallest
    relative gap over every comparison it decided (the margin).  A query whose
    margin exceeds DECIDE took no decision that float32 can take differently, so
    the GPU must return the same result set, the same distance-computation and
    expansion counts, and the same order up to swaps of distances within 1e-5.
    Every other query must still return a valid list: distinct ids, ascending
    distances equal to the float64 distance of each returned id within 1e-5,
    -1 / +inf padding.
"""
import numpy as np

REL = 1e-5
DECIDE = 3e-6


def d64(X, Q, ids):
    """float64 distances of Q[r] to X[ids[r, c]] (inf where ids < 0)."""
    ok = ids >= 0
    diff = X[np.where(ok, ids, 0)].astype(np.float64) - Q[:, None, :].astype(np.float64)
    out = np.sqrt((diff * diff).sum(2))
    out[~ok] = np.inf
    return out


def assert_valid_lists(ids, dist, X, Q, rel=REL):
    """Distinct ids per row, -1 / +inf padding at the end only, distances ascending
    and equal to the float64 distance of each returned id within `rel`."""
    for r in range(len(ids)):
        row = ids[r]
        m = int((row >= 0).sum())
        assert (row[:m] >= 0).all() and (row[m:] == -1).all(), (r, row)
        assert len(set(row[:m].tolist())) == m, (r, row)
        assert np.isinf(dist[r, m:]).all(), r
        assert (np.diff(dist[r, :m]) >= 0).all(), (r, dist[r])
    want = d64(X, Q, ids)
    ok = ids >= 0
    np.testing.assert_allclose(dist[ok], want[ok], rtol=rel)


def assert_rows_near(ids, lens, o_ids, o_lens, rel=REL):
    """Rows equal except for ids whose competing distances are within `rel`:
    position by position the distances agree within `rel`."""
    assert ids.shape == o_ids.shape
    fin = np.isfinite(o_lens)
    assert np.array_equal(np.isfinite(lens), fin)
    np.testing.assert_allclose(lens[fin], o_lens[fin], rtol=rel)
    assert np.array_equal(ids[~fin], o_ids[~fin])


def assert_search_parity(ids, dist, st, o_ids, o_dist, o_st, margin, X, Q, min_tie_free=0.5, counts=True,
                         rel=REL):
    """The margin rule for float data (module docstring).  Returns the fraction of
    queries the oracle decided without a near-tie."""
    assert_valid_lists(ids, dist, X, Q, rel)
    tf = margin > DECIDE
    frac = float(tf.mean())
    assert frac >= min_tie_free, f"only {frac:.2f} of the queries are tie-free"
    for r in np.nonzero(tf)[0]:
        a, b = ids[r], o_ids[r]
        assert set(a[a >= 0].tolist()) == set(b[b >= 0].tolist()), (r, a, b)
        np.testing.assert_allclose(dist[r][a >= 0], o_dist[r][b >= 0], rtol=rel)
    if counts:
        assert np.array_equal(st[tf, 0], o_st[tf, 0]), "distance computations differ on tie-free queries"
        assert np.array_equal(st[tf, 1], o_st[tf, 1]), "expansions differ on tie-free queries"
    return frac


def assert_reranked(ids, dist, cand, X, Q, k, rel=REL):
    """The rerank of a reduced-precision search, for queries whose candidate
    search was tie-free: `cand` [nq, k_rerank] are the oracle's kept candidates;
    the GPU's k results must be the k nearest of them in float64, up to swaps of
    distances within `rel`."""
    dc = d64(X, Q, cand)
    order = np.lexsort((np.where(cand >= 0, cand, np.iinfo(np.int32).max), dc), axis=1)[:, :k]
    want_ids = np.take_along_axis(cand, order, 1)
    want_d = np.take_along_axis(dc, order, 1)
    assert_valid_lists(ids, dist, X, Q, rel)
    for r in range(len(ids)):
        got = ids[r][ids[r] >= 0]
        assert set(got.tolist()) <= set(cand[r][cand[r] >= 0].tolist()), r
    assert_rows_near(ids, dist.astype(np.float64), want_ids, want_d, rel)
