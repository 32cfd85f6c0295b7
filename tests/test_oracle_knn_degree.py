"""Pins of the oracle's exact kNN graph and static degree adjustment (Algorithm 2).

Each check compares against something other than the oracle itself: scipy's
k-d tree, hand-built point sets, scipy.sparse transposes for the special graphs
KNNG / TKNNG / BKNNG of Sec. 2.1, and a sequential transcription of Algorithm 2.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.spatial import cKDTree

from paper_1810_07355_gb300 import synth


def test_knn_matches_kdtree(oracle_lib):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(600, 8)).astype(np.float32)
    Q = rng.normal(size=(40, 8)).astype(np.float32)
    ids, dist = oracle_lib.knn(X, Q, 12)
    td, ti = cKDTree(X.astype(np.float64)).query(Q.astype(np.float64), k=12)
    assert np.array_equal(ids, ti)
    np.testing.assert_allclose(dist, td, rtol=1e-12)


def test_knng_excludes_self_matches_kdtree(oracle_lib):
    X = synth.gaussian_mixture(500, d=16, components=5, sigma=3.0, seed=11)
    ids, dist = oracle_lib.knng(X, 10)
    td, ti = cKDTree(X.astype(np.float64)).query(X.astype(np.float64), k=11)
    # continuous data: the nearest point of every row is itself
    assert np.array_equal(ti[:, 0], np.arange(500))
    assert np.array_equal(ids, ti[:, 1:])
    np.testing.assert_allclose(dist, td[:, 1:], rtol=1e-12)


def test_knn_line_ties_and_duplicates(oracle_lib):
    # points on a line: 0, 1, 2, 2 (duplicate), 5
    X = np.array([[0], [1], [2], [2], [5]], np.float32)
    ids, dist = oracle_lib.knng(X, 3)
    # node 1: nodes 0, 2, 3 all at distance 1 -> id order
    assert ids[1].tolist() == [0, 2, 3]
    # node 2: its duplicate 3 at distance 0 is a neighbour (self excluded by id only)
    assert ids[2].tolist() == [3, 1, 0]
    assert dist[2].tolist() == [0.0, 1.0, 2.0]
    assert ids[4].tolist() == [2, 3, 1]
    # k larger than n - 1 pads with -1 / inf
    ids, dist = oracle_lib.knng(X[:3], 4)
    assert ids[0].tolist() == [1, 2, -1, -1]
    assert np.isinf(dist[0, 2:]).all()


def _csr(ptr, col, ln, n):
    return sp.csr_matrix((ln, col, ptr), shape=(n, n))


def _knng_matrix(ids, dist, m):
    n = ids.shape[0]
    rows = np.repeat(np.arange(n), m)
    return sp.csr_matrix((dist[:, :m].ravel(), (rows, ids[:, :m].ravel())), shape=(n, n))


def _check_sorted_unique(ptr, col, ln):
    for i in range(len(ptr) - 1):
        c, l = col[ptr[i]:ptr[i + 1]], ln[ptr[i]:ptr[i + 1]]
        assert len(set(c.tolist())) == len(c), "duplicate edge"
        assert i not in set(c.tolist()), "self loop"
        order = np.lexsort((c, l))
        assert np.array_equal(order, np.arange(len(c))), "not sorted by (len, id)"


@pytest.fixture(scope="module")
def small_graph(oracle_lib):
    X = synth.gaussian_mixture(300, d=12, components=4, sigma=4.0, seed=5)
    ids, dist = oracle_lib.knng(X, 16)
    return X, ids, dist


def test_degree_knng_special_case(oracle_lib, small_graph):
    _, ids, dist = small_graph
    ptr, col, ln = oracle_lib.adjust_degree(ids, dist, 10, 0)
    assert np.array_equal(np.diff(ptr), np.full(300, 10))
    assert np.array_equal(col.reshape(300, 10), ids[:, :10])
    np.testing.assert_array_equal(ln.reshape(300, 10), dist[:, :10])


def test_degree_tknng_is_transpose(oracle_lib, small_graph):
    _, ids, dist = small_graph
    n, k = ids.shape
    ptr, col, ln = oracle_lib.adjust_degree(ids, dist, 0, k)
    got = _csr(ptr, col, ln, n)
    want = _knng_matrix(ids, dist, k).T.tocsr()
    assert (got != want).nnz == 0
    _check_sorted_unique(ptr, col, ln)


def test_degree_bknng_is_union(oracle_lib, small_graph):
    _, ids, dist = small_graph
    n, k = ids.shape
    h = k // 2
    ptr, col, ln = oracle_lib.adjust_degree(ids, dist, h, h)
    A = _knng_matrix(ids, dist, h)
    want = A.maximum(A.T).tocsr()  # symmetric distances: same value either way
    got = _csr(ptr, col, ln, n)
    assert (got != want).nnz == 0
    _check_sorted_unique(ptr, col, ln)


def _alg2_sequential(ids, dist, e_o, e_i):
    """Algorithm 2 walked node by node with loop bound p <= max(e_o, e_i)."""
    n, k = ids.shape
    adj = [dict() for _ in range(n)]
    for o in range(n):
        for p in range(1, min(k, max(e_o, e_i)) + 1):
            nb, ln = int(ids[o, p - 1]), float(dist[o, p - 1])
            if p <= e_o:
                adj[o][nb] = ln  # a forward edge keeps its own length
            if p <= e_i and o not in adj[nb]:
                adj[nb][o] = ln
    return adj


@pytest.mark.parametrize("e_o,e_i", [(3, 7), (8, 2), (5, 5), (16, 16), (0, 4)])
def test_degree_matches_sequential_alg2(oracle_lib, small_graph, e_o, e_i):
    _, ids, dist = small_graph
    n, k = ids.shape
    ptr, col, ln = oracle_lib.adjust_degree(ids, dist, e_o, e_i)
    adj = _alg2_sequential(ids, dist, e_o, e_i)
    for o in range(n):
        got = dict(zip(col[ptr[o]:ptr[o + 1]].tolist(), ln[ptr[o]:ptr[o + 1]].tolist()))
        assert got == adj[o]
    _check_sorted_unique(ptr, col, ln)
    outdeg = np.diff(ptr)
    indeg = np.bincount(col, minlength=n)
    assert (outdeg >= min(e_o, k)).all()
    assert (indeg >= min(e_i, k)).all()


def test_degree_row_subset(oracle_lib, small_graph):
    _, ids, dist = small_graph
    full = oracle_lib.adjust_degree(ids, dist, 6, 9)
    rows = np.array([299, 0, 17, 150])
    ptr, col, ln = oracle_lib.adjust_degree(ids, dist, 6, 9, rows=rows)
    for r, i in enumerate(rows):
        a = full[1][full[0][i]:full[0][i + 1]]
        b = col[ptr[r]:ptr[r + 1]]
        assert np.array_equal(a, b)


def _rows(ptr, col, ln):
    return [list(zip(col[ptr[i]:ptr[i + 1]].tolist(), ln[ptr[i]:ptr[i + 1]].tolist())) for i in range(len(ptr) - 1)]


def test_sac_hand_traced_line(oracle_lib):
    """Algorithm 3 on five points of a line, x = 0, 1, 3, 6, 10, with k = 2:
    N_k = 0:[1,2] 1:[0,2] 2:[1,0] 3:[2,4] 4:[3,2] (ties by id).
    (e_o, e_i) = (1, 1): G_t = 0:{1} 1:{0,2} 2:{3} 3:{4} 4:{}; order 4, 0, 2, 3, 1;
    step 2 adds 0->1, 2->3, 3->4, 1->0, 1->2 (n = 2 has no in-edge yet, so the
    out-degree limit does not apply); step 3 gives node 4 its nearest, 3.
    (e_o, e_i) = (1, 2): order 3, 4, 0, 1, 2; step 2 adds 3->4, 4->3, 0->1, 0->2,
    1->0, 2->1 and skips the rest (n has an in-edge and o has e_o out-edges)."""
    x = np.array([0.0, 1.0, 3.0, 6.0, 10.0])
    nbr = np.array([[1, 2], [0, 2], [1, 0], [2, 4], [3, 2]], dtype=np.int32)
    ln = np.abs(x[nbr] - x[:, None])
    got = _rows(*oracle_lib.adjust_degree_sac(nbr, ln, 1, 1))
    assert got == [[(1, 1.0)], [(0, 1.0), (2, 2.0)], [(3, 3.0)], [(4, 4.0)], [(3, 4.0)]]
    got = _rows(*oracle_lib.adjust_degree_sac(nbr, ln, 1, 2))
    assert got == [[(1, 1.0), (2, 3.0)], [(0, 1.0)], [(1, 2.0)], [(4, 4.0)], [(3, 4.0)]]


def test_sac_special_cases_and_invariants(oracle_lib):
    rng = np.random.default_rng(3)
    X = rng.normal(size=(400, 6))
    nbr, ln = oracle_lib.knng(X.astype(np.float32), 12)
    n = len(X)
    # e_i = 0: no reversed edges, the result is the kNN graph truncated to e_o
    ptr, col, l = oracle_lib.adjust_degree_sac(nbr, ln, 5, 0)
    assert np.array_equal(ptr, np.arange(n + 1) * 5)
    assert np.array_equal(col.reshape(n, 5), nbr[:, :5])
    # e_o = 0: exactly one incoming edge per node, from one of its first e_i neighbours
    ptr, col, l = oracle_lib.adjust_degree_sac(nbr, ln, 0, 4)
    src = np.repeat(np.arange(n), np.diff(ptr))
    assert len(col) == n and np.array_equal(np.sort(col), np.arange(n))
    assert all(src[t] in nbr[col[t], :4] for t in range(len(col)))
    # general case: every node has an in-edge; out-degree >= e_o; in-degree from the
    # reversed pass is <= e_i; no self loops or duplicates; rows sorted by (len, id)
    e_o, e_i = 4, 6
    ptr, col, l = oracle_lib.adjust_degree_sac(nbr, ln, e_o, e_i)
    src = np.repeat(np.arange(n), np.diff(ptr))
    assert set(col.tolist()) == set(range(n))
    assert np.all(np.diff(ptr) >= e_o) and np.all(col != src)
    for i in range(n):
        row = list(zip(l[ptr[i]:ptr[i + 1]], col[ptr[i]:ptr[i + 1]]))
        assert row == sorted(row) and len(set(c for _, c in row)) == len(row)
    # an edge o->n is either a kNN edge of o or a reversed edge (o among n's first e_i)
    fwd = {(i, j) for i in range(n) for j in nbr[i]}
    rev = {(j, i) for i in range(n) for j in nbr[i, :e_i]}
    assert all((s, c) in fwd or (s, c) in rev for s, c in zip(src.tolist(), col.tolist()))
    # lengths are the stored kNN lengths of the edge's pair
    d = {(i, j): ln[i, p] for i in range(n) for p, j in enumerate(nbr[i])}
    assert all(np.isclose(lv, d.get((s, c), d.get((c, s)))) for s, c, lv in zip(src, col, l))


def _sac_per_edge(nbr, ln, e_o, e_i):
    """Algorithm 3 evaluated per edge (the form the GPU computes): o keeps the
    members of N(G_t, o) at positions < e_o, and a later member n when o is the
    first, in increasing (|N(G_t, x)|, x), of the nodes x that meet n (the valid
    ids of n's first e_i kNN entries); nodes left below e_o then take their
    nearest kNN neighbours not yet in the list."""
    n, k = nbr.shape
    fi = min(e_i, k)
    members = [[] for _ in range(n)]
    for y in range(n):
        for p in range(fi):
            if nbr[y, p] >= 0:
                members[nbr[y, p]].append((ln[y, p], y))
    for o in range(n):
        members[o].sort()
    first = [min(((len(members[o]), o) for o in nbr[y, :fi] if o >= 0), default=(0, -1))[1] for y in range(n)]
    ptr, col, lens = [0], [], []
    for o in range(n):
        row = [(l, y) for p, (l, y) in enumerate(members[o]) if p < e_o or first[y] == o]
        if len(members[o]) < e_o:
            have = {y for _, y in members[o]}
            for p in range(k):
                if nbr[o, p] < 0 or len(row) >= e_o:
                    break
                if nbr[o, p] not in have:
                    row.append((ln[o, p], nbr[o, p]))
        row.sort()
        col += [y for _, y in row]
        lens += [l for l, _ in row]
        ptr.append(len(col))
    return np.array(ptr), np.array(col, dtype=np.int32), np.array(lens)


@pytest.mark.parametrize("e_o,e_i", [(5, 10), (10, 5), (0, 8), (8, 0), (3, 3), (12, 12), (20, 30)])
def test_sac_sequential_pass_equals_per_edge_rule(oracle_lib, e_o, e_i):
    """The sequential greedy pass of Algorithm 3 (the oracle) and its per-edge
    reading agree edge for edge, on tie-heavy integer points and on float data:
    a node is met only by its own first e_i kNN entries, so the in-degree limit
    e_i never refuses an edge and each decision depends on one edge alone."""
    for X, k in ((synth.small_integers(700, 4, high=4, seed=3), 12),
                 (synth.workload("gmm10k", n=900, nq=1)[0], 12)):
        nbr, ln = oracle_lib.knng(X, k)
        o = oracle_lib.adjust_degree_sac(nbr, ln, e_o, e_i)
        c = _sac_per_edge(nbr, ln, e_o, e_i)
        assert np.array_equal(o[0], c[0]) and np.array_equal(o[1], c[1]) and np.array_equal(o[2], c[2])
