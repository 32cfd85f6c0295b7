"""Pins of the oracle's path adjustment (Algorithms 4 and 5, Sec. 2.3, Fig. 2).

The Fig. 2 cases are realised as small 2-D point sets; the general rule is
checked against a dense-matrix brute force over all (i, m, j) triples, and the
invariants the reading guarantees (out-degree >= 1, reachability, idempotence)
are checked with scipy.sparse.csgraph.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

from paper_1810_07355_gb300 import synth


def _graph_from_edges(P, edges):
    """CSR with Euclidean lengths of directed edges among points P, rows by (len, id)."""
    n = len(P)
    rows = [[] for _ in range(n)]
    for a, b in edges:
        rows[a].append((float(np.linalg.norm(P[a] - P[b])), b))
    ptr, col, ln = [0], [], []
    for r in rows:
        r.sort()
        col += [b for _, b in r]
        ln += [l for l, _ in r]
        ptr.append(len(col))
    return np.array(ptr, np.int64), np.array(col, np.int32), np.array(ln, np.float64)


def _edges(ptr, col):
    return {(i, int(c)) for i in range(len(ptr) - 1) for c in col[ptr[i]:ptr[i + 1]]}


def test_fig2_case_a_three_edge_path_kept(oracle_lib):
    # n_s=0 -> n_d=3 with only the 3-edge alternative 0 -> 1 -> 2 -> 3
    P = np.array([[0, 0], [1, 0.5], [2, 0.5], [3, 0]], np.float64)
    g = _graph_from_edges(P, [(0, 3), (0, 1), (1, 2), (2, 3)])
    out = oracle_lib.adjust_path(*g)
    assert (0, 3) in _edges(out[0], out[1])
    assert _edges(out[0], out[1]) == _edges(g[0], g[1])


def test_fig2_case_b_two_edge_path_removed(oracle_lib):
    # n_s=0 -> n_d=2 with alternative 0 -> 1 -> 2, both hops shorter
    P = np.array([[0, 0], [1, 0.3], [2, 0]], np.float64)
    g = _graph_from_edges(P, [(0, 2), (0, 1), (1, 2)])
    out = oracle_lib.adjust_path(*g, witnesses=True)
    assert (0, 2) not in _edges(out[0], out[1])
    assert _edges(out[0], out[1]) == {(0, 1), (1, 2)}
    # the witness of the removed edge is node 1
    wit = out[3]
    assert wit[list(g[1][g[0][0]:g[0][1]]).index(2)] == 1


def test_fig2_case_c_longer_hop_kept(oracle_lib):
    # alternative 0 -> 1 -> 2 exists but hop 1 -> 2 is longer than 0 -> 2
    P = np.array([[0, 0], [0.5, 1.8], [2, 0]], np.float64)
    g = _graph_from_edges(P, [(0, 2), (0, 1), (1, 2)])
    assert np.linalg.norm(P[1] - P[2]) > np.linalg.norm(P[0] - P[2])
    out = oracle_lib.adjust_path(*g)
    assert (0, 2) in _edges(out[0], out[1])


def _brute(ptr, col, ln):
    n = len(ptr) - 1
    A = np.zeros((n, n), bool)
    L = np.full((n, n), np.inf)
    for i in range(n):
        A[i, col[ptr[i]:ptr[i + 1]]] = True
        L[i, col[ptr[i]:ptr[i + 1]]] = ln[ptr[i]:ptr[i + 1]]
    keep = A.copy()
    for i in range(n):
        for j in np.nonzero(A[i])[0]:
            m = A[i] & A[:, j] & (L[i] < L[i, j]) & (L[:, j] < L[i, j])
            m[j] = False
            if m.any():
                keep[i, j] = False
    return keep


@pytest.fixture(scope="module")
def degree_graph(oracle_lib):
    X = synth.gaussian_mixture(120, d=6, components=3, sigma=3.0, seed=21)
    ids, dist = oracle_lib.knng(X, 12)
    return oracle_lib.adjust_degree(ids, dist, 6, 8)


def test_path_matches_bruteforce(oracle_lib, degree_graph):
    ptr, col, ln = degree_graph
    out = oracle_lib.adjust_path(ptr, col, ln)
    keep = _brute(ptr, col, ln)
    assert _edges(out[0], out[1]) == {tuple(e) for e in np.argwhere(keep).tolist()}
    # kept edges stay in their (len, id) order
    for i in range(len(ptr) - 1):
        l = out[2][out[0][i]:out[0][i + 1]]
        assert (np.diff(l) >= 0).all()


def test_path_invariants(oracle_lib, degree_graph):
    ptr, col, ln = degree_graph
    n = len(ptr) - 1
    out = oracle_lib.adjust_path(ptr, col, ln, witnesses=True)
    # every node that had an edge keeps its shortest one
    assert (np.diff(out[0]) >= 1).all()
    # reachability is unchanged
    A = sp.csr_matrix((np.ones(len(col)), col, ptr), shape=(n, n))
    B = sp.csr_matrix((np.ones(len(out[1])), out[1], out[0]), shape=(n, n))
    assert np.array_equal(np.isfinite(shortest_path(A, unweighted=True)),
                          np.isfinite(shortest_path(B, unweighted=True)))
    # idempotence
    again = oracle_lib.adjust_path(*out[:3])
    assert np.array_equal(again[0], out[0]) and np.array_equal(again[1], out[1])
    # witnesses really witness: i->m and m->j exist with both hops shorter
    wit = out[3]
    L = {(i, int(c)): float(l) for i in range(n) for c, l in
         zip(col[ptr[i]:ptr[i + 1]], ln[ptr[i]:ptr[i + 1]])}
    e = 0
    for i in range(n):
        for c in col[ptr[i]:ptr[i + 1]]:
            m = int(wit[e])
            if m >= 0:
                assert L[(i, m)] < L[(i, int(c))] and L[(m, int(c))] < L[(i, int(c))]
            e += 1
    # the removal is substantial on clustered data (the paper reports about half)
    assert out[0][-1] < 0.8 * ptr[-1]


def test_path_row_subset(oracle_lib, degree_graph):
    ptr, col, ln = degree_graph
    full = oracle_lib.adjust_path(ptr, col, ln)
    rows = np.array([5, 119, 0])
    sub = oracle_lib.adjust_path(ptr, col, ln, rows=rows)
    for r, i in enumerate(rows):
        assert np.array_equal(full[1][full[0][i]:full[0][i + 1]], sub[1][sub[0][r]:sub[0][r + 1]])


def test_alg4_literal_keeps_superset(oracle_lib, degree_graph):
    """Algorithm 4 tests paths in its partial output, so it removes no edge that
    the order-free reading keeps (continuous data: no equal lengths)."""
    ptr, col, ln = degree_graph
    r2 = _edges(*oracle_lib.adjust_path(ptr, col, ln)[:2])
    a4 = _edges(*oracle_lib.adjust_path_alg4(ptr, col, ln)[:2])
    assert r2 <= a4 <= _edges(ptr, col)
    P = np.array([[0, 0], [1, 0.3], [2, 0]], np.float64)
    g = _graph_from_edges(P, [(0, 2), (0, 1), (1, 2)])
    assert _edges(*oracle_lib.adjust_path_alg4(*g)[:2]) == {(0, 1), (1, 2)}


def _alg4_case(order):
    """Points A = (0, 0), B = (5, 1), C = (10, 0), D = (5, 2) with edges A->B, A->C,
    B->D, B->C: |AB| = |BC| = sqrt(26) < |AC| = 10 and |BD| = 1 < |BC|, so the order-free
    rule drops A->C (witness B).  `order` gives the node ids of A, B, C, D."""
    pts = {"A": (0, 0), "B": (5, 1), "C": (10, 0), "D": (5, 2)}
    ids = dict(zip("ABCD", order))
    P = np.zeros((4, 2), np.float64)
    for k, v in pts.items():
        P[ids[k]] = v
    edges = [(ids[a], ids[b]) for a, b in ("AB", "AC", "BD", "BC")]
    return ids, _graph_from_edges(P, edges)


def test_alg4_literal_rounds_and_ascending_ids_by_hand(oracle_lib):
    """Algorithm 4 taken literally (rounds; inside a round, nodes by ascending id).
    Round 1 adds A->B and B->D.  In round 2, A tests A->C against the partial graph:
    B->C is there only if B came before A in that round.  Traced by hand:
    B before A drops A->C; A before B keeps it, while the order-free rule drops it in
    both cases."""
    for order, drop in (((1, 0, 2, 3), True), ((0, 1, 2, 3), False)):
        ids, g = _alg4_case(order)
        a, b, c, d = (ids[k] for k in "ABCD")
        full = {(a, b), (a, c), (b, d), (b, c)}
        assert _edges(*oracle_lib.adjust_path(*g)[:2]) == full - {(a, c)}
        assert _edges(*oracle_lib.adjust_path_alg4(*g)[:2]) == (full - {(a, c)} if drop else full)


def test_alg4_literal_witness_added_too_late_by_hand(oracle_lib):
    """The witness edge 2->1 is node 2's third edge (after 2->3 and 2->4), so it enters
    the partial graph in round 3, after node 0 has kept 0->1 in round 2; the
    order-free rule drops 0->1 (|02| = |21| = sqrt(26) < |01| = 10)."""
    P = np.array([[0, 0], [10, 0], [5, 1], [5, 2], [5, 3.5]], np.float64)
    g = _graph_from_edges(P, [(0, 2), (0, 1), (2, 3), (2, 4), (2, 1)])
    full = {(0, 2), (0, 1), (2, 3), (2, 4), (2, 1)}
    assert _edges(*oracle_lib.adjust_path(*g)[:2]) == full - {(0, 1)}
    assert _edges(*oracle_lib.adjust_path_alg4(*g)[:2]) == full
    # lists come out in the order edges were added: ascending length per node
    ptr, col, ln = oracle_lib.adjust_path_alg4(*g)[:3]
    assert col[ptr[2]:ptr[3]].tolist() == [3, 4, 1]
    assert np.allclose(ln[ptr[0]:ptr[1]], [np.sqrt(26.0), 10.0])
