"""Pins of the oracle's graph statistics (Table 4, Sec. 3.1): a star graph whose
values follow by hand, a ceil(5 %) case, and an independent numpy / scipy.sparse
computation on random graphs."""
import numpy as np
import pytest

import oracle


def csr(n, edges):
    """CSR of (src, dst, length) triples, rows ordered by (length, id)."""
    edges = sorted(edges, key=lambda e: (e[0], e[2], e[1]))
    ptr = np.zeros(n + 1, np.int64)
    for s, _, _ in edges:
        ptr[s + 1] += 1
    ptr = np.cumsum(ptr)
    col = np.array([e[1] for e in edges], np.int32)
    ln = np.array([e[2] for e in edges], np.float64)
    return ptr, col, ln


def test_star_by_hand():
    # node 0 -> every other node j with length j; every j -> 0 with length j
    n = 20
    edges = [(0, j, float(j)) for j in range(1, n)] + [(j, 0, float(j)) for j in range(1, n)]
    st = oracle.graph_stats(*csr(n, edges))
    assert st["mean_out"] == pytest.approx(38 / 20)
    # m = ceil(20 / 20) = 1: the largest outdegree (19) and the smallest indegree (1)
    assert st["top5_out"] == 19 and st["bottom5_in"] == 1
    assert st["max_out"] == 19 and st["max_in"] == 19 and st["zero_in"] == 0
    # node 0 keeps its 10 shortest incoming (1..10, sum 55); node j keeps its one (length j)
    assert st["in_dist10"] == pytest.approx((55 + sum(range(1, 20))) / (10 + 19))


def test_five_percent_rounds_up_and_isolated_nodes():
    # n = 30: m = ceil(1.5) = 2.  Node i (i < 6) has i out-edges to nodes 10.. ;
    # nodes 6..9 and 20..29 receive nothing.
    n = 30
    edges = [(i, 10 + t, 1.0 + t) for i in range(6) for t in range(i)]
    st = oracle.graph_stats(*csr(n, edges))
    assert st["top5_out"] == pytest.approx((5 + 4) / 2)
    assert st["bottom5_in"] == 0
    # indegree of node 10 + t is the number of i in (t, 5]: 5, 4, 3, 2, 1
    assert st["max_in"] == 5 and st["zero_in"] == n - 5
    assert st["mean_out"] == pytest.approx(15 / 30)
    # all incoming lists are shorter than 10: every edge counts once
    assert st["in_dist10"] == pytest.approx(np.mean([1.0 + t for i in range(6) for t in range(i)]))


def test_no_edges():
    st = oracle.graph_stats(np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0))
    assert st["mean_out"] == 0 and st["top5_out"] == 0 and st["bottom5_in"] == 0 and st["zero_in"] == 7
    assert np.isnan(st["in_dist10"])


@pytest.mark.parametrize("n,seed", [(57, 1), (400, 2), (1000, 3)])
def test_random_graphs_against_scipy(n, seed):
    import scipy.sparse as sp
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, 40, n)
    deg[rng.integers(0, n, 3)] = rng.integers(100, 300, 3)  # a few hubs
    edges = []
    for i in range(n):
        dst = rng.choice(np.delete(np.arange(n), i), size=min(deg[i], n - 1), replace=False)
        for j in dst:
            edges.append((i, int(j), float(rng.integers(1, 50))))  # integer lengths: many ties
    ptr, col, ln = csr(n, edges)
    st = oracle.graph_stats(ptr, col, ln)
    out = np.diff(ptr)
    ind = np.bincount(col, minlength=n)
    m = -(-n // 20)
    assert st["top5_out"] == pytest.approx(np.sort(out)[::-1][:m].mean())
    assert st["bottom5_in"] == pytest.approx(np.sort(ind)[:m].mean())
    assert st["max_in"] == ind.max() and st["zero_in"] == (ind == 0).sum()
    t = sp.csr_matrix((ln + 1.0, col, ptr), shape=(n, n)).T.tocsr()  # +1 keeps zeros out of the sparsity
    kept = [np.sort(t.data[t.indptr[j]:t.indptr[j + 1]] - 1.0)[:10] for j in range(n)]
    allk = np.concatenate(kept)
    assert st["in_dist10"] == pytest.approx(allk.mean(), rel=1e-12)
