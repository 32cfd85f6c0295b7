"""GPU parity: every CUDA step against the CPU FP64 oracle on the same inputs.

Integer-valued inputs (the image-descriptor workload) are ranked exactly in
float32, so graphs, seeds and search results must match the oracle bit for bit.
Float inputs follow the near-tie rules of parity_helpers (1e-5 relative).  Each
step is fed the same input on both sides (stepwise parity).
"""
import numpy as np
import pytest

import oracle
from paper_1810_07355_gb300 import synth
from parity_helpers import (DECIDE, REL, assert_reranked, assert_rows_near, assert_search_parity,  # noqa: F401
                            assert_valid_lists)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def onng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07355_gb300 import onng as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


def assert_rows_match(ids, lens, o_ids, o_lens, exact=True):
    """Rows equal; without `exact`, an id may differ only where the competing
    distances are within 1e-5 relative (position by position)."""
    if exact:
        assert np.array_equal(ids, o_ids)
        np.testing.assert_allclose(lens, o_lens, rtol=1e-6)
        return
    assert_rows_near(ids, lens.astype(np.float64), o_ids, o_lens)
    assert (ids != o_ids).any(1).mean() <= 0.05


# ----------------------------------------------------------------------------- kNN graph

@pytest.mark.parametrize("n,k", [(3000, 10), (1037, 40), (2500, 100), (700, 200)])
def test_knng_integer_exact(onng, n, k):
    X, _ = synth.workload("sift1m", n=n, nq=1)
    nbr, ln = onng.build_knng(dev(X), k)
    o_ids, o_len = oracle.knng(X, k)
    assert_rows_match(host(nbr), host(ln), o_ids, o_len)


def test_knng_tie_heavy_and_duplicates(onng):
    X = synth.small_integers(1500, 8, high=3, seed=4)  # many duplicate points and equal distances
    nbr, ln = onng.build_knng(dev(X), 24)
    o_ids, o_len = oracle.knng(X, 24)
    assert_rows_match(host(nbr), host(ln), o_ids, o_len)


@pytest.mark.parametrize("d", [64, 128])
def test_knng_tensor_core_ties(onng, d):
    """Integer data at d = 64 / 128 goes through the tcgen05 path; heavy ties and
    duplicate points must still come out in (distance, id) order."""
    X = synth.small_integers(2000, d, high=3, seed=d)
    nbr, ln = onng.build_knng(dev(X), 30)
    o_ids, o_len = oracle.knng(X, 30)
    assert_rows_match(host(nbr), host(ln), o_ids, o_len)


def test_knn_tensor_core_ragged_and_self(onng):
    """Row and column counts that are not multiples of the tile (256 query rows in
    two blocks of 128, 128 base columns), a last CTA with one row block, queries
    that are base rows (self excluded) and queries that are not."""
    X, Q = synth.workload("sift1m", n=1000 + 77, nq=131)
    ids, ln = onng.knn(dev(X), dev(X[300:300 + 131]), 17, self_offset=300)
    o_ids, o_len = oracle.knn(X, X[300:300 + 131], 17, self_ids=np.arange(300, 431))
    assert_rows_match(host(ids), host(ln), o_ids, o_len)
    ids, ln = onng.knn(dev(X), dev(Q), 100)
    o_ids, o_len = oracle.knn(X, Q, 100)
    assert_rows_match(host(ids), host(ln), o_ids, o_len)


def test_knng_float_near_ties_only(onng):
    X, _ = synth.workload("gmm10k", n=2000, nq=1)
    nbr, ln = onng.build_knng(dev(X), 40)
    o_ids, o_len = oracle.knng(X, 40)
    assert_rows_match(host(nbr), host(ln), o_ids, o_len, exact=False)


def test_knng_float_split_tensor_core_offset(onng):
    """Float data far from the origin (every coordinate + 1000) takes the split
    bfloat16 tensor-core sweep, which centres both sets on the base mean first:
    the ranking error scales with the spread of the data, not with its offset."""
    X, _ = synth.workload("gmm10k", n=3000, nq=1)
    X = (X + 1000.0).astype(np.float32)
    nbr, ln = onng.build_knng(dev(X), 40)
    o_ids, o_len = oracle.knng(X, 40)
    assert_rows_match(host(nbr), host(ln), o_ids, o_len, exact=False)


def test_knn_float_simt_sweep(onng):
    """Float inputs below the tensor-core paths' sizes (d < 32; fewer than 128
    queries) take the float32 SIMT sweep."""
    rng = np.random.default_rng(5)
    X = rng.random((2500, 16), dtype=np.float32)
    nbr, ln = onng.build_knng(dev(X), 20)
    o_ids, o_len = oracle.knng(X, 20)
    assert_rows_match(host(nbr), host(ln), o_ids, o_len, exact=False)
    Xg, Qg = synth.workload("gmm10k", n=3000, nq=60)
    ids, ln = onng.knn(dev(Xg), dev(Qg), 10)
    o_ids, o_len = oracle.knn(Xg, Qg, 10)
    assert_rows_match(host(ids), host(ln), o_ids, o_len, exact=False)


def test_knn_queries_ground_truth(onng):
    X, Q = synth.workload("sift1m", n=4000, nq=300)
    ids, ln = onng.knn(dev(X), dev(Q), 10)
    o_ids, o_len = oracle.knn(X, Q, 10)
    assert_rows_match(host(ids), host(ln), o_ids, o_len)


def test_knn_padding_small_base(onng):
    X = synth.small_integers(20, 4, high=50, seed=2)
    ids, ln = onng.build_knng(dev(X), 19)
    o_ids, o_len = oracle.knng(X, 19)
    assert_rows_match(host(ids), host(ln), o_ids, o_len)


# ----------------------------------------------------------------------------- adjustment

def _csr_equal(g, o):
    ptr, col, ln = (host(t) for t in g)
    assert np.array_equal(ptr, o[0])
    assert np.array_equal(col, o[1])
    np.testing.assert_array_equal(ln.astype(np.float64), o[2])


@pytest.fixture(scope="module")
def sift_knng(onng):
    X, Q = synth.workload("sift1m", n=6000, nq=200)
    nbr, ln = onng.build_knng(dev(X), 40)
    return X, Q, nbr, ln


@pytest.mark.parametrize("e_o,e_i", [(10, 30), (40, 0), (0, 40), (20, 20), (5, 13)])
def test_degree_stepwise(onng, sift_knng, e_o, e_i):
    _, _, nbr, ln = sift_knng
    g = onng.adjust_degree(nbr, ln, e_o, e_i)
    o = oracle.adjust_degree(host(nbr), host(ln).astype(np.float64), e_o, e_i)
    _csr_equal(g, o)


def _hub_knng(onng, n=3000):
    # a dense cluster with a few central points that sit in almost every list
    rng = np.random.default_rng(5)
    X = np.rint(rng.normal(100, 20, size=(n, 16))).clip(0, 255).astype(np.float32)
    X[:3] = 100.0
    nbr, ln = onng.build_knng(dev(X), 40)
    return X, nbr, ln


def test_degree_hub_rows(onng):
    _, nbr, ln = _hub_knng(onng)
    g = onng.adjust_degree(nbr, ln, 10, 40)
    deg = np.diff(host(g[0]))
    assert deg.max() > 512  # exercises the CTA sort
    o = oracle.adjust_degree(host(nbr), host(ln).astype(np.float64), 10, 40)
    _csr_equal(g, o)


@pytest.mark.parametrize("e_o,e_i", [(10, 30), (40, 0), (0, 40), (20, 20), (5, 13), (30, 60)])
def test_sac_stepwise(onng, sift_knng, e_o, e_i):
    """Algorithm 3 (SAC) on the GPU equals the oracle's sequential pass bit for bit."""
    _, _, nbr, ln = sift_knng
    g = onng.adjust_degree_sac(nbr, ln, e_o, e_i)
    o = oracle.adjust_degree_sac(host(nbr), host(ln).astype(np.float64), e_o, e_i)
    _csr_equal(g, o)


def test_sac_hub_rows_and_ties(onng):
    """Hub nodes (long G_t lists, the CTA sort) and a tie-heavy graph."""
    _, nbr, ln = _hub_knng(onng)
    g = onng.adjust_degree_sac(nbr, ln, 10, 40)
    o = oracle.adjust_degree_sac(host(nbr), host(ln).astype(np.float64), 10, 40)
    _csr_equal(g, o)
    X = synth.small_integers(1200, 4, high=4, seed=9)
    nbr, ln = onng.build_knng(dev(X), 16)
    for e_o, e_i in ((4, 8), (0, 16), (16, 0)):
        g = onng.adjust_degree_sac(nbr, ln, e_o, e_i)
        o = oracle.adjust_degree_sac(host(nbr), host(ln).astype(np.float64), e_o, e_i)
        _csr_equal(g, o)


@pytest.mark.parametrize("e_o,e_i", [(10, 30), (20, 20)])
def test_path_stepwise(onng, sift_knng, e_o, e_i):
    _, _, nbr, ln = sift_knng
    g = onng.adjust_degree(nbr, ln, e_o, e_i)
    p = onng.adjust_path(*g, witnesses=True)
    o = oracle.adjust_path(host(g[0]), host(g[1]), host(g[2]).astype(np.float64), witnesses=True)
    _csr_equal(p[:3], o[:3])
    assert np.array_equal(host(p[3]), o[3])


def test_path_hub_rows(onng):
    _, nbr, ln = _hub_knng(onng)
    g = onng.adjust_degree(nbr, ln, 10, 40)
    assert np.diff(host(g[0])).max() > 256  # exercises the CTA kernel
    p = onng.adjust_path(*g, witnesses=True)
    o = oracle.adjust_path(host(g[0]), host(g[1]), host(g[2]).astype(np.float64), witnesses=True)
    _csr_equal(p[:3], o[:3])
    assert np.array_equal(host(p[3]), o[3])


def test_path_hub_row_beyond_shared_memory(onng):
    """A hub of about 8,000 edges: points on a sphere around one centre point all
    list the centre first, so its row is far beyond the warp kernel's 256 edges
    and takes the CTA kernel (its hash in global scratch)."""
    n, d = 8000, 64
    rng = np.random.default_rng(12)
    U = rng.normal(size=(n, d))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    X = np.rint(128.0 + 60.0 * U).clip(0, 255).astype(np.float32)
    X[0] = 128.0
    nbr, ln = onng.build_knng(dev(X), 40)
    g = onng.adjust_degree(nbr, ln, 10, 40)
    assert np.diff(host(g[0])).max() > 6144
    p = onng.adjust_path(*g, witnesses=True)
    o = oracle.adjust_path(host(g[0]), host(g[1]), host(g[2]).astype(np.float64), witnesses=True)
    _csr_equal(p[:3], o[:3])
    assert np.array_equal(host(p[3]), o[3])


@pytest.mark.parametrize("e_o,e_i", [(10, 30), (20, 20), (5, 13)])
def test_path_literal_alg4_stepwise(onng, sift_knng, e_o, e_i):
    """Algorithm 4 taken literally on the GPU equals the oracle's round-robin pass
    (ascending ids inside a round) bit for bit."""
    _, _, nbr, ln = sift_knng
    g = onng.adjust_degree(nbr, ln, e_o, e_i)
    p = onng.adjust_path_literal(*g)
    o = oracle.adjust_path_alg4(host(g[0]), host(g[1]), host(g[2]).astype(np.float64))
    _csr_equal(p, o)


def test_path_literal_alg4_hubs_ties_and_floats(onng):
    """Hub rows (many rounds for a few nodes), tie-heavy lengths (same-round
    dependencies between nodes that share targets) and float lengths."""
    _, nbr, ln = _hub_knng(onng)
    g = onng.adjust_degree(nbr, ln, 10, 40)
    _csr_equal(onng.adjust_path_literal(*g), oracle.adjust_path_alg4(host(g[0]), host(g[1]),
                                                                      host(g[2]).astype(np.float64)))
    X = synth.small_integers(1500, 4, high=5, seed=11)
    nbr, ln = onng.build_knng(dev(X), 20)
    g = onng.adjust_degree(nbr, ln, 8, 16)
    _csr_equal(onng.adjust_path_literal(*g), oracle.adjust_path_alg4(host(g[0]), host(g[1]),
                                                                      host(g[2]).astype(np.float64)))
    X, _ = synth.workload("gmm10k", n=2500, nq=1)
    nbr, ln = onng.build_knng(dev(X), 30)
    g = onng.adjust_degree(nbr, ln, 10, 20)
    _csr_equal(onng.adjust_path_literal(*g), oracle.adjust_path_alg4(host(g[0]), host(g[1]),
                                                                      host(g[2]).astype(np.float64)))


def test_path_float_lengths(onng):
    X, _ = synth.workload("gmm10k", n=3000, nq=1)
    nbr, ln = onng.build_knng(dev(X), 30)
    g = onng.adjust_degree(nbr, ln, 10, 20)
    p = onng.adjust_path(*g)
    o = oracle.adjust_path(host(g[0]), host(g[1]), host(g[2]).astype(np.float64))
    _csr_equal(p, o)


# ----------------------------------------------------------------------------- seeds

def test_seeds_random_bit_exact(onng):
    for n, ns in [(1000, 10), (10**6, 64), (7, 3), (5, 5)]:
        s = onng.seeds_random(77, 500, n, ns)
        assert np.array_equal(host(s), oracle.seeds_random(77, 500, n, ns))


def test_seeds_pivot_integer_exact(onng):
    X, Q = synth.workload("sift1m", n=20000, nq=300)
    s = onng.seeds_pivot(dev(X), dev(Q), 1024, 10)
    assert np.array_equal(host(s), oracle.seeds_pivot(X, Q, 1024, 10))
    s = onng.seeds_pivot(dev(X[:50]), dev(Q), 1024, 64)  # fewer pivots than seeds: -1 padded
    assert np.array_equal(host(s), oracle.seeds_pivot(X[:50], Q, 1024, 64))


@pytest.mark.parametrize("d,P,nq,n_seed", [(260, 200, 37, 12), (8, 64, 16, 64), (128, 2048, 5, 1)])
def test_seeds_pivot_tiles_and_ragged_edges(onng, d, P, nq, n_seed):
    """Several coordinate chunks, a ragged last pivot tile and query group, and
    many equal distances (small integers): ids equal the oracle's, ties by pivot index."""
    X = synth.small_integers(3000, d, high=4, seed=d)
    Q = synth.small_integers(nq, d, high=4, seed=d + 1)
    s = onng.seeds_pivot(dev(X), dev(Q), P, n_seed)
    assert np.array_equal(host(s), oracle.seeds_pivot(X, Q, P, n_seed))


@pytest.mark.parametrize("d,P,n_seed", [(100, 16384, 10), (128, 5000, 64)])
def test_seeds_pivot_many_pivots(onng, d, P, n_seed):
    """More pivots than one query's distances would fit in shared memory: the
    running best list gives the oracle's ids (ties by pivot index)."""
    X = synth.small_integers(40000, d, high=6, seed=d + 5)
    Q = synth.small_integers(70, d, high=6, seed=d + 6)
    s = onng.seeds_pivot(dev(X), dev(Q), P, n_seed)
    assert np.array_equal(host(s), oracle.seeds_pivot(X, Q, P, n_seed))


# ----------------------------------------------------------------------------- search

@pytest.fixture(scope="module")
def sift_graph(onng, sift_knng):
    X, Q, nbr, ln = sift_knng
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    seeds = onng.seeds_pivot(dev(X), dev(Q), 512, 10)
    return X, Q, g, seeds


@pytest.mark.parametrize("k,e_s,eps,padded", [(10, 10, 0.0, False), (10, 10, 0.1, True), (10, 0, 0.05, False),
                                              (1, 5, 0.2, True), (1, 5, 0.2, False), (10, 10, 0.2, True),
                                              (10, 5, 0.3, False), (100, 20, 0.05, True),
                                              (10, 10, float("inf"), False), (128, 0, 0.0, False),
                                              (10, 40, 0.1, True)])
def test_search_integer_exact(onng, sift_graph, k, e_s, eps, padded):
    """Bit-exact against Algorithm 1 in float64, including the searches whose
    candidate set outgrows the shared-memory pool (eps >= 0.2 spills to global)."""
    X, Q, g, seeds = sift_graph
    idx = onng.Index(g[0], g[1], dev(X))
    if padded:
        idx.with_adjacency(max(e_s, 1))
    ids, dist, st = onng.search(idx, dev(Q), k, e_s, eps, seeds)
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, k, e_s, np.float32(eps), host(seeds))
    assert np.array_equal(host(ids), o_ids)
    np.testing.assert_allclose(host(dist), o_dist, rtol=1e-6)
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])  # distance computations
    assert np.array_equal(host(st)[:, 1], o_st[:, 1])  # expansions
    assert (host(st)[:, 3] == 0).all()


@pytest.mark.parametrize("cap,prec", [(1, 0), (9, 0), (60, 0), (60, 1)])
def test_search_expansion_cap_integer_exact(onng, sift_graph, cap, prec):
    """A per-query expansion cap (the bench's capped form): the ids, distance
    computations, expansions and the LIMIT flag equal the capped oracle's; bf16 is
    exact on these byte-valued vectors, so its reranked lists match too."""
    X, Q, g, seeds = sift_graph
    idx = onng.Index(g[0], g[1], dev(X)).with_adjacency(20).with_bf16()
    kw = dict(precision=onng.PREC_BF16, k_rerank=10) if prec else {}
    ids, dist, st = onng.search(idx, dev(Q), 10, 20, 0.12, seeds, max_expansions=cap, **kw)
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, 10, 20, np.float32(0.12), host(seeds),
                                        max_exp=cap)
    assert np.array_equal(host(ids), o_ids)
    np.testing.assert_allclose(host(dist), o_dist, rtol=1e-6)
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])
    assert np.array_equal(host(st)[:, 1], o_st[:, 1])
    assert np.array_equal(host(st)[:, 3] & onng.FLAG_LIMIT, o_st[:, 3])
    assert (host(st)[:, 1] <= cap).all()


def test_search_unbounded_is_exact_knn(onng, sift_graph):
    """eps = inf with every edge scanned visits every node of a strongly
    connected graph, so the search returns the exact k nearest neighbours."""
    X, Q, g, seeds = sift_graph
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    n = len(X)
    A = sp.csr_matrix((np.ones(len(host(g[1]))), host(g[1]), host(g[0])), shape=(n, n))
    ncomp, _ = connected_components(A, directed=True, connection="strong")
    assert ncomp == 1
    ids, dist, st = onng.search(onng.Index(g[0], g[1], dev(X)), dev(Q), 10, 0, float("inf"), seeds)
    gt, gd = oracle.knn(X, Q, 10)
    assert np.array_equal(host(ids), gt)
    np.testing.assert_allclose(host(dist), gd, rtol=1e-6)
    assert (host(st)[:, 0] == n).all()
    assert (host(st)[:, 3] == 0).all()


def test_search_float_data(onng):
    X, Q = synth.workload("gmm10k", n=4000, nq=150)
    nbr, ln = onng.build_knng(dev(X), 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    seeds = onng.seeds_pivot(dev(X), dev(Q), 1024, 10)
    idx = onng.Index(g[0], g[1], dev(X))
    for eps in (0.0, 0.05, 0.1):
        ids, dist, st = onng.search(idx, dev(Q), 10, 10, eps, seeds)
        o = oracle.search(host(g[0]), host(g[1]), X, Q, 10, 10, np.float32(eps), host(seeds), margin=True)
        assert_search_parity(host(ids), host(dist), host(st), *o, X, Q, min_tie_free=0.6)


def test_search_edge_cases(onng, sift_graph):
    X, Q, g, seeds = sift_graph
    idx = onng.Index(g[0], g[1], dev(X))
    # no queries
    ids, dist, st = onng.search(idx, dev(Q[:0]), 10, 10, 0.1, seeds[:0])
    assert ids.shape == (0, 10)
    # invalid / repeated seeds are skipped; a query with no valid seed returns padding
    s = host(seeds).copy()
    s[0, :] = -1
    s[1, 1:] = s[1, 0]
    s[2, 3] = len(X) + 5
    ids, dist, st = onng.search(idx, dev(Q), 10, 10, 0.1, dev(s))
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, 10, 10, np.float32(0.1),
                                        np.where(s >= len(X), -1, s))
    assert (host(ids)[0] == -1).all() and np.isinf(host(dist)[0]).all()
    assert np.array_equal(host(ids), o_ids)
    # per-query eps / e_s arrays equal separate calls
    eq = torch.tensor([0.0, 0.2] * 100, dtype=torch.float32, device="cuda")
    es = torch.tensor([5, 20] * 100, dtype=torch.int32, device="cuda")
    ids2, _, st2 = onng.search(idx, dev(Q), 10, 10, 0.1, seeds, eps_q=eq, es_q=es)
    a, _, _ = onng.search(idx, dev(Q[0::2]), 10, 5, 0.0, seeds[0::2])
    b, _, _ = onng.search(idx, dev(Q[1::2]), 10, 20, 0.2, seeds[1::2])
    assert torch.equal(ids2[0::2], a) and torch.equal(ids2[1::2], b)
    # expansion cap: flagged
    _, _, st3 = onng.search(idx, dev(Q), 10, 10, 0.2, seeds, max_expansions=3)
    assert ((host(st3)[:, 3] & onng.FLAG_LIMIT) != 0).any()
    assert (host(st3)[:, 1] <= 3).all()


def test_pad_adjacency(onng, sift_graph):
    _, _, g, _ = sift_graph
    adj = host(onng.pad_adjacency(g[0], g[1], 12))
    ptr, col = host(g[0]), host(g[1])
    for i in range(0, len(ptr) - 1, 97):
        row = col[ptr[i]:ptr[i + 1]][:12]
        assert np.array_equal(adj[i, :len(row)], row) and (adj[i, len(row):] == -1).all()


def test_search_visited_spill(onng):
    """Queries that visit more nodes than the shared-memory table holds continue in
    the global bitmap and still match the oracle; the warps reuse their bitmaps
    for later queries, so a wrong clear would show up as missing visits."""
    X, Q = synth.workload("sift1m", n=10000, nq=20)
    nbr, ln = onng.build_knng(dev(X), 40)
    g = onng.adjust_degree(nbr, ln, 20, 40)
    seeds = onng.seeds_pivot(dev(X), dev(Q), 256, 10)
    ids, dist, st = onng.search(onng.Index(g[0], g[1], dev(X)), dev(Q), 100, 0, 0.5, seeds)
    o_ids, _, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, 100, 0, np.float32(0.5), host(seeds))
    assert (host(st)[:, 0] > 2048).sum() >= 5
    assert np.array_equal(host(ids), o_ids)
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])


def test_search_bf16_rerank(onng, sift_graph):
    """Integer data is exact in bfloat16, so the bf16 pass with an FP32 rerank of
    k_rerank candidates equals the FP32 search with k_rerank results, truncated."""
    X, Q, g, seeds = sift_graph
    idx = onng.Index(g[0], g[1], dev(X))
    ids, dist, st = onng.search(idx, dev(Q), 10, 10, 0.05, seeds, precision=onng.PREC_BF16, k_rerank=20)
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, 20, 10, np.float32(0.05), host(seeds))
    assert np.array_equal(host(ids), o_ids[:, :10])
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])


@pytest.mark.parametrize("name,n", [("sift1m", 20000), ("gmm10k", 5000)])
def test_to_fp8_matches_oracle(onng, name, n):
    """Per-dimension scales and e4m3 codes: the same float32 division and the
    same rounding decision on both sides, so both are bit-exact."""
    X, _ = synth.workload(name, n=n, nq=1)
    X[:, 3] = 0.0  # an all-zero column takes scale 1
    scale, codes = onng.to_fp8(dev(X))
    o_scale, o_codes, _ = oracle.fp8_quantize(X)
    assert np.array_equal(host(scale), o_scale)
    assert np.array_equal(host(codes), o_codes)


@pytest.mark.parametrize("name", ["sift1m", "gmm10k"])
def test_search_fp8_follows_oracle_on_dequantised_vectors(onng, name):
    """The FP8 pass follows the oracle run on the dequantised vectors
    scale_j * e4m3 (float32 products), then the float32 rerank of k_rerank
    candidates against the exact vectors."""
    X, Q = synth.workload(name, n=4000, nq=150)
    nbr, ln = onng.build_knng(dev(X), 30)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 20))
    seeds = onng.seeds_pivot(dev(X), dev(Q), 512, 10)
    idx = onng.Index(g[0], g[1], dev(X))
    ids, dist, st = onng.search(idx, dev(Q), 10, 10, 0.05, seeds, precision=onng.PREC_FP8, k_rerank=32)
    _, _, xq = oracle.fp8_quantize(X)
    cand, _, o_st, mg = oracle.search(host(g[0]), host(g[1]), xq, Q, 32, 10, np.float32(0.05), host(seeds),
                                      margin=True)
    ids, dist, st = host(ids), host(dist), host(st)
    assert_valid_lists(ids, dist, X, Q)
    tf = mg > DECIDE
    assert tf.mean() >= 0.5
    # tie-free candidate searches do the same work and keep the same candidates
    assert np.array_equal(st[tf, 0], o_st[tf, 0]) and np.array_equal(st[tf, 1], o_st[tf, 1])
    assert_reranked(ids[tf], dist[tf], cand[tf], X, Q[tf], 10)


def test_search_bf16_float_data(onng):
    """On float data the bf16 pass follows the oracle run on bf16-rounded vectors;
    the rerank then uses the exact vectors."""
    X, Q = synth.workload("gmm10k", n=3000, nq=100)
    nbr, ln = onng.build_knng(dev(X), 30)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 20))
    seeds = onng.seeds_pivot(dev(X), dev(Q), 512, 10)
    idx = onng.Index(g[0], g[1], dev(X))
    ids, dist, st = onng.search(idx, dev(Q), 10, 10, 0.05, seeds, precision=onng.PREC_BF16, k_rerank=32)
    Xb = oracle.bf16_round(X)
    cand, _, o_st, mg = oracle.search(host(g[0]), host(g[1]), Xb, Q, 32, 10, np.float32(0.05), host(seeds),
                                      margin=True)
    ids, dist, st = host(ids), host(dist), host(st)
    assert_valid_lists(ids, dist, X, Q)
    tf = mg > DECIDE
    assert tf.mean() >= 0.5
    assert np.array_equal(st[tf, 0], o_st[tf, 0]) and np.array_equal(st[tf, 1], o_st[tf, 1])
    # the rerank of the oracle's bf16 candidates with exact float64 distances
    assert_reranked(ids[tf], dist[tf], cand[tf], X, Q[tf], 10)
    assert torch.equal(onng.to_bf16(dev(X)).float().cpu(), torch.from_numpy(Xb))
