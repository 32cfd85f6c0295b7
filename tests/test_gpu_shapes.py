"""GPU parity at the text- and GIST-shaped dimensions (d = 100 and d = 960).

The search kernels read a vector as float4 chunks, one per lane and round:
d = 100 leaves a ragged last round (25 of 32 lanes), d = 960 takes eight rounds
(240 chunks).  The kNN graph of float data at these d goes through the split
bfloat16 tensor-core sweep (queries fewer than 128: the float32 SIMT sweep).  Integer-valued inputs whose squared distances stay below 2^24 are
exact in float32, so there graphs and searches must equal the float64 oracle bit
for bit at every eps; float inputs follow the near-tie rules of parity_helpers.

Inputs are the generators of the text-embedding (unit vectors, Zipf cluster
sizes) and GIST-like (|centre + noise|) workloads with fewer clusters than the
full-size sets, so that a few thousand points still form dense clusters.
"""
import numpy as np
import pytest

import oracle
from paper_1810_07355_gb300 import synth
from parity_helpers import (DECIDE, REL, assert_reranked, assert_rows_near, assert_search_parity, assert_valid_lists,
                            d64)

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


def text_like(n, nq):
    kw = dict(d=100, directions=20, centers_seed=1903)
    return synth.text_embeddings(n, seed=1904, **kw), synth.text_embeddings(nq, seed=1905, **kw)


def gist_like(n, nq):
    kw = dict(d=960, clusters=10, centers_seed=1906)
    return synth.gist_like(n, seed=1907, **kw), synth.gist_like(nq, seed=1908, **kw)


def int_like(n, nq, d):
    """Image-descriptor integers; at d = 960 divided by 4 (0..63) so that squared
    distances stay below 2^24 and float32 is exact."""
    kw = dict(d=d, clusters=40, centers_seed=1909)
    X = synth.image_descriptors(n, seed=1910, **kw)
    Q = synth.image_descriptors(nq, seed=1911, **kw)
    if d > 128:
        X, Q = np.floor(X / 4), np.floor(Q / 4)
    return X.astype(np.float32), Q.astype(np.float32)


def graph(onng, X, k=30, e_o=10, e_i=20):
    nbr, ln = onng.build_knng(dev(X), k)
    return onng.adjust_path(*onng.adjust_degree(nbr, ln, e_o, e_i))


# ----------------------------------------------------------------------------- kNN

@pytest.mark.parametrize("d", [100, 960])
def test_knng_integer_exact_at_d(onng, d):
    X, _ = int_like(1500 if d == 960 else 2500, 1, d)
    nbr, ln = onng.build_knng(dev(X), 24)
    o_ids, o_len = oracle.knng(X, 24)
    assert np.array_equal(host(nbr), o_ids)
    np.testing.assert_allclose(host(ln), o_len, rtol=1e-6)


@pytest.mark.parametrize("shape", ["text", "gist"])
def test_knng_float_near_ties_at_d(onng, shape):
    X, _ = text_like(3000, 1) if shape == "text" else gist_like(1500, 1)
    nbr, ln = onng.build_knng(dev(X), 30)
    o_ids, o_len = oracle.knng(X, 30)
    ids, lens = host(nbr), host(ln).astype(np.float64)
    assert_rows_near(ids, lens, o_ids, o_len)
    # every returned length is the float64 distance of the returned id
    np.testing.assert_allclose(lens, d64(X, X, ids), rtol=REL)
    # differing ids only inside near-ties: most rows are identical
    assert (ids == o_ids).all(1).mean() > 0.9


@pytest.mark.parametrize("shape", ["text", "gist"])
def test_knn_queries_at_d(onng, shape):
    X, Q = text_like(2500, 200) if shape == "text" else gist_like(1200, 100)
    ids, ln = onng.knn(dev(X), dev(Q), 10)
    o_ids, o_len = oracle.knn(X, Q, 10)
    assert_rows_near(host(ids), host(ln).astype(np.float64), o_ids, o_len)


# ----------------------------------------------------------------------------- search, integer data

@pytest.fixture(scope="module", params=[100, 960])
def int_graph(onng, request):
    d = request.param
    X, Q = int_like(3000 if d == 100 else 2000, 160, d)
    g = graph(onng, X)
    seeds = onng.seeds_pivot(dev(X), dev(Q), 256, 10)
    return X, Q, g, seeds


@pytest.mark.parametrize("k,e_s,eps,padded", [(10, 10, 0.0, False), (10, 10, 0.1, True), (10, 0, 0.2, False),
                                              (1, 5, 0.05, True), (100, 20, 0.05, True),
                                              (10, 10, float("inf"), False)])
def test_search_integer_exact_at_d(onng, int_graph, k, e_s, eps, padded):
    """ids, distances and counts bit-exact against Algorithm 1 in float64 at
    d = 100 (ragged last chunk round) and d = 960 (eight rounds)."""
    X, Q, g, seeds = int_graph
    idx = onng.Index(g[0], g[1], dev(X))
    if padded:
        idx.with_adjacency(max(e_s, 1))
    ids, dist, st = onng.search(idx, dev(Q), k, e_s, eps, seeds)
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, k, e_s, np.float32(eps), host(seeds))
    assert np.array_equal(host(ids), o_ids)
    np.testing.assert_allclose(host(dist), o_dist, rtol=1e-6)
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])
    assert np.array_equal(host(st)[:, 1], o_st[:, 1])
    assert (host(st)[:, 3] == 0).all()


def test_search_integer_bf16_at_d(onng, int_graph):
    """Integers up to 256 are exact in bfloat16: the bf16 pass with an float32
    rerank of k_rerank candidates equals the float32 search with k_rerank results."""
    X, Q, g, seeds = int_graph
    idx = onng.Index(g[0], g[1], dev(X))
    ids, dist, st = onng.search(idx, dev(Q), 10, 10, 0.05, seeds, precision=onng.PREC_BF16, k_rerank=24)
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, 24, 10, np.float32(0.05), host(seeds))
    assert np.array_equal(host(ids), o_ids[:, :10])
    np.testing.assert_allclose(host(dist), o_dist[:, :10], rtol=1e-6)
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])


def test_search_integer_fp8_at_d(onng, int_graph):
    """FP8: the search follows the oracle run on the dequantised vectors (float
    values, so the margin rule applies), then the float32 rerank."""
    X, Q, g, seeds = int_graph
    idx = onng.Index(g[0], g[1], dev(X))
    ids, dist, st = onng.search(idx, dev(Q), 10, 10, 0.05, seeds, precision=onng.PREC_FP8, k_rerank=32)
    _, _, xq = oracle.fp8_quantize(X)
    cand, o_d, o_st, mg = oracle.search(host(g[0]), host(g[1]), xq, Q, 32, 10, np.float32(0.05), host(seeds),
                                        margin=True)
    ids, dist, st = host(ids), host(dist), host(st)
    assert_valid_lists(ids, dist, X, Q)
    tf = mg > DECIDE
    assert tf.mean() >= 0.5
    assert np.array_equal(st[tf, 0], o_st[tf, 0]) and np.array_equal(st[tf, 1], o_st[tf, 1])
    assert_reranked(ids[tf], dist[tf], cand[tf], X, Q[tf], 10)


# ----------------------------------------------------------------------------- search, float data

@pytest.fixture(scope="module", params=["text", "gist"])
def float_graph(onng, request):
    X, Q = text_like(4000, 200) if request.param == "text" else gist_like(3000, 150)
    g = graph(onng, X)
    seeds = onng.seeds_pivot(dev(X), dev(Q), 512, 10)
    return request.param, X, Q, g, seeds


def _eps_for(shape):
    # GIST-like distances crowd into a band about 1 % wide, so at larger eps
    # nearly every run meets a near-tie; the integer tests cover those eps exactly
    return (0.0, 0.02) if shape == "gist" else (0.0, 0.05)


def test_search_float_at_d(onng, float_graph):
    shape, X, Q, g, seeds = float_graph
    idx = onng.Index(g[0], g[1], dev(X))
    for eps in _eps_for(shape):
        ids, dist, st = onng.search(idx, dev(Q), 10, 10, eps, seeds)
        o = oracle.search(host(g[0]), host(g[1]), X, Q, 10, 10, np.float32(eps), host(seeds), margin=True)
        assert_search_parity(host(ids), host(dist), host(st), *o, X, Q, min_tie_free=0.3)


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_search_reduced_float_at_d(onng, float_graph, prec):
    """bf16 / FP8 candidate search against the oracle run on the rounded
    (dequantised) vectors, then the float32 rerank against the exact vectors."""
    shape, X, Q, g, seeds = float_graph
    idx = onng.Index(g[0], g[1], dev(X))
    p = onng.PREC_BF16 if prec == "bf16" else onng.PREC_FP8
    Xr = oracle.bf16_round(X) if prec == "bf16" else oracle.fp8_quantize(X)[2]
    for eps in _eps_for(shape):
        ids, dist, st = onng.search(idx, dev(Q), 10, 10, eps, seeds, precision=p, k_rerank=32)
        cand, _, o_st, mg = oracle.search(host(g[0]), host(g[1]), Xr, Q, 32, 10, np.float32(eps), host(seeds),
                                          margin=True)
        ids, dist, st = host(ids), host(dist), host(st)
        assert_valid_lists(ids, dist, X, Q)
        tf = mg > DECIDE
        assert tf.mean() >= 0.3, tf.mean()
        assert np.array_equal(st[tf, 0], o_st[tf, 0]) and np.array_equal(st[tf, 1], o_st[tf, 1])
        assert_reranked(ids[tf], dist[tf], cand[tf], X, Q[tf], 10)
