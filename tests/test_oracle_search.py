"""Pins of the oracle's KnnSearch (Algorithm 1), visited set (Set / IsSet), seed
rules, bfloat16 rounding and the predictor network.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

from paper_1810_07355_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_chain_trace(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "chain_search.json")))
    X = np.array(g["X"], np.float32)
    n = len(X)
    rows = [[c for c in (i - 1, i + 1) if 0 <= c < n] for i in range(n)]
    ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col = np.array(sum(rows, []), np.int32)
    Q = np.array([g["query"]], np.float32)
    seeds = np.array([g["seeds"]], np.int32)
    for c in g["cases"]:
        ids, dist, st = oracle_lib.search(ptr, col, X, Q, g["k"], c["e_s"], g["eps"], seeds)
        assert ids[0].tolist() == c["ids"]
        np.testing.assert_allclose(dist[0], c["dist"], rtol=1e-6)
        assert st[0, 0] == c["distance_computations"]
        assert st[0, 1] == c["expansions"]


def _chain(g):
    X = np.array(g["X"], np.float32)
    n = len(X)
    rows = [[c for c in (i - 1, i + 1) if 0 <= c < n] for i in range(n)]
    ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col = np.array(sum(rows, []), np.int32)
    return X, ptr, col


def test_chain_margin(oracle_lib):
    """The smallest relative gap among the comparisons Algorithm 1 decided,
    traced by hand on the chain (golden values), including an exact tie (0)."""
    g = json.load(open(os.path.join(GOLDEN, "chain_search.json")))
    X, ptr, col = _chain(g)
    Q = np.array([g["query"]], np.float32)
    for c in g["cases"]:
        _, _, _, mg = oracle_lib.search(ptr, col, X, Q, g["k"], c["e_s"], g["eps"], np.array([g["seeds"]], np.int32),
                                        margin=True)
        np.testing.assert_allclose(mg, [c["margin"]], rtol=1e-6)
    m = json.load(open(os.path.join(GOLDEN, "chain_margin.json")))
    ids, dist, st, mg = oracle_lib.search(ptr, col, X, np.array([m["query"]], np.float32), m["k"], m["e_s"], m["eps"],
                                          np.array([m["seeds"]], np.int32), margin=True)
    assert ids[0].tolist() == m["ids"]
    np.testing.assert_allclose(dist[0], m["dist"], rtol=1e-6)
    assert st[0, 0] == m["distance_computations"] and st[0, 1] == m["expansions"]
    np.testing.assert_allclose(mg, [m["margin"]], rtol=1e-6)
    t = m["tie_case"]
    _, _, _, mg = oracle_lib.search(ptr, col, X, np.array([t["query"]], np.float32), t["k"], t["e_s"], t["eps"],
                                    np.array([t["seeds"]], np.int32), margin=True)
    assert mg[0] == t["margin"]


def test_margin_leaves_results_unchanged(oracle_lib):
    """Asking for the margin changes no result or count, and a run whose
    distances are all integers at least one apart has a margin of at least
    1 / (largest distance compared)."""
    X, Q = synth.workload("gmm10k", n=1500, nq=40)
    ids, dist = oracle_lib.knng(X, 20)
    ptr, col, _ = oracle_lib.adjust_degree(ids, dist, 8, 16)
    seeds = oracle_lib.seeds_pivot(X, Q, 64, 5)
    a = oracle_lib.search(ptr, col, X, Q, 10, 8, 0.1, seeds)
    b = oracle_lib.search(ptr, col, X, Q, 10, 8, 0.1, seeds, margin=True)
    for u, v in zip(a, b[:3]):
        assert np.array_equal(u, v)
    assert (b[3] >= 0).all() and np.isfinite(b[3]).all()
    # 1-D points at even integers, queries at odd integers + 0.5: every distance
    # is an integer + 0.5 and every bound r * 1 too, so two compared values that
    # differ do so by >= 1
    P = (2 * np.arange(200, dtype=np.float32))[:, None]
    rows = [[c for c in (i - 1, i + 1) if 0 <= c < 200] for i in range(200)]
    ptr1 = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col1 = np.array(sum(rows, []), np.int32)
    Q1 = (2 * np.arange(5, 195, 9, dtype=np.float32) + 0.5)[:, None]
    s1 = np.full((len(Q1), 1), 0, np.int32)
    _, d1, _, mg = oracle_lib.search(ptr1, col1, P, Q1, 3, 0, 0.0, s1, margin=True)
    assert (mg >= 1.0 / 400.0).all()


@pytest.fixture(scope="module")
def one_cluster(oracle_lib):
    X = synth.gaussian_mixture(800, d=16, components=1, sigma=5.0, seed=31)
    Q = synth.gaussian_mixture(30, d=16, components=1, sigma=5.0, seed=32)
    ids, dist = oracle_lib.knng(X, 12)
    ptr, col, ln = oracle_lib.adjust_degree(ids, dist, 6, 12)
    return X, Q, (ptr, col, ln)


def test_unbounded_search_is_exact(oracle_lib, one_cluster):
    """eps = inf and e_s = inf on a strongly connected graph visit every node."""
    X, Q, (ptr, col, _) = one_cluster
    n = len(X)
    A = sp.csr_matrix((np.ones(len(col)), col, ptr), shape=(n, n))
    assert connected_components(A, directed=True, connection="strong")[0] == 1
    seeds = oracle_lib.seeds_random(5, len(Q), n, 3)
    ids, dist, st = oracle_lib.search(ptr, col, X, Q, 10, 0, np.inf, seeds)
    td, ti = cKDTree(X.astype(np.float64)).query(Q.astype(np.float64), k=10)
    assert np.array_equal(ids, ti)
    np.testing.assert_allclose(dist, td, rtol=1e-12)
    assert (st[:, 0] == n).all()


def test_complete_graph_is_exact(oracle_lib):
    rng = np.random.default_rng(8)
    X = rng.normal(size=(60, 5)).astype(np.float32)
    Q = rng.normal(size=(10, 5)).astype(np.float32)
    n = len(X)
    col = np.concatenate([[j for j in range(n) if j != i] for i in range(n)]).astype(np.int32)
    ptr = np.arange(0, n * (n - 1) + 1, n - 1, dtype=np.int64)
    seeds = np.zeros((len(Q), 1), np.int32)
    ids, dist, _ = oracle_lib.search(ptr, col, X, Q, 7, 0, 0.0, seeds)
    td, ti = cKDTree(X.astype(np.float64)).query(Q.astype(np.float64), k=7)
    assert np.array_equal(ids, ti)


def test_results_are_valid(oracle_lib, one_cluster):
    X, Q, (ptr, col, _) = one_cluster
    seeds = oracle_lib.seeds_random(9, len(Q), len(X), 4)
    for eps in (0.0, 0.05):
        ids, dist, st = oracle_lib.search(ptr, col, X, Q, 10, 4, eps, seeds)
        for q in range(len(Q)):
            got = ids[q][ids[q] >= 0]
            assert len(set(got.tolist())) == len(got)
            rec = np.linalg.norm(X[got].astype(np.float64) - Q[q].astype(np.float64), axis=1)
            np.testing.assert_allclose(dist[q][:len(got)], rec, rtol=1e-12)
            assert (np.diff(dist[q][:len(got)]) >= 0).all()
        assert (st[:, 0] >= st[:, 1]).all()


def test_small_k_pads(oracle_lib):
    X = np.array([[0.0], [1.0], [5.0]], np.float32)
    ptr = np.array([0, 1, 2, 2], np.int64)
    col = np.array([1, 0], np.int32)
    ids, dist, _ = oracle_lib.search(ptr, col, X, np.array([[0.2]], np.float32), 3, 0, 0.0,
                                     np.array([[0]], np.int32))
    assert ids[0].tolist() == [0, 1, -1] and np.isinf(dist[0, 2])


def test_recall_grows_with_eps(oracle_lib):
    X, Q = synth.workload("gmm10k", n=4000, nq=100)
    ids, dist = oracle_lib.knng(X, 40)
    g = oracle_lib.adjust_path(*oracle_lib.adjust_degree(ids, dist, 10, 30))
    seeds = oracle_lib.seeds_pivot(X, Q, 1024, 10)
    gt, _ = oracle_lib.knn(X, Q, 10)
    rec = []
    for eps in (0.0, 0.02, 0.05, 0.1, 0.2):
        r, _, _ = oracle_lib.search(g[0], g[1], X, Q, 10, 10, eps, seeds)
        rec.append(np.mean([len(set(a) & set(b)) / 10 for a, b in zip(r, gt)]))
    assert all(b >= a - 0.01 for a, b in zip(rec, rec[1:]))
    assert rec[-1] > 0.9


def test_hash_size_formula(oracle_lib):
    # s = 2^floor((floor(log2 n) + 11) / 2)
    assert oracle_lib.hash_size(10_000) == 4096
    assert oracle_lib.hash_size(1_000_000) == 32768
    assert oracle_lib.hash_size(1_200_000) == 32768
    assert oracle_lib.hash_size(1 << 20) == 1 << 15
    assert oracle_lib.hash_size(2) == 1 << 6


def test_hash_set_isset_is_a_set(oracle_lib):
    rng = np.random.default_rng(4)
    n = 10_000  # s = 4096: plenty of collisions in 20k draws from 2^20 ids
    ids = rng.integers(0, 1 << 20, size=20_000).astype(np.int32)
    got = oracle_lib.hash_selftest(ids, n)
    seen, want = set(), []
    for i in ids.tolist():
        want.append(i in seen)
        seen.add(i)
    assert got.tolist() == want


def test_splitmix64_published_vectors(oracle_lib):
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    for v in g["vectors"]:
        assert oracle_lib.splitmix64(v["state"], len(v["outputs"])) == [int(x, 0) for x in v["outputs"]]


def test_random_seeds_from_published_draws(oracle_lib):
    """The random rule maps the published SplitMix64 outputs z to floor(z * n / 2^64)
    and redraws repeats; query q starts at state global_seed + q * 2^32."""
    g = json.load(open(os.path.join(GOLDEN, "splitmix64.json")))
    z0 = [int(x, 0) for x in g["vectors"][0]["outputs"]]  # state 0
    z1 = [int(x, 0) for x in g["vectors"][1]["outputs"]]  # state 1234567
    assert oracle_lib.seeds_random(0, 1, 1000, 3)[0].tolist() == [(z * 1000) >> 64 for z in z0]
    # query 1 of global seed 1234567 - 2^32 starts at state 1234567
    gs = (1234567 - (1 << 32)) % (1 << 64)
    assert oracle_lib.seeds_random(gs, 2, 10**6, 5)[1].tolist() == [(z * 10**6) >> 64 for z in z1]
    # n = 8: the published draws map to 2, 1, 4, 1, 7; the repeated 1 is redrawn
    assert [(z * 8) >> 64 for z in z1] == [2, 1, 4, 1, 7]
    assert oracle_lib.seeds_random(1234567, 1, 8, 4)[0].tolist() == [2, 1, 4, 7]


def test_random_seeds_properties(oracle_lib):
    s = oracle_lib.seeds_random(123, 4000, 1000, 10)
    assert s.min() >= 0 and s.max() < 1000
    assert all(len(set(r.tolist())) == 10 for r in s)
    counts = np.bincount(s.ravel(), minlength=1000)
    chi2 = ((counts - 40.0) ** 2 / 40.0).sum()
    assert chi2 < 1000 + 6 * np.sqrt(2000)  # df = 999
    assert not np.array_equal(s[0], s[1])
    assert np.array_equal(oracle_lib.seeds_random(123, 4000, 1000, 10), s)
    assert oracle_lib.seeds_random(1, 2, 5, 3).tolist() == [[0, 1, 2], [0, 1, 2]]


def test_pivot_seeds_match_kdtree(oracle_lib):
    rng = np.random.default_rng(6)
    X = rng.normal(size=(5000, 6)).astype(np.float32)
    Q = rng.normal(size=(50, 6)).astype(np.float32)
    s = oracle_lib.seeds_pivot(X, Q, 256, 5)
    piv = (np.arange(256) * 5000) // 256
    _, ti = cKDTree(X[piv].astype(np.float64)).query(Q.astype(np.float64), k=5)
    assert np.array_equal(s, piv[ti])


def test_bf16_round_matches_torch(oracle_lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(size=5000) * 10 ** rng.uniform(-30, 30, 5000),
                        np.arange(-300, 300), [0.0, -0.0, np.inf, -np.inf]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(oracle_lib.bf16_round(x), want)
    # integers 0..256 are exact in bfloat16
    ints = np.arange(0, 257, dtype=np.float32)
    assert np.array_equal(oracle_lib.bf16_round(ints), ints)


def test_mlp_forward_matches_torch(oracle_lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    P = rng.normal(size=oracle_lib.MLP_NPARAM) * 0.3
    x = rng.normal(size=(17, 16))
    sizes = [64 * 16, 64, 64 * 64, 64, 2 * 64, 2]
    W1, b1, W2, b2, W3, b3 = [torch.from_numpy(a) for a in np.split(P, np.cumsum(sizes)[:-1])]
    h = torch.relu(torch.from_numpy(x) @ W1.reshape(64, 16).T + b1)
    h = torch.relu(h @ W2.reshape(64, 64).T + b2)
    y = h @ W3.reshape(2, 64).T + b3
    np.testing.assert_allclose(oracle_lib.mlp_forward(P, x), y.numpy(), rtol=1e-12, atol=1e-12)


def test_mlp_gradient_finite_difference(oracle_lib):
    rng = np.random.default_rng(9)
    P = rng.normal(size=oracle_lib.MLP_NPARAM) * 0.3
    x = rng.normal(size=(9, 16))
    t = rng.normal(size=(9, 2))
    loss, G = oracle_lib.mlp_loss_grad(P, x, t)
    h = 1e-6
    idx = rng.choice(oracle_lib.MLP_NPARAM, size=300, replace=False)
    idx = np.concatenate([idx, np.arange(oracle_lib.MLP_NPARAM - 130, oracle_lib.MLP_NPARAM)])
    for i in idx:
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (oracle_lib.mlp_loss_grad(Pp, x, t)[0] - oracle_lib.mlp_loss_grad(Pm, x, t)[0]) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(G[i])), (i, fd, G[i])
    y = oracle_lib.mlp_forward(P, x)
    assert abs(loss - 0.5 * ((y - t) ** 2).sum() / 9) < 1e-12


def test_adam_matches_torch(oracle_lib):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(12)
    P = rng.normal(size=50)
    m, v = np.zeros(50), np.zeros(50)
    tp = torch.nn.Parameter(torch.from_numpy(P.copy()))
    opt = torch.optim.Adam([tp], lr=0.01)
    for t in range(1, 6):
        G = rng.normal(size=50)
        oracle_lib.adam_step(P, G, m, v, t, 0.01)
        tp.grad = torch.from_numpy(G)
        opt.step()
    np.testing.assert_allclose(P, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_probe_features_chain(oracle_lib):
    """Probe after one hop of the chain trace (Algorithm 1 stopped before the
    second expansion): node 0 expanded, node 1 visited, R = {1, 0}."""
    g = json.load(open(os.path.join(GOLDEN, "chain_search.json")))
    X = np.array(g["X"], np.float32)
    n = len(X)
    rows = [[c for c in (i - 1, i + 1) if 0 <= c < n] for i in range(n)]
    ptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    col = np.array(sum(rows, []), np.int32)
    Q = np.array([g["query"]], np.float32)
    f, st = oracle_lib.search_probe(ptr, col, X, Q, 2, 0, 0.0, np.array([g["seeds"]], np.int32), 1, 0.9)
    e6 = 1e-6
    want = [0.9, np.log(6.4 + e6), 0.0, 0.0, np.log((5.4 + e6) / (6.4 + e6)), np.log((6.4 + e6) / (5.4 + e6)),
            0.0, 2 / 2, 1.0, np.log1p(2), 1 / 2, 1.0, 0.0, np.log1p(1), 1.0, np.log(1) / 8]
    np.testing.assert_allclose(f[0], want, atol=1e-6)
    assert st[0, 0] == 2 and st[0, 1] == 1
    # a cap beyond the search length changes nothing: the probe is the full search
    f, st = oracle_lib.search_probe(ptr, col, X, Q, 2, 0, 0.0, np.array([g["seeds"]], np.int32), 100, 0.9)
    assert st[0, 1] == 8 and f[0, 14] == 0.0 and abs(f[0, 8] - 0.08) < 1e-12


def test_e4m3_matches_torch_float8(oracle_lib):
    """The oracle's e4m3 encode / decode against torch's float8_e4m3fn (round to
    nearest even) on random values, every midpoint between neighbouring codes,
    and all 256 codes."""
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    rng = np.random.default_rng(5)
    codes = np.arange(256, dtype=np.uint8)
    want = torch.from_numpy(codes).view(torch.float8_e4m3fn).float().numpy()
    got = oracle_lib.e4m3_decode(codes)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    assert np.array_equal(got[~np.isnan(got)], want[~np.isnan(want)])
    pos = np.sort(got[:0x7F])
    mids = ((pos[1:].astype(np.float64) + pos[:-1]) / 2).astype(np.float32)
    x = np.concatenate([rng.uniform(-448, 448, 50_000), rng.uniform(-1, 1, 50_000), rng.uniform(-0.02, 0.02, 20_000),
                        mids, -mids, pos, [0.0, -0.0, 448.0, -448.0]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(oracle_lib.e4m3_encode(x), want)
    # saturation (torch gives NaN there): the largest finite code
    big = np.array([449.0, 464.0, 1e6, 3e38, -500.0], dtype=np.float32)
    assert np.array_equal(oracle_lib.e4m3_encode(big), [0x7E, 0x7E, 0x7E, 0x7E, 0xFE])


def test_fp8_quantize_scales_and_error_bound(oracle_lib):
    """c_j = max |x_ij| / 448 (1 for a zero column); every dequantised value is
    within half a step of e4m3 (2^-4 relative, 2^-10 c_j absolute near zero)."""
    rng = np.random.default_rng(6)
    X = rng.normal(0, 3, size=(500, 24)).astype(np.float32)
    X[:, 5] = 0.0
    X[:, 7] = np.abs(X[:, 7]) * 1e-4
    scale, codes, xq = oracle_lib.fp8_quantize(X)
    mx = np.abs(X).max(0)
    assert np.array_equal(scale, np.where(mx > 0, mx / np.float32(448.0), np.float32(1.0)).astype(np.float32))
    assert np.array_equal(xq, (scale[None, :] * oracle_lib.e4m3_decode(codes)).astype(np.float32))
    err = np.abs(xq.astype(np.float64) - X)
    bound = np.maximum(np.abs(X) * 2.0 ** -4, scale[None, :] * 2.0 ** -10) * (1 + 1e-6)
    assert np.all(err <= bound)
    assert np.all(xq[:, 5] == 0.0)
    # the column maximum is stored exactly (it scales to 448, a code)
    j = np.abs(X).argmax(0)
    assert np.allclose(np.abs(xq[j, np.arange(24)]), mx, rtol=1e-6)


def test_expansion_cap(oracle_lib, one_cluster):
    """The capped search: a cap no query reaches changes nothing; with a cap of one
    expansion and eps = inf the result is the k nearest of the seeds and the first
    e_s neighbours of the nearest seed (brute force), flagged 4 when a candidate
    was left; expansion counts never exceed the cap."""
    X, Q, (ptr, col, _) = one_cluster
    n = len(X)
    seeds = oracle_lib.seeds_random(11, len(Q), n, 3)
    ids, dist, st = oracle_lib.search(ptr, col, X, Q, 10, 6, 0.1, seeds)
    c_ids, c_dist, c_st = oracle_lib.search(ptr, col, X, Q, 10, 6, 0.1, seeds, max_exp=int(st[:, 1].max()) + 1)
    assert np.array_equal(ids, c_ids) and np.array_equal(st[:, :2], c_st[:, :2]) and (c_st[:, 3] == 0).all()
    c_ids, c_dist, c_st = oracle_lib.search(ptr, col, X, Q, 10, 6, np.inf, seeds, max_exp=1)
    assert (c_st[:, 1] == 1).all()
    X64, Q64 = X.astype(np.float64), Q.astype(np.float64)
    for q in range(len(Q)):
        sd = np.sqrt(((X64[seeds[q]] - Q64[q]) ** 2).sum(1))
        first = seeds[q][np.lexsort((seeds[q], sd))[0]]
        cand = np.unique(np.concatenate([seeds[q], col[ptr[first]:ptr[first] + 6]]))
        cd = np.sqrt(((X64[cand] - Q64[q]) ** 2).sum(1))
        order = np.lexsort((cand, cd))[:10]
        want = np.full(10, -1)
        want[:len(order)] = cand[order]
        assert np.array_equal(c_ids[q], want), q
        assert c_st[q, 3] == (4 if len(cand) > 1 else 0)
    for cap in (2, 5):
        _, _, c_st = oracle_lib.search(ptr, col, X, Q, 10, 6, 0.1, seeds, max_exp=cap)
        assert (c_st[:, 1] <= cap).all()


def _capped_best_first(X64, q, ptr, col, seeds, k, e_s, cap):
    """Brute force of Algorithm 1 at eps = inf stopped after `cap` expansions:
    every scanned neighbour enters the candidates, so the run pops nodes in
    (distance, id) order from everything seen and the results are the k nearest
    of everything seen.  Returns (ids, distance computations, expansions,
    candidate left)."""
    seen = {}
    for s in seeds:
        seen.setdefault(int(s), float(np.sqrt(((X64[s] - q) ** 2).sum())))
    cand = dict(seen)
    expansions = 0
    while cand and expansions < cap:
        node = min(cand, key=lambda i: (cand[i], i))
        del cand[node]
        expansions += 1
        for nb in col[ptr[node]:min(ptr[node] + e_s, ptr[node + 1])]:
            nb = int(nb)
            if nb not in seen:
                seen[nb] = float(np.sqrt(((X64[nb] - q) ** 2).sum()))
                cand[nb] = seen[nb]
    ids = sorted(seen, key=lambda i: (seen[i], i))[:k]
    return ids + [-1] * (k - len(ids)), len(seen), expansions, bool(cand)


def test_expansion_cap_against_brute_force(oracle_lib, one_cluster):
    """Caps of 2, 3 and 7 expansions at eps = inf: ids, distance computations,
    expansions and the limit flag equal a brute-force best-first run stopped at
    the cap."""
    X, Q, (ptr, col, _) = one_cluster
    seeds = oracle_lib.seeds_random(13, len(Q), len(X), 3)
    X64 = X.astype(np.float64)
    for cap in (2, 3, 7):
        ids, _, st = oracle_lib.search(ptr, col, X, Q, 10, 6, np.inf, seeds, max_exp=cap)
        for qi in range(len(Q)):
            want, dc, ex, left = _capped_best_first(X64, Q[qi].astype(np.float64), ptr, col, seeds[qi], 10, 6,
                                                    cap)
            assert ids[qi].tolist() == want, (cap, qi)
            assert (st[qi, 0], st[qi, 1], st[qi, 3]) == (dc, ex, 4 if left else 0), (cap, qi)
