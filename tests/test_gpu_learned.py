"""GPU parity of the learned-parameter path: the predictor network's forward,
gradient, Adam and fused training kernels against the float64 oracle, the
probe features against the oracle's probe, and the per-query search against
the oracle run with the same per-query parameters."""
import numpy as np
import pytest

import oracle
from paper_1810_07355_gb300 import synth

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


def _params(seed=1):
    rng = np.random.default_rng(seed)
    return rng.normal(size=oracle.MLP_NPARAM) * 0.25


def test_mlp_forward_matches_oracle(onng):
    P = _params()
    X = np.random.default_rng(2).normal(size=(333, 16))
    Y = host(onng.mlp_forward(dev(P.astype(np.float32)), dev(X.astype(np.float32))))
    np.testing.assert_allclose(Y, oracle.mlp_forward(P.astype(np.float32).astype(np.float64),
                                                       X.astype(np.float32).astype(np.float64)), rtol=1e-4, atol=1e-5)


def test_mlp_gradient_matches_oracle(onng):
    P = _params(3).astype(np.float32)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(1000, 16)).astype(np.float32)
    T = rng.normal(size=(1000, 2)).astype(np.float32)
    loss, G = onng.mlp_loss_grad(dev(P), dev(X), dev(T))
    o_loss, o_G = oracle.mlp_loss_grad(P.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(float(loss) - o_loss) <= 1e-4 * abs(o_loss)
    g = host(G).astype(np.float64)
    # within 1e-4 relative of the float64 gradient (as a vector), and element by
    # element up to the float32 rounding of a 1000-term mean
    assert np.linalg.norm(g - o_G) <= 1e-4 * np.linalg.norm(o_G)
    np.testing.assert_allclose(g, o_G, rtol=1e-4, atol=1e-5 * np.abs(o_G).max())


def test_mlp_adam_and_fused_training_match_oracle(onng):
    rng = np.random.default_rng(5)
    P0 = _params(6).astype(np.float32)
    X = rng.normal(size=(96, 16)).astype(np.float32)
    T = rng.normal(size=(96, 2)).astype(np.float32)
    # oracle: 6 steps on consecutive batches of 32 (wrapping)
    P, m, v = P0.astype(np.float64), np.zeros(oracle.MLP_NPARAM), np.zeros(oracle.MLP_NPARAM)
    for t in range(1, 7):
        b = [((t - 1) * 32 + j) % 96 for j in range(32)]
        _, G = oracle.mlp_loss_grad(P, X[b].astype(np.float64), T[b].astype(np.float64))
        oracle.adam_step(P, G, m, v, t, 1e-2)
    # separate gradient + Adam kernels
    Pd, Md, Vd = dev(P0.copy()), torch.zeros(oracle.MLP_NPARAM, device="cuda"), torch.zeros(oracle.MLP_NPARAM, device="cuda")
    for t in range(1, 7):
        b = torch.tensor([((t - 1) * 32 + j) % 96 for j in range(32)], device="cuda")
        _, G = onng.mlp_loss_grad(Pd, dev(X)[b], dev(T)[b])
        onng.mlp_adam(Pd, G, Md, Vd, t, 1e-2)
    np.testing.assert_allclose(host(Pd), P, rtol=1e-3, atol=1e-4)
    # fused single-kernel training
    Pf, Mf, Vf = dev(P0.copy()), torch.zeros(oracle.MLP_NPARAM, device="cuda"), torch.zeros(oracle.MLP_NPARAM, device="cuda")
    L = onng.mlp_train(Pf, Mf, Vf, dev(X), dev(T), steps=6, batch=32, lr=1e-2, losses=True)
    np.testing.assert_allclose(host(Pf), P, rtol=1e-3, atol=1e-4)
    assert L.shape == (6,) and torch.isfinite(L).all()


def test_mlp_predict_bf16(onng):
    P = _params(7).astype(np.float32) * 0.2
    X = np.random.default_rng(8).normal(size=(200, 16)).astype(np.float32)
    eps, es = onng.mlp_predict(dev(P), dev(X), alpha=1.5, es_min=6, es_max=20)
    Pb, Xb = oracle.bf16_round(P).astype(np.float64), oracle.bf16_round(X).astype(np.float64)
    y = oracle.mlp_forward(Pb, Xb)
    want_eps = np.maximum(0.0, np.exp(y[:, 0]) - 0.01) * 1.5
    np.testing.assert_allclose(host(eps), want_eps, rtol=2e-3, atol=1e-5)
    want_es = np.clip(np.rint(np.exp(y[:, 1])), 6, 20)
    near_half = np.abs(np.exp(y[:, 1]) - np.floor(np.exp(y[:, 1])) - 0.5) < 1e-3
    assert (host(es)[~near_half] == want_es[~near_half]).all()


@pytest.fixture(scope="module")
def graph(onng):
    X, Q = synth.workload("sift1m", n=8000, nq=300)
    nbr, ln = onng.build_knng(dev(X), 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    seeds = onng.seeds_pivot(dev(X), dev(Q), 512, 10)
    return X, Q, g, seeds


@pytest.mark.parametrize("h,eps", [(1, 0.0), (3, 0.05), (8, 0.0), (500, 0.1)])
def test_probe_features_match_oracle(onng, graph, h, eps):
    X, Q, g, seeds = graph
    idx = onng.Index(g[0], g[1], dev(X)).with_adjacency(20)
    f, st = onng.search_probe(idx, dev(Q), 10, 20, eps, seeds, h, 0.95)
    of, ost = oracle.search_probe(host(g[0]), host(g[1]), X, Q, 10, 20, np.float32(eps), host(seeds), h, 0.95)
    assert np.array_equal(host(st)[:, 0], ost[:, 0]) and np.array_equal(host(st)[:, 1], ost[:, 1])
    np.testing.assert_allclose(host(f), of, rtol=1e-5, atol=2e-6)


def test_per_query_parameters_match_oracle(onng, graph):
    X, Q, g, seeds = graph
    idx = onng.Index(g[0], g[1], dev(X)).with_adjacency(20)
    rng = np.random.default_rng(3)
    eq = rng.choice([0.0, 0.03, 0.1], size=len(Q)).astype(np.float32)
    es = rng.choice([6, 12, 20], size=len(Q)).astype(np.int32)
    ids, _, st = onng.search(idx, dev(Q), 10, 20, 0.0, seeds, eps_q=dev(eq), es_q=dev(es))
    for e in np.unique(eq):
        for s in np.unique(es):
            sel = np.nonzero((eq == e) & (es == s))[0]
            if len(sel) == 0:
                continue
            o_ids, _, o_st = oracle.search(host(g[0]), host(g[1]), X, Q[sel], 10, int(s), np.float32(e),
                                           host(seeds)[sel])
            assert np.array_equal(host(ids)[sel], o_ids)
            assert np.array_equal(host(st)[sel, 0], o_st[:, 0])


def test_labels_equal_oracle_labels(onng, graph):
    """Labels from the GPU sweep equal labels from the oracle's sweep (subset)."""
    from paper_1810_07355_gb300 import learned
    X, Q, g, seeds = graph
    idx = onng.Index(g[0], g[1], dev(X)).with_adjacency(20)
    gt, _ = onng.knn(dev(X), dev(Q), 10)
    eps_grid, es_grid = (0.0, 0.02, 0.1), (6, 12)
    rec, cost = learned.sweep(idx, dev(Q), gt, seeds, 10, eps_grid, es_grid)
    sub = np.arange(0, len(Q), 10)
    o_rec = np.empty((len(sub), len(es_grid), len(eps_grid)))
    o_cost = np.empty_like(o_rec)
    gt_h = host(gt)[sub]
    for a, s in enumerate(es_grid):
        for b, e in enumerate(eps_grid):
            o_ids, _, o_st = oracle.search(host(g[0]), host(g[1]), X, Q[sub], 10, s, np.float32(e), host(seeds)[sub])
            o_rec[:, a, b] = [len(set(r) & set(t)) / 10 for r, t in zip(o_ids, gt_h)]
            o_cost[:, a, b] = o_st[:, 0]
    for t in (0.9, 1.0):
        e1, s1 = learned.labels_from_sweep(rec[sub], cost[sub], t, eps_grid, es_grid)
        e2, s2 = learned.labels_from_sweep(torch.from_numpy(o_rec).float().cuda(),
                                           torch.from_numpy(o_cost).float().cuda(), t, eps_grid, es_grid)
        assert torch.equal(e1, e2) and torch.equal(s1, s2)


def test_learned_search_trains_and_runs(onng, graph):
    """The trained network fits its labels better than their mean, and the learned
    search returns valid, sorted results."""
    from paper_1810_07355_gb300 import learned
    X, Q, g, seeds = graph
    idx = onng.Index(g[0], g[1], dev(X)).with_adjacency(20)
    gt, _ = onng.knn(dev(X), dev(Q), 10)
    pred, (Xtr, Ttr) = learned.train(idx, dev(Q), gt, seeds, 10, steps=1500, batch=128)
    Y = onng.mlp_forward(pred.P, Xtr)
    mse = float(((Y - Ttr) ** 2).mean())
    base = float(((Ttr - Ttr.mean(0)) ** 2).mean())
    assert mse < base
    idx.with_bf16()
    ids, dist, st, eps_q, es_q = learned.learned_search(pred, idx, dev(Q), 10, seeds, 1.0, 1.0, k_rerank=20)
    d = host(dist)
    assert (np.diff(d, axis=1) >= 0).all() and (host(ids) >= 0).all()
    assert (host(es_q) >= 6).all() and (host(es_q) <= 20).all()


def test_learned_against_fixed_and_eq1_policies(onng):
    """What the trained network gains over the method without it, on held-out
    queries at a target mean recall of 0.9: distance computations per query
    (probe included) of the network's policy at each shrinkage beta, of one
    global eps (the fixed policy) and of the paper's Eq. 1 policy (e_s tied to
    eps by e_p = floor(10^(20 eps)) + 30, eps bisected).  Every reported policy
    reaches the target; the table is printed.  The network's choice is the
    cheapest of its rows; whether it beats the fixed policy is what the bench
    reports, not something this test assumes."""
    from scipy.stats import spearmanr

    from paper_1810_07355_gb300 import learned
    X, Q = synth.workload("sift1m", n=20000, nq=1200)
    nbr, ln = onng.build_knng(dev(X), 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    idx = onng.Index(g[0], g[1], dev(X)).with_adjacency(20)
    Qd = dev(Q)
    gt, _ = onng.knn(dev(X), Qd, 10)
    seeds = onng.seeds_pivot(dev(X), Qd, 512, 10)
    tr, ho = slice(0, 800), slice(800, 1200)
    target = 0.9
    pred, _ = learned.train(idx, Qd[tr], gt[tr], seeds[tr], 10, targets=(0.9, 1.0), h=4, steps=2000)
    best, ybar, table = learned.select_shrinkage(pred, idx, Qd[ho], gt[ho], seeds[ho], 10, target, 1.0,
                                                 es_options=(20,), precision=onng.PREC_FP32)
    fixed = [r for r in table if r["beta"] is None][0]
    net = [r for r in table if r["beta"] is not None and r["recall"] >= target - 1e-9]
    # Eq. 1 on the same held-out queries
    idx_csr = onng.Index(g[0], g[1], dev(X))

    def eq1_run(eps):
        ids, _, st = onng.search(idx_csr, Qd[ho], 10, learned.eq1_policy(eps), eps, seeds[ho])
        return float(learned.recall_per_query(ids, gt[ho]).mean()), float(st[:, 0].float().mean())
    lo, hi = 0.0, 0.2
    if eq1_run(lo)[0] >= target:
        hi = lo
    for _ in range(14):
        if hi == lo:
            break
        mid = 0.5 * (lo + hi)
        lo, hi = (lo, mid) if eq1_run(mid)[0] >= target else (mid, hi)
    eq1_rec, eq1_dc = eq1_run(hi)
    print("\npolicy                      dc/query  recall")
    for r in table:
        print(f"{'fixed eps' if r['beta'] is None else 'network beta=' + str(r['beta']):26s}  {r['dc']:8.1f}  "
              f"{r['recall']:.4f}")
    print(f"{'Eq. 1 (eps=%.4f, e_s=%d)' % (hi, learned.eq1_policy(hi)):26s}  {eq1_dc:8.1f}  {eq1_rec:.4f}")
    assert fixed["recall"] >= target - 1e-9 and eq1_rec >= target
    assert net, "no network setting reaches the target"
    assert best is not None and best["recall"] >= target - 1e-9
    # the network's own eps (beta = 1) against the held-out labels
    rec, cost = learned.sweep(idx, Qd[ho], gt[ho], seeds[ho], 10)
    eps_lab, _ = learned.labels_from_sweep(rec, cost, 1.0)
    feat, _ = onng.search_probe(idx, Qd[ho], 10, pred.probe_es, 0.0, seeds[ho], pred.h, 1.0)
    y = onng.mlp_forward(pred.P, feat)[:, 0]
    rho = spearmanr(host(y), host(eps_lab)).correlation
    print("held-out rank correlation of predicted and label eps:", round(float(rho), 3))
    assert np.isfinite(rho)
