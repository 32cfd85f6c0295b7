"""Learned per-query (eps, e_s): labels, training and the three-kernel search.

The paper fixes the number of scanned edges as a function of eps (Eq. 1,
e_p = 10^(w_e eps) + e_0) and uses one eps for every query.  Here a small
network predicts, per query, the eps and e_s that reach a requested recall at
the fewest distance computations, from features of the query's first h hops:

  1. probe   - the search kernel stopped after h expansions writes 16 features
               (onng_search_probe),
  2. predict - the network, evaluated in bfloat16 (onng_mlp_predict), maps them
               to eps_q = max(0, exp(y0) - 0.01) * alpha and e_s,q,
  3. search  - the search kernel runs with the per-query eps_q / e_s,q.

Labels come from sweeps of the plain search over an (eps, e_s) grid.  On
integer-valued data the plain GPU search equals Algorithm 1 run in float64 bit
for bit (tested), so these labels are the ones the CPU oracle gives; a test
checks that on a subset.  Two label forms are provided:
  - per-query targets (what the benchmark trains on, t in {0.9, 1.0}): the
    cheapest cell whose recall@k reaches t.  Per-query recall@10 takes only the
    values 0, 0.1, ..., 1, so t = 0.95 and 0.99 both mean 10 of 10.  Feature 0
    of the network input is t; a mean recall such as 0.95 is then reached by
    calibrating the eps scale alpha (calibrate_alpha);
  - cost-aware (train's default when no targets are given): for a price lambda
    on a distance computation, the cell maximising recall_q - lambda * cost_q.
    Over a query set this is the allocation with the fewest distance
    computations for its mean recall, so a mean recall is reached by
    calibrating lambda alone (calibrate_lambda); easy queries then stop early
    and hopeless ones are not chased.  Feature 0 is log10(lambda).
Everything here except the three kernels is preparation (labels, calibration),
not the search path.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import onng

EPS_GRID = (0.0, 0.01, 0.02, 0.035, 0.05, 0.07, 0.1, 0.14, 0.2, 0.3)
ES_GRID = (8, 12, 16, 20)
EPS_FLOOR = 0.01
LAMBDAS = tuple(float(x) for x in np.logspace(-5.5, -3.0, 6))


def recall_per_query(ids: torch.Tensor, gt: torch.Tensor) -> torch.Tensor:
    hit = (ids[:, :, None] == gt[:, None, :]) & (gt[:, None, :] >= 0)
    return hit.any(2).sum(1).float() / gt.shape[1]


def sweep(index, Q, gt, seeds, k, eps_grid=EPS_GRID, es_grid=ES_GRID):
    """recall [nq, |es|, |eps|] and distance computations [nq, |es|, |eps|] of the plain search."""
    nq = Q.shape[0]
    rec = torch.empty((nq, len(es_grid), len(eps_grid)), device=Q.device)
    cost = torch.empty((nq, len(es_grid), len(eps_grid)), device=Q.device)
    for a, es in enumerate(es_grid):
        for b, eps in enumerate(eps_grid):
            ids, _, st = onng.search(index, Q, k, es, eps, seeds)
            rec[:, a, b] = recall_per_query(ids, gt)
            cost[:, a, b] = st[:, 0].float()
    return rec, cost


def labels_from_sweep(rec, cost, target, eps_grid=EPS_GRID, es_grid=ES_GRID):
    """Cheapest grid cell reaching `target` per query: (eps* [nq], e_s* [nq]).

    Queries that reach it nowhere get the most expensive cell (largest e_s, eps).
    """
    ok = rec >= target - 1e-6
    c = torch.where(ok, cost, torch.full_like(cost, float("inf")))
    flat = c.reshape(c.shape[0], -1)
    best = flat.argmin(1)
    none = ~ok.reshape(ok.shape[0], -1).any(1)
    best = torch.where(none, torch.full_like(best, flat.shape[1] - 1), best)
    es_i, eps_i = best // len(eps_grid), best % len(eps_grid)
    eps = torch.tensor(eps_grid, device=rec.device)[eps_i]
    es = torch.tensor(es_grid, device=rec.device, dtype=torch.float32)[es_i]
    return eps, es


def labels_lagrange(rec, cost, lam, eps_grid=EPS_GRID, es_grid=ES_GRID):
    """Per query, the grid cell maximising recall - lam * cost (ties: cheaper cell)."""
    score = rec - lam * cost - 1e-12 * cost
    best = score.reshape(score.shape[0], -1).argmax(1)
    es_i, eps_i = best // len(eps_grid), best % len(eps_grid)
    eps = torch.tensor(eps_grid, device=rec.device)[eps_i]
    es = torch.tensor(es_grid, device=rec.device, dtype=torch.float32)[es_i]
    return eps, es


@dataclass
class Predictor:
    """Trained network plus the settings it was trained with."""
    P: torch.Tensor
    h: int = 8
    probe_es: int = 20
    probe_eps: float = 0.0
    es_min: int = min(ES_GRID)
    es_max: int = max(ES_GRID)
    losses: list = field(default_factory=list)


def train(index, Qtr, gt, seeds, k, targets=None, h=8, steps=3000, batch=128, lr=2e-3, seed=0,
          sweep_result=None, lambdas=LAMBDAS):
    """Labels from the plain-search sweep, features from the probe, GPU training.

    The features are standardised for training (mean 0, variance 1 over the
    training set); the standardisation is then folded into the first layer
    (W1 / sigma, b1 - W1 mu / sigma), so the network takes raw probe features."""
    rec, cost = sweep_result if sweep_result is not None else sweep(index, Qtr, gt, seeds, k)
    feat, _ = onng.search_probe(index, Qtr, k, max(ES_GRID), 0.0, seeds, h, 0.0)
    X, T = [], []
    keys = [("t", t) for t in targets] if targets is not None else [("lam", l) for l in lambdas]
    for kind, v in keys:
        eps, es = labels_from_sweep(rec, cost, v) if kind == "t" else labels_lagrange(rec, cost, v)
        f = feat.clone()
        f[:, 0] = v if kind == "t" else float(np.log10(v))
        X.append(f)
        T.append(torch.stack([torch.log(eps + EPS_FLOOR), torch.log(es)], 1))
    X = torch.cat(X)
    T = torch.cat(T)
    g = torch.Generator(device="cpu").manual_seed(seed)
    perm = torch.randperm(X.shape[0], generator=g).to(X.device)
    X, T = X[perm].contiguous(), T[perm].contiguous()
    mu = X.mean(0)
    sd = X.std(0).clamp_min(1e-3)
    Xn = ((X - mu) / sd).contiguous()
    P = onng.mlp_init(seed, X.device)
    M = torch.zeros_like(P)
    V = torch.zeros_like(P)
    L = onng.mlp_train(P, M, V, Xn, T, steps, batch, lr, losses=True)
    W1 = P[:16 * 64].view(64, 16)
    b1 = P[16 * 64:16 * 64 + 64]
    b1 -= (W1 * (mu / sd)).sum(1)
    W1 /= sd
    return Predictor(P, h=h, probe_es=max(ES_GRID), losses=L.cpu().tolist()), (X, T)


def learned_search(pred: Predictor, index, Q, k, seeds, target, alpha=1.0, precision=onng.PREC_BF16, k_rerank=0,
                   out=None):
    """probe -> bfloat16 predictor -> search with per-query (eps, e_s)."""
    feat, _ = onng.search_probe(index, Q, k, pred.probe_es, pred.probe_eps, seeds, pred.h, target)
    eps_q, es_q = onng.mlp_predict(pred.P, feat, alpha, pred.es_min, pred.es_max)
    ids, dist, st = onng.search(index, Q, k, pred.es_max, 0.0, seeds, precision=precision, k_rerank=k_rerank,
                                eps_q=eps_q, es_q=es_q, out=out)
    return ids, dist, st, eps_q, es_q


_OW3, _OB3 = 16 * 64 + 64 + 64 * 64 + 64, 16 * 64 + 64 + 64 * 64 + 64 + 2 * 64


def shrink(pred: Predictor, beta: float, ybar: float, es_fixed: int | None = None) -> Predictor:
    """The network with its eps output pulled toward the constant ybar:
    y0' = ybar + beta (y0 - ybar), folded into the last layer (W3[0] *= beta,
    b3[0] = beta b3[0] + (1 - beta) ybar).  beta = 0 is one eps for every query
    (the fixed policy, scaled by alpha); beta = 1 is the network as trained.
    es_fixed, if given, pins e_s for every query."""
    P = pred.P.clone()
    P[_OW3:_OW3 + 64] *= beta
    P[_OB3] = beta * P[_OB3] + (1.0 - beta) * ybar
    lo, hi = (es_fixed, es_fixed) if es_fixed is not None else (pred.es_min, pred.es_max)
    return Predictor(P, h=pred.h, probe_es=pred.probe_es, probe_eps=pred.probe_eps, es_min=lo, es_max=hi,
                     losses=pred.losses)


def select_shrinkage(pred, index, Q, gt, seeds, k, target_recall, t, betas=(0.0, 0.25, 0.5, 0.75, 1.0),
                     es_options=(None,), **kw):
    """On a held-out query set, for each (beta, e_s option): calibrate alpha to the
    target mean recall and count distance computations per query, of the search
    and of the probe.  Rows that miss the target (alpha at its upper bound) are
    kept in the table but never chosen.  beta = 0 without the probe is the fixed
    policy (one eps for all queries); it is the row {"beta": None}.

    Returns (best row, ybar, table); best["beta"] is None when the fixed policy
    is cheapest."""
    feat, _ = onng.search_probe(index, Q, k, pred.probe_es, pred.probe_eps, seeds, pred.h, t)
    ybar = float(onng.mlp_forward(pred.P, feat)[:, 0].mean())
    table = []
    for es_fixed in es_options:
        for beta in betas:
            pb = shrink(pred, beta, ybar, es_fixed)
            alpha = calibrate_alpha(pb, index, Q, gt, seeds, k, target_recall, t, **kw)
            ids, _, st, _, _ = learned_search(pb, index, Q, k, seeds, t, alpha, **kw)
            _, pst = onng.search_probe(index, Q, k, pb.probe_es, pb.probe_eps, seeds, pb.h, t)
            row = {"beta": beta, "es_fixed": es_fixed, "alpha": alpha, "recall": float(recall_per_query(ids, gt).mean()),
                   "dc_search": float(st[:, 0].float().mean()), "dc_probe": float(pst[:, 0].float().mean())}
            row["dc"] = row["dc_search"] + row["dc_probe"]
            table.append(row)
            if beta == 0.0 and es_fixed is not None:
                table.append(dict(row, beta=None, dc_probe=0.0, dc=row["dc_search"]))
    ok = [r for r in table if r["recall"] >= target_recall - 1e-9]
    best = min(ok, key=lambda r: r["dc"]) if ok else None
    return best, ybar, table


def calibrate_lambda(pred, index, Q, gt, seeds, k, target_recall, lo=-7.0, hi=-2.0, iters=12, **kw):
    """Largest price lambda (bisection on log10 lambda) whose mean recall@k reaches
    target_recall; returns the feature value log10(lambda)."""
    def rec(l10):
        ids = learned_search(pred, index, Q, k, seeds, l10, 1.0, **kw)[0]
        return float(recall_per_query(ids, gt).mean())
    if rec(lo) < target_recall:
        return lo
    if rec(hi) >= target_recall:
        return hi
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if rec(mid) >= target_recall:
            lo = mid
        else:
            hi = mid
    return lo


def calibrate_alpha(pred, index, Q, gt, seeds, k, target_recall, t, lo=0.05, hi=8.0, iters=14, **kw):
    """Smallest alpha (bisection, log scale) whose mean recall@k reaches target_recall."""
    def rec(al):
        ids = learned_search(pred, index, Q, k, seeds, t, al, **kw)[0]
        return float(recall_per_query(ids, gt).mean())
    if rec(hi) < target_recall:
        return hi
    if rec(lo) >= target_recall:
        return lo
    for _ in range(iters):
        mid = float(np.sqrt(lo * hi))
        if rec(mid) >= target_recall:
            hi = mid
        else:
            lo = mid
    return hi


def eq1_policy(eps: float, e0: int = 30, we: float = 20.0) -> int:
    """Eq. 1 of the paper, e_p = 10^(w_e eps) + e_0, rounded down (the paper is silent)."""
    return int(np.floor(10.0 ** (we * eps))) + e0
