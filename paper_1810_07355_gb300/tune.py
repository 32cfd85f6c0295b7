"""Choosing the expected degrees (e_o, e_i) by the loss of Eq. 2 and hill climbing.

The paper scores a degree-adjusted graph by the mean log10 number of distance
computations over a target precision range [p_l, p_u] (Eq. 2),

    L(e_o, e_i, p_l, p_u) = integral_{p_l}^{p_u} log10 C(e_o, e_i, x) dx / (p_u - p_l),

where C(e_o, e_i, p) is the mean number of distance computations per query at
precision p (precision = recall@k here: the search returns k results).  The
integral is estimated from searches (Sec. 2.6): a binary search on eps finds eps_l
with precision in (p_l - 0.005, p_l] and eps_u with precision in [p_u, p_u + 0.005);
[eps_l, eps_u] is cut into 9 equal parts, the 10 eps values are searched, and the
trapezoidal rule integrates log10 C over the measured precisions.  Since L is
convex in (e_o, e_i) (the paper's Fig. 3(b)), a hill climb with a step of 5 edges (Sec. 3)
finds the minimum.

Readings (the paper is silent or garbled): the upper bracket is read as
[p_u, p_u + 0.005) (the text prints p_l + 0.005 there); the piecewise-linear
interpolant of the 10 (precision, log10 C) samples, sorted by precision, is
integrated over exactly [p_l, p_u]; the climb moves to the best of the four
neighbours (e_o +- step, e_i +- step) while that lowers L, within the given bounds.

The arithmetic here (the integral, the climb) is host-side bookkeeping over the
library's kernels: every graph and every search runs on the GPU.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def eq2_loss(precisions, costs, p_l: float, p_u: float) -> float:
    """Eq. 2 from samples: the mean over [p_l, p_u] of the piecewise-linear
    interpolant of log10(cost) against precision (samples sorted by precision;
    the interpolant is held constant beyond the sampled range)."""
    if not p_u > p_l:
        raise ValueError("need p_u > p_l")
    p = np.asarray(precisions, dtype=np.float64)
    y = np.log10(np.asarray(costs, dtype=np.float64))
    if p.size < 2:
        raise ValueError("need at least two samples")
    o = np.argsort(p, kind="stable")
    p, y = p[o], y[o]
    # merge equal precisions (their mean cost), so the interpolant is a function
    up, inv = np.unique(p, return_inverse=True)
    uy = np.bincount(inv, weights=y) / np.bincount(inv)
    knots = np.concatenate([[p_l], up[(up > p_l) & (up < p_u)], [p_u]])
    vals = np.interp(knots, up, uy)
    area = float(np.sum(0.5 * (vals[1:] + vals[:-1]) * np.diff(knots)))  # trapezoidal rule
    return area / (p_u - p_l)


def bracket_eps(precision_at, target: float, side: str, lo: float = 0.0, hi: float = 1.0, tol: float = 0.005,
                iters: int = 40):
    """Binary search for an eps whose precision lies in (target - tol, target]
    (side "low") or in [target, target + tol) (side "high"); precision_at(eps)
    is non-decreasing in eps.  Returns (eps, precision); the closest eps found
    if the window is never hit."""
    p_hi = precision_at(hi)
    while p_hi < target and hi < 64.0:
        lo, hi = hi, hi * 2.0
        p_hi = precision_at(hi)
    best = None
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        p = precision_at(mid)
        inside = (target - tol < p <= target) if side == "low" else (target <= p < target + tol)
        if inside:
            return mid, p
        if best is None or abs(p - target) < abs(best[1] - target):
            best = (mid, p)
        if p < target or (side == "low" and p == target):
            lo = mid
        else:
            hi = mid
    return best


def loss_of_search(run, p_l: float, p_u: float, samples: int = 10):
    """Eq. 2 for one graph.  run(eps) -> (precision, mean distance computations)."""
    e_l, _ = bracket_eps(lambda e: run(e)[0], p_l, "low")
    e_u, _ = bracket_eps(lambda e: run(e)[0], p_u, "high", lo=e_l)
    eps = np.linspace(e_l, e_u, samples)
    pc = [run(float(e)) for e in eps]
    return eq2_loss([a for a, _ in pc], [b for _, b in pc], p_l, p_u), list(zip(eps.tolist(), pc))


@dataclass
class Climb:
    best: tuple
    loss: float
    path: list = field(default_factory=list)     # (e_o, e_i, loss) of each accepted point
    evaluated: dict = field(default_factory=dict)


def hill_climb(loss_fn, start, step: int = 5, lo=(0, 0), hi=(10 ** 9, 10 ** 9), max_moves: int = 100) -> Climb:
    """Steepest-descent hill climb over integer (e_o, e_i) on a grid of `step`."""
    cache = {}

    def f(x):
        if x not in cache:
            cache[x] = float(loss_fn(*x))
        return cache[x]

    cur = (int(start[0]), int(start[1]))
    cur_l = f(cur)
    path = [(cur[0], cur[1], cur_l)]
    for _ in range(max_moves):
        nbrs = [(cur[0] + dx, cur[1] + dy) for dx, dy in ((step, 0), (-step, 0), (0, step), (0, -step))]
        nbrs = [x for x in nbrs if lo[0] <= x[0] <= hi[0] and lo[1] <= x[1] <= hi[1] and x != (0, 0)]
        if not nbrs:
            break
        cand = min(nbrs, key=lambda x: (f(x), x))
        if f(cand) >= cur_l:
            break
        cur, cur_l = cand, f(cand)
        path.append((cur[0], cur[1], cur_l))
    return Climb(cur, cur_l, path, dict(cache))


def graph_loss(onng, knn, X, Q, gt, seeds, k: int, e_o: int, e_i: int, p_l: float, p_u: float, e_s: int = 0,
               path: bool = True):
    """Eq. 2 of the graph built from the kNN lists `knn` = (nbr, len) with
    (e_o, e_i) (degree adjustment, then path adjustment unless path=False),
    searched with Q against ground truth gt (recall@k as precision)."""
    import torch
    nbr, ln = knn
    g = onng.adjust_degree(nbr, ln, e_o, e_i)
    if path:
        g = onng.adjust_path(*g)
    idx = onng.Index(g[0], g[1], X)
    valid = gt >= 0

    def run(eps):
        ids, _, st = onng.search(idx, Q, k, e_s, eps, seeds)
        hit = (ids[:, :, None] == gt[:, None, :]) & valid[:, None, :]
        prec = float(hit.any(2).sum(1).float().mean() / k)
        return prec, float(st[:, 0].double().mean())
    with torch.no_grad():
        return loss_of_search(run, p_l, p_u)


def optimize_degrees(onng, X, Q, k: int, knn_k: int, start=(20, 60), p_l: float = 0.90, p_u: float = 0.98,
                     step: int = 5, e_s: int = 0, n_pivot: int = 1024, n_seed: int = 10, path: bool = True,
                     max_moves: int = 100):
    """The paper's degree optimisation on the GPU: the exact kNN graph once, then
    a hill climb over (e_o, e_i) in [0, knn_k] scored by Eq. 2 on queries Q."""
    nbr, ln = onng.build_knng(X, knn_k)
    gt, _ = onng.knn(X, Q, k)
    seeds = onng.seeds_pivot(X, Q, n_pivot, n_seed)
    return hill_climb(lambda eo, ei: graph_loss(onng, (nbr, ln), X, Q, gt, seeds, k, eo, ei, p_l, p_u, e_s, path)[0],
                      start, step=step, lo=(0, 0), hi=(knn_k, knn_k), max_moves=max_moves)


__all__ = ["eq2_loss", "bracket_eps", "loss_of_search", "hill_climb", "graph_loss", "optimize_degrees", "Climb"]
