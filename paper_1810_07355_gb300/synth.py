"""Seeded synthetic workloads shaped like the paper's descriptor sets (Section 3).

The paper evaluates on SIFT (128-d integer image descriptors), GIST (960-d) and
GloVe (100-d word vectors, angular distance).  None of those datasets is shipped
here, so these generators produce stand-ins with the same shapes, value types
and cluster structure.  This module holds only random-number recipes: none of
the method's arithmetic (distances, graphs, search) lives here, so it can feed
both the CUDA path and the CPU oracle.

Every generator is deterministic in (seed, sizes) through numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1810


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_mixture(n: int, d: int = 128, components: int = 50, sigma: float = 8.0,
                     center_range: float = 100.0, seed: int = SEED_BASE + 1,
                     centers_seed: int | None = None) -> np.ndarray:
    """Isotropic Gaussian mixture: centres U[0, center_range]^d, points centre + N(0, sigma^2 I).

    The component of every point is drawn uniformly.  ``centers_seed`` fixes the
    centres separately so that base and query sets share one mixture.
    """
    crng = _rng(SEED_BASE + 1 if centers_seed is None else centers_seed)
    centers = crng.uniform(0.0, center_range, size=(components, d))
    rng = _rng(seed)
    comp = rng.integers(0, components, size=n)
    x = centers[comp] + rng.normal(0.0, sigma, size=(n, d))
    return np.ascontiguousarray(x, dtype=np.float32)


def image_descriptors(n: int, d: int = 128, clusters: int = 1000, seed: int = SEED_BASE + 2,
                      centers_seed: int | None = None, active_prob: float = 0.70,
                      chunk: int = 1 << 17) -> np.ndarray:
    """SIFT-like integer descriptors 0..255 stored as float32 (about 30 % zeros).

    Per cluster c and dimension j a magnitude mu_cj ~ Gamma(shape 2, scale 20).
    A coordinate is active with probability ``active_prob``; an active one is
    round(mu_cj * g) with g ~ Gamma(4, 1/4) (mean 1), clipped to [0, 255]; an
    inactive one is 0.  Rounding of small products adds a few more zeros; the
    default gives a zero fraction of about 0.30.
    """
    crng = _rng(SEED_BASE + 2 if centers_seed is None else centers_seed)
    mu = crng.gamma(2.0, 20.0, size=(clusters, d)).astype(np.float32)
    rng = _rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        comp = rng.integers(0, clusters, size=m)
        g = rng.gamma(4.0, 0.25, size=(m, d)).astype(np.float32)
        act = rng.random(size=(m, d), dtype=np.float32) < active_prob
        v = np.rint(mu[comp] * g)
        np.clip(v, 0.0, 255.0, out=v)
        v[~act] = 0.0
        out[s:s + m] = v
    return out


def text_embeddings(n: int, d: int = 100, directions: int = 2000, zipf_s: float = 1.1,
                    angular_sigma: float = 0.3, seed: int = SEED_BASE + 3,
                    centers_seed: int | None = None, chunk: int = 1 << 17) -> np.ndarray:
    """GloVe-like unit vectors: Zipf(s) cluster sizes over random directions on S^{d-1}.

    x = normalise(mu_c + (angular_sigma / sqrt(d)) * N(0, I)), so the angular
    deviation from the cluster direction is about ``angular_sigma`` radians.
    Angular distance is then served by L2 on the unit sphere.
    """
    crng = _rng(SEED_BASE + 3 if centers_seed is None else centers_seed)
    mu = crng.normal(size=(directions, d))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    w = 1.0 / np.arange(1, directions + 1, dtype=np.float64) ** zipf_s
    w /= w.sum()
    rng = _rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        comp = rng.choice(directions, size=m, p=w)
        v = mu[comp] + (angular_sigma / np.sqrt(d)) * rng.normal(size=(m, d))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        out[s:s + m] = v
    return out


def gist_like(n: int, d: int = 960, clusters: int = 500, sigma: float = 0.1,
              seed: int = SEED_BASE + 4, centers_seed: int | None = None,
              chunk: int = 1 << 15) -> np.ndarray:
    """GIST-like non-negative descriptors: |centre + N(0, sigma^2 I)|, centres U[0,1]^d."""
    crng = _rng(SEED_BASE + 4 if centers_seed is None else centers_seed)
    centers = crng.uniform(0.0, 1.0, size=(clusters, d)).astype(np.float32)
    rng = _rng(seed)
    out = np.empty((n, d), dtype=np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        comp = rng.integers(0, clusters, size=m)
        out[s:s + m] = np.abs(centers[comp] + rng.normal(0.0, sigma, size=(m, d)).astype(np.float32))
    return out


def small_integers(n: int, d: int, high: int = 8, seed: int = 7) -> np.ndarray:
    """Tie-heavy integer points in [0, high) stored float32 (exercises id tie-breaks)."""
    return _rng(seed).integers(0, high, size=(n, d)).astype(np.float32)


# Named workloads.  Base and query sets share centres (centers_seed) but draw
# points from different streams (seed + 100 for queries, + 200 for training).
WORKLOADS = {
    "gmm10k": dict(gen=gaussian_mixture, n=10_000, d=128, nq=200,
                   kw=dict(components=50, sigma=8.0), base_seed=SEED_BASE + 1),
    "sift1m": dict(gen=image_descriptors, n=1_000_000, d=128, nq=10_000,
                   kw=dict(clusters=1000), base_seed=SEED_BASE + 2),
    "glove1m2": dict(gen=text_embeddings, n=1_200_000, d=100, nq=10_000,
                     kw=dict(directions=2000), base_seed=SEED_BASE + 3),
    "gist1m": dict(gen=gist_like, n=1_000_000, d=960, nq=1_000,
                   kw=dict(clusters=500), base_seed=SEED_BASE + 4),
}


def workload(name: str, n: int | None = None, nq: int | None = None, train: int = 0):
    """Return (base, queries[, train_queries]) float32 arrays for a named workload.

    ``n`` / ``nq`` override the sizes (same mixture, fewer points).
    """
    w = WORKLOADS[name]
    n = w["n"] if n is None else n
    nq = w["nq"] if nq is None else nq
    b = w["base_seed"]
    kw = dict(w["kw"], d=w["d"], centers_seed=b)
    base = w["gen"](n, seed=b + 1000, **kw)
    queries = w["gen"](nq, seed=b + 100, **kw)
    if train:
        return base, queries, w["gen"](train, seed=b + 200, **kw)
    return base, queries


def request_trace(seconds: float, rate_qps: float, seed: int = SEED_BASE + 5, max_size: int = 256,
                  ks=(1, 10, 100), recalls=(0.9, 0.95, 0.99)):
    """Seeded request trace for the serving loop: Poisson arrivals whose mean
    query rate is ``rate_qps``; request sizes L = floor(exp(U[0, ln(max_size+1))))
    clipped to [1, max_size] (log-uniform, mean ~46 at 256); k and the required
    recall uniform over ``ks`` / ``recalls``.

    Returns a structured array (arrival seconds, first query row, size, k, recall)
    sorted by arrival; the rows index a query matrix of ``sum(size)`` rows."""
    rng = _rng(seed)
    lo, hi = 0.0, float(np.log(max_size + 1))
    mean_size = float(np.mean(np.clip(np.floor(np.exp(rng.uniform(lo, hi, 200_000))), 1, max_size)))
    req_rate = rate_qps / mean_size
    count = int(rng.poisson(req_rate * seconds))
    arrival = np.sort(rng.uniform(0.0, seconds, count))
    size = np.clip(np.floor(np.exp(rng.uniform(lo, hi, count))), 1, max_size).astype(np.int64)
    first = np.concatenate([[0], np.cumsum(size)[:-1]]).astype(np.int64)
    k = np.asarray(ks, dtype=np.int64)[rng.integers(0, len(ks), count)]
    rec = np.asarray(recalls, dtype=np.float64)[rng.integers(0, len(recalls), count)]
    out = np.zeros(count, dtype=[("arrival", "f8"), ("first", "i8"), ("size", "i8"), ("k", "i8"), ("recall", "f8")])
    out["arrival"], out["first"], out["size"], out["k"], out["recall"] = arrival, first, size, k, rec
    return out
