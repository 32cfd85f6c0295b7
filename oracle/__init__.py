"""CPU FP64 oracle (test infrastructure only).

A plain C implementation of the paper's algorithms, compiled with gcc and called
through ctypes with numpy arrays.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg use it; the CUDA library never imports it and
shares no code with it.  See ``onng_oracle.c`` for the passage each function
follows and for the readings taken where the paper is silent.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, library routines (scipy's k-d tree, scipy.sparse
transposes), hand-built graphs and brute force; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "onng_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to the source (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            i64, i32, dbl, vp = C.c_int64, C.c_int, C.c_double, C.c_void_p
            lib.oracle_knn.argtypes = [vp, i64, i32, vp, i64, vp, i32, vp, vp, i32]
            lib.oracle_knn.restype = i32
            lib.oracle_adjust_degree.argtypes = [vp, vp, i64, i32, i32, i32, vp, i64, vp, vp, vp, i64]
            lib.oracle_adjust_degree.restype = i64
            lib.oracle_adjust_path.argtypes = [vp, vp, vp, i64, vp, i64, vp, vp, vp, i64, vp]
            lib.oracle_adjust_path.restype = i64
            lib.oracle_adjust_path_alg4.argtypes = [vp, vp, vp, i64, vp, vp, vp, i64]
            lib.oracle_adjust_path_alg4.restype = i64
            lib.oracle_seeds_random.argtypes = [C.c_uint64, i64, i64, i32, vp]
            lib.oracle_seeds_random.restype = i32
            lib.oracle_seeds_pivot.argtypes = [vp, i64, i32, vp, i64, i32, i32, vp, i32]
            lib.oracle_seeds_pivot.restype = i32
            lib.oracle_splitmix64.argtypes = [vp]
            lib.oracle_splitmix64.restype = C.c_uint64
            lib.oracle_hash_size.argtypes = [i64]
            lib.oracle_hash_size.restype = i64
            lib.oracle_hash_selftest.argtypes = [vp, i64, i64, vp]
            lib.oracle_hash_selftest.restype = i32
            lib.oracle_search.argtypes = [vp, vp, vp, i64, i32, vp, i64, i32, i32, dbl, vp, i32,
                                          vp, vp, vp, i32]
            lib.oracle_search.restype = i32
            lib.oracle_search_capped.argtypes = [vp, vp, vp, i64, i32, vp, i64, i32, i32, dbl, vp, i32, i64,
                                                 vp, vp, vp, i32]
            lib.oracle_search_capped.restype = i32
            lib.oracle_search_margin.argtypes = [vp, vp, vp, i64, i32, vp, i64, i32, i32, dbl, vp, i32,
                                                 vp, vp, vp, vp, i32]
            lib.oracle_search_margin.restype = i32
            lib.oracle_search_probe.argtypes = [vp, vp, vp, i64, i32, vp, i64, i32, i32, dbl, vp, i32,
                                                i64, dbl, vp, vp, i32]
            lib.oracle_search_probe.restype = i32
            lib.oracle_bf16_round.argtypes = [vp, i64, vp]
            lib.oracle_bf16_round.restype = None
            lib.oracle_adjust_degree_sac.argtypes = [vp, vp, i64, i32, i32, i32, vp, vp, vp, i64]
            lib.oracle_adjust_degree_sac.restype = i64
            lib.oracle_e4m3_encode.argtypes = [vp, i64, vp]
            lib.oracle_e4m3_encode.restype = None
            lib.oracle_e4m3_decode.argtypes = [vp, i64, vp]
            lib.oracle_e4m3_decode.restype = None
            lib.oracle_fp8_quantize.argtypes = [vp, i64, i32, vp, vp, vp]
            lib.oracle_fp8_quantize.restype = None
            lib.oracle_mlp_nparam.restype = i32
            lib.oracle_mlp_forward.argtypes = [vp, vp, i64, vp]
            lib.oracle_mlp_forward.restype = None
            lib.oracle_mlp_loss_grad.argtypes = [vp, vp, vp, i64, vp]
            lib.oracle_mlp_loss_grad.restype = dbl
            lib.oracle_adam_step.argtypes = [vp, vp, vp, vp, i64, i64, dbl, dbl, dbl, dbl]
            lib.oracle_adam_step.restype = None
            lib.oracle_graph_stats.argtypes = [vp, vp, vp, i64, vp]
            lib.oracle_graph_stats.restype = i32
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def knn(base, queries, k: int, self_ids=None, threads: int = 0):
    """Exact k nearest base points of every query row, (distance, id) order.

    Returns (ids int32 [nq,k], dist float64 [nq,k]); padded with -1 / inf.
    ``self_ids[r]`` (optional) is excluded from row r.
    """
    base = _c(base, np.float32)
    queries = _c(queries, np.float32)
    n, d = base.shape
    nq = queries.shape[0]
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float64)
    si = None if self_ids is None else _c(self_ids, np.int64)
    rc = _load().oracle_knn(_p(base), n, d, _p(queries), nq, None if si is None else _p(si),
                            k, _p(ids), _p(dist), threads)
    assert rc == 0, rc
    return ids, dist


def knng(X, k: int, rows=None, threads: int = 0):
    """Exact kNN graph of X (self excluded by id); optionally only ``rows``."""
    X = _c(X, np.float32)
    rows = np.arange(X.shape[0]) if rows is None else np.asarray(rows)
    return knn(X, X[rows], k, self_ids=rows, threads=threads)


def adjust_degree(nbr, length, e_o: int, e_i: int, rows=None):
    """Algorithm 2 (set form).  Returns CSR (ptr int64, col int32, len float64)."""
    nbr = _c(nbr, np.int32)
    length = _c(length, np.float64)
    n, k = nbr.shape
    nrows = n if rows is None else len(rows)
    r = None if rows is None else _c(rows, np.int64)
    cap = nrows * min(e_o, k) + int(n) * min(e_i, k) + 1
    ptr = np.empty(nrows + 1, np.int64)
    col = np.empty(cap, np.int32)
    ln = np.empty(cap, np.float64)
    m = _load().oracle_adjust_degree(_p(nbr), _p(length), n, k, e_o, e_i,
                                     None if r is None else _p(r), nrows, _p(ptr), _p(col), _p(ln), cap)
    assert m >= 0
    return ptr, col[:m].copy(), ln[:m].copy()


def adjust_degree_sac(nbr, length, e_o: int, e_i: int):
    """Algorithm 3 (degree adjustment with constraints).  CSR (ptr, col, len float64)."""
    nbr = _c(nbr, np.int32)
    length = _c(length, np.float64)
    n, k = nbr.shape
    cap = int(n) * (min(e_i, k) + min(e_o, k)) + 1
    ptr = np.empty(n + 1, np.int64)
    col = np.empty(cap, np.int32)
    ln = np.empty(cap, np.float64)
    m = _load().oracle_adjust_degree_sac(_p(nbr), _p(length), n, k, e_o, e_i, _p(ptr), _p(col), _p(ln), cap)
    assert m >= 0
    return ptr, col[:m].copy(), ln[:m].copy()


def adjust_path(ptr, col, length, rows=None, witnesses: bool = False):
    """Path adjustment (order-free reading).  Returns CSR (+ witness per input edge)."""
    ptr = _c(ptr, np.int64)
    col = _c(col, np.int32)
    length = _c(length, np.float64)
    n = ptr.shape[0] - 1
    nrows = n if rows is None else len(rows)
    r = None if rows is None else _c(rows, np.int64)
    if rows is None:
        cap = int(ptr[-1]) + 1
    else:
        cap = int(sum(ptr[i + 1] - ptr[i] for i in rows)) + 1
    optr = np.empty(nrows + 1, np.int64)
    ocol = np.empty(cap, np.int32)
    olen = np.empty(cap, np.float64)
    wit = np.empty(cap, np.int32) if witnesses else None
    m = _load().oracle_adjust_path(_p(ptr), _p(col), _p(length), n, None if r is None else _p(r), nrows,
                                   _p(optr), _p(ocol), _p(olen), cap, None if wit is None else _p(wit))
    assert m >= 0
    out = (optr, ocol[:m].copy(), olen[:m].copy())
    if witnesses:
        return out + (wit[:cap - 1].copy(),)
    return out


def adjust_path_alg4(ptr, col, length):
    """Algorithm 4 taken literally (reported variant, not the parity target)."""
    ptr = _c(ptr, np.int64)
    col = _c(col, np.int32)
    length = _c(length, np.float64)
    n = ptr.shape[0] - 1
    cap = int(ptr[-1]) + 1
    optr = np.empty(n + 1, np.int64)
    ocol = np.empty(cap, np.int32)
    olen = np.empty(cap, np.float64)
    m = _load().oracle_adjust_path_alg4(_p(ptr), _p(col), _p(length), n, _p(optr), _p(ocol), _p(olen), cap)
    assert m >= 0
    return optr, ocol[:m].copy(), olen[:m].copy()


def seeds_random(global_seed: int, nq: int, n: int, n_seed: int):
    """The random seed rule (SplitMix64 stream per query).  int32 [nq, n_seed]."""
    out = np.empty((nq, n_seed), np.int32)
    rc = _load().oracle_seeds_random(C.c_uint64(global_seed), nq, n, n_seed, _p(out))
    assert rc == 0
    return out


def seeds_pivot(X, Q, n_pivot: int, n_seed: int, threads: int = 0):
    """The pivot seed rule: the n_seed nearest of the pivots floor(t*n/P).  int32 [nq, n_seed]."""
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    out = np.empty((Q.shape[0], n_seed), np.int32)
    rc = _load().oracle_seeds_pivot(_p(X), X.shape[0], X.shape[1], _p(Q), Q.shape[0], n_pivot, n_seed,
                                    _p(out), threads)
    assert rc == 0
    return out


def splitmix64(state: int, count: int):
    """``count`` successive SplitMix64 outputs from ``state``."""
    st = np.array([state], dtype=np.uint64)
    return [int(_load().oracle_splitmix64(_p(st))) for _ in range(count)]


def hash_size(n: int) -> int:
    """Visited-table size s = 2^floor((floor(log2 n) + 11) / 2)."""
    return int(_load().oracle_hash_size(n))


def hash_selftest(ids, n: int):
    """Replays Set/IsSet over ``ids``: returns IsSet(i) before each Set(i)."""
    ids = _c(ids, np.int32)
    out = np.empty(ids.shape[0], np.uint8)
    assert _load().oracle_hash_selftest(_p(ids), ids.shape[0], n, _p(out)) == 0
    return out.astype(bool)


def search(ptr, col, X, Q, k: int, e_s: int, eps: float, seeds, threads: int = 0, margin: bool = False,
           max_exp: int = 0):
    """Algorithm 1 for every query.  Returns (ids int32, dist float64, stats int64 [nq,4]).

    With ``margin`` also returns, per query, the smallest relative gap of any
    comparison the run decided (float64 [nq]; inf when it compared nothing): a
    run whose margin exceeds another arithmetic's relative rounding error takes
    every decision the same way in that arithmetic."""
    ptr = _c(ptr, np.int64)
    col = _c(col, np.int32)
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    seeds = _c(seeds, np.int32)
    n, d = X.shape
    nq = Q.shape[0]
    ids = np.empty((nq, k), np.int32)
    dist = np.empty((nq, k), np.float64)
    stats = np.empty((nq, 4), np.int64)
    if margin:
        mg = np.empty(nq, np.float64)
        rc = _load().oracle_search_margin(_p(ptr), _p(col), _p(X), n, d, _p(Q), nq, k, e_s, float(eps),
                                          _p(seeds), seeds.shape[1], _p(ids), _p(dist), _p(stats), _p(mg),
                                          threads)
        assert rc == 0, rc
        return ids, dist, stats, mg
    if max_exp > 0:
        rc = _load().oracle_search_capped(_p(ptr), _p(col), _p(X), n, d, _p(Q), nq, k, e_s, float(eps),
                                          _p(seeds), seeds.shape[1], max_exp, _p(ids), _p(dist), _p(stats), threads)
        assert rc == 0, rc
        return ids, dist, stats
    rc = _load().oracle_search(_p(ptr), _p(col), _p(X), n, d, _p(Q), nq, k, e_s, float(eps),
                               _p(seeds), seeds.shape[1], _p(ids), _p(dist), _p(stats), threads)
    assert rc == 0, rc
    return ids, dist, stats


def search_probe(ptr, col, X, Q, k: int, e_s: int, eps: float, seeds, h: int, target: float, threads: int = 0):
    """Algorithm 1 stopped after h expansions; returns (features float64 [nq,16], stats int64 [nq,4])."""
    ptr = _c(ptr, np.int64)
    col = _c(col, np.int32)
    X = _c(X, np.float32)
    Q = _c(Q, np.float32)
    seeds = _c(seeds, np.int32)
    n, d = X.shape
    nq = Q.shape[0]
    feat = np.empty((nq, 16), np.float64)
    stats = np.empty((nq, 4), np.int64)
    rc = _load().oracle_search_probe(_p(ptr), _p(col), _p(X), n, d, _p(Q), nq, k, e_s, float(eps), _p(seeds),
                                     seeds.shape[1], h, float(target), _p(feat), _p(stats), threads)
    assert rc == 0, rc
    return feat, stats


def e4m3_encode(x):
    """FP8 e4m3 codes (uint8): nearest finite value, ties to even, saturating at 448."""
    x = _c(x, np.float32)
    y = np.empty(x.shape, dtype=np.uint8)
    _load().oracle_e4m3_encode(_p(x), x.size, _p(y))
    return y


def e4m3_decode(codes):
    """float32 values of FP8 e4m3 codes."""
    c = _c(codes, np.uint8)
    y = np.empty(c.shape, dtype=np.float32)
    _load().oracle_e4m3_decode(_p(c), c.size, _p(y))
    return y


def fp8_quantize(X):
    """(scale float32 [d], codes uint8 [n, d], dequantised float32 [n, d]) with
    c_j = max_i |x_ij| / 448 and code = e4m3(x_ij / c_j)."""
    X = _c(X, np.float32)
    n, d = X.shape
    scale = np.empty(d, dtype=np.float32)
    codes = np.empty((n, d), dtype=np.uint8)
    xq = np.empty((n, d), dtype=np.float32)
    _load().oracle_fp8_quantize(_p(X), n, d, _p(scale), _p(codes), _p(xq))
    return scale, codes, xq


def bf16_round(x):
    """bfloat16 round-to-nearest-even, returned as float32."""
    x = _c(x, np.float32)
    y = np.empty_like(x)
    _load().oracle_bf16_round(_p(x), x.size, _p(y))
    return y


MLP_NPARAM = 16 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2


def mlp_forward(P, x):
    P = _c(P, np.float64)
    x = _c(x, np.float64)
    y = np.empty((x.shape[0], 2), np.float64)
    _load().oracle_mlp_forward(_p(P), _p(x), x.shape[0], _p(y))
    return y


def mlp_loss_grad(P, x, t):
    P = _c(P, np.float64)
    x = _c(x, np.float64)
    t = _c(t, np.float64)
    G = np.empty(MLP_NPARAM, np.float64)
    loss = _load().oracle_mlp_loss_grad(_p(P), _p(x), _p(t), x.shape[0], _p(G))
    return loss, G


def adam_step(P, G, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays P, m, v."""
    _load().oracle_adam_step(_p(P), _p(_c(G, np.float64)), _p(m), _p(v), P.size, t, lr, beta1, beta2, eps)


GRAPH_STATS = ("mean_out", "top5_out", "bottom5_in", "in_dist10", "max_out", "max_in", "zero_in")


def graph_stats(ptr, col, length) -> dict:
    """Table 4's graph statistics of a CSR graph (keys: GRAPH_STATS)."""
    ptr = _c(ptr, np.int64)
    col = _c(col, np.int32)
    length = _c(length, np.float64)
    out = np.empty(7, np.float64)
    rc = _load().oracle_graph_stats(_p(ptr), _p(col), _p(length), ptr.shape[0] - 1, _p(out))
    assert rc == 0
    return dict(zip(GRAPH_STATS, out.tolist()))
