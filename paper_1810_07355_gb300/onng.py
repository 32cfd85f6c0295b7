"""Python binding of the onng C ABI (``include/onng.h``).

Argument marshalling only: every step runs in ``libonng.so``'s CUDA kernels.
Tensors are torch CUDA tensors; the current torch stream is passed to every call.
If the library cannot be loaded the calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading
from dataclasses import dataclass

import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

ONNG_OK, ONNG_E_INVAL, ONNG_E_WORKSPACE, ONNG_E_CUDA, ONNG_E_LIMIT, ONNG_E_UNSUPPORTED, ONNG_E_AGAIN = range(7)
FLAG_S_OVERFLOW, FLAG_VISIT_OVERFLOW, FLAG_LIMIT, FLAG_CHECK = 1, 2, 4, 8
PREC_FP32, PREC_BF16, PREC_FP8 = 0, 1, 2


class OnngError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"onng status {status}: {msg}")
        self.status = status


class _Index(C.Structure):
    _fields_ = [("row_ptr", C.c_void_p), ("col", C.c_void_p), ("X", C.c_void_p), ("X_bf16", C.c_void_p),
                ("adj", C.c_void_p), ("n", C.c_int64), ("d", C.c_int32), ("adj_width", C.c_int32),
                ("X_fp8", C.c_void_p), ("fp8_scale", C.c_void_p)]


class _GraphStats(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("max_out", C.c_int64), ("max_in", C.c_int64),
                ("zero_in", C.c_int64), ("mean_out", C.c_double), ("top5_out", C.c_double),
                ("bottom5_in", C.c_double), ("in_dist10", C.c_double)]


class _ServeConfig(C.Structure):
    _fields_ = [("precision", C.c_int32), ("k_rerank", C.c_int32), ("n_pivot", C.c_int32), ("n_seed", C.c_int32),
                ("max_queries", C.c_int32), ("k_max", C.c_int32), ("slots", C.c_int32), ("timeout_ms", C.c_int32)]


class _Params(C.Structure):
    _fields_ = [("k", C.c_int32), ("e_s", C.c_int32), ("eps", C.c_float), ("precision", C.c_int32),
                ("k_rerank", C.c_int32), ("max_expansions", C.c_int32), ("pool_cap", C.c_int32)]


def library_path() -> str:
    """The library this process loads: ``libonng.so``, or the one the
    ONNG_LIBRARY environment variable names (e.g. the bounds-checked build)."""
    return os.environ.get("ONNG_LIBRARY") or _build.LIB


def load(build_if_missing: bool = True):
    """Loads (building first if needed) ``libonng.so`` and declares its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if build_if_missing and path == _build.LIB:
            _build.build()
        elif build_if_missing and os.path.abspath(path) == _build.LIB_CHECK:
            _build.build_checked()
        if not os.path.exists(path):
            raise RuntimeError(f"onng CUDA library not found at {path}")
        lib = C.CDLL(path)
        i32, i64, u64, sz, vp, f32 = C.c_int32, C.c_int64, C.c_uint64, C.c_size_t, C.c_void_p, C.c_float
        sig = {
            "onng_last_error": ([], C.c_char_p),
            "onng_version": ([], C.c_int),
            "onng_knn_workspace_bytes": ([i64, i32, i64, i32], sz),
            "onng_knn": ([vp, i64, i32, vp, i64, i32, i64, vp, vp, vp, sz, vp], C.c_int),
            "onng_build_knng": ([vp, i64, i32, i32, vp, vp, vp, sz, vp], C.c_int),
            "onng_adjust_degree_workspace_bytes": ([i64, i32], sz),
            "onng_adjust_degree_count": ([vp, vp, i64, i32, i32, i32, vp, vp, vp, sz, vp], C.c_int),
            "onng_adjust_degree": ([vp, vp, i64, i32, i32, i32, vp, vp, vp, vp, sz, vp], C.c_int),
            "onng_adjust_degree_sac_workspace_bytes": ([i64, i32], sz),
            "onng_adjust_degree_sac_count": ([vp, vp, i64, i32, i32, i32, vp, vp, vp, sz, vp], C.c_int),
            "onng_adjust_degree_sac": ([vp, vp, i64, i32, i32, i32, vp, vp, vp, vp, sz, vp], C.c_int),
            "onng_adjust_path_workspace_bytes": ([i64, i64], sz),
            "onng_adjust_path_literal_workspace_bytes": ([i64, i64], sz),
            "onng_adjust_path_literal": ([vp, vp, vp, i64, vp, vp, vp, vp, vp, sz, vp], C.c_int),
            "onng_adjust_path": ([vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, sz, vp], C.c_int),
            "onng_seeds_random": ([u64, i64, i64, i32, vp, vp], C.c_int),
            "onng_seeds_pivot_workspace_bytes": ([i64, i32, i32], sz),
            "onng_seeds_pivot": ([vp, i64, i32, vp, i64, i32, i32, vp, vp, sz, vp], C.c_int),
            "onng_search_workspace_bytes": ([i64, C.POINTER(_Index), C.POINTER(_Params)], sz),
            "onng_search": ([C.POINTER(_Index), vp, i64, C.POINTER(_Params), vp, i32, vp, vp, vp, vp, vp, vp, sz, vp],
                            C.c_int),
            "onng_to_bf16": ([vp, i64, vp, vp], C.c_int),
            "onng_to_fp8": ([vp, i64, i32, vp, vp, vp], C.c_int),
            "onng_pad_adjacency": ([vp, vp, i64, i32, vp, vp], C.c_int),
            "onng_search_probe": ([C.POINTER(_Index), vp, i64, C.POINTER(_Params), vp, i32, f32, vp, vp, vp, sz, vp],
                                  C.c_int),
            "onng_search_noalloc": ([C.POINTER(_Index), vp, i64, C.POINTER(_Params), vp, i32, vp, vp, vp, vp, vp, vp],
                                    C.c_int),
            "onng_mlp_nparam": ([], C.c_int),
            "onng_mlp_forward": ([vp, vp, i64, vp, vp], C.c_int),
            "onng_mlp_loss_grad": ([vp, vp, vp, i64, vp, vp, vp], C.c_int),
            "onng_mlp_adam": ([vp, vp, vp, vp, i64, f32, f32, f32, f32, vp], C.c_int),
            "onng_mlp_train": ([vp, vp, vp, vp, vp, i64, i32, i64, i64, f32, vp, vp, vp], C.c_int),
            "onng_mlp_predict": ([vp, vp, i64, f32, i32, i32, vp, vp, vp], C.c_int),
            "onng_graph_stats_workspace_bytes": ([i64, i64], sz),
            "onng_graph_stats": ([vp, vp, vp, i64, C.POINTER(_GraphStats), vp, sz, vp], C.c_int),
            "onng_index_save": ([C.c_char_p, vp, vp, vp, vp, i64, i32, vp], C.c_int),
            "onng_index_check": ([C.c_char_p, vp, vp, vp, vp], C.c_int),
            "onng_index_load": ([C.c_char_p, i64, i32, i64, vp, vp, vp, vp, vp], C.c_int),
            "onng_crc32": ([C.c_uint32, vp, sz], C.c_uint32),
            "onng_serve_create": ([C.POINTER(_Index), C.POINTER(_ServeConfig), C.POINTER(vp)], C.c_int),
            "onng_serve_submit": ([vp, vp, i32, i32, f32, i32, C.POINTER(C.c_uint64)], C.c_int),
            "onng_serve_poll": ([vp, C.c_uint64, vp, vp, i32], C.c_int),
            "onng_serve_destroy": ([vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def exported_symbols():
    """Names of the entry points declared in the header."""
    return [
        "onng_last_error", "onng_version", "onng_knn_workspace_bytes", "onng_knn", "onng_build_knng",
        "onng_adjust_degree_workspace_bytes", "onng_adjust_degree_count", "onng_adjust_degree",
        "onng_adjust_path_workspace_bytes", "onng_adjust_path", "onng_seeds_random",
        "onng_seeds_pivot_workspace_bytes", "onng_seeds_pivot", "onng_search_workspace_bytes", "onng_search",
        "onng_to_bf16", "onng_pad_adjacency", "onng_search_probe", "onng_mlp_nparam", "onng_mlp_forward",
        "onng_mlp_loss_grad", "onng_mlp_adam", "onng_mlp_train", "onng_mlp_predict", "onng_search_noalloc", "onng_to_fp8",
        "onng_adjust_degree_sac_workspace_bytes", "onng_adjust_degree_sac_count", "onng_adjust_degree_sac",
        "onng_adjust_path_literal_workspace_bytes", "onng_adjust_path_literal",
        "onng_graph_stats_workspace_bytes", "onng_graph_stats", "onng_index_save", "onng_index_check",
        "onng_index_load", "onng_crc32", "onng_serve_create", "onng_serve_submit", "onng_serve_poll",
        "onng_serve_destroy",
    ]


def _check(status: int):
    if status != ONNG_OK:
        raise OnngError(status, load().onng_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ws(nbytes: int, device):
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def _dev(t: torch.Tensor, dtype) -> torch.Tensor:
    if not t.is_cuda:
        raise ValueError("onng expects CUDA tensors")
    return t.to(dtype).contiguous()


# ----------------------------------------------------------------------------- kNN graph

def knn(X: torch.Tensor, Q: torch.Tensor, k: int, self_offset: int = -1):
    """Exact k nearest rows of X for every row of Q: (ids int32 [nq,k], lengths float32 [nq,k])."""
    X = _dev(X, torch.float32)
    Q = _dev(Q, torch.float32)
    n, d = X.shape
    nq = Q.shape[0]
    lib = load()
    nbr = torch.empty((nq, k), dtype=torch.int32, device=X.device)
    ln = torch.empty((nq, k), dtype=torch.float32, device=X.device)
    ws = _ws(lib.onng_knn_workspace_bytes(n, d, nq, k), X.device)
    _check(lib.onng_knn(_ptr(X), n, d, _ptr(Q), nq, k, self_offset, _ptr(nbr), _ptr(ln), _ptr(ws), ws.numel(),
                        _stream()))
    return nbr, ln


def build_knng(X: torch.Tensor, k: int):
    """Exact kNN graph of X (self excluded): (nbr int32 [n,k], len float32 [n,k])."""
    X = _dev(X, torch.float32)
    n, d = X.shape
    lib = load()
    nbr = torch.empty((n, k), dtype=torch.int32, device=X.device)
    ln = torch.empty((n, k), dtype=torch.float32, device=X.device)
    ws = _ws(lib.onng_knn_workspace_bytes(n, d, n, k), X.device)
    _check(lib.onng_build_knng(_ptr(X), n, d, k, _ptr(nbr), _ptr(ln), _ptr(ws), ws.numel(), _stream()))
    return nbr, ln


# ----------------------------------------------------------------------------- adjustment

def adjust_degree(nbr: torch.Tensor, length: torch.Tensor, e_o: int, e_i: int):
    """Algorithm 2 (set form) on the GPU: CSR (row_ptr int64, col int32, len float32)."""
    nbr = _dev(nbr, torch.int32)
    length = _dev(length, torch.float32)
    n, k = nbr.shape
    lib = load()
    dev = nbr.device
    ws = _ws(lib.onng_adjust_degree_workspace_bytes(n, k), dev)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(0)
    _check(lib.onng_adjust_degree_count(_ptr(nbr), _ptr(length), n, k, e_o, e_i, _ptr(row_ptr), C.byref(nnz),
                                        _ptr(ws), ws.numel(), _stream()))
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    ln = torch.empty(max(nnz.value, 1), dtype=torch.float32, device=dev)
    _check(lib.onng_adjust_degree(_ptr(nbr), _ptr(length), n, k, e_o, e_i, _ptr(row_ptr), _ptr(col), _ptr(ln),
                                  _ptr(ws), ws.numel(), _stream()))
    return row_ptr, col[:nnz.value], ln[:nnz.value]


def adjust_degree_sac(nbr: torch.Tensor, length: torch.Tensor, e_o: int, e_i: int):
    """Algorithm 3 (degree adjustment with constraints) on the GPU: CSR (row_ptr int64, col int32, len float32)."""
    nbr = _dev(nbr, torch.int32)
    length = _dev(length, torch.float32)
    n, k = nbr.shape
    lib = load()
    dev = nbr.device
    ws = _ws(lib.onng_adjust_degree_sac_workspace_bytes(n, k), dev)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
    nnz = C.c_int64(0)
    _check(lib.onng_adjust_degree_sac_count(_ptr(nbr), _ptr(length), n, k, e_o, e_i, _ptr(row_ptr), C.byref(nnz),
                                            _ptr(ws), ws.numel(), _stream()))
    col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device=dev)
    ln = torch.empty(max(nnz.value, 1), dtype=torch.float32, device=dev)
    _check(lib.onng_adjust_degree_sac(_ptr(nbr), _ptr(length), n, k, e_o, e_i, _ptr(row_ptr), _ptr(col), _ptr(ln),
                                      _ptr(ws), ws.numel(), _stream()))
    return row_ptr, col[:nnz.value], ln[:nnz.value]


def adjust_path(row_ptr: torch.Tensor, col: torch.Tensor, length: torch.Tensor, witnesses: bool = False):
    """Order-free path adjustment on the GPU: CSR (+ witness node per input edge, -1 if kept)."""
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    length = _dev(length, torch.float32)
    n = row_ptr.numel() - 1
    m = col.numel()
    lib = load()
    dev = row_ptr.device
    ws = _ws(lib.onng_adjust_path_workspace_bytes(n, m), dev)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    oc = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    ol = torch.empty(max(m, 1), dtype=torch.float32, device=dev)
    wit = torch.empty(max(m, 1), dtype=torch.int32, device=dev) if witnesses else None
    nnz = C.c_int64(0)
    _check(lib.onng_adjust_path(_ptr(row_ptr), _ptr(col), _ptr(length), n, _ptr(rp), _ptr(oc), _ptr(ol),
                                C.byref(nnz), _ptr(wit), _ptr(ws), ws.numel(), _stream()))
    out = (rp, oc[:nnz.value], ol[:nnz.value])
    return out + (wit[:m],) if witnesses else out


def adjust_path_literal(row_ptr: torch.Tensor, col: torch.Tensor, length: torch.Tensor):
    """Algorithm 4 taken literally (rounds over the partial output, ascending ids
    inside a round) on the GPU: CSR (row_ptr int64, col int32, len float32)."""
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    length = _dev(length, torch.float32)
    n = row_ptr.numel() - 1
    m = col.numel()
    lib = load()
    dev = row_ptr.device
    ws = _ws(lib.onng_adjust_path_literal_workspace_bytes(n, m), dev)
    rp = torch.empty(n + 1, dtype=torch.int64, device=dev)
    oc = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    ol = torch.empty(max(m, 1), dtype=torch.float32, device=dev)
    nnz = C.c_int64(0)
    _check(lib.onng_adjust_path_literal(_ptr(row_ptr), _ptr(col), _ptr(length), n, _ptr(rp), _ptr(oc), _ptr(ol),
                                        C.byref(nnz), _ptr(ws), ws.numel(), _stream()))
    return rp, oc[:nnz.value], ol[:nnz.value]


def graph_stats(row_ptr: torch.Tensor, col: torch.Tensor, length: torch.Tensor) -> dict:
    """Table 4's graph statistics (top-5 % outdegree, bottom-5 % indegree, mean
    indegree distance over the 10 shortest incoming edges) and the degree extremes."""
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    length = _dev(length, torch.float32)
    n = row_ptr.numel() - 1
    lib = load()
    ws = _ws(lib.onng_graph_stats_workspace_bytes(n, col.numel()), row_ptr.device)
    out = _GraphStats()
    _check(lib.onng_graph_stats(_ptr(row_ptr), _ptr(col), _ptr(length), n, C.byref(out), _ptr(ws), ws.numel(),
                                _stream()))
    return {name: getattr(out, name) for name, _ in _GraphStats._fields_}


# ----------------------------------------------------------------------------- index files

def crc32(data: bytes, crc: int = 0) -> int:
    """The CRC-32 the index files carry (reflected, polynomial 0xEDB88320)."""
    buf = C.create_string_buffer(bytes(data), len(data))
    return int(load().onng_crc32(crc, C.cast(buf, C.c_void_p), len(data)))


def index_check(path: str) -> dict:
    """Header fields of an index file after a full size and CRC check (host only)."""
    n, d, nnz, has_len = C.c_int64(0), C.c_int32(0), C.c_int64(0), C.c_int32(0)
    _check(load().onng_index_check(os.fsencode(path), C.byref(n), C.byref(d), C.byref(nnz), C.byref(has_len)))
    return {"n": n.value, "d": d.value, "nnz": nnz.value, "has_len": bool(has_len.value)}


def save_index(index: "Index", path: str):
    """Writes the graph (with its lengths when the index has them) and the float32
    vectors; the reduced-precision copies and the padded table are rebuilt on load."""
    _check(load().onng_index_save(os.fsencode(path), _ptr(index.row_ptr), _ptr(index.col), _ptr(index.length),
                                  _ptr(index.X), index.n, index.d, _stream()))


def load_index(path: str, device="cuda") -> "Index":
    """Reads an index file written by save_index into new device tensors."""
    h = index_check(path)
    rp = torch.empty(h["n"] + 1, dtype=torch.int64, device=device)
    col = torch.empty(max(h["nnz"], 1), dtype=torch.int32, device=device)
    ln = torch.empty(max(h["nnz"], 1), dtype=torch.float32, device=device) if h["has_len"] else None
    X = torch.empty((h["n"], h["d"]), dtype=torch.float32, device=device)
    _check(load().onng_index_load(os.fsencode(path), h["n"], h["d"], h["nnz"], _ptr(rp), _ptr(col), _ptr(ln),
                                  _ptr(X), _stream()))
    return Index(rp, col[:h["nnz"]], X, None, None if ln is None else ln[:h["nnz"]])


# ----------------------------------------------------------------------------- seeds

def seeds_random(global_seed: int, nq: int, n: int, n_seed: int, device="cuda"):
    out = torch.empty((nq, n_seed), dtype=torch.int32, device=device)
    _check(load().onng_seeds_random(global_seed, nq, n, n_seed, _ptr(out), _stream()))
    return out


def seeds_pivot(X: torch.Tensor, Q: torch.Tensor, n_pivot: int, n_seed: int):
    X = _dev(X, torch.float32)
    Q = _dev(Q, torch.float32)
    out = torch.empty((Q.shape[0], n_seed), dtype=torch.int32, device=X.device)
    lib = load()
    ws = _ws(lib.onng_seeds_pivot_workspace_bytes(X.shape[0], X.shape[1], n_pivot), X.device)
    _check(lib.onng_seeds_pivot(_ptr(X), X.shape[0], X.shape[1], _ptr(Q), Q.shape[0], n_pivot, n_seed, _ptr(out),
                                _ptr(ws), ws.numel(), _stream()))
    return out


def pad_adjacency(row_ptr: torch.Tensor, col: torch.Tensor, width: int) -> torch.Tensor:
    """adj [n, width] int32: the first `width` entries of every row, -1 past its end."""
    row_ptr = _dev(row_ptr, torch.int64)
    col = _dev(col, torch.int32)
    n = row_ptr.numel() - 1
    adj = torch.empty((n, width), dtype=torch.int32, device=row_ptr.device)
    _check(load().onng_pad_adjacency(_ptr(row_ptr), _ptr(col), n, width, _ptr(adj), _stream()))
    return adj


def to_bf16(X: torch.Tensor) -> torch.Tensor:
    """bfloat16 (round to nearest even) copy made by the library's kernel."""
    X = _dev(X, torch.float32)
    out = torch.empty(X.shape, dtype=torch.bfloat16, device=X.device)
    _check(load().onng_to_bf16(_ptr(X), X.numel(), _ptr(out), _stream()))
    return out


def to_fp8(X: torch.Tensor):
    """(scale float32 [d], codes uint8 [n, d]): the library's e4m3 copy with
    per-dimension scales max|x_j| / 448."""
    X = _dev(X, torch.float32)
    n, d = X.shape
    scale = torch.empty(d, dtype=torch.float32, device=X.device)
    out = torch.empty((n, d), dtype=torch.uint8, device=X.device)
    _check(load().onng_to_fp8(_ptr(X), n, d, _ptr(scale), _ptr(out), _stream()))
    return scale, out


# ----------------------------------------------------------------------------- search

@dataclass
class Index:
    """A device-resident index: adjusted graph (CSR) and vectors."""
    row_ptr: torch.Tensor
    col: torch.Tensor
    X: torch.Tensor
    X_bf16: torch.Tensor | None = None
    length: torch.Tensor | None = None
    adj: torch.Tensor | None = None
    X_fp8: torch.Tensor | None = None
    fp8_scale: torch.Tensor | None = None

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    def with_bf16(self) -> "Index":
        if self.X_bf16 is None:
            self.X_bf16 = to_bf16(self.X)
        return self

    def with_fp8(self) -> "Index":
        if self.X_fp8 is None:
            self.fp8_scale, self.X_fp8 = to_fp8(self.X)
        return self

    def with_adjacency(self, width: int) -> "Index":
        """Adds the padded first-`width` adjacency table the search reads when e_s <= width."""
        if self.adj is None or self.adj.shape[1] != width:
            self.adj = pad_adjacency(self.row_ptr, self.col, width)
        return self

    def _c(self) -> _Index:
        return _Index(self.row_ptr.data_ptr(), self.col.data_ptr(), self.X.data_ptr(),
                      0 if self.X_bf16 is None else self.X_bf16.data_ptr(),
                      0 if self.adj is None else self.adj.data_ptr(), self.n, self.d,
                      0 if self.adj is None else self.adj.shape[1],
                      0 if self.X_fp8 is None else self.X_fp8.data_ptr(),
                      0 if self.fp8_scale is None else self.fp8_scale.data_ptr())


def build_index(X: torch.Tensor, k: int, e_o: int, e_i: int, path: bool = True) -> Index:
    """Algorithm ConstructGraph with the exact kNN graph: kNNG -> degree -> path adjustment."""
    X = _dev(X, torch.float32)
    nbr, ln = build_knng(X, k)
    g = adjust_degree(nbr, ln, e_o, e_i)
    if path:
        g = adjust_path(*g)
    return Index(g[0], g[1], X, None, g[2])


class SearchWorkspace:
    """Reusable device workspace for ``search`` (grows on demand)."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes: int, device):
        if self.buf is None or self.buf.numel() < nbytes or self.buf.device != torch.device(device):
            self.buf = torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)
        return self.buf


_default_ws = SearchWorkspace()


def search(index: Index, Q: torch.Tensor, k: int, e_s: int, eps: float, seeds: torch.Tensor,
           precision: int = PREC_FP32, k_rerank: int = 0, eps_q: torch.Tensor | None = None,
           es_q: torch.Tensor | None = None, max_expansions: int = 0, stats: bool = True,
           workspace: SearchWorkspace | None = None, out=None, pool_cap: int = 0):
    """Algorithm 1 for every query row: (ids int32 [nq,k], dist float32 [nq,k], stats int32 [nq,4] or None).

    ``pool_cap`` sets the per-warp candidate spill-pool entries (0: the library default)."""
    Q = _dev(Q, torch.float32)
    seeds = _dev(seeds, torch.int32)
    nq = Q.shape[0]
    dev = Q.device
    lib = load()
    if precision == PREC_BF16:
        index.with_bf16()
    elif precision == PREC_FP8:
        index.with_fp8()
    p = _Params(k, e_s, float(eps) if math.isfinite(eps) else math.inf, precision, k_rerank, max_expansions, pool_cap)
    ic = index._c()
    need = lib.onng_search_workspace_bytes(nq, C.byref(ic), C.byref(p))
    ws = (workspace or _default_ws).get(need, dev)
    if out is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=dev)
        dist = torch.empty((nq, k), dtype=torch.float32, device=dev)
        st = torch.empty((nq, 4), dtype=torch.int32, device=dev) if stats else None
    else:
        ids, dist, st = out
    eq = None if eps_q is None else _dev(eps_q, torch.float32)
    sq = None if es_q is None else _dev(es_q, torch.int32)
    _check(lib.onng_search(C.byref(ic), _ptr(Q), nq, C.byref(p), _ptr(seeds), seeds.shape[1], _ptr(eq), _ptr(sq),
                           _ptr(ids), _ptr(dist), _ptr(st), _ptr(ws), ws.numel(), _stream()))
    return ids, dist, st


def search_noalloc(index: Index, Q: torch.Tensor, k: int, e_s: int, eps: float, seeds: torch.Tensor,
                   precision: int = PREC_FP32, k_rerank: int = 0, eps_q: torch.Tensor | None = None,
                   es_q: torch.Tensor | None = None, max_expansions: int = 0, out=None):
    """``search`` through onng_search_noalloc: the library allocates nothing and
    uses its fixed per-device scratch instead of a workspace.

    For callers that cannot allocate device memory per call.  ``out`` =
    (ids [nq,k] int32, dist [nq,k] float32, stats [nq,4] int32 or None) lets the
    caller pass the result buffers too; otherwise they are allocated here, by
    torch, before the call.  Calls that can overlap on the GPU race on the shared
    scratch; keep them on one stream."""
    Q = _dev(Q, torch.float32)
    seeds = _dev(seeds, torch.int32)
    nq = Q.shape[0]
    dev = Q.device
    lib = load()
    if precision == PREC_BF16:
        index.with_bf16()
    elif precision == PREC_FP8:
        index.with_fp8()
    p = _Params(k, e_s, float(eps) if math.isfinite(eps) else math.inf, precision, k_rerank, max_expansions)
    ic = index._c()
    if out is None:
        out = (torch.empty((nq, k), dtype=torch.int32, device=dev), torch.empty((nq, k), dtype=torch.float32, device=dev),
               torch.empty((nq, 4), dtype=torch.int32, device=dev))
    ids, dist, st = out
    eq = None if eps_q is None else _dev(eps_q, torch.float32)
    sq = None if es_q is None else _dev(es_q, torch.int32)
    _check(lib.onng_search_noalloc(C.byref(ic), _ptr(Q), nq, C.byref(p), _ptr(seeds), seeds.shape[1], _ptr(eq),
                                   _ptr(sq), _ptr(ids), _ptr(dist), _ptr(st), _stream()))
    return ids, dist, st


def search_probe(index: Index, Q: torch.Tensor, k: int, e_s: int, eps: float, seeds: torch.Tensor, h: int,
                 target: float, workspace: SearchWorkspace | None = None):
    """Algorithm 1 stopped after h expansions: (features float32 [nq,16], stats int32 [nq,4])."""
    Q = _dev(Q, torch.float32)
    seeds = _dev(seeds, torch.int32)
    nq = Q.shape[0]
    lib = load()
    p = _Params(k, e_s, float(eps), PREC_FP32, 0, h)
    ic = index._c()
    ws = (workspace or _default_ws).get(lib.onng_search_workspace_bytes(nq, C.byref(ic), C.byref(p)), Q.device)
    feat = torch.empty((nq, 16), dtype=torch.float32, device=Q.device)
    st = torch.empty((nq, 4), dtype=torch.int32, device=Q.device)
    _check(lib.onng_search_probe(C.byref(ic), _ptr(Q), nq, C.byref(p), _ptr(seeds), seeds.shape[1], float(target),
                                 _ptr(feat), _ptr(st), _ptr(ws), ws.numel(), _stream()))
    return feat, st


# ----------------------------------------------------------------------------- predictor network

MLP_NPARAM = 16 * 64 + 64 + 64 * 64 + 64 + 2 * 64 + 2


def mlp_init(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-initialised parameters (flat float32 vector, biases zero)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for fan_in, fan_out in ((16, 64), (64, 64), (64, 2)):
        parts.append(torch.randn(fan_out * fan_in, generator=g) * (2.0 / fan_in) ** 0.5)
        parts.append(torch.zeros(fan_out))
    return torch.cat(parts).to(device=device, dtype=torch.float32)


def mlp_forward(P: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    X = _dev(X, torch.float32)
    Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
    _check(load().onng_mlp_forward(_ptr(_dev(P, torch.float32)), _ptr(X), X.shape[0], _ptr(Y), _stream()))
    return Y


def mlp_loss_grad(P: torch.Tensor, X: torch.Tensor, T: torch.Tensor):
    X = _dev(X, torch.float32)
    T = _dev(T, torch.float32)
    G = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    _check(load().onng_mlp_loss_grad(_ptr(_dev(P, torch.float32)), _ptr(X), _ptr(T), X.shape[0], _ptr(G), _ptr(loss),
                                     _stream()))
    return loss, G


def mlp_adam(P, G, M, V, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam step on float32 CUDA tensors P, M, V."""
    _check(load().onng_mlp_adam(_ptr(P), _ptr(G), _ptr(M), _ptr(V), t, lr, beta1, beta2, eps, _stream()))


def mlp_train(P, M, V, X, T, steps: int, batch: int, lr: float, t0: int = 0, losses: bool = False):
    """`steps` Adam steps on consecutive mini-batches, in one kernel; returns the per-step losses if asked."""
    X = _dev(X, torch.float32)
    T = _dev(T, torch.float32)
    G = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
    L = torch.empty(max(steps, 1), dtype=torch.float32, device=X.device) if losses else None
    _check(load().onng_mlp_train(_ptr(P), _ptr(M), _ptr(V), _ptr(X), _ptr(T), X.shape[0], batch, steps, t0, lr,
                                 _ptr(G), _ptr(L), _stream()))
    return L


def mlp_predict(P, X, alpha: float = 1.0, es_min: int = 1, es_max: int = 32):
    """bfloat16 evaluation: (eps float32 [B], e_s int32 [B])."""
    X = _dev(X, torch.float32)
    B = X.shape[0]
    eps = torch.empty(B, dtype=torch.float32, device=X.device)
    es = torch.empty(B, dtype=torch.int32, device=X.device)
    _check(load().onng_mlp_predict(_ptr(_dev(P, torch.float32)), _ptr(X), B, float(alpha), es_min, es_max, _ptr(eps),
                                   _ptr(es), _stream()))
    return eps, es


# ----------------------------------------------------------------------------- serving service

class Service:
    """The library's own serving loop (onng_serve_*): a native worker thread batches
    submitted requests by (k, eps, e_s) class over `slots` CUDA streams.  Queries
    are host float32 arrays; results come back as host arrays."""

    def __init__(self, index: "Index", precision: int = PREC_FP32, k_rerank: int = 0, n_pivot: int = 1024,
                 n_seed: int = 10, max_queries: int = 1024, k_max: int = 100, slots: int = 4,
                 timeout_ms: int = 10000):
        self.index = index  # its tensors must outlive the service
        self._ix = index._c()
        cfg = _ServeConfig(precision, k_rerank, n_pivot, n_seed, max_queries, k_max, slots, timeout_ms)
        self._h = C.c_void_p()
        self._shape = {}
        _check(load().onng_serve_create(C.byref(self._ix), C.byref(cfg), C.byref(self._h)))

    def submit(self, Q, k: int, eps: float, e_s: int) -> int:
        import numpy as np
        Q = np.ascontiguousarray(Q, dtype=np.float32)
        t = C.c_uint64(0)
        _check(load().onng_serve_submit(self._h, Q.ctypes.data_as(C.c_void_p), Q.shape[0], k, eps, e_s,
                                        C.byref(t)))
        self._shape[t.value] = (Q.shape[0], k)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = 10000):
        """(ids, dist) as numpy arrays [nq, k], or None if not done within timeout_ms."""
        import numpy as np
        nq, k = self._shape[ticket]
        ids = np.empty((nq, k), np.int32)
        dist = np.empty((nq, k), np.float32)
        st = load().onng_serve_poll(self._h, ticket, ids.ctypes.data_as(C.c_void_p),
                                    dist.ctypes.data_as(C.c_void_p), timeout_ms)
        if st == ONNG_E_AGAIN:
            return None
        del self._shape[ticket]
        _check(st)
        return ids, dist

    def close(self):
        if self._h:
            load().onng_serve_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
