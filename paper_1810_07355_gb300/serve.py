"""Request loop with continuous batching over a device-resident index.

Requests (a few queries each, with their own k and required recall) arrive over
time.  The loop groups pending requests by (k, recall) class, since one search
launch runs one k and one eps, and keeps up to `slots` launches in flight, each
on its own CUDA stream with its own fixed workspace, query, seed and result
buffers.  A slot is free again once its launch's results are back on the host;
requests that arrived meanwhile are admitted into the next free slot, so the
work of several batches overlaps on the device.  Admission is bounded by device
memory: the workspace budget is split across the slots, and the search sizes
its grid to the workspace it is given (a smaller workspace means fewer resident
warps, never a failure).

Each query's result depends only on the query, its seeds, k, eps, e_s and the
precision, never on what it is batched with; the tests check that every
request's result equals the same request searched alone.

Everything on the device runs in the library's kernels (pivot seeds, search);
this module only moves bytes and keeps time.  Run as
``python -m paper_1810_07355_gb300.serve`` for the serving measurement.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json
import time
from collections import OrderedDict, deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import onng


@dataclass
class Batch:
    cls: tuple            # (k, recall)
    reqs: list            # trace row indices, in admission order
    rows: list            # (first, size) per request in the trace's query matrix
    nq: int


class Scheduler:
    """Pending requests per (k, recall) class, FIFO within a class; the next
    batch comes from the class whose oldest request arrived first and takes
    that class's requests in order while they fit in `max_queries`."""

    def __init__(self):
        self.pending = OrderedDict()

    def add(self, rid: int, arrival: float, first: int, size: int, k: int, recall: float):
        self.pending.setdefault((int(k), float(recall)), deque()).append((arrival, rid, int(first), int(size)))

    def __len__(self):
        return sum(len(q) for q in self.pending.values())

    def next_batch(self, max_queries: int) -> Batch | None:
        live = [(q[0][0], c) for c, q in self.pending.items() if q]
        if not live:
            return None
        _, cls = min(live)
        q = self.pending[cls]
        reqs, rows, nq = [], [], 0
        while q and (nq == 0 or nq + q[0][3] <= max_queries):
            _, rid, first, size = q.popleft()
            reqs.append(rid)
            rows.append((first, size))
            nq += size
        return Batch(cls, reqs, rows, nq)


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    ws: torch.Tensor
    q_host: torch.Tensor
    q_dev: torch.Tensor
    seeds: torch.Tensor
    ids_dev: torch.Tensor
    dist_dev: torch.Tensor
    ids_host: torch.Tensor
    dist_host: torch.Tensor
    event: torch.cuda.Event = None
    batch: Batch = None


@dataclass
class ServeResult:
    ids: dict = field(default_factory=dict)      # request -> int32 [size, k]
    dist: dict = field(default_factory=dict)     # request -> float32 [size, k]
    latency: dict = field(default_factory=dict)  # request -> seconds from arrival to results on the host
    launches: int = 0
    wall: float = 0.0

    def summary(self, trace) -> dict:
        lat = np.array([self.latency[i] for i in range(len(trace))]) * 1e3
        queries = int(trace["size"].sum())
        return {"requests": len(trace), "queries": queries, "launches": self.launches,
                "queries_per_s": round(queries / self.wall, 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "wall_s": round(self.wall, 3)}


class Server:
    """Continuous-batching search server over one index on the current device."""

    def __init__(self, index: onng.Index, eps_table: dict, e_s: int, n_pivot: int = 256, n_seed: int = 10,
                 precision: int = onng.PREC_FP32, k_rerank: int = 0, slots: int = 4, ws_budget: int = 1 << 30,
                 max_queries: int = 4096, k_max: int = 100):
        self.lib = onng.load()
        self.index = (index.with_bf16() if precision == onng.PREC_BF16 else
                      index.with_fp8() if precision == onng.PREC_FP8 else index)
        self.eps_table, self.e_s = dict(eps_table), e_s
        self.n_pivot, self.n_seed = n_pivot, n_seed
        self.precision, self.k_rerank = precision, k_rerank
        self.max_queries, self.k_max = max_queries, k_max
        dev = index.X.device
        d = index.X.shape[1]
        ic = self.index._c()
        p = onng._Params(k_max, e_s, 0.0, precision, max(k_rerank, k_max), 0)
        # eps_table values: eps (with e_s) or (eps, e_s) per (k, recall) class
        full = self.lib.onng_search_workspace_bytes(max_queries, C.byref(ic), C.byref(p))
        one_cta = self.lib.onng_search_workspace_bytes(1, C.byref(ic), C.byref(p))
        self.ws_bytes = int(min(full, ws_budget // slots))
        if self.ws_bytes < one_cta:
            raise ValueError(f"workspace budget {ws_budget} B over {slots} slots is below one search CTA "
                             f"({one_cta} B per slot)")
        self.slots = []
        for _ in range(slots):
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(device=dev),
                ws=torch.empty(self.ws_bytes, dtype=torch.uint8, device=dev),
                q_host=torch.empty((max_queries, d), dtype=torch.float32).pin_memory(),
                q_dev=torch.empty((max_queries, d), dtype=torch.float32, device=dev),
                seeds=torch.empty(max_queries * n_seed, dtype=torch.int32, device=dev),
                ids_dev=torch.empty(max_queries * k_max, dtype=torch.int32, device=dev),
                dist_dev=torch.empty(max_queries * k_max, dtype=torch.float32, device=dev),
                ids_host=torch.empty(max_queries * k_max, dtype=torch.int32).pin_memory(),
                dist_host=torch.empty(max_queries * k_max, dtype=torch.float32).pin_memory()))

    def _launch(self, s: _Slot, b: Batch, Q: np.ndarray):
        k, recall = b.cls
        eps, e_s = self._params(k, recall)
        qh = s.q_host.numpy()
        o = 0
        for first, size in b.rows:
            qh[o:o + size] = Q[first:first + size]
            o += size
        X = self.index.X
        ic = self.index._c()
        p = onng._Params(k, e_s, eps, self.precision, max(self.k_rerank, k) if self.precision else 0, 0)
        st = C.c_void_p(s.stream.cuda_stream)
        with torch.cuda.stream(s.stream):
            s.q_dev[:b.nq].copy_(s.q_host[:b.nq], non_blocking=True)
            onng._check(self.lib.onng_seeds_pivot(onng._ptr(X), X.shape[0], X.shape[1], onng._ptr(s.q_dev), b.nq,
                                                  self.n_pivot, self.n_seed, onng._ptr(s.seeds), None, 0, st))
            onng._check(self.lib.onng_search(C.byref(ic), onng._ptr(s.q_dev), b.nq, C.byref(p), onng._ptr(s.seeds),
                                             self.n_seed, None, None, onng._ptr(s.ids_dev), onng._ptr(s.dist_dev),
                                             None, onng._ptr(s.ws), self.ws_bytes, st))
            s.ids_host[:b.nq * k].copy_(s.ids_dev[:b.nq * k], non_blocking=True)
            s.dist_host[:b.nq * k].copy_(s.dist_dev[:b.nq * k], non_blocking=True)
            s.event = torch.cuda.Event()
            s.event.record(s.stream)
        s.batch = b

    def _params(self, k, recall):
        v = self.eps_table[(int(k), float(recall))]
        return (float(v[0]), int(v[1])) if isinstance(v, tuple) else (float(v), self.e_s)

    def _collect(self, s: _Slot, out: ServeResult, trace, now: float):
        b = s.batch
        k = b.cls[0]
        ids = s.ids_host[:b.nq * k].numpy().reshape(b.nq, k)
        dist = s.dist_host[:b.nq * k].numpy().reshape(b.nq, k)
        o = 0
        for rid, (_, size) in zip(b.reqs, b.rows):
            out.ids[rid] = ids[o:o + size].copy()
            out.dist[rid] = dist[o:o + size].copy()
            out.latency[rid] = now - trace["arrival"][rid]
            o += size
        s.batch, s.event = None, None

    def run(self, trace, Q: np.ndarray) -> ServeResult:
        """Serves `trace` (synth.request_trace rows) in real time; Q holds the queries."""
        if len(trace) and int(trace["size"].max()) > self.max_queries:
            raise ValueError("a request is larger than the batch capacity")
        if len(trace) and int(trace["k"].max()) > self.k_max:
            raise ValueError("a request's k exceeds k_max")
        out, sched = ServeResult(), Scheduler()
        n, nxt, done = len(trace), 0, 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while done < n:
            now = time.perf_counter() - t0
            while nxt < n and trace["arrival"][nxt] <= now:
                r = trace[nxt]
                sched.add(nxt, float(r["arrival"]), r["first"], r["size"], r["k"], r["recall"])
                nxt += 1
            progress = False
            for s in self.slots:
                if s.batch is not None and s.event.query():
                    done += len(s.batch.reqs)
                    self._collect(s, out, trace, time.perf_counter() - t0)
                    progress = True
            for s in self.slots:
                if s.batch is None and len(sched):
                    self._launch(s, sched.next_batch(self.max_queries), Q)
                    out.launches += 1
                    progress = True
            if not progress:
                time.sleep(2e-5)
        out.wall = time.perf_counter() - t0
        return out

    def search_alone(self, Q: np.ndarray, k: int, recall: float):
        """One request by itself through the same C-ABI calls (the reference for the
        alone-versus-in-the-mix test)."""
        s = self.slots[0]
        b = Batch((int(k), float(recall)), [0], [(0, len(Q))], len(Q))
        self._launch(s, b, Q)
        s.event.synchronize()
        ids = s.ids_host[:b.nq * k].numpy().reshape(b.nq, k).copy()
        dist = s.dist_host[:b.nq * k].numpy().reshape(b.nq, k).copy()
        s.batch, s.event = None, None
        return ids, dist


def calibrate_eps(index, Q, k_values, recalls, e_s_options, n_pivot, n_seed, precision=onng.PREC_FP32, k_rerank=0,
                  iters=12, eps_max=2.0):
    """For each (k, recall): the first e_s of `e_s_options` (0 = every edge) at which
    eps_max reaches the recall on calibration queries Q, and there the smallest eps
    (bisection) that does.  Classes that no option reaches get the last option at
    eps_max.  Returns {(k, recall): (eps, e_s)}."""
    from .learned import recall_per_query
    Qd = torch.as_tensor(Q, device=index.X.device)
    seeds = onng.seeds_pivot(index.X, Qd, n_pivot, n_seed)
    table = {}
    for k in k_values:
        gt, _ = onng.knn(index.X, Qd, k)

        def rec(eps, es):
            kw = dict(precision=precision, k_rerank=max(k_rerank, k)) if precision else {}
            ids = onng.search(index, Qd, k, es, eps, seeds, **kw)[0]
            return float(recall_per_query(ids, gt).mean())
        for target in recalls:
            es = next((e for e in e_s_options if rec(eps_max, e) >= target), None)
            if es is None:
                table[(k, target)] = (eps_max, e_s_options[-1])
                continue
            lo, hi = 0.0, eps_max
            if rec(lo, es) >= target:
                table[(k, target)] = (lo, es)
                continue
            for _ in range(iters):
                mid = 0.5 * (lo + hi)
                if rec(mid, es) >= target:
                    hi = mid
                else:
                    lo = mid
            table[(k, target)] = (hi, es)
    return table


def main():
    from . import synth
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--seconds", type=float, default=10.0)
    ap.add_argument("--rate", type=float, default=100_000.0, help="mean offered queries/s")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--ws-mb", type=int, default=1024, help="device workspace budget over all slots (MB)")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--e-s", type=int, default=10, help="first e_s tried per class (then 2x, 4x, every edge)")
    ap.add_argument("--k-rerank", type=int, default=32, help="float32 rerank of max(k, this) in bf16 / fp8")
    ap.add_argument("--capacity-rate", type=float, default=2_000_000.0,
                    help="offered load of a second, saturating run (0: skip)")
    a = ap.parse_args()
    dev = torch.device("cuda")
    X, Qcal = synth.workload("gmm10k", nq=2000)
    trace = synth.request_trace(a.seconds, a.rate)
    queries = int(trace["size"].sum())
    _, Q = synth.workload("gmm10k", nq=queries)
    Xd = torch.from_numpy(X).to(dev)
    nbr, ln = onng.build_knng(Xd, 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    index = onng.Index(g[0], g[1], Xd).with_adjacency(a.e_s)
    prec = {"fp32": onng.PREC_FP32, "bf16": onng.PREC_BF16, "fp8": onng.PREC_FP8}[a.precision]
    ks, recalls = (1, 10, 100), (0.9, 0.95, 0.99)
    es_opts = (a.e_s, 2 * a.e_s, 4 * a.e_s, 0)
    kr = a.k_rerank if prec != onng.PREC_FP32 else 0
    table = calibrate_eps(index, Qcal, ks, recalls, es_opts, 256, 10, prec, kr)
    table32 = calibrate_eps(index, Qcal, ks, recalls, es_opts, 256, 10)
    budget = a.ws_mb << 20
    srv = Server(index, table, a.e_s, precision=prec, k_rerank=kr, slots=a.slots, ws_budget=budget)
    srv.run(trace[: min(len(trace), 200)], Q)  # warm-up
    res = srv.run(trace, Q)
    base = Server(index, table32, a.e_s, slots=1, ws_budget=budget)
    base.run(trace[: min(len(trace), 200)], Q)
    res0 = base.run(trace, Q)
    # a sample of requests searched alone must give the same results as in the mix
    rng = np.random.default_rng(0)
    same = 0
    sample = rng.choice(len(trace), size=min(200, len(trace)), replace=False)
    for rid in sample:
        r = trace[rid]
        ids, dist = srv.search_alone(Q[r["first"]:r["first"] + r["size"]], int(r["k"]), float(r["recall"]))
        same += int(np.array_equal(ids, res.ids[rid]) and np.array_equal(dist, res.dist[rid]))
    capacity = None
    if a.capacity_rate > 0:
        ctrace = synth.request_trace(min(a.seconds, 2.0), a.capacity_rate, seed=synth.SEED_BASE + 6)
        _, CQ = synth.workload("gmm10k", nq=int(ctrace["size"].sum()))
        capacity = {"offered_qps": a.capacity_rate, "served": srv.run(ctrace, CQ).summary(ctrace),
                    "batched_fp32_one_slot": base.run(ctrace, CQ).summary(ctrace)}
    line = {"metric": "serving: queries/s and p50/p99 request latency, continuous batching",
            "index": "gmm10k n=10000 d=128 (k=40 graph, e_o=10, e_i=30, path adjustment)",
            "trace": {"seconds": a.seconds, "offered_qps": a.rate, "requests": len(trace), "queries": queries,
                      "sizes": "log-uniform 1..256", "k": list(ks), "recall": list(recalls)},
            "served": dict(res.summary(trace), precision=a.precision, k_rerank=kr, slots=a.slots, ws_mb=a.ws_mb,
                           ws_bytes_per_slot=srv.ws_bytes),
            "batched_fp32_one_slot": res0.summary(trace), "capacity": capacity,
            "eps_e_s_table": {f"k={k},recall={t}": [round(v[0], 4), v[1]] for (k, t), v in table.items()},
            "same_alone_and_in_mix": f"{same}/{len(sample)}"}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
