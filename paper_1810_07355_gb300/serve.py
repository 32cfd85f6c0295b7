"""Request loop with continuous batching over a device-resident index.

Requests (a few queries each, with their own k and required recall) arrive over
time.  The loop groups pending requests by (k, recall) class, since one search
launch runs one k and one eps, and keeps up to `slots` launches in flight, each
on its own CUDA stream with its own query, seed and result buffers.  A slot is
free again once its launch's results are back on the host; requests that
arrived meanwhile are admitted into the next free slot, so the work of several
batches overlaps on the device.

Admission is by device workspace: all launches draw their search workspace from
one budget (a first-fit pool over a single device buffer).  A batch is admitted
when the pool can give it the workspace its grid needs (the library's
onng_search_workspace_bytes for that batch); when nothing else is in flight it
takes what the pool has, down to one CTA's worth (the search then runs fewer
warps, never fails).  The pool returns a launch's range when its results are on
the host.

A host watchdog bounds every launch: one whose results have not arrived within
`timeout_s` stops the loop with ServeTimeout, naming the batch.

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


class ServeTimeout(RuntimeError):
    """A launch did not complete within the watchdog's limit."""


class WorkspacePool:
    """First-fit allocator over `budget` bytes of one device buffer (offsets
    aligned to 256 bytes).  alloc returns an offset or None; free returns a range."""

    def __init__(self, budget: int, device):
        self.budget = int(budget) // 256 * 256
        self.buf = torch.empty(max(self.budget, 256), dtype=torch.uint8, device=device)
        self.free_list = [(0, self.budget)]  # sorted (offset, size)

    def alloc(self, nbytes: int):
        need = (int(nbytes) + 255) // 256 * 256
        for i, (off, size) in enumerate(self.free_list):
            if size >= need:
                rest = (off + need, size - need)
                self.free_list[i:i + 1] = [rest] if rest[1] else []
                return off
        return None

    def largest(self) -> int:
        return max((size for _, size in self.free_list), default=0)

    def free(self, off: int, nbytes: int):
        need = (int(nbytes) + 255) // 256 * 256
        fl = sorted(self.free_list + [(off, need)])
        merged = []
        for o, sz in fl:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + sz)
            else:
                merged.append((o, sz))
        self.free_list = merged

    def in_use(self) -> int:
        return self.budget - sum(size for _, size in self.free_list)


@dataclass
class _Slot:
    stream: torch.cuda.Stream
    q_host: torch.Tensor
    q_dev: torch.Tensor
    seeds: torch.Tensor
    ids_dev: torch.Tensor
    dist_dev: torch.Tensor
    ids_host: torch.Tensor
    dist_host: torch.Tensor
    event: torch.cuda.Event = None
    batch: Batch = None
    ws_off: int = -1
    ws_bytes: int = 0
    deadline: float = 0.0


@dataclass
class ServeResult:
    ids: dict = field(default_factory=dict)      # request -> int32 [size, k]
    dist: dict = field(default_factory=dict)     # request -> float32 [size, k]
    latency: dict = field(default_factory=dict)  # request -> seconds from arrival to results on the host
    launches: int = 0
    wall: float = 0.0
    ws_peak: int = 0        # most workspace bytes in use at once
    ws_waits: int = 0       # times a batch waited for workspace

    def summary(self, trace) -> dict:
        lat = np.array([self.latency[i] for i in range(len(trace))]) * 1e3
        queries = int(trace["size"].sum())
        return {"requests": len(trace), "queries": queries, "launches": self.launches,
                "queries_per_s": round(queries / self.wall, 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                "p99_ms": round(float(np.percentile(lat, 99)), 3), "wall_s": round(self.wall, 3),
                "workspace_peak_bytes": self.ws_peak, "workspace_waits": self.ws_waits}


class Server:
    """Continuous-batching search server over one index on the current device."""

    def __init__(self, index: onng.Index, eps_table: dict, e_s: int, n_pivot: int = 1024, n_seed: int = 10,
                 precision: int = onng.PREC_FP32, k_rerank: int = 0, slots: int = 4, ws_budget: int = 1 << 30,
                 max_queries: int = 4096, k_max: int = 100, timeout_s: float = 10.0):
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
        self.timeout_s = timeout_s
        p = onng._Params(k_max, e_s, 0.0, precision, max(k_rerank, k_max), 0)
        # eps_table values: eps (with e_s) or (eps, e_s) per (k, recall) class
        self.one_cta = int(self.lib.onng_search_workspace_bytes(1, C.byref(ic), C.byref(p)))
        if ws_budget < self.one_cta:
            raise ValueError(f"workspace budget {ws_budget} B is below one search CTA ({self.one_cta} B)")
        self.pool = WorkspacePool(ws_budget, dev)
        self.slots = []
        for _ in range(slots):
            self.slots.append(_Slot(
                stream=torch.cuda.Stream(device=dev),
                q_host=torch.empty((max_queries, d), dtype=torch.float32).pin_memory(),
                q_dev=torch.empty((max_queries, d), dtype=torch.float32, device=dev),
                seeds=torch.empty(max_queries * n_seed, dtype=torch.int32, device=dev),
                ids_dev=torch.empty(max_queries * k_max, dtype=torch.int32, device=dev),
                dist_dev=torch.empty(max_queries * k_max, dtype=torch.float32, device=dev),
                ids_host=torch.empty(max_queries * k_max, dtype=torch.int32).pin_memory(),
                dist_host=torch.empty(max_queries * k_max, dtype=torch.float32).pin_memory()))

    def _need(self, b: Batch) -> int:
        """Workspace bytes the search grid of batch b needs."""
        k, recall = b.cls
        eps, e_s = self._params(k, recall)
        p = onng._Params(k, e_s, eps, self.precision, max(self.k_rerank, k) if self.precision else 0, 0)
        ic = self.index._c()
        return int(self.lib.onng_search_workspace_bytes(b.nq, C.byref(ic), C.byref(p)))

    def _reserve(self, b: Batch, idle: bool):
        """(offset, bytes) of workspace for batch b, or None to wait: the grid's
        full need, or, when nothing is in flight, the largest free range (at least
        one CTA's worth)."""
        need = self._need(b)
        off = self.pool.alloc(need)
        if off is not None:
            return off, need
        if idle:
            got = min(need, self.pool.largest())
            if got >= self.one_cta:
                return self.pool.alloc(got), got
        return None

    def _launch(self, s: _Slot, b: Batch, Q: np.ndarray, ws_off: int, ws_bytes: int):
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
            ws = C.c_void_p(self.pool.buf.data_ptr() + ws_off)
            onng._check(self.lib.onng_search(C.byref(ic), onng._ptr(s.q_dev), b.nq, C.byref(p), onng._ptr(s.seeds),
                                             self.n_seed, None, None, onng._ptr(s.ids_dev), onng._ptr(s.dist_dev),
                                             None, ws, ws_bytes, st))
            s.ids_host[:b.nq * k].copy_(s.ids_dev[:b.nq * k], non_blocking=True)
            s.dist_host[:b.nq * k].copy_(s.dist_dev[:b.nq * k], non_blocking=True)
            s.event = torch.cuda.Event()
            s.event.record(s.stream)
        s.batch, s.ws_off, s.ws_bytes = b, ws_off, ws_bytes

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
        self.pool.free(s.ws_off, s.ws_bytes)
        s.batch, s.event, s.ws_off, s.ws_bytes = None, None, -1, 0

    def run(self, trace, Q: np.ndarray) -> ServeResult:
        """Serves `trace` (synth.request_trace rows) in real time; Q holds the queries."""
        if len(trace) and int(trace["size"].max()) > self.max_queries:
            raise ValueError("a request is larger than the batch capacity")
        if len(trace) and int(trace["k"].max()) > self.k_max:
            raise ValueError("a request's k exceeds k_max")
        out, sched = ServeResult(), Scheduler()
        n, nxt, done = len(trace), 0, 0
        held = None  # a batch taken from the scheduler that waits for workspace
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
                if s.batch is None:
                    continue
                if s.event.query():
                    done += len(s.batch.reqs)
                    self._collect(s, out, trace, time.perf_counter() - t0)
                    progress = True
                elif time.perf_counter() > s.deadline:
                    raise ServeTimeout(f"batch of {s.batch.nq} queries (class {s.batch.cls}, requests "
                                       f"{s.batch.reqs[:4]}...) not done after {self.timeout_s} s")
            for s in self.slots:
                if s.batch is not None or (held is None and not len(sched)):
                    continue
                b = held if held is not None else sched.next_batch(self.max_queries)
                idle = all(x.batch is None for x in self.slots)
                got = self._reserve(b, idle)
                if got is None:
                    if held is None:
                        out.ws_waits += 1
                    held = b
                    break
                held = None
                self._launch(s, b, Q, *got)
                s.deadline = time.perf_counter() + self.timeout_s
                out.launches += 1
                out.ws_peak = max(out.ws_peak, self.pool.in_use())
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
        got = self._reserve(b, True)
        self._launch(s, b, Q, *got)
        s.event.synchronize()
        ids = s.ids_host[:b.nq * k].numpy().reshape(b.nq, k).copy()
        dist = s.dist_host[:b.nq * k].numpy().reshape(b.nq, k).copy()
        self.pool.free(s.ws_off, s.ws_bytes)
        s.batch, s.event, s.ws_off, s.ws_bytes = None, None, -1, 0
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


def run_native(index, table: dict, trace, Q: np.ndarray, precision: int, k_rerank: int, slots: int,
               n_pivot: int = 1024, timeout_ms: int = 10_000) -> ServeResult:
    """The same trace through the library's native service (onng_serve_*): a host
    thread submits each request at its arrival time with its class's (eps, e_s);
    this thread polls the tickets in arrival order and takes the moment a poll
    returns as the request's completion (so a request that finished before an
    earlier one was collected counts the wait)."""
    import threading
    n = len(trace)
    out = ServeResult(ids=[None] * n, dist=[None] * n, latency={}, launches=0, wall=0.0)
    tickets = [None] * n
    ready = threading.Condition()
    import sys
    switch = sys.getswitchinterval()
    sys.setswitchinterval(2e-4)  # the two host threads hand over the interpreter often
    with onng.Service(index, precision=precision, k_rerank=k_rerank, n_pivot=n_pivot, max_queries=4096,
                      k_max=100, slots=slots, timeout_ms=timeout_ms) as svc:
        t0 = time.perf_counter()

        def submitter():
            for rid in range(n):
                r = trace[rid]
                delay = float(r["arrival"]) - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
                eps, es = table[(int(r["k"]), float(r["recall"]))]
                t = svc.submit(Q[r["first"]:r["first"] + r["size"]], int(r["k"]), float(eps), int(es))
                with ready:
                    tickets[rid] = t
                    ready.notify()

        th = threading.Thread(target=submitter)
        th.start()
        for rid in range(n):
            with ready:
                ready.wait_for(lambda: tickets[rid] is not None)
            res = None
            while res is None:
                res = svc.poll(tickets[rid], timeout_ms)
            out.latency[rid] = time.perf_counter() - t0 - trace["arrival"][rid]
            out.ids[rid], out.dist[rid] = res
        th.join()
        out.wall = time.perf_counter() - t0
    sys.setswitchinterval(switch)
    return out


def serve_spec(seconds: float = 60.0, rate: float = 100_000.0, precisions=("fp8", "bf16"), slots: int = 4,
               ws_mb: int = 1024, e_s: int = 10, k_rerank: int = 32, capacity_rate: float = 0.0,
               timeout_s: float = 10.0) -> dict:
    """The serving measurement: the 10k x 128 Gaussian-mixture index (k = 40
    graph, e_o = 10, e_i = 30, path adjustment) with bfloat16 and FP8 copies, a
    seeded Poisson trace of `seconds` at `rate` queries/s (requests of 1-256
    queries, log-uniform; k in {1, 10, 100}; recall in {0.9, 0.95, 0.99}), served
    in real time by the continuous-batching loop in each reduced precision and by
    one-slot batched fp32 search; per run queries/s and p50 / p99 request latency,
    and a sample of requests searched alone for the same-in-the-mix check."""
    from . import synth
    dev = torch.device("cuda")
    X, Qcal = synth.workload("gmm10k", nq=2000)
    trace = synth.request_trace(seconds, rate)
    queries = int(trace["size"].sum())
    _, Q = synth.workload("gmm10k", nq=queries)
    Xd = torch.from_numpy(X).to(dev)
    nbr, ln = onng.build_knng(Xd, 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    index = onng.Index(g[0], g[1], Xd).with_adjacency(e_s)
    ks, recalls = (1, 10, 100), (0.9, 0.95, 0.99)
    es_opts = (e_s, 2 * e_s, 4 * e_s, 0)
    budget = ws_mb << 20
    codes = {"fp32": onng.PREC_FP32, "bf16": onng.PREC_BF16, "fp8": onng.PREC_FP8}
    runs, tables, same = {}, {}, {}
    rng = np.random.default_rng(0)
    sample = rng.choice(len(trace), size=min(200, len(trace)), replace=False)
    for name in tuple(precisions) + ("fp32",):
        prec = codes[name]
        kr = k_rerank if prec != onng.PREC_FP32 else 0
        table = calibrate_eps(index, Qcal, ks, recalls, es_opts, 1024, 10, prec, kr)
        srv = Server(index, table, e_s, precision=prec, k_rerank=kr, slots=1 if name == "fp32" else slots,
                     ws_budget=budget, timeout_s=timeout_s)
        srv.run(trace[: min(len(trace), 200)], Q)  # warm-up
        res = srv.run(trace, Q)
        key = "batched_fp32_one_slot" if name == "fp32" else name
        runs[key] = dict(res.summary(trace), precision=name, k_rerank=kr, slots=len(srv.slots), ws_budget_mb=ws_mb)
        tables[name] = {f"k={k},recall={t}": [round(v[0], 4), v[1]] for (k, t), v in table.items()}
        ok = 0
        for rid in sample:
            r = trace[rid]
            ids, dist = srv.search_alone(Q[r["first"]:r["first"] + r["size"]], int(r["k"]), float(r["recall"]))
            ok += int(np.array_equal(ids, res.ids[rid]) and np.array_equal(dist, res.dist[rid]))
        same[key] = f"{ok}/{len(sample)}"
        if name == "bf16":
            # the same trace through the native service (worker thread in the library)
            run_native(index, table, trace[: min(len(trace), 200)], Q, prec, kr, slots)  # warm-up
            nat = run_native(index, table, trace, Q, prec, kr, slots)
            nsum = nat.summary(trace)
            nsum.pop("launches", None)
            nsum.pop("workspace_peak_bytes", None)
            nsum.pop("workspace_waits", None)
            ok_n = sum(int(np.array_equal(nat.ids[rid], res.ids[rid]) and np.array_equal(nat.dist[rid], res.dist[rid]))
                       for rid in sample)
            runs["bf16_native_service"] = dict(nsum, precision=name, k_rerank=kr, slots=slots,
                                               same_as_python_loop=f"{ok_n}/{len(sample)}")
        if capacity_rate > 0 and name != "fp32":
            ctrace = synth.request_trace(min(seconds, 2.0), capacity_rate, seed=synth.SEED_BASE + 6)
            _, CQ = synth.workload("gmm10k", nq=int(ctrace["size"].sum()))
            runs[key]["capacity"] = {"offered_qps": capacity_rate, "served": srv.run(ctrace, CQ).summary(ctrace)}
        del srv
    return {"metric": "serving: queries/s and p50/p99 request latency, continuous batching",
            "index": "gmm10k n=10000 d=128 (k=40 graph, e_o=10, e_i=30, path adjustment) + bf16 and FP8 copies",
            "trace": {"seconds": seconds, "offered_qps": rate, "requests": len(trace), "queries": queries,
                      "sizes": "log-uniform 1..256", "k": list(ks), "recall": list(recalls), "seed": synth.SEED_BASE + 5},
            "runs": runs, "eps_e_s_table": tables, "same_alone_and_in_mix": same,
            "admission": f"one {ws_mb} MB workspace pool; a batch takes what its grid needs"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--seconds", type=float, default=60.0)
    ap.add_argument("--rate", type=float, default=100_000.0, help="mean offered queries/s")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--ws-mb", type=int, default=1024, help="device workspace budget over all slots (MB)")
    ap.add_argument("--precisions", default="fp8,bf16", help="reduced precisions served (fp32 one-slot is the baseline)")
    ap.add_argument("--e-s", type=int, default=10, help="first e_s tried per class (then 2x, 4x, every edge)")
    ap.add_argument("--k-rerank", type=int, default=32, help="float32 rerank of max(k, this) in bf16 / fp8")
    ap.add_argument("--capacity-rate", type=float, default=0.0, help="offered load of a short saturating run (0: skip)")
    a = ap.parse_args()
    line = serve_spec(a.seconds, a.rate, tuple(p for p in a.precisions.split(",") if p), a.slots, a.ws_mb, a.e_s,
                      a.k_rerank, a.capacity_rate)
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
