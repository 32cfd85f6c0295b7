"""Serving loop: request trace, class batching, workspace admission, the host
watchdog, and results that do not depend on what a request is batched with
(continuous batching over several streams)."""
import numpy as np
import pytest

from paper_1810_07355_gb300 import synth

torch = pytest.importorskip("torch")


def test_request_trace_shape_and_seed():
    t = synth.request_trace(2.0, 50_000)
    assert np.all(np.diff(t["arrival"]) >= 0) and t["arrival"].min() >= 0 and t["arrival"].max() <= 2.0
    assert t["size"].min() >= 1 and t["size"].max() <= 256
    assert np.array_equal(t["first"], np.concatenate([[0], np.cumsum(t["size"])[:-1]]))
    assert set(np.unique(t["k"])) <= {1, 10, 100} and set(np.unique(t["recall"])) <= {0.9, 0.95, 0.99}
    # offered load within 10 % of the requested mean rate (Poisson, ~2,300 requests)
    assert abs(t["size"].sum() / 2.0 - 50_000) < 5_000
    assert np.array_equal(t, synth.request_trace(2.0, 50_000))


def test_scheduler_batches_by_class_oldest_first():
    from paper_1810_07355_gb300.serve import Scheduler
    s = Scheduler()
    s.add(0, 0.10, 0, 5, 10, 0.9)
    s.add(1, 0.20, 5, 3, 1, 0.95)
    s.add(2, 0.30, 8, 4, 10, 0.9)
    s.add(3, 0.40, 12, 9, 10, 0.9)
    b = s.next_batch(10)
    assert b.cls == (10, 0.9) and b.reqs == [0, 2] and b.nq == 9 and b.rows == [(0, 5), (8, 4)]
    b = s.next_batch(10)
    assert b.cls == (1, 0.95) and b.reqs == [1]
    b = s.next_batch(4)  # a request larger than the capacity still goes alone
    assert b.reqs == [3] and b.nq == 9
    assert s.next_batch(10) is None and len(s) == 0


def test_workspace_pool_first_fit_and_merge():
    from paper_1810_07355_gb300.serve import WorkspacePool
    p = WorkspacePool(4096, "cpu")
    a = p.alloc(1000)  # rounded to 1024
    b = p.alloc(1024)
    c = p.alloc(2048)
    assert (a, b, c) == (0, 1024, 2048) and p.alloc(1) is None and p.in_use() == 4096
    p.free(b, 1024)
    assert p.largest() == 1024 and p.alloc(2000) is None
    p.free(a, 1000)  # merges with the free range after it
    assert p.free_list == [(0, 2048)] and p.alloc(2048) == 0
    p.free(0, 2048)
    p.free(c, 2048)
    assert p.free_list == [(0, 4096)] and p.in_use() == 0


@pytest.mark.gpu
def test_watchdog_stops_a_stalled_launch():
    """A launch whose completion never shows on the host (a stall injected on the
    host: its event reports unfinished forever) stops the loop with ServeTimeout
    after the watchdog's limit; the device work itself completes normally."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time

    from paper_1810_07355_gb300 import onng
    from paper_1810_07355_gb300.serve import Server, ServeTimeout
    X, _ = synth.workload("gmm10k", n=3000)
    trace = synth.request_trace(0.05, 20_000, seed=12)
    _, Q = synth.workload("gmm10k", nq=int(trace["size"].sum()))
    Xd = torch.from_numpy(X).cuda()
    nbr, ln = onng.build_knng(Xd, 20)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 20))
    index = onng.Index(g[0], g[1], Xd)
    eps = {(k, r): 0.05 for k in (1, 10, 100) for r in (0.9, 0.95, 0.99)}
    srv = Server(index, eps, 10, slots=2, ws_budget=64 << 20, timeout_s=0.5)

    class Stalled:
        def query(self):
            return False

    real = srv._launch

    def stalled_launch(s, b, Q_, off, nbytes):
        real(s, b, Q_, off, nbytes)
        s.event.synchronize()
        s.event = Stalled()
    srv._launch = stalled_launch
    t0 = time.perf_counter()
    with pytest.raises(ServeTimeout):
        srv.run(trace, Q)
    assert 0.4 < time.perf_counter() - t0 < 5.0


@pytest.mark.gpu
def test_serving_results_equal_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07355_gb300 import onng
    from paper_1810_07355_gb300.serve import Server
    X, _ = synth.workload("gmm10k")
    trace = synth.request_trace(0.25, 40_000, seed=11)
    _, Q = synth.workload("gmm10k", nq=int(trace["size"].sum()))
    Xd = torch.from_numpy(X).cuda()
    nbr, ln = onng.build_knng(Xd, 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    index = onng.Index(g[0], g[1], Xd).with_adjacency(10)
    eps = {(k, r): e for k in (1, 10, 100) for r, e in ((0.9, 0.02), (0.95, 0.05), (0.99, 0.1))}
    for prec in (onng.PREC_FP32, onng.PREC_BF16, onng.PREC_FP8):
        # a small workspace budget: three slots with clamped grids
        srv = Server(index, eps, 10, precision=prec, k_rerank=20 if prec else 0, slots=3, ws_budget=48 << 20,
                     max_queries=1024)
        res = srv.run(trace, Q)
        assert len(res.ids) == len(trace) and res.launches < len(trace)
        for rid in range(len(trace)):
            r = trace[rid]
            q = Q[r["first"]:r["first"] + r["size"]]
            ids, dist = srv.search_alone(q, int(r["k"]), float(r["recall"]))
            assert np.array_equal(ids, res.ids[rid]) and np.array_equal(dist, res.dist[rid]), rid
        # and through the plain binding (its own workspace and grid) for a few requests
        for rid in range(0, len(trace), max(1, len(trace) // 8)):
            r = trace[rid]
            q = torch.from_numpy(Q[r["first"]:r["first"] + r["size"]]).cuda()
            k = int(r["k"])
            s = onng.seeds_pivot(Xd, q, srv.n_pivot, 10)
            kw = dict(precision=prec, k_rerank=max(20, k)) if prec else {}
            ids, dist, _ = onng.search(index, q, k, 10, eps[(k, float(r["recall"]))], s, **kw)
            assert np.array_equal(ids.cpu().numpy(), res.ids[rid]), rid
        if prec == onng.PREC_FP32:
            # served fp32 requests against Algorithm 1 in float64 (near-tie rule)
            import oracle
            from parity_helpers import assert_search_parity
            ptr, col = g[0].cpu().numpy(), g[1].cpu().numpy()
            for rid in range(0, len(trace), max(1, len(trace) // 12)):
                r = trace[rid]
                q = Q[r["first"]:r["first"] + r["size"]]
                k = int(r["k"])
                s = onng.seeds_pivot(Xd, torch.from_numpy(q).cuda(), srv.n_pivot, 10).cpu().numpy()
                o = oracle.search(ptr, col, X, q, k, 10, np.float32(eps[(k, float(r["recall"]))]), s, margin=True)
                st = np.zeros((len(q), 4), np.int64)
                assert_search_parity(res.ids[rid], res.dist[rid], st, *o, X, q, min_tie_free=0.0, counts=False)
