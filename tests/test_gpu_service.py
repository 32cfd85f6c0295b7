"""The native serving loop (onng_serve_*): every request served in a batch equals
the same request searched alone (pivot seeds + search with its k, eps and e_s),
with requests submitted from several host threads; and the watchdog stops the
service when a launch outlives its limit (a long but finite search, no fault)."""
import threading

import numpy as np
import pytest

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


@pytest.fixture(scope="module")
def setup(onng):
    X, Q = synth.workload("sift1m", n=20000, nq=3000)
    Xd = torch.from_numpy(X).cuda()
    index = onng.build_index(Xd, 40, 10, 30).with_adjacency(16).with_bf16()
    return X, Q, index


@pytest.mark.parametrize("prec", [0, 1])
def test_service_equals_alone(onng, setup, prec):
    X, Q, index = setup
    classes = [(10, 0.05, 16), (10, 0.1, 16), (1, 0.0, 8), (50, 0.08, 0)]
    rng = np.random.default_rng(prec)
    reqs = []
    first = 0
    for i in range(240):
        nq = int(rng.integers(1, 40))
        if first + nq > len(Q):
            first = 0
        reqs.append((first, nq, classes[i % len(classes)]))
        first += nq
    results = {}
    with onng.Service(index, precision=prec, k_rerank=20, n_pivot=512, max_queries=256, k_max=50,
                      slots=3) as svc:
        def client(part):
            for i in part:
                f, nq, (k, eps, es) = reqs[i]
                t = svc.submit(Q[f:f + nq], k, eps, es)
                results[i] = (t, None)
            for i in part:
                out = None
                while out is None:
                    out = svc.poll(results[i][0], 5000)
                results[i] = (results[i][0], out)
        threads = [threading.Thread(target=client, args=(list(range(j, len(reqs), 3)),)) for j in range(3)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
    kw = dict(precision=prec, k_rerank=20) if prec else {}
    for i, (f, nq, (k, eps, es)) in enumerate(reqs):
        q = torch.from_numpy(Q[f:f + nq]).cuda()
        seeds = onng.seeds_pivot(index.X, q, 512, 10)
        ids, dist, _ = onng.search(index, q, k, es, eps, seeds, **{**kw, "k_rerank": max(20, k)} if prec else {})
        got_ids, got_dist = results[i][1]
        assert np.array_equal(got_ids, ids.cpu().numpy()), i
        assert np.array_equal(got_dist, dist.cpu().numpy()), i


def test_service_watchdog(onng, setup):
    X, Q, index = setup
    big = np.ascontiguousarray(np.tile(Q, (2, 1))[:4096])
    svc = onng.Service(index, max_queries=4096, k_max=50, slots=1, timeout_ms=1)
    try:
        t = svc.submit(big, 50, 1.0, 0)  # every edge, eps 1: a long search
        with pytest.raises(onng.OnngError) as e:
            out = None
            while out is None:
                out = svc.poll(t, 5000)
        assert e.value.status == onng.ONNG_E_LIMIT
        with pytest.raises(onng.OnngError):
            svc.submit(Q[:4], 10, 0.1, 16)
    finally:
        svc.close()
