"""onng_search_noalloc: the search for callers that cannot allocate device memory.

A query loop that must not stall (cudaMalloc and cudaFree may synchronise the
whole device), a process whose device memory is already taken by the index, or
plain C code without an allocator cannot hand the search a workspace per call.
onng_search_noalloc takes its scratch from one fixed array per device instead.
These tests check that it returns exactly what onng_search returns, on several
calls in a row (the array keeps the previous call's contents, so each call must
clear what has to start empty), that it reserves no device memory, and that an
index too large for the array is refused with a clear error.

The file is named so that pytest collects it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1810_07355_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def onng():
    from paper_1810_07355_gb300 import onng as m
    m.load()
    return m


def test_noalloc_refuses_index_beyond_its_scratch(onng):
    """Checked before any CUDA call, so it runs without a GPU."""
    lib = onng.load()
    p = onng._Params(10, 20, 0.1, onng.PREC_FP32, 0, 0)
    ix = onng._Index(None, None, None, None, None, 100_000_000, 128, 0)
    st = lib.onng_search_noalloc(C.byref(ix), None, 5, C.byref(p), None, 4, None, None, None, None, None, None)
    assert st == onng.ONNG_E_WORKSPACE
    msg = lib.onng_last_error().decode()
    assert "onng_search_noalloc" in msg and "n = 100000000" in msg and str(32 << 20) in msg


@pytest.fixture(scope="module")
def case(onng):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    X, Q = synth.workload("sift1m", n=20000, nq=1500)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    nbr, ln = onng.build_knng(Xd, 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    idx = onng.Index(g[0], g[1], Xd).with_adjacency(20).with_bf16()
    seeds = onng.seeds_pivot(Xd, Qd, 256, 8)
    return idx, Qd, seeds


def _forms(onng, nq):
    g = torch.Generator(device="cpu").manual_seed(7)
    eps_q = (torch.rand(nq, generator=g) * 0.2).cuda()
    es_q = torch.randint(8, 21, (nq,), generator=g, dtype=torch.int32).cuda()
    return [
        dict(k=10, e_s=20, eps=0.1),
        dict(k=10, e_s=20, eps=0.0, precision=onng.PREC_BF16, k_rerank=20, eps_q=eps_q, es_q=es_q),
        dict(k=50, e_s=0, eps=0.3),
        dict(k=10, e_s=20, eps=0.1),
    ]


@pytest.mark.gpu
def test_noalloc_matches_search_on_calls_in_a_row(onng, case):
    idx, Q, seeds = case
    nq = Q.shape[0]
    forms = _forms(onng, nq)
    want = [onng.search(idx, Q, seeds=seeds, **f) for f in forms]
    for _ in range(2):
        for f, (w_ids, w_dist, w_st) in zip(forms, want):
            out = (torch.full((nq, f["k"]), -7, dtype=torch.int32, device=Q.device),
                   torch.full((nq, f["k"]), -7.0, dtype=torch.float32, device=Q.device),
                   torch.full((nq, 4), -7, dtype=torch.int32, device=Q.device))
            ids, dist, st = onng.search_noalloc(idx, Q, seeds=seeds, out=out, **f)
            torch.cuda.synchronize()
            assert torch.equal(ids, w_ids), f
            assert torch.equal(dist, w_dist), f
            assert torch.equal(st, w_st), f


@pytest.mark.gpu
def test_noalloc_reserves_no_device_memory(onng, case):
    idx, Q, seeds = case
    nq = Q.shape[0]
    out = (torch.empty((nq, 10), dtype=torch.int32, device=Q.device),
           torch.empty((nq, 10), dtype=torch.float32, device=Q.device),
           torch.empty((nq, 4), dtype=torch.int32, device=Q.device))
    onng.search_noalloc(idx, Q, 10, 20, 0.1, seeds, out=out)  # first call on the device: address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    used0 = torch.cuda.memory_allocated()
    for _ in range(3):
        onng.search_noalloc(idx, Q, 10, 20, 0.1, seeds, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == used0
    w_ids, w_dist, _ = onng.search(idx, Q, 10, 20, 0.1, seeds)
    assert torch.equal(out[0], w_ids) and torch.equal(out[1], w_dist)
