"""The search's soft limits on the GPU: a candidate spill pool that fills up,
and a visited-id log that overflows (the whole bitmap is then cleared).

Neither may write outside the caller's workspace or output rows (canary bytes
past their ends stay untouched), a query that the limit cannot have touched must
still equal the float64 oracle bit for bit, and a query that did hit it returns
a valid list and a flag.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1810_07355_gb300 import synth
from parity_helpers import assert_valid_lists

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CANARY = 0xA5


@pytest.fixture(scope="module")
def onng():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07355_gb300 import onng as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


class FixedWorkspace:
    """A workspace of exactly `nbytes` followed by `tail` canary bytes."""

    def __init__(self, nbytes, tail=1 << 20):
        self.nbytes = int(nbytes)
        self.full = torch.full((self.nbytes + tail,), CANARY, dtype=torch.uint8, device="cuda")

    def get(self, need, device):
        # whatever the call asks for, it gets `nbytes`: the library sizes its grid to it
        return self.full[:self.nbytes]

    def tail_intact(self):
        return bool((self.full[self.nbytes:] == CANARY).all().item())


def canaried_out(nq, k, extra=64):
    ids = torch.full((nq * k + extra,), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((nq * k + extra,), -7.0, dtype=torch.float32, device="cuda")
    st = torch.full((nq * 4 + extra,), -7, dtype=torch.int32, device="cuda")
    views = (ids[:nq * k].view(nq, k), dist[:nq * k].view(nq, k), st[:nq * 4].view(nq, 4))

    def intact():
        return bool((ids[nq * k:] == -7).all() and (dist[nq * k:] == -7.0).all() and (st[nq * 4:] == -7).all())
    return views, intact


def ws_bytes(onng, idx, nq, k, pool_cap=0):
    p = onng._Params(k, 0, 0.0, onng.PREC_FP32, 0, 0, pool_cap)
    ic = idx._c()
    return onng.load().onng_search_workspace_bytes(nq, C.byref(ic), C.byref(p))


@pytest.fixture(scope="module")
def sift6k(onng):
    X, Q = synth.workload("sift1m", n=6000, nq=200)
    nbr, ln = onng.build_knng(dev(X), 40)
    g = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
    seeds = onng.seeds_pivot(dev(X), dev(Q), 512, 10)
    return X, Q, g, seeds


def test_pool_overflow_is_flagged_and_stays_in_bounds(onng, sift6k):
    """pool_cap = 64: the register head (32 keys) and the shared overflow (128
    keys) hold 160 candidates before the pool is touched, so every query whose
    oracle candidate set never exceeds 150 must be unflagged and exact; at
    eps = 0.3 every candidate set outgrows the pool."""
    X, Q, g, seeds = sift6k
    idx = onng.Index(g[0], g[1], dev(X))
    nq, k, cap = len(Q), 10, 64
    for eps, must_flag in ((0.08, False), (0.3, True)):
        ws = FixedWorkspace(ws_bytes(onng, idx, nq, k, cap))
        out, intact = canaried_out(nq, k)
        ids, dist, st = onng.search(idx, dev(Q), k, 0, eps, seeds, workspace=ws, out=out, pool_cap=cap)
        torch.cuda.synchronize()
        assert ws.tail_intact() and intact()
        o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, k, 0, np.float32(eps), host(seeds))
        ids, dist, st = host(ids), host(dist), host(st)
        flagged = (st[:, 3] & onng.FLAG_S_OVERFLOW) != 0
        small = o_st[:, 2] <= 150
        assert not flagged[small].any()
        assert np.array_equal(ids[small], o_ids[small])
        assert np.array_equal(st[small, 0], o_st[small, 0])
        assert np.array_equal(ids[~flagged], o_ids[~flagged])
        assert_valid_lists(ids, dist, X, Q, rel=1e-6)
        if must_flag:
            assert flagged.sum() >= nq // 2
        else:
            assert small.mean() > 0.7


def test_visited_log_overflow_clears_the_bitmap(onng):
    """eps = inf with every edge scanned visits all 30,000 nodes, past the
    16,384-id log, so each warp clears its whole bitmap after such a query.  One
    CTA (4 warps) serves 12 queries, so every warp reuses its bitmap: a wrong
    clear would hide nodes from the next query."""
    rng = np.random.default_rng(17)
    n = 30000
    # uniform 8-d integer points: one strongly connected graph, so every query
    # reaches every node (the largest candidate set, about 11,000, fits the pool)
    X = rng.integers(0, 256, size=(n, 8)).astype(np.float32)
    Q = rng.integers(0, 256, size=(12, 8)).astype(np.float32)
    nbr, ln = onng.build_knng(dev(X), 16)
    g = onng.adjust_degree(nbr, ln, 8, 16)
    seeds = onng.seeds_random(5, len(Q), n, 4)
    idx = onng.Index(g[0], g[1], dev(X))
    ws = FixedWorkspace(ws_bytes(onng, idx, 4, 10))  # room for one CTA of 4 warps
    out, intact = canaried_out(len(Q), 10)
    ids, dist, st = onng.search(idx, dev(Q), 10, 0, float("inf"), seeds, workspace=ws, out=out)
    torch.cuda.synchronize()
    assert ws.tail_intact() and intact()
    o_ids, o_dist, o_st = oracle.search(host(g[0]), host(g[1]), X, Q, 10, 0, np.inf, host(seeds))
    assert (o_st[:, 0] == n).all()
    assert np.array_equal(host(ids), o_ids)
    assert np.array_equal(host(st)[:, 0], o_st[:, 0])
    assert np.array_equal(host(st)[:, 1], o_st[:, 1])
    assert (host(st)[:, 3] == 0).all()
