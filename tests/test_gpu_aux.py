"""GPU checks of the auxiliary entry points: the graph statistics of Table 4
against the oracle, and index files written and read back through the device."""
import struct
import zlib

import numpy as np
import pytest

import oracle
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


INT_KEYS = ("max_out", "max_in", "zero_in")


def assert_stats_equal(got, want):
    for key in INT_KEYS:
        assert got[key] == want[key], key
    # degree sums are exact integers; the length mean is summed in another order
    for key in ("mean_out", "top5_out", "bottom5_in"):
        assert got[key] == pytest.approx(want[key], rel=1e-15, abs=0), key
    if np.isnan(want["in_dist10"]):
        assert np.isnan(got["in_dist10"])
    else:
        assert got["in_dist10"] == pytest.approx(want["in_dist10"], rel=1e-12)


def random_csr(n, seed, hubs=3, max_deg=40):
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, min(max_deg, n) + 1, n)
    if n >= 8:
        deg[rng.integers(0, n, hubs)] = rng.integers(n // 4, n // 2, hubs)
    ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    col = np.concatenate([rng.choice(n, size=d, replace=False) for d in deg]).astype(np.int32)
    ln = rng.integers(1, 30, ptr[-1]).astype(np.float32)  # integer lengths: many ties
    return ptr, col, ln


@pytest.mark.parametrize("n,seed", [(1, 0), (37, 1), (2000, 2), (70001, 3)])
def test_graph_stats_random(onng, n, seed):
    ptr, col, ln = random_csr(n, seed)
    got = onng.graph_stats(dev(ptr), dev(col), dev(ln))
    assert got["n"] == n and got["nnz"] == ptr[-1]
    assert_stats_equal(got, oracle.graph_stats(ptr, col, ln))


def test_graph_stats_adjusted_graphs(onng):
    X, _ = synth.workload("sift1m", n=6000, nq=1)
    nbr, ln = onng.build_knng(dev(X), 40)
    for g in (onng.adjust_degree(nbr, ln, 10, 30), onng.adjust_path(*onng.adjust_degree(nbr, ln, 20, 40))):
        got = onng.graph_stats(*g)
        want = oracle.graph_stats(*(t.cpu().numpy() for t in g))
        assert_stats_equal(got, want)
    # the 1-NNG's indegrees (Sec. 3, Fig. 3(c)): every node has one out-edge
    one = onng.adjust_degree(nbr, ln, 1, 0)
    got = onng.graph_stats(*one)
    assert got["mean_out"] == 1.0 and got["top5_out"] == 1.0
    assert_stats_equal(got, oracle.graph_stats(*(t.cpu().numpy() for t in one)))


def test_graph_stats_rejects_bad_ids(onng):
    ptr = np.array([0, 2, 3], np.int64)
    col = np.array([1, 5, 0], np.int32)
    with pytest.raises(onng.OnngError):
        onng.graph_stats(dev(ptr), dev(col), dev(np.ones(3, np.float32)))


def test_index_file_round_trip(onng, tmp_path):
    X, Q = synth.workload("sift1m", n=5000, nq=64)
    index = onng.build_index(dev(X), 30, 10, 30)
    path = str(tmp_path / "idx.onng")
    onng.save_index(index, path)
    raw = open(path, "rb").read()
    # the file follows the documented layout
    magic, ver, flags, n, d, crc, nnz = struct.unpack("<8sIIqiIq", raw[:40])
    assert (magic, ver, flags, n, d, nnz) == (b"ONNGIDX\0", 1, 1, 5000, 128, index.col.numel())
    assert crc == zlib.crc32(raw[64:]) and raw[40:64] == bytes(24)
    off = 64
    for t, dt in ((index.row_ptr, "<i8"), (index.col, "<i4"), (index.length, "<f4"), (index.X, "<f4")):
        a = t.cpu().numpy().reshape(-1)
        assert np.array_equal(np.frombuffer(raw, dt, a.size, off), a)
        off += a.nbytes
    assert off == len(raw)
    back = onng.load_index(path)
    for name in ("row_ptr", "col", "length", "X"):
        assert torch.equal(getattr(back, name), getattr(index, name)), name
    # the loaded index searches exactly as the original
    seeds = onng.seeds_random(7, 64, 5000, 10)
    Qd = dev(Q)
    a = onng.search(index, Qd, 10, 20, 0.1, seeds)
    b = onng.search(back, Qd, 10, 20, 0.1, seeds)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    # a corrupted copy is refused and leaves the destination untouched
    bad = str(tmp_path / "bad.onng")
    broken = bytearray(raw)
    broken[-1] ^= 0x40
    open(bad, "wb").write(bytes(broken))
    with pytest.raises(onng.OnngError):
        onng.load_index(bad)
    keep = torch.full((5001,), -7, dtype=torch.int64, device="cuda")
    lib = onng.load()
    st = lib.onng_index_load(bad.encode(), 5000, 128, index.col.numel(), keep.data_ptr(), index.col.data_ptr(),
                             None, index.X.data_ptr(), None)
    assert st == onng.ONNG_E_INVAL and bool((keep == -7).all())
