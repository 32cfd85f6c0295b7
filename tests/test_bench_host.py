"""Host-side pieces of the benchmark: clock-sample parsing, the algorithmic-byte
count behind the roofline, recall@k, the precision-error and near-tie helpers."""
import types

import pytest

torch = pytest.importorskip("torch")
import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1300.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2000, 2070, 1250.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = c.summary()
    assert s == {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.lines.append("0, 1500, 2070, 1300.0, 0x8, Active, Not Active, Active, Not Active")
    assert c.summary()["reasons"] == ["hw_slowdown", "sw_power_cap", "sw_thermal_slowdown"]
    assert bench.Clocks(0).summary() is None


def test_search_bytes_closed_form():
    # stats rows: distance computations, expansions, adjacency entries scanned, flags
    st = torch.tensor([[100, 10, 200, 0], [50, 5, 100, 0]], dtype=torch.int32)
    a = types.SimpleNamespace(nq=2, n_seed=10, k=10, k_rerank=20)
    d = 128
    b, ndc = bench.search_bytes(st, d, a, 2, True)
    want = 150 * d * 2 + 300 * 4 + 15 * 16 + 2 * d * 4 + 2 * 10 * 4 + 2 * 10 * 8 + 2 * 20 * d * 4
    assert b == want and ndc == 75.0
    b32, _ = bench.search_bytes(st, d, a, 4, False)
    assert b32 == 150 * d * 4 + 300 * 4 + 15 * 16 + 2 * d * 4 + 2 * 10 * 4 + 2 * 10 * 8


def test_recall_at_counts_hits_and_ignores_padding():
    ids = torch.tensor([[1, 2, 3], [4, 5, 6]])
    gt = torch.tensor([[3, 2, 9], [4, -1, -1]])
    # query 0: 2 of 3; query 1: 1 hit (padding never matches) -> (2/3 + 1/3) / 2
    assert bench.recall_at(ids, gt) == pytest.approx(0.5)
    assert bench.recall_at(gt.clamp_min(0), gt.clamp_min(0)) == pytest.approx(1.0)


def test_cpu_baseline_times_whole_passes(oracle_lib):
    """The CPU baseline leg runs the oracle over whole passes of the query batch."""
    from paper_1810_07355_gb300 import synth
    X, Q = synth.workload("gmm10k", n=1500, nq=40)
    nbr, ln = oracle_lib.knng(X, 10)
    ptr, col, _ = oracle_lib.adjust_degree(nbr, ln, 5, 10)
    seeds = torch.from_numpy(oracle_lib.seeds_pivot(X, Q, 64, 5))
    idx = types.SimpleNamespace(row_ptr=torch.from_numpy(ptr), col=torch.from_numpy(col))
    a = types.SimpleNamespace(k=10, e_s=10)
    r = bench.cpu_baseline(a, idx, X, Q, seeds, 0.1, min_wall=0.05, max_reps=3)
    assert r["kind"] == "oracle" and r["value"] > 0 and r["cores"] >= 1
    assert "pass(es) over all 40 queries" in r["sample"]


def test_path_bytes_by_hand():
    """Node 0 -> 1 (1.0), 2 (2.0); node 1 -> 2 (1.5); node 2 -> 0 (3.0), 1 (1.0),
    with 4 output edges.  Edges shorter than their row's longest: (0,1) reads the
    list of 1 (one entry) and (2,1) the list of 1: 2 entries of 8 bytes; plus
    5 input + 4 output edges and two row-pointer arrays of 4 entries."""
    ptr = torch.tensor([0, 2, 3, 5])
    col = torch.tensor([1, 2, 2, 0, 1], dtype=torch.int32)
    ln = torch.tensor([1.0, 2.0, 1.5, 3.0, 1.0])
    assert bench.path_bytes(torch, ptr, col, ln, 4) == 2 * 8 + (5 + 4) * 8 + 2 * 4 * 8


def test_parse_defaults_name_the_metric_workload():
    a = bench.parse([])
    assert (a.workload, a.n, a.nq, a.k, a.knn_k, a.e_o, a.e_i) == ("sift1m", 1_000_000, 10_000, 10, 100, 20, 60)
    assert bench.parse(["--workload", "gist1m"]).nq == 1000
    assert bench.parse(["--workload", "glove1m2"]).n == 1_200_000
    c = bench.common_config(a, 0.1, 1)
    assert c["workload"].startswith("sift-like n=1000000 d=128") and c["eps_fp32"] == 0.1


def test_precision_error_by_hand():
    """bfloat16 keeps 8 significant bits: 257 rounds (ties to even) to 256, so a
    query at the origin sees 256 for a true 257, relative error 1/257; an FP8 e4m3
    code of 17 (scale 1) decodes to 16 (steps of 2 at that exponent), error 1/17.
    Byte-valued coordinates up to 256 are exact in bfloat16.  Padding ids (-1) are
    not counted."""
    X = torch.tensor([[257.0, 0.0], [17.0, 0.0], [200.0, 3.0]])
    Q = torch.zeros((1, 2))
    ids = torch.tensor([[0, 2, -1]])
    e = bench.precision_error(torch, X, Q, ids)
    assert e["pairs"] == 2 and e["max_rel"] == pytest.approx(1 / 257, rel=1e-12)
    assert e["mean_rel"] == pytest.approx(0.5 / 257, rel=1e-12)
    assert bench.precision_error(torch, X[2:], Q, torch.tensor([[0]]))["max_rel"] == 0.0
    scale = torch.ones(2)
    codes = X.to(torch.float8_e4m3fn).view(torch.uint8)
    e8 = bench.precision_error(torch, X, Q, torch.tensor([[1]]), scale, codes)
    assert e8["max_rel"] == pytest.approx(1 / 17, rel=1e-12)


def test_rows_near_accepts_only_near_ties():
    """A row passes when its ids equal the oracle's, or when every position's
    distance agrees within 1e-5 relative (so swapped ids sit at near-equal
    distances); an extra infinite pad must be infinite on both sides."""
    import numpy as np
    o_ids = np.array([[1, 2, 3], [1, 2, 3], [1, 2, -1]])
    o_len = np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 3.0], [1.0, 2.0, np.inf]])
    ids = np.array([[1, 2, 3], [1, 3, 2], [1, 2, -1]])
    near = np.array([[1.0, 2.0, 3.0], [1.0, 2.0 + 1e-6, 3.0], [1.0, 2.0, np.inf]])
    assert bench.rows_near(ids, near, o_ids, o_len).tolist() == [True, True, True]
    far = near.copy()
    far[1, 1] = 2.1
    assert bench.rows_near(ids, far, o_ids, o_len).tolist() == [True, False, True]
    pad = near.copy()
    pad[2, 2] = 5.0
    assert bench.rows_near(np.array([[1, 2, 3], [1, 3, 2], [1, 2, 4]]), pad, o_ids, o_len).tolist() == \
        [True, True, False]
