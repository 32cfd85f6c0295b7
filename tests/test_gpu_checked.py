"""The bounds-checked build (-DONNG_CHECK) and determinism re-runs.

The checked library runs in a child process (ONNG_LIBRARY names it), so the
parent never loads it.  It must give the plain build's results on a valid
graph, and on a graph with ids outside [0, n) or rows outside the column array
it must skip those entries and flag the queries ONNG_FLAG_CHECK: every such
id is turned into "no id" where it is read, before any access uses it.  The
plain library is never given a corrupted graph."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import numpy as np, torch
import oracle
from paper_1810_07355_gb300 import onng, synth
assert onng.library_path().endswith("libonng_check.so")
X, Q = synth.workload("sift1m", n=4000, nq=200)
Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
nbr, ln = onng.build_knng(Xd, 30)
rp, col, length = onng.adjust_path(*onng.adjust_degree(nbr, ln, 10, 30))
seeds = onng.seeds_random(3, 200, 4000, 10)
# a valid graph: the oracle's results, no check flag
ids, dist, st = onng.search(onng.Index(rp, col, Xd), Qd, 10, 16, 0.1, seeds)
o_ids, _, o_st = oracle.search(rp.cpu().numpy(), col.cpu().numpy(), X, Q, 10, 16, np.float32(0.1),
                               seeds.cpu().numpy())
assert np.array_equal(ids.cpu().numpy(), o_ids)
assert np.array_equal(st[:, :2].cpu().numpy(), o_st[:, :2])
assert not (st[:, 3] & onng.FLAG_CHECK).any()
# ids outside [0, n) in every tenth row, read through the CSR and the padded table
bad = col.clone()
rows = torch.arange(0, 4000, 10, device="cuda")
bad[rp[rows]] = 4000 + 5
bad[rp[rows] + 1] = -3
for index in (onng.Index(rp, bad, Xd), onng.Index(rp, bad, Xd).with_adjacency(16),
              onng.Index(rp, bad, Xd).with_adjacency(32)):
    ids, dist, st = onng.search(index, Qd, 10, 16, 0.1, seeds)
    got = ids.cpu().numpy()
    assert ((got >= -1) & (got < 4000)).all()
    assert (st[:, 3] & onng.FLAG_CHECK).any()
    ok = got >= 0
    d64 = np.sqrt(((X[np.where(ok, got, 0)].astype(np.float64) - Q[:, None, :]) ** 2).sum(2))
    np.testing.assert_allclose(dist.cpu().numpy()[ok], d64[ok], rtol=1e-5)
# rows outside col (no padded table: it would read them)
rp2 = rp.clone()
rp2[rows[1:]] = rp[-1] + 1000
ids, dist, st = onng.search(onng.Index(rp2, col, Xd), Qd, 10, 16, 0.1, seeds)
assert (st[:, 3] & onng.FLAG_CHECK).any()
assert ((ids.cpu().numpy() >= -1) & (ids.cpu().numpy() < 4000)).all()
print("checked build ok")
"""


def test_checked_build_flags_bad_graphs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07355_gb300 import build
    lib = build.build_checked()
    env = dict(os.environ, ONNG_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "checked build ok" in r.stdout


def test_search_is_deterministic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07355_gb300 import onng, synth
    X, Q = synth.workload("sift1m", n=6000, nq=500)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    index = onng.build_index(Xd, 40, 10, 30).with_adjacency(20).with_bf16()
    seeds = onng.seeds_pivot(Xd, Qd, 256, 10)
    for kw in (dict(), dict(precision=onng.PREC_BF16, k_rerank=20)):
        a = onng.search(index, Qd, 10, 20, 0.08, seeds, **kw)
        b = onng.search(index, Qd, 10, 20, 0.08, seeds, **kw)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    # the build is deterministic too
    again = onng.build_index(Xd, 40, 10, 30)
    assert torch.equal(again.row_ptr, index.row_ptr) and torch.equal(again.col, index.col)
