"""Eq. 2 loss and the hill climb over (e_o, e_i): the arithmetic on CPU against
closed forms and brute force, and one GPU run over a small graph."""
import numpy as np
import pytest

from paper_1810_07355_gb300 import synth
from paper_1810_07355_gb300.tune import bracket_eps, eq2_loss, hill_climb

torch = pytest.importorskip("torch")


def test_eq2_constant_and_linear_costs():
    # constant cost: L = log10 C
    assert eq2_loss([0.85, 0.9, 0.95, 0.99], [100.0] * 4, 0.90, 0.98) == pytest.approx(2.0)
    # log10 C linear in precision: L = its value at the middle of [p_l, p_u]
    p = np.linspace(0.89, 0.99, 10)
    c = 10 ** (2 + (p - 0.89) / 0.10)
    assert eq2_loss(p, c, 0.90, 0.98) == pytest.approx(2.5)
    # unsorted samples and repeated precisions give the same value
    o = np.random.default_rng(0).permutation(10)
    assert eq2_loss(p[o], c[o], 0.90, 0.98) == pytest.approx(2.5)


def test_eq2_matches_dense_integration():
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = np.sort(rng.uniform(0.85, 1.0, 10))
        c = 10 ** rng.uniform(2, 4, 10)
        xs = np.linspace(0.90, 0.98, 200_001)
        v = np.interp(xs, p, np.log10(c))
        want = np.sum(0.5 * (v[1:] + v[:-1]) * np.diff(xs)) / 0.08  # dense sampling of the interpolant
        assert eq2_loss(p, c, 0.90, 0.98) == pytest.approx(want, abs=1e-7)


def test_bracket_eps_windows():
    prec = lambda e: min(1.0, 0.5 + e)  # noqa: E731
    e, p = bracket_eps(prec, 0.9, "low")
    assert 0.895 < p <= 0.9 and 0.395 < e <= 0.4 + 1e-12
    e, p = bracket_eps(prec, 0.98, "high")
    assert 0.98 <= p < 0.985
    # a step function: the closest reachable point is returned
    e, p = bracket_eps(lambda x: 0.5 if x < 0.3 else 1.0, 0.9, "low")
    assert p in (0.5, 1.0)


def test_hill_climb_finds_the_minimum_of_a_convex_function():
    f = lambda eo, ei: (eo - 35) ** 2 + 2 * (ei - 80) ** 2  # noqa: E731
    c = hill_climb(f, (20, 60), step=5, lo=(0, 0), hi=(100, 100))
    assert c.best == (35, 80) and c.loss == 0
    assert all(a[2] > b[2] for a, b in zip(c.path, c.path[1:]))  # every move lowers the loss
    # the bounds hold
    c = hill_climb(f, (20, 60), step=5, lo=(0, 0), hi=(30, 70))
    assert c.best == (30, 70)


@pytest.mark.gpu
def test_degree_optimisation_runs_on_the_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1810_07355_gb300 import onng
    from paper_1810_07355_gb300.tune import graph_loss, optimize_degrees
    X, Q = synth.workload("gmm10k", n=4000, nq=200)
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    knn = onng.build_knng(Xd, 40)
    gt, _ = onng.knn(Xd, Qd, 10)
    seeds = onng.seeds_pivot(Xd, Qd, 256, 10)
    L, samples = graph_loss(onng, knn, Xd, Qd, gt, seeds, 10, 10, 30, 0.90, 0.98)
    precs = np.array([pc[0] for _, pc in samples])
    logc = np.log10([pc[1] for _, pc in samples])
    assert len(samples) == 10 and np.all((precs >= 0) & (precs <= 1)) and np.all(np.isfinite(logc))
    # a mean of the interpolant lies within the sampled values
    assert np.isfinite(L) and logc.min() - 1e-9 <= L <= logc.max() + 1e-9
    c = optimize_degrees(onng, Xd, Qd, 10, 40, start=(10, 30), step=5, n_pivot=256, max_moves=2)
    assert c.loss <= c.evaluated[(10, 30)] and len(c.evaluated) >= 3
