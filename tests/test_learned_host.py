"""Host logic of the learned form: the shrinkage fold into the last layer, and
label selection from sweep tables (hand-computed cases)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def test_shrink_folds_into_the_last_layer(oracle_lib):
    """The shrunk network's first output is ybar + beta (y0 - ybar) and its second
    output is unchanged (evaluated by the oracle's float64 network)."""
    from paper_1810_07355_gb300 import learned, onng
    P = onng.mlp_init(3, "cpu")
    P[16 * 64:16 * 64 + 64] = 0.1  # non-zero biases everywhere
    P[-2:] = torch.tensor([0.3, -0.2])
    x = np.random.default_rng(4).normal(size=(50, 16))
    y = oracle_lib.mlp_forward(P.double().numpy(), x)
    pred = learned.Predictor(P)
    for beta, ybar in ((0.0, -2.0), (0.5, 1.5), (1.0, 0.7)):
        ps = learned.shrink(pred, beta, ybar, es_fixed=20)
        ys = oracle_lib.mlp_forward(ps.P.double().numpy(), x)
        np.testing.assert_allclose(ys[:, 0], ybar + beta * (y[:, 0] - ybar), rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(ys[:, 1], y[:, 1], rtol=1e-12)
        assert ps.es_min == ps.es_max == 20
    assert torch.equal(pred.P, P)  # the original is untouched


def test_labels_from_sweep_and_lagrange_by_hand():
    from paper_1810_07355_gb300 import learned
    eps_grid, es_grid = (0.0, 0.1, 0.2), (8, 16)
    # one query: rec / cost over [e_s][eps]
    rec = torch.tensor([[[0.5, 0.9, 1.0], [0.8, 1.0, 1.0]]])
    cost = torch.tensor([[[10.0, 40.0, 90.0], [20.0, 60.0, 120.0]]])
    # cheapest cell reaching 1.0: (e_s 16, eps 0.1) at 60 beats (8, 0.2) at 90
    e, s = learned.labels_from_sweep(rec, cost, 1.0, eps_grid, es_grid)
    assert float(e[0]) == pytest.approx(0.1) and float(s[0]) == 16
    # reaching 0.9: (8, 0.1) at 40
    e, s = learned.labels_from_sweep(rec, cost, 0.9, eps_grid, es_grid)
    assert float(e[0]) == pytest.approx(0.1) and float(s[0]) == 8
    # unreachable: the most expensive cell
    e, s = learned.labels_from_sweep(rec * 0.5, cost, 1.0, eps_grid, es_grid)
    assert float(e[0]) == pytest.approx(0.2) and float(s[0]) == 16
    # Lagrangian: lam = 0.001 -> maximise rec - 0.001 cost: (16, 0.1) = 0.94 beats (8, 0.2) = 0.91
    e, s = learned.labels_lagrange(rec, cost, 0.001, eps_grid, es_grid)
    assert float(e[0]) == pytest.approx(0.1) and float(s[0]) == 16
    # a high price prefers the cheapest cell
    e, s = learned.labels_lagrange(rec, cost, 0.1, eps_grid, es_grid)
    assert float(e[0]) == pytest.approx(0.0) and float(s[0]) == 8


def test_eq1_policy_anchors():
    """Eq. 1 with the paper's GIST setting e_0 = 30, w_e = 20, rounded down:
    10^0 + 30, 10^1 + 30, 10^2 + 30."""
    from paper_1810_07355_gb300 import learned
    assert learned.eq1_policy(0.0) == 31
    assert learned.eq1_policy(0.05) == 40
    assert learned.eq1_policy(0.1) == 130
    assert learned.eq1_policy(0.02) == 32  # floor(10^0.4) = 2
    assert learned.eq1_policy(0.1, e0=10, we=10.0) == 20
