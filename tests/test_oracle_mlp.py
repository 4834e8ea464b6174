"""Pins for the MLP oracle (CPU, fp64): central finite differences of the
loss, closed forms of a first Adam step and of a zero network, and the
paper's switching rule on hand-made inputs."""
import numpy as np
import pytest

from oracle import mlp


def _data(n=40, seed=1):
    rs = np.random.RandomState(seed)
    raw = rs.uniform(0, 15, (n, mlp.IN))
    tgt = rs.normal(9, 2, (n, mlp.OUT))
    mask = (rs.uniform(size=(n, mlp.OUT)) > 0.2).astype(np.float64)
    return raw, tgt, mask


def test_layout_size():
    assert mlp.OUT == 9
    assert mlp.NW == 12 + 32 * 6 + 32 + 32 * 32 + 32 + 9 * 32 + 9 == 1589


def test_gradient_matches_central_differences():
    raw, tgt, mask = _data()
    w = mlp.init_weights(raw.mean(0), raw.std(0), seed=3)
    w[mlp.OFF_B1:mlp.OFF_W2] = np.random.RandomState(4).normal(0, 0.1, 32)
    loss, g = mlp.loss_and_grad(w, raw, tgt, mask)
    rs = np.random.RandomState(5)
    idx = np.concatenate([rs.choice(np.arange(mlp.OFF_W1, mlp.NW), 60, replace=False),
                          [mlp.OFF_B3, mlp.OFF_W3, mlp.OFF_B1, mlp.NW - 1]])
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, raw, tgt, mask)[0] - mlp.loss_and_grad(wm, raw, tgt, mask)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    assert np.all(g[:mlp.OFF_W1] == 0)


def test_zero_network_predicts_bias_and_mse():
    raw, tgt, mask = _data(10)
    w = np.zeros(mlp.NW)
    w[mlp.OFF_ISTD:mlp.OFF_ISTD + 6] = 1.0
    w[mlp.OFF_B3:] = np.arange(1, mlp.OUT + 1)
    y, _ = mlp.forward(w, raw)
    assert np.array_equal(y, np.tile(np.arange(1, mlp.OUT + 1), (10, 1)).astype(float))
    loss, g = mlp.loss_and_grad(w, raw, tgt, mask)
    r = (y - tgt) * mask
    assert abs(loss - (r ** 2).sum() / mask.sum()) < 1e-12
    assert np.allclose(g[mlp.OFF_B3:], 2 * r.sum(0) / mask.sum(), rtol=1e-12)
    assert np.all(g[mlp.OFF_W1:mlp.OFF_B2 + 32] == 0)    # tanh(0) = 0 blocks earlier layers


def test_first_adam_step_is_signed_lr():
    """At t = 1 the bias-corrected moments are g and g^2, so each step is
    -lr * g / (|g| + eps)."""
    w = np.ones(mlp.NW)
    g = np.linspace(-3, 3, mlp.NW)
    w2, m, v = mlp.adam_step(w, g, np.zeros(mlp.NW), np.zeros(mlp.NW), 1, lr=0.01)
    exp = w.copy()
    exp[mlp.OFF_W1:] -= 0.01 * g[mlp.OFF_W1:] / (np.abs(g[mlp.OFF_W1:]) + 1e-8)
    assert np.allclose(w2, exp, rtol=0, atol=1e-15)
    assert np.array_equal(w2[:mlp.OFF_W1], w[:mlp.OFF_W1])


def test_training_reduces_loss():
    raw, tgt, mask = _data(200, seed=7)
    tgt = np.stack([raw[:, 0] * 0.5 + k for k in range(mlp.OUT)], 1)
    w = mlp.init_weights(raw.mean(0), raw.std(0), seed=1)
    m = np.zeros(mlp.NW)
    v = np.zeros(mlp.NW)
    l0 = mlp.loss_and_grad(w, raw, tgt, mask)[0]
    for t in range(1, 301):
        _, g = mlp.loss_and_grad(w, raw, tgt, mask)
        w, m, v = mlp.adam_step(w, g, m, v, t, lr=0.01)
    assert mlp.loss_and_grad(w, raw, tgt, mask)[0] < 0.05 * l0


def test_heuristic_rule():
    # eager + TC graph, no switching: always mode 1
    assert mlp.heuristic_choose(0, 1, 0, 10, [5, 1e9], [1, 1]).tolist() == [1, 1]
    # lazy CC graph with switching: bottom-up exactly when unvisited < 10 |Q|
    assert mlp.heuristic_choose(1, 0, 1, 10, [99, 100, 101], [10, 10, 10]).tolist() == [4, 2, 2]


def test_regret_definition():
    t = np.array([[1.0, 2.0], [5.0, 3.0]])
    assert mlp.regret(t, [0, 1]) == 0.0
    assert mlp.regret(t, [1, 0]) == pytest.approx((2 + 5) / 4 - 1)


def test_raw_features():
    f = mlp.raw_features([0, 10], [3, 7], [100, -5], [256, 0], [1, 4], 16.0)
    assert f.shape == (2, 6)
    assert np.allclose(f[0], np.log1p([0, 3, 100, 256, 1, 16]))
    assert f[1, 2] == 0.0


def test_bottom_up_guard():
    """Bottom-up (choice 4) is skipped exactly when log1p(unvisited) >
    log1p(frontier out-arcs) + log 16, i.e. more than about 16 unvisited
    vertices per frontier arc; otherwise the plain argmin stands.  The
    scheduled slots play no part."""
    w = np.zeros(mlp.NW)
    w[mlp.OFF_ISTD:mlp.OFF_ISTD + 6] = 1.0
    w[mlp.OFF_B3:] = [5, 5, 5, 5, 1, 5, 5, 5, 2]          # bottom-up predicted fastest, choice 8 next
    raw = mlp.raw_features([10, 10, 10], [1e6, 1e4, 1e6], [1000, 1e6, 16e6], [40, 1e9, 40], [3, 3, 3], 4.0)
    assert mlp.choose(w, raw).tolist() == [4, 8, 4]
    # 16e6 + 1 < 16 (1e6 + 1): just inside; 16 (1e6 + 1) + 100 unvisited: outside
    raw2 = mlp.raw_features([10], [1e6], [16e6 + 116], [40], [3], 4.0)
    assert mlp.choose(w, raw2).tolist() == [8]
