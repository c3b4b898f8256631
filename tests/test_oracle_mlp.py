"""Pins for the float64 network reference (no GPU): finite differences,
closed forms, bfloat16 rounding against torch's conversion, and the
feature histogram on hand-worked values."""
import numpy as np
import pytest
import torch

from oracle import mlp


def _params(rng, scale=0.3):
    W1 = rng.normal(0, scale, (mlp.N_HIDDEN, mlp.N_FEATURES))
    b1 = rng.normal(0, scale, mlp.N_HIDDEN)
    w2 = rng.normal(0, scale, mlp.N_HIDDEN)
    b2 = float(rng.normal())
    return W1, b1, w2, b2


@pytest.mark.parametrize("seed", range(3))
def test_gradients_match_central_differences(seed):
    rng = np.random.default_rng(seed)
    W1, b1, w2, b2 = _params(rng)
    x = rng.normal(0, 1, (7, mlp.N_FEATURES))
    t = rng.normal(3, 2, 7)
    y, cache = mlp.forward(x, W1, b1, w2, b2)
    g = mlp.backward(y, t, cache, W1, w2)

    def L(W1_, b1_, w2_, b2_):
        return mlp.loss(mlp.forward(x, W1_, b1_, w2_, b2_)[0], t)

    h = 1e-6
    for idx in [(0, 0), (5, 17), (127, 63), (64, 1)]:
        Wp, Wm = W1.copy(), W1.copy()
        Wp[idx] += h
        Wm[idx] -= h
        fd = (L(Wp, b1, w2, b2) - L(Wm, b1, w2, b2)) / (2 * h)
        assert abs(fd - g[0][idx]) <= 1e-6 * max(1.0, abs(fd))
    for j in [0, 31, 127]:
        bp, bm = b1.copy(), b1.copy()
        bp[j] += h
        bm[j] -= h
        fd = (L(W1, bp, w2, b2) - L(W1, bm, w2, b2)) / (2 * h)
        assert abs(fd - g[1][j]) <= 1e-6 * max(1.0, abs(fd))
        wp, wm = w2.copy(), w2.copy()
        wp[j] += h
        wm[j] -= h
        fd = (L(W1, b1, wp, b2) - L(W1, b1, wm, b2)) / (2 * h)
        assert abs(fd - g[2][j]) <= 1e-6 * max(1.0, abs(fd))
    fd = (L(W1, b1, w2, b2 + h) - L(W1, b1, w2, b2 - h)) / (2 * h)
    assert abs(fd - g[3]) <= 1e-6 * max(1.0, abs(fd))


def test_closed_form_constant_hidden_layer():
    # W1 = 0: every hidden unit equals relu(b1), so y = w2 . relu(b1) + b2
    rng = np.random.default_rng(1)
    b1 = rng.normal(size=mlp.N_HIDDEN)
    w2 = rng.normal(size=mlp.N_HIDDEN)
    x = rng.normal(size=(4, mlp.N_FEATURES))
    y, _ = mlp.forward(x, np.zeros((mlp.N_HIDDEN, mlp.N_FEATURES)), b1, w2, 0.5)
    assert np.allclose(y, np.dot(w2, np.maximum(b1, 0)) + 0.5, rtol=0, atol=1e-12)
    # loss gradient w.r.t. b2 is mean(y - t)
    t = np.arange(4.0)
    g = mlp.backward(y, t, mlp.forward(x, np.zeros((128, 64)), b1, w2, 0.5)[1],
                     np.zeros((128, 64)), w2)
    assert np.isclose(g[3], np.mean(y - t))
    # units with negative pre-activation pass no gradient to their weights
    dead = b1 < 0
    assert np.all(g[0][dead] == 0) and np.all(g[1][dead] == 0)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([0.3, -2.0, 1e-3])
    theta, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), step=1, lr=0.01, eps=0.0)
    assert np.allclose(theta, -0.01 * np.sign(g))
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_bf16_rounding_hand_values_and_torch():
    one = 1.0
    cases = {one: one, one + 2 ** -8: one, one + 3 * 2 ** -8: one + 2 ** -6,
             -(one + 2 ** -7): -(one + 2 ** -7), 0.0: 0.0}
    for a, want in cases.items():
        assert float(mlp.bf16_round(np.float32(a))) == want
    rng = np.random.default_rng(2)
    x = (rng.normal(size=10000) * 10.0 ** rng.integers(-8, 8, 10000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_feature_histogram_hand_values():
    df = np.array([0, 1, 2, 3, 4, 1023, 1024, 2 ** 40])
    x = mlp.features(df, np.array([0, 8]))
    want = np.zeros(64)
    for b in (0, 1, 2, 2, 3, 10, 11, 41):
        want[b] += 1
    assert np.array_equal(x[0], want * mlp.FEATURE_SCALE)
    assert np.array_equal(mlp.floor_log2(np.array([1, 2, 3, 4, 7, 8, 2 ** 33 - 1])),
                          [0, 1, 1, 2, 2, 3, 32])
