"""Pins of the oracle's learned coefficient predictor (CPU only)."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp


def test_bf16_round_on_bit_patterns():
    cases = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -1.5 - 2.0 ** -9,
                      3.0e38, 1.0e-40, 0.0, -0.0], dtype=np.float32)
    got = mlp.bf16_round(cases)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -7, -1.5, 3.0e38, 1.0e-40, 0.0, -0.0], dtype=np.float32)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even -> 1.
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == np.float32(1.0 + 2.0 ** -7)
    assert got[3] == np.float32(-1.5)
    assert np.isnan(mlp.bf16_round(np.array([np.nan], dtype=np.float32)))[0]
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(10000) * 10.0 ** rng.uniform(-6, 6, 10000)).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-12)
    assert mlp.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5)
    u = np.linspace(-3, 3, 13)
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(u), fd, rtol=1e-6, atol=1e-9)


def test_shift_into_current_window():
    y = np.arange(1.0, 6.0)
    np.testing.assert_array_equal(mlp.shift(y, 2), [3.0, 4.0, 5.0, 0.0, 0.0])
    np.testing.assert_array_equal(mlp.shift(y, 5), np.zeros(5))


def test_features_layout():
    M, s = 20, 80
    rng = np.random.default_rng(1)
    W = rng.standard_normal((s, M + 1))
    prev = [rng.standard_normal(M) for _ in range(4)]
    f = mlp.features(W, M, prev)
    assert f.shape == (4 * M + s,)
    np.testing.assert_array_equal(f[:M], mlp.shift(prev[0], 1))
    e = np.zeros(M)
    e[-1], e[-2] = 2.0, -1.0
    np.testing.assert_allclose(f[4 * M:], (W[:, :M] @ e - W[:, M]) / np.linalg.norm(W[:, M]))


def _small_params(rng, dt=np.float64):
    p = mlp.Params(rng.standard_normal((mlp.HID, mlp.IN)).astype(dt) * 0.1,
                   rng.standard_normal(mlp.HID).astype(dt) * 0.1,
                   rng.standard_normal((mlp.HID, mlp.HID)).astype(dt) * 0.06,
                   rng.standard_normal(mlp.HID).astype(dt) * 0.1,
                   rng.standard_normal((mlp.OUT, mlp.HID)).astype(dt) * 0.06,
                   rng.standard_normal(mlp.OUT).astype(dt) * 0.1,
                   rng.standard_normal(mlp.IN).astype(dt), 1.0 + rng.random(mlp.IN).astype(dt),
                   0.5 + rng.random(mlp.OUT).astype(dt))
    return p


def _batch(rng, B):
    F = rng.standard_normal((B, mlp.IN))
    T = rng.standard_normal((B, mlp.OUT))
    Q = rng.standard_normal((B, mlp.OUT, mlp.OUT))
    G = np.einsum("bij,bkj->bik", Q, Q)
    nb = 0.5 + rng.random(B)
    return F, T, G, nb


def test_backward_matches_finite_differences_fp64():
    rng = np.random.default_rng(2)
    p = _small_params(rng)
    F, T, G, nb = _batch(rng, 5)
    loss, grads = mlp.loss_and_grad(p, F, T, G, nb, dtype=np.float64, round_bf16=False)
    h = 1e-6
    names = ["W1", "b1", "W2", "b2", "W3", "b3"]
    for name, g in zip(names, grads):
        arr = getattr(p, name)
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(6)]:
            old = arr[idx]
            arr[idx] = old + h
            lp, _ = mlp.loss_and_grad(p, F, T, G, nb, dtype=np.float64, round_bf16=False)
            arr[idx] = old - h
            lm, _ = mlp.loss_and_grad(p, F, T, G, nb, dtype=np.float64, round_bf16=False)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, idx)


def test_loss_is_zero_at_the_target():
    rng = np.random.default_rng(3)
    p = _small_params(rng)
    F, _, G, nb = _batch(rng, 4)
    y, _ = mlp.forward(p, F, dtype=np.float64, round_bf16=False)
    loss, grads = mlp.loss_and_grad(p, F, y, G, nb, dtype=np.float64, round_bf16=False)
    assert abs(loss) < 1e-20
    assert all(np.abs(g).max() < 1e-12 for g in grads)


def test_adam_reduces_a_quadratic():
    w = [np.array([3.0, -2.0], dtype=np.float32)]
    m = [np.zeros(2, np.float32)]
    v = [np.zeros(2, np.float32)]
    for t in range(1, 3001):
        mlp.adam_update(w, [2 * w[0]], m, v, t, lr=1e-2)
    assert np.abs(w[0]).max() < 1e-2


def test_he_uniform_bounds_and_moments():
    W = mlp.he_uniform(11, 256, 160, 0)
    b = math.sqrt(6 / 160)
    assert W.shape == (256, 160) and np.abs(W).max() <= b
    assert abs(W.mean()) < 0.01 * b and abs(W.var() - b * b / 3) < 0.05 * b * b / 3


def test_loss_is_the_excess_squared_relative_residual():
    """With G = (AX)^T (AX) and the target y* = argmin ||A X y - b||, the loss of
    a prediction y equals (||A X y - b||^2 - ||A X y* - b||^2) / ||b||^2, formed
    here from explicit residuals; so it is never negative, and the net's
    residual is never below the least-squares one."""
    rng = np.random.default_rng(5)
    p = _small_params(rng)
    B, n, M = 3, 60, mlp.OUT
    F = rng.standard_normal((B, mlp.IN))
    y, _ = mlp.forward(p, F, dtype=np.float64, round_bf16=False)
    T, G, nb, excess = [], [], [], []
    for k in range(B):
        AX = rng.standard_normal((n, M))
        b = rng.standard_normal(n)
        ys = np.linalg.lstsq(AX, b, rcond=None)[0]
        T.append(ys)
        G.append(AX.T @ AX)
        nb.append(np.linalg.norm(b))
        r_net = np.linalg.norm(AX @ y[k] - b)
        r_opt = np.linalg.norm(AX @ ys - b)
        assert r_net >= r_opt
        excess.append((r_net ** 2 - r_opt ** 2) / nb[-1] ** 2)
    loss, _ = mlp.loss_and_grad(p, F, np.array(T), np.array(G), np.array(nb), dtype=np.float64,
                                round_bf16=False)
    assert loss == pytest.approx(float(np.mean(excess)), rel=1e-9)
    assert loss > 0
