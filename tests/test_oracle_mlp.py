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


# ---- Adam (Kingma and Ba, 2015): closed forms that a mistake in the update fails ----

def _adam_run(grads, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, w0=0.0):
    """Apply adam_update to one float64 scalar parameter for the gradient
    sequence `grads`; returns the parameter after every step."""
    w = [np.array([w0], dtype=np.float64)]
    m = [np.zeros(1)]
    v = [np.zeros(1)]
    out = []
    for t, g in enumerate(grads, start=1):
        mlp.adam_update(w, [np.array([g])], m, v, t, lr=lr, b1=b1, b2=b2, eps=eps)
        out.append(float(w[0][0]))
    return out


@pytest.mark.parametrize("g", [3.0, -0.25, 1e-8, -2e-9, 1e3])
def test_adam_first_step_is_lr_times_g_over_abs_g_plus_eps(g):
    """From zero moments the bias-corrected estimates after one step are g and
    g^2 exactly, so the step is lr g / (|g| + eps).  Fails without the bias
    correction (the step becomes about 3.16 lr sign(g)), with eps under the
    square root (tiny g: g / sqrt(g^2 + eps) is far from g / (|g| + eps)), or
    with a sign step lr sign(g)."""
    lr, eps = 1e-3, 1e-8
    w1 = _adam_run([g], lr=lr, eps=eps)[0]
    assert w1 == pytest.approx(-lr * g / (abs(g) + eps), rel=1e-12)


@pytest.mark.parametrize("g", [0.7, -5.0, 1e-8])
def test_adam_constant_gradient_moves_at_a_constant_rate(g):
    """A constant gradient keeps both bias-corrected moments exact (m_hat = g,
    v_hat = g^2: the correction divides out the geometric weights), so every
    step is the same lr g / (|g| + eps) and w_T = -T lr g / (|g| + eps).
    Fails if beta1 and beta2 are swapped in either the decay or the correction."""
    lr, eps, T = 1e-2, 1e-8, 40
    ws = _adam_run([g] * T, lr=lr, eps=eps)
    step = lr * g / (abs(g) + eps)
    for t, w in enumerate(ws, start=1):
        assert w == pytest.approx(-t * step, rel=1e-10)


def test_adam_alternating_gradient_closed_form():
    """g_t = (-1)^t c.  Then v_hat_t = c^2 (g^2 is constant) and, summing the
    geometric series of the first moment,
        m_hat_t = c (-1)^t (1 - b1) (1 - (-b1)^t) / ((1 + b1) (1 - b1^t)),
    so the step at t is lr m_hat_t / (|c| + eps).  Pins beta1 on the first
    moment and beta2 on the second: exchanging them, or decaying the second
    moment with beta1, changes v_hat away from c^2."""
    lr, b1, b2, eps, c, T = 1e-2, 0.9, 0.999, 1e-8, 0.5, 12
    ws = _adam_run([(-1) ** t * c for t in range(1, T + 1)], lr=lr, b1=b1, b2=b2, eps=eps)
    prev = 0.0
    for t, w in enumerate(ws, start=1):
        mhat = c * (-1) ** t * (1 - b1) * (1 - (-b1) ** t) / ((1 + b1) * (1 - b1 ** t))
        assert (w - prev) == pytest.approx(-lr * mhat / (abs(c) + eps), rel=1e-9, abs=1e-15)
        prev = w
    # The first step is a full lr step against g_1 = -c; the second, against +c,
    # is only a fraction of lr because the first moment still remembers -c.
    assert ws[0] == pytest.approx(lr * c / (c + eps), rel=1e-12)
    assert 0 < ws[0] - ws[1] < 0.1 * lr


def test_adam_second_step_uses_normalised_moving_averages():
    """After two steps with gradients a then c, each bias-corrected moment is
    the average of the two samples with weights (beta, 1) normalised to sum 1:
    m_hat = (b1 a + c) / (1 + b1) and v_hat = (b2 a^2 + c^2) / (1 + b2).
    Gradients of different magnitude separate beta1 from beta2 in the second
    moment (decaying and correcting it with beta1 fails here)."""
    lr, b1, b2, eps, a, c = 1e-3, 0.9, 0.999, 1e-8, 1.0, 3.0
    w1, w2 = _adam_run([a, c], lr=lr, b1=b1, b2=b2, eps=eps)
    mhat = (b1 * a + c) / (1 + b1)
    vhat = (b2 * a * a + c * c) / (1 + b2)
    assert w2 - w1 == pytest.approx(-lr * mhat / (math.sqrt(vhat) + eps), rel=1e-9)


def test_adam_float32_arrays_update_in_place():
    """The update works in place on float32 parameter arrays (the GPU keeps
    FP32 master weights) and leaves their dtype unchanged."""
    w = [np.array([1.0, -1.0], dtype=np.float32)]
    m = [np.zeros(2, np.float32)]
    v = [np.zeros(2, np.float32)]
    ref = w[0]
    mlp.adam_update(w, [np.array([0.5, -0.5], np.float32)], m, v, 1, lr=0.1)
    assert w[0] is ref and w[0].dtype == np.float32
    assert np.allclose(w[0], [0.9, -0.9], rtol=1e-6)


# ---- He-uniform initialisation: stream layout and distribution ----

def test_he_uniform_stream_layout():
    """Entry (i, j) of a fan_out x fan_in block takes SplitMix64 output
    stream_offset + 1 + i fan_in + j: a block equals the rows of a longer
    draw, row i of it equals row 0 of the draw offset by i fan_in, and the
    scale is sqrt(6 / fan_in) on a common unit draw."""
    W = mlp.he_uniform(7, 6, 10, 100)
    flat = mlp.he_uniform(7, 1, 60, 100)                   # same outputs, other bound
    scale = math.sqrt(6 / 10) / math.sqrt(6 / 60)
    assert np.allclose(W.reshape(-1), flat.reshape(-1) * scale, rtol=1e-6, atol=0)
    for i in range(6):
        row = mlp.he_uniform(7, 1, 10, 100 + 10 * i)
        assert np.array_equal(W[i], row[0])
    assert not np.array_equal(mlp.he_uniform(8, 6, 10, 100), W)   # the seed matters


def test_he_uniform_is_uniform_on_its_interval():
    """Kolmogorov-Smirnov against U(-b, b), b = sqrt(6 / fan_in), on 40,960
    draws; the variance is b^2 / 3 = 2 / fan_in (He et al., 2015)."""
    from scipy import stats
    fan_in = 160
    W = mlp.he_uniform(123, 256, fan_in, 0).astype(np.float64).reshape(-1)
    b = math.sqrt(6 / fan_in)
    assert stats.kstest(W, stats.uniform(loc=-b, scale=2 * b).cdf).pvalue > 1e-3
    assert W.var() == pytest.approx(2 / fan_in, rel=0.03)
