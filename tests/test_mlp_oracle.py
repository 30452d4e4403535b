"""Pins of the MLP oracle (oracle/mlp_oracle.py), the reference the engine's
surrogate kernels are checked against (the paper has no learned part):
gradients against central finite differences, bfloat16 rounding and GELU
against library implementations, Adam's first step against its closed form."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def _params(seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(M.N_PARAMS) * scale * 0.2).astype(np.float32)


def test_parameter_count():
    assert M.N_PARAMS == 33793


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = _params(1).astype(np.float64)
    x = rng.standard_normal((7, 4))
    t = rng.standard_normal(7)
    loss, g = M.loss_and_grad(theta, x, t, bf16=False)
    idx = rng.choice(M.N_PARAMS, 40, replace=False)
    idx = np.concatenate([idx, [0, 511, 512, 33791, 33792]])   # W1, b1 ends, w4, b4
    h = 1e-6
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        fd = (M.loss_and_grad(tp, x, t, bf16=False)[0] - M.loss_and_grad(tm, x, t, bf16=False)[0]) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-8), i


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.standard_normal(5000).astype(np.float32) * 10.0 ** rng.integers(-8, 8, 5000),
                        np.array([1.0, 1.00390625, 1.01171875, -2.5, 0.0, 65504.0], np.float32)])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(M.bf16_round(v), ref)


def test_gelu_matches_torch():
    torch = pytest.importorskip("torch")
    z = np.linspace(-6, 6, 2001)
    ref = torch.nn.functional.gelu(torch.from_numpy(z), approximate="none").numpy()
    assert np.allclose(M.gelu(z), ref, rtol=1e-12, atol=1e-14)
    # derivative by central differences
    h = 1e-6
    assert np.allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), atol=1e-7)


def test_adam_first_step_moves_by_the_learning_rate():
    theta = _params(3)
    g = np.random.default_rng(4).standard_normal(M.N_PARAMS)
    new, m, v = M.adam_step(theta, np.zeros_like(g), np.zeros_like(g), g, 1, lr=1e-3)
    # bias-corrected first step: m_hat = g, v_hat = g^2, so the step is lr g / (|g| + eps)
    assert np.allclose(new - theta, -1e-3 * g / (np.abs(g) + 1e-8), atol=1e-7)
