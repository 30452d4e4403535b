"""The surrogate's hand-written MLP kernels against the float64 oracle
(oracle/mlp_oracle.py: bfloat16-rounded weights, GELU, mean squared error,
Adam). The engine accumulates in float32, so values agree to a tolerance."""
import numpy as np
import pytest

from oracle import mlp_oracle as M
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    engine()
    from paper_1204_5072_gb300 import surrogate
    return surrogate


def _data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, 4)).astype(np.float32)
    t = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 3] ** 2).astype(np.float32)
    return x, t


def test_forward_matches_oracle(S):
    theta = S.init_params(1)
    x, _ = _data(1000, 2)
    m = S.MLP(theta)
    y = m.predict(x)
    ref = M.forward(theta, x)
    assert np.max(np.abs(y - ref)) <= 2e-4 * np.max(np.abs(ref)) + 1e-5
    m.close()


def test_gradient_matches_oracle(S):
    theta = S.init_params(3)
    x, t = _data(700, 4)          # several tiles and a ragged last tile
    m = S.MLP(theta)
    loss, g = m.loss_grad(x, t)
    rl, rg = M.loss_and_grad(theta, x, t)
    assert loss == pytest.approx(rl, rel=1e-4)
    for name, shape in M.SHAPES:
        a = M.unflatten(g)[name].ravel()
        b = M.unflatten(rg)[name].ravel()
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b) + 1e-7, name
    m.close()


def test_adam_trajectory_matches_oracle(S):
    theta0 = S.init_params(5)
    x, t = _data(512, 6)
    m = S.MLP(theta0)
    order = np.arange(512, dtype=np.uint32)
    import ctypes
    from paper_1204_5072_gb300._lib import _ptr, load
    lr = 1e-3
    out = ctypes.c_float()
    assert load().kpz_mlp_train(m._m, _ptr(x), _ptr(t), 512, _ptr(np.tile(order, 4)), 4, 512,
                                ctypes.c_float(lr), ctypes.byref(out)) == 0
    got = m.params()
    th, mm, vv = theta0.copy(), np.zeros(M.N_PARAMS), np.zeros(M.N_PARAMS)
    for step in range(1, 5):
        _, g = M.loss_and_grad(th, x, t)
        th, mm, vv = M.adam_step(th, mm, vv, g, step, lr)
    moved = np.linalg.norm(th - theta0)
    assert np.linalg.norm(got - th) <= 0.05 * moved
    m.close()


def test_training_is_deterministic_and_learns(S):
    x, t = _data(4096, 7)
    res = []
    for _ in range(2):
        m = S.MLP(S.init_params(8))
        l0, _ = m.loss_grad(x, t)
        m.train(x, t, epochs=30, batch=256, lr=3e-3, seed=9)
        l1, _ = m.loss_grad(x, t)
        res.append((m.params(), l0, l1))
        m.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][2] < 0.2 * res[0][1]
