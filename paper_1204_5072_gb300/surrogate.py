"""Learned surrogate of the roughness curve W^2(t; L, p, q) and its use by the
ensemble batcher (not part of the paper; the paper runs every realisation
for a fixed time, Sec. 4).

The network (kpz_mlp_* in include/kpz.h) maps scaled features
(log2 L, log t, p, q) to log W^2. It is trained on the W^2 curves the batched
simulator produces, by the library's own forward, backward and Adam kernels.
Its curves give the saturation time t_x(L, p, q): the time the predicted
log W^2 comes within `sat_tol` of its plateau. The batcher can then run each
realisation for `factor * t_x` sweeps instead of a fixed rule such as
4 L^1.6; the plain simulation stays the fallback and the measure of the error.
"""
from __future__ import annotations

import ctypes
import math
import warnings

import numpy as np

from . import _lib
from ._lib import _ptr, check, load

N_PARAMS = 33793
WIDTH = 128


def _bind(L):
    if getattr(L, "_mlp_bound", False):
        return
    c = ctypes
    vp = c.c_void_p
    L.kpz_mlp_create.argtypes = [c.POINTER(vp), vp, vp]
    L.kpz_mlp_params.argtypes = [vp, vp]
    L.kpz_mlp_predict.argtypes = [vp, vp, c.c_uint32, vp]
    L.kpz_mlp_loss_grad.argtypes = [vp, vp, vp, c.c_uint32, c.POINTER(c.c_float), vp]
    L.kpz_mlp_train.argtypes = [vp, vp, vp, c.c_uint32, vp, c.c_uint32, c.c_uint32, c.c_float,
                                c.POINTER(c.c_float)]
    L.kpz_mlp_free.argtypes = [vp]
    L.kpz_mlp_free.restype = None
    for fn in ("kpz_mlp_create", "kpz_mlp_params", "kpz_mlp_predict", "kpz_mlp_loss_grad", "kpz_mlp_train"):
        getattr(L, fn).restype = c.c_int
    L._mlp_bound = True


def init_params(seed: int = 0) -> np.ndarray:
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in [(4, WIDTH), (WIDTH, WIDTH), (WIDTH, WIDTH)]:
        a = math.sqrt(6.0 / fan_in)
        parts += [rng.uniform(-a, a, (fan_out, fan_in)).ravel(), np.zeros(fan_out)]
    parts += [rng.uniform(-math.sqrt(3.0 / WIDTH), math.sqrt(3.0 / WIDTH), WIDTH), np.zeros(1)]
    out = np.concatenate(parts).astype(np.float32)
    assert out.size == N_PARAMS
    return out


class MLP:
    """The engine's MLP (bfloat16 weights, float32 arithmetic) through the C ABI."""

    def __init__(self, params: np.ndarray | None = None, seed: int = 0, stream=None):
        lib = load()
        _bind(lib)
        p = np.ascontiguousarray(init_params(seed) if params is None else params, np.float32)
        assert p.size == N_PARAMS
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        self._m = ctypes.c_void_p()
        check(lib.kpz_mlp_create(ctypes.byref(self._m), _ptr(p), ctypes.c_void_p(stream or 0)))

    def params(self) -> np.ndarray:
        out = np.zeros(N_PARAMS, np.float32)
        check(load().kpz_mlp_params(self._m, _ptr(out)))
        return out

    def predict(self, x: np.ndarray) -> np.ndarray:
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 4)
        y = np.zeros(len(x), np.float32)
        check(load().kpz_mlp_predict(self._m, _ptr(x), len(x), _ptr(y)))
        return y

    def loss_grad(self, x: np.ndarray, t: np.ndarray):
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, np.float32)
        g = np.zeros(N_PARAMS, np.float32)
        loss = ctypes.c_float()
        check(load().kpz_mlp_loss_grad(self._m, _ptr(x), _ptr(t), len(x), ctypes.byref(loss), _ptr(g)))
        return float(loss.value), g

    def train(self, x, t, epochs=200, batch=512, lr=1e-3, seed=0, lr_final=None) -> float:
        """Adam over shuffled minibatches (one upload per epoch); returns the
        last minibatch loss. With lr_final the rate decays geometrically."""
        x = np.ascontiguousarray(x, np.float32).reshape(-1, 4)
        t = np.ascontiguousarray(t, np.float32)
        n = len(x)
        rng = np.random.default_rng(seed)
        steps = max(1, n // batch)
        last = float("nan")
        for e in range(epochs):
            rate = lr if lr_final is None else lr * (lr_final / lr) ** (e / max(1, epochs - 1))
            order = rng.permutation(n)[: steps * batch].astype(np.uint32)
            if len(order) < steps * batch:
                order = np.resize(order, steps * batch).astype(np.uint32)
            out = ctypes.c_float()
            check(load().kpz_mlp_train(self._m, _ptr(x), _ptr(t), n, _ptr(order), steps, batch,
                                       ctypes.c_float(rate), ctypes.byref(out)))
            last = float(out.value)
        return last

    def close(self):
        if getattr(self, "_m", None):
            load().kpz_mlp_free(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------- #
def features(L, t, p, q) -> np.ndarray:
    """Scaled inputs of the network: (log2 L, log t, p, q) centred on the
    ranges of the batched ensembles (L 2^7..2^13, t 1..1e5, p, q in [0, 1])."""
    L, t, p, q = (np.asarray(v, np.float64) for v in np.broadcast_arrays(L, t, p, q))
    f = np.stack([(np.log2(L) - 10.0) / 2.0, (np.log(np.maximum(t, 1.0)) - 6.0) / 3.0,
                  (p - 0.75) / 0.2, (q - 0.25) / 0.2], axis=-1)
    return f.astype(np.float32)


def ensemble_curves(specs, times, w2, p_bin=0.05):
    """Ensemble means of the realisations' W^2 curves: realisations of one L
    whose p falls in the same bin of width p_bin are averaged (at every time
    all of them reached), and the mean curve is placed at their mean (p, q).
    The network is then fitted to log of the ensemble mean, which is the
    quantity it is judged on; fitted to single realisations it would learn
    the mean of log W^2, lower by about half the variance of log W^2 (a few
    per cent where a realisation's W^2 fluctuates by 20 %). p_bin = 0 keeps
    every curve as it is (for curves that are ensemble means already)."""
    groups = {}
    for k, (L, p, q, _seed, _sample, n) in enumerate(specs):
        key = (L, int(p // p_bin)) if p_bin > 0 else (L, k)
        groups.setdefault(key, []).append(k)
    out_specs, out_w2 = [], []
    for key in sorted(groups):
        ks = groups[key]
        n = min(specs[k][5] for k in ks)
        with warnings.catch_warnings():   # times past every run's end: all-NaN columns
            warnings.simplefilter("ignore", RuntimeWarning)
            m = np.nanmean(np.asarray(w2, np.float64)[ks], axis=0)
        p = float(np.mean([specs[k][1] for k in ks]))
        q = float(np.mean([specs[k][2] for k in ks]))
        out_specs.append((key[0], p, q, 0, 0, n))
        out_w2.append(m)
    return out_specs, np.array(out_w2)


def curves_to_samples(specs, times, w2):
    """Training rows from W^2 curves: every (curve, time > 0) with a W^2."""
    X, Y = [], []
    for (L, p, q, _seed, _sample, n), row in zip(specs, w2):
        for t, w in zip(times, row):
            if 0 < t <= n and np.isfinite(w) and w > 0:
                X.append((L, t, p, q))
                Y.append(math.log(w))
    X = np.array(X, np.float64)
    return features(X[:, 0], X[:, 1], X[:, 2], X[:, 3]), np.array(Y, np.float32)


class Surrogate:
    """Trained network plus the curve and saturation-time queries the batcher uses."""

    def __init__(self, mlp: MLP):
        self.mlp = mlp

    @classmethod
    def fit(cls, specs, times, w2, epochs=300, batch=512, lr=3e-3, seed=0, p_bin=0.0) -> "Surrogate":
        """Train on the W^2 curves of the realisations `specs` (L, p, q, seed,
        sample, n) sampled at `times`; with p_bin > 0 realisations are first
        averaged into ensemble means (ensemble_curves)."""
        if p_bin > 0:
            specs, w2 = ensemble_curves(specs, times, w2, p_bin)
        x, y = curves_to_samples(specs, times, w2)
        m = MLP(seed=seed)
        m.train(x, y, epochs=epochs, batch=batch, lr=lr, seed=seed, lr_final=lr / 30)
        return cls(m)

    def w2(self, L, t, p, q) -> np.ndarray:
        """Predicted W^2 at the given (broadcast) points."""
        return np.exp(self.mlp.predict(features(L, t, p, q)).astype(np.float64))

    def t_sat(self, L, p, q, t_max=1e5, sat_tol=0.1, n=256) -> float:
        """Saturation time: first t (log grid up to t_max) at which the
        predicted log W^2 is within sat_tol of its maximum over the grid."""
        t = np.unique(np.round(np.logspace(0, math.log10(t_max), n)))
        lw = np.log(self.w2(L, t, p, q))
        plateau = lw.max()
        return float(t[np.argmax(lw >= plateau - sat_tol)])

    def plan(self, specs, factor=2.0, cap=100_000, t_max=1e5):
        """Run lengths min(cap, factor * t_sat) for (L, p, q, seed, sample, n) specs."""
        out = []
        for (L, p, q, seed, sample, _n) in specs:
            T = int(min(cap, math.ceil(factor * self.t_sat(L, p, q, t_max=t_max))))
            out.append((L, p, q, seed, sample, max(T, 1)))
        return out

    def planned_batch(self, specs, factor=2.0, cap=100_000, t_max=1e5, **batch_opts):
        """The realisations (L, p, q, seed, sample, n) as one persistent batch
        (kpz_batch_create) with the planned run lengths min(cap, factor t_x)
        instead of n; the batch queues them longest planned run first, so the
        realisations the surrogate predicts to be the most expensive start
        first and short ones fill in behind them. Returns (Batch, planned specs)."""
        from ._lib import Batch
        planned = self.plan(specs, factor=factor, cap=cap, t_max=t_max)
        return Batch(planned, **batch_opts), planned

    def t_x_fit(self, Ls, p, q, t_max=1e5):
        """Saturation times t_x(L) predicted for the sizes Ls and the exponent
        z of a power-law fit t_x ~ L^z over them (the KPZ class has z ~ 1.6)."""
        tx = np.array([self.t_sat(L, p, q, t_max=t_max) for L in Ls])
        z = float(np.polyfit(np.log(np.asarray(Ls, float)), np.log(tx), 1)[0]) if len(Ls) > 1 else float("nan")
        return tx, z

    def close(self):
        self.mlp.close()
