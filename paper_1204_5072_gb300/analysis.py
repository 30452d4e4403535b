"""Analysis of roughness curves W^2(t) from the engine's ensembles: the
statistics arXiv:1204.5072 defers to its companion papers (Sec. 2.1 defines
W^2; KPZ scaling in 2+1 dimensions, W ~ t^beta before saturation and
W_sat ~ L^alpha, crossover t_x ~ L^z after it).

Post-processing of a few hundred curves of a few dozen points each, so plain
numpy on the host; the curves themselves come from the CUDA kernels
(Batch.w2, Lattice.roughness).

  ensemble_mean(w2)            mean and standard error over realisations
  beta_eff(t, w2)              effective growth exponent between sample times
  fit_beta(t, w2, t0, t1)      log-log fit of W^2 ~ t^(2 beta) on [t0, t1]
  plateau(t, w2, t_sat)        saturated W^2 (mean over t >= t_sat)
  crossover_time(t, w2, ...)   first time W^2 reaches a fraction of its plateau
  fit_power(x, y)              exponent and prefactor of y ~ x^a (least squares
                               in log-log), used for W^2_sat ~ L^(2 alpha) and
                               t_x ~ L^z
"""
from __future__ import annotations

import math

import numpy as np


def ensemble_mean(w2):
    """Mean, standard error and count over realisations (axis 0) of a
    (n_realisations, n_times) array; NaN entries (times past a run's end)
    are left out."""
    a = np.asarray(w2, np.float64)
    n = np.sum(np.isfinite(a), axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.nansum(a, axis=0) / n
        dev = np.where(np.isfinite(a), a - mean, 0.0)
        var = np.sum(dev * dev, axis=0) / (n - 1)
        err = np.sqrt(var / n)
    mean = np.where(n > 0, mean, np.nan)
    err = np.where(n > 1, err, np.nan)
    return mean, err, n


def beta_eff(t, w2):
    """Effective exponent between consecutive sample times: with W ~ t^beta,
    beta_eff = (ln W^2(t_{k+1}) - ln W^2(t_k)) / (2 (ln t_{k+1} - ln t_k)),
    reported at the geometric mean time. Times <= 0 are skipped."""
    t = np.asarray(t, np.float64)
    w = np.asarray(w2, np.float64)
    keep = (t > 0) & np.isfinite(w) & (w > 0)
    t, w = t[keep], w[keep]
    lt, lw = np.log(t), np.log(w)
    tm = np.sqrt(t[1:] * t[:-1])
    return tm, (lw[1:] - lw[:-1]) / (2.0 * (lt[1:] - lt[:-1]))


def fit_power(x, y, sigma_y=None):
    """Least-squares fit of ln y = a ln x + ln c; returns (a, c, err_a). With
    sigma_y (standard errors of y) the points are weighted by (y / sigma_y)^2,
    the inverse variance of ln y; err_a is then the fit's standard error."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    lx, ly = np.log(x), np.log(y)
    if sigma_y is None:
        wts = np.ones_like(lx)
    else:
        s = np.asarray(sigma_y, np.float64) / y
        wts = 1.0 / np.maximum(s, 1e-300) ** 2
    W = wts.sum()
    mx, my = (wts * lx).sum() / W, (wts * ly).sum() / W
    sxx = (wts * (lx - mx) ** 2).sum()
    a = (wts * (lx - mx) * (ly - my)).sum() / sxx
    c = math.exp(my - a * mx)
    if sigma_y is not None:
        err = math.sqrt(1.0 / sxx)
    elif len(x) > 2:
        res = ly - (a * lx + my - a * mx)
        err = math.sqrt((res * res).sum() / (len(x) - 2) / sxx)
    else:
        err = float("nan")
    return a, c, err


def fit_beta(t, w2, t0, t1, err=None):
    """Growth exponent beta from W^2 ~ t^(2 beta) on t0 <= t <= t1; returns
    (beta, err_beta)."""
    t = np.asarray(t, np.float64)
    w = np.asarray(w2, np.float64)
    m = (t >= t0) & (t <= t1) & np.isfinite(w) & (w > 0)
    a, _, e = fit_power(t[m], w[m], None if err is None else np.asarray(err)[m])
    return a / 2.0, e / 2.0


def plateau(t, w2, t_sat, err=None):
    """Saturated W^2: the mean of the curve over t >= t_sat, and its standard
    error (from the spread of those points, or from err if given)."""
    t = np.asarray(t, np.float64)
    w = np.asarray(w2, np.float64)
    m = (t >= t_sat) & np.isfinite(w)
    if not m.any():
        return float("nan"), float("nan")
    v = w[m]
    if err is not None:
        e = np.asarray(err, np.float64)[m]
        return float(v.mean()), float(np.sqrt((e * e).sum()) / m.sum())
    return float(v.mean()), float(v.std(ddof=1) / math.sqrt(m.sum())) if m.sum() > 1 else float("nan")


def crossover_time(t, w2, w2_sat, frac=0.9):
    """First sample time at which W^2 reaches frac * w2_sat, interpolated
    linearly in (ln t, ln W^2) between the bracketing samples."""
    t = np.asarray(t, np.float64)
    w = np.asarray(w2, np.float64)
    target = frac * w2_sat
    for k in range(1, len(t)):
        if t[k - 1] > 0 and w[k - 1] < target <= w[k]:
            u = (math.log(target) - math.log(w[k - 1])) / (math.log(w[k]) - math.log(w[k - 1]))
            return float(math.exp(math.log(t[k - 1]) + u * (math.log(t[k]) - math.log(t[k - 1]))))
    return float("nan")
