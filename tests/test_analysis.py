"""Pins of the roughness analysis (paper_1204_5072_gb300/analysis.py) against
closed forms: exact power laws, a Family-Vicsek scaling form with known
exponents, and the textbook mean / standard error."""
import math

import numpy as np
import pytest

from paper_1204_5072_gb300 import analysis as A


def test_ensemble_mean_and_standard_error_with_missing_points():
    rng = np.random.default_rng(3)
    a = rng.normal(5.0, 2.0, (40, 7))
    a[30:, 5:] = np.nan                       # runs that ended early
    mean, err, n = A.ensemble_mean(a)
    for k in range(7):
        col = a[:, k][np.isfinite(a[:, k])]
        assert n[k] == col.size
        assert mean[k] == pytest.approx(col.mean(), rel=1e-12)
        assert err[k] == pytest.approx(col.std(ddof=1) / math.sqrt(col.size), rel=1e-12)


def test_beta_eff_of_an_exact_power_law_is_the_exponent():
    t = np.unique(np.round(np.logspace(0, 5, 40)))
    for beta in (0.24, 0.5, 0.125):
        tm, b = A.beta_eff(t, 3.0 * t ** (2 * beta))
        assert np.allclose(b, beta, rtol=0, atol=1e-12)
        assert np.allclose(tm, np.sqrt(t[1:] * t[:-1]))


def test_fit_power_recovers_exponent_and_prefactor():
    x = np.array([128, 256, 512, 1024, 2048], np.float64)
    a, c, e = A.fit_power(x, 0.7 * x ** 0.78)
    assert a == pytest.approx(0.78, abs=1e-12) and c == pytest.approx(0.7, rel=1e-12) and e < 1e-10
    # equal weights give the unweighted fit; noisy data lands within a few errors
    a2, c2, _ = A.fit_power(x, 0.7 * x ** 0.78, sigma_y=0.01 * 0.7 * x ** 0.78)
    assert a2 == pytest.approx(a, abs=1e-12) and c2 == pytest.approx(c, rel=1e-12)
    rng = np.random.default_rng(1)
    y = 2.0 * x ** 1.6 * np.exp(rng.normal(0, 0.02, x.size))
    a3, _, e3 = A.fit_power(x, y)
    assert abs(a3 - 1.6) < 4 * e3 + 1e-3


def test_family_vicsek_form_gives_alpha_beta_z():
    """W^2(L, t) = L^(2 alpha) min((t / L^z)^(2 beta), 1) with alpha = beta z:
    growth t^(2 beta), plateau L^(2 alpha), crossover at 0.9^(1/2beta) L^z."""
    beta, z = 0.24, 1.61
    alpha = beta * z
    t = np.unique(np.round(np.logspace(0, 7, 300)))
    Ls = np.array([128, 256, 512, 1024])
    sat, tx = [], []
    for L in Ls:
        w2 = L ** (2 * alpha) * np.minimum((t / L ** z) ** (2 * beta), 1.0)
        b, _ = A.fit_beta(t, w2, 10, 0.5 * L ** z)
        assert b == pytest.approx(beta, abs=1e-9)
        s, _ = A.plateau(t, w2, 2 * L ** z)
        sat.append(s)
        tx.append(A.crossover_time(t, w2, s, frac=0.9))
    a2, _, _ = A.fit_power(Ls, sat)
    zz, _, _ = A.fit_power(Ls, tx)
    assert a2 / 2 == pytest.approx(alpha, abs=1e-9)
    assert zz == pytest.approx(z, abs=1e-9)


def test_crossover_interpolates_in_log_log():
    t = np.array([1, 10, 80, 100, 1000], np.float64)
    w2 = np.minimum(t, 100.0)
    assert A.crossover_time(t, w2, 100.0, frac=0.9) == pytest.approx(90.0, rel=1e-12)
    assert math.isnan(A.crossover_time(t, w2, 1e4))
