"""Roughness analysis on ensembles from the batched engine: the KPZ case
(p = 1, q = 0) grows and saturates with exponents near the 2+1-dimensional
KPZ values (beta ~ 0.24, alpha ~ 0.39, z ~ 1.61; small L bias them), and the
lambda = 0 case (p = q, Edwards-Wilkinson class) saturates with a far smaller
alpha (logarithmic in L)."""
import numpy as np
import pytest

from paper_1204_5072_gb300 import analysis as A
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu
N = 32


def _curves(eng, p, q, Ls, T_of):
    specs = [(L, p, q, 11, k, int(T_of(L))) for L in Ls for k in range(N)]
    b = eng.Batch(specs, n_samples=80, run=4)
    b.run()
    t = b.times().astype(np.float64)
    w = b.w2()
    b.close()
    return t, [A.ensemble_mean(w[N * i: N * (i + 1)])[:2] for i in range(len(Ls))]


def test_kpz_exponents_from_batched_ensembles():
    eng = engine()
    Ls = [128, 256, 512]
    t, curves = _curves(eng, 1.0, 0.0, Ls, lambda L: 6 * L ** 1.6)
    sat, sat_e, tx = [], [], []
    for L, (m, e) in zip(Ls, curves):
        s, se = A.plateau(t, m, 2.5 * L ** 1.6, err=e)
        sat.append(s)
        sat_e.append(se)
        tx.append(A.crossover_time(t, m, s, frac=0.5))
    beta, beta_err = A.fit_beta(t, curves[-1][0], 20, 0.05 * 512 ** 1.6, err=curves[-1][1])
    alpha = A.fit_power(Ls, sat, sigma_y=sat_e)[0] / 2
    z = A.fit_power(Ls, tx)[0]
    assert 0.19 < beta < 0.26, (beta, beta_err)
    assert sat[0] < sat[1] < sat[2]
    assert 0.33 < alpha < 0.48, alpha
    assert 1.35 < z < 2.2, z
    # effective exponent before saturation stays in the KPZ range, not the EW one (0)
    tm, be = A.beta_eff(t, curves[-1][0])
    mid = (tm > 50) & (tm < 0.05 * 512 ** 1.6)
    assert np.all((be[mid] > 0.15) & (be[mid] < 0.3)), be[mid]


def test_edwards_wilkinson_case_saturates_logarithmically():
    eng = engine()
    Ls = [128, 256]
    t, curves = _curves(eng, 0.5, 0.5, Ls, lambda L: 3 * L ** 2)
    sat = [A.plateau(t, m, 1.5 * L ** 2, err=e)[0] for L, (m, e) in zip(Ls, curves)]
    alpha = A.fit_power(Ls, sat)[0] / 2
    assert sat[0] < sat[1]
    assert 0.0 < alpha < 0.2, (alpha, sat)


def test_edwards_wilkinson_to_kpz_crossover_in_lambda():
    """The nonlinearity lambda = 2p/(p+q) - 1 (Sec. 2.1) with p + q = 1:
    lambda = 0 is the Edwards-Wilkinson class (W^2 ~ ln t in 2+1 dimensions,
    an effective beta near 0.05 over t in [20, 1100]), lambda = 1 the KPZ
    class (beta ~ 0.24); in between the growth crosses over from the first to
    the second, later for smaller lambda, so the effective exponent over a
    fixed window rises monotonically with lambda (measured at L = 512: 0.062,
    0.068, 0.096, 0.162, 0.215 for lambda = 0, 0.25, 0.5, 0.75, 1)."""
    eng = engine()
    L, T, n = 512, 1100, 16
    betas = []
    for lam in (0.0, 0.25, 0.5, 0.75, 1.0):
        p = (1 + lam) / 2
        b = eng.Batch([(L, p, 1 - p, 21, k, T) for k in range(n)], n_samples=60, run=4)
        b.run()
        t = b.times().astype(np.float64)
        w = b.w2()
        b.close()
        m, e = A.ensemble_mean(w)[:2]
        betas.append(A.fit_beta(t, m, 20, T, err=e)[0])
    assert all(b1 < b2 for b1, b2 in zip(betas, betas[1:])), betas
    assert 0.03 < betas[0] < 0.09 and 0.19 < betas[-1] < 0.26, betas
    assert betas[2] - betas[0] > 0.015 and betas[-1] - betas[2] > 0.06, betas
