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
