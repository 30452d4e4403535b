"""The L = 4096 workload as an ensemble: 16 realisations (seeds 1..16) to 10^4
sweeps at (p, q) = (1, 0) and (0.95, 0.05), each rate in one persistent batch.

* Realisation 1 of the batch equals the oracle's stored trajectory
  (tests/golden/l4096_*.txt) at every W^2 sampling time: exact S1, S2, and the
  final height of site (0,0).
* The growth exponent of the ensemble mean W^2(t) ~ t^(2 beta) over
  t in [100, 10^4] (far below saturation at L = 4096) is the 2+1-dimensional
  KPZ value at both rates (lambda = 1 and 0.9).
* Random-sequential updates without decomposition (exact, on the GPU) at
  L = 512 give the same beta over t in [50, 2000] as the decomposed dynamics.
"""
import numpy as np
import pytest

from paper_1204_5072_gb300 import analysis as A
from synth import inputs as I
from tests.gpu_util import engine
from tests.test_gpu_fullsize import _golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    return engine()


@pytest.mark.parametrize("w", ["L4096_P1", "L4096_P095"])
def test_ensemble_member_matches_oracle_and_beta_is_kpz(eng, w):
    W = getattr(I, w)
    specs = [(W.L, W.p, W.q, seed, W.sample, W.mcs) for seed in range(1, 17)]
    b = eng.Batch(specs, n_samples=64)
    b.run()
    t = b.times().astype(np.int64)
    s1, s2, h00 = b.sums()
    w2 = b.w2()
    b.close()
    rec = _golden(w)
    assert list(t) == [r[0] for r in rec]
    for k, (tt, g1, g2, _, _) in enumerate(rec):
        assert (int(s1[0, k]), int(s2[0, k])) == (g1, g2), (w, tt)
    assert int(h00[0]) == rec[-1][3]
    m, e = A.ensemble_mean(w2)[:2]
    beta, beta_err = A.fit_beta(t.astype(np.float64), m, 100, W.mcs, err=e)
    assert 0.21 < beta < 0.26, (w, beta, beta_err)


def test_beta_of_decomposed_and_random_sequential_updates_agree(eng):
    L, T, n = 512, 2000, 12
    ts = [t for t in I.sample_times(T) if t >= 1]
    betas = {}
    for dec in (0, 4):
        W = np.zeros((n, len(ts)))
        for k in range(n):
            lat = eng.Lattice(L, 1.0, 0.0, seed=51, sample=k, decomposition=dec)
            t0 = 0
            for j, tt in enumerate(ts):
                lat.run(tt - t0)
                t0 = tt
                W[k, j] = lat.roughness()["w2"]
            lat.close()
        m, e = A.ensemble_mean(W)[:2]
        betas[dec] = A.fit_beta(np.array(ts, np.float64), m, 50, T, err=e)[0]
    assert abs(betas[0] - betas[4]) < 0.03, betas
    assert 0.19 < betas[4] < 0.27, betas
