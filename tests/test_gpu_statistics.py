"""Statistics of the decomposed dynamics on the GPU (arXiv:1204.5072, Sec. 3:
the decomposition must not change the physics).

* Growth exponent: W^2 ~ t^(2 beta) in the growth regime; for the 2+1-d KPZ
  class beta ~ 0.24 (p = 1, q = 0, L = 512, t in [50, 2000]).
* Random-sequential reference: the ensemble mean of W^2(t) from the GPU
  agrees with the oracle's random-sequential-update runs (no decomposition)
  within the early-time offset of single-hit double tiling (about 3-5 % for
  t <= 64, measured with the oracle at L = 128-256 for tile sizes 16-128) and
  within errors later.
* lambda = 0 (p = q): Edwards-Wilkinson class, much slower (logarithmic) growth.
"""
import numpy as np
import pytest

from oracle import oracle as O
from synth import inputs as I
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    return engine()


def _ensemble(eng, L, p, q, ts, n, seed=1, decomposition=0):
    W = np.zeros((n, len(ts)))
    for k in range(n):
        lat = eng.Lattice(L, p, q, seed=seed, sample=k, decomposition=decomposition)
        t0 = 0
        for j, t in enumerate(ts):
            if t > t0:
                lat.run(t - t0)
            W[k, j] = lat.roughness()["w2"]
            t0 = t
        lat.close()
    return W


def test_growth_exponent_beta(eng):
    ts = [t for t in I.sample_times(2000) if t >= 50]
    W = _ensemble(eng, 512, 1.0, 0.0, ts, 16)
    m = W.mean(axis=0)
    slope = np.polyfit(np.log(ts), np.log(m), 1)[0]
    beta = slope / 2
    assert 0.20 < beta < 0.27, beta


def test_matches_random_sequential_reference(eng):
    L, ts, n = 128, [1, 2, 4, 8, 16, 32, 64, 128], 24
    gpu = _ensemble(eng, L, 1.0, 0.0, ts, 64, seed=11)
    rsu = np.zeros((n, len(ts)))
    for k in range(n):
        st = O.State.flat(L)
        for j, t in enumerate(ts):
            st.rsu(t - st.t, 1.0, 0.0, seed=12, sample=k)
            rsu[k, j] = st.w2()
    mg, mr = gpu.mean(0), rsu.mean(0)
    err = np.sqrt(gpu.var(0, ddof=1) / gpu.shape[0] + rsu.var(0, ddof=1) / n)
    rel = mg / mr - 1
    assert np.all(np.abs(rel) < 0.07), rel
    assert np.all(np.abs(mg - mr) < 0.07 * mr + 4 * err)
    # growth exponents over t in [8, 128] agree
    sel = slice(3, None)
    bg = np.polyfit(np.log(ts[sel]), np.log(mg[sel]), 1)[0] / 2
    br = np.polyfit(np.log(ts[sel]), np.log(mr[sel]), 1)[0] / 2
    assert abs(bg - br) < 0.03, (bg, br)


@pytest.mark.parametrize("p,q,band", [(0.95, 0.05, 0.07), (0.6, 0.3, 0.03)])
def test_general_rates_match_random_sequential_reference(eng, p, q, band):
    """General rates (the acceptance path of eq. rule): the GPU ensemble's
    W^2(t) against the oracle's random-sequential updates at the same (p, q).
    The single-hit offset shrinks as the rates drop (measured with the
    oracle at L = 128, 96 realisations each: about -3 % at (0.95, 0.05),
    under 1 % at (0.6, 0.3), -3 to -6 % at p = 1), so the band is 7 % and
    3 %; a wrong acceptance probability (e.g. one level of U reused, which
    moves P(accept) from 0.95 to 0.6) would move W^2 far outside it."""
    L, ts, n = 128, [1, 2, 4, 8, 16, 32, 64, 128], 24
    gpu = _ensemble(eng, L, p, q, ts, 64, seed=41)
    rsu = np.zeros((n, len(ts)))
    for k in range(n):
        st = O.State.flat(L)
        for j, t in enumerate(ts):
            st.rsu(t - st.t, p, q, seed=42, sample=k)
            rsu[k, j] = st.w2()
    mg, mr = gpu.mean(0), rsu.mean(0)
    err = np.sqrt(gpu.var(0, ddof=1) / gpu.shape[0] + rsu.var(0, ddof=1) / n)
    assert np.all(np.abs(mg - mr) < band * mr + 4 * err), (p, q, mg / mr - 1, err / mr)
    sel = slice(3, None)
    bg = np.polyfit(np.log(ts[sel]), np.log(mg[sel]), 1)[0] / 2
    br = np.polyfit(np.log(ts[sel]), np.log(mr[sel]), 1)[0] / 2
    assert abs(bg - br) < 0.04, (p, q, bg, br)


def test_edwards_wilkinson_grows_slower(eng):
    ts = [8, 512]
    kpz = _ensemble(eng, 256, 1.0, 0.0, ts, 4).mean(0)
    ew = _ensemble(eng, 256, 0.5, 0.5, ts, 4).mean(0)
    assert ew[1] / ew[0] < 0.6 * kpz[1] / kpz[0]


def test_both_device_layers_against_random_sequential_updates(eng):
    """Dead-border tiles (the paper's KPZ scheme), the tile-set double tiling
    (no dead border) and dead borders at both layers (the earlier scheme) at
    L = 256 against random-sequential updates: all stay within the
    early-time offset of single hits (the oracle at L = 128: -3 to -6 % for
    the paper's scheme, -2 to -4 % for dead borders at both layers) and grow
    with the same exponent; the first two agree with each other within
    errors (the offset comes from the work-group layer)."""
    L, ts, n = 256, [1, 2, 4, 8, 16, 32, 64], 16
    rsu = np.zeros((n, len(ts)))
    for k in range(n):
        st = O.State.flat(L)
        for j, t in enumerate(ts):
            st.rsu(t - st.t, 1.0, 0.0, seed=12, sample=k)
            rsu[k, j] = st.w2()
    mr = rsu.mean(0)
    means = {}
    for dec in (0, 1, 3):
        W = _ensemble(eng, L, 1.0, 0.0, ts, 48, seed=21 + dec, decomposition=dec)
        mg = W.mean(0)
        means[dec] = (mg, W.var(0, ddof=1) / W.shape[0])
        rel = mg / mr - 1
        assert np.all(np.abs(rel) < 0.07), (dec, rel)
        bg = np.polyfit(np.log(ts[3:]), np.log(mg[3:]), 1)[0] / 2
        br = np.polyfit(np.log(ts[3:]), np.log(mr[3:]), 1)[0] / 2
        assert abs(bg - br) < 0.04, (dec, bg, br)
    (m0, v0), (m1, v1) = means[0], means[1]
    assert np.all(np.abs(m0 - m1) < 0.02 * m0 + 4 * np.sqrt(v0 + v1)), (m0, m1)
