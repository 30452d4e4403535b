"""Pins of the oracle's random-sequential reference (one attempt at a time at
a uniformly random site, no decomposition; each sweep L^2 attempts, rule of
Sec. 2.1, eq. rule): the p = q = 0 identity, valid surfaces, a replay of one
sweep from the Philox stream and the single-site update, and uniform sites."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_schedule import _check_valid

TAG_RSU = 4


def _site_stream(L, seed, sample, s, n):
    """Sites and acceptance numbers of attempts 0..n-1 of sweep s: counter
    (4 << 28 | a >> 32, a, s, sample), site (w0 mod L, w1 mod L), U = w2 >> 16."""
    out = []
    for a in range(n):
        w = O.philox([(TAG_RSU << 28) | (a >> 32), a, s, sample], [seed & 0xFFFFFFFF, seed >> 32])
        out.append((int(w[0]) & (L - 1), int(w[1]) & (L - 1), int(w[2]) >> 16))
    return out


def test_no_rates_no_change_and_valid_surfaces():
    z = O.State.flat(32).rsu(3, 0.0, 0.0, seed=4)
    assert np.array_equal(z.packed(), O.State.flat(32).packed()) and z.t == 3
    st = O.State.flat(32)
    for p, q in [(1.0, 0.0), (0.7, 0.4), (0.0, 1.0)]:
        st.rsu(2, p, q, seed=6, sample=1)
        _check_valid(st)


@pytest.mark.parametrize("p,q", [(1.0, 0.0), (0.8, 0.3)])
def test_replay_of_one_sweep(p, q):
    L, seed, sample = 16, 9, 2
    st = O.State.flat(L).rsu(2, p, q, seed=seed, sample=sample)   # sweeps 0 and 1
    ref = O.State.flat(L).rsu(1, p, q, seed=seed, sample=sample)  # sweep 0
    Tp, Tq = O.threshold(p), O.threshold(q)
    h00 = ref.h00
    for i, j, U in _site_stream(L, seed, sample, 1, L * L):
        dh = ref.attempt(i, j, U < Tp, U < Tq)
        if (i, j) == (0, 0):
            h00 += dh
    assert np.array_equal(ref.sx, st.sx) and np.array_equal(ref.sy, st.sy)
    assert h00 == st.h00


def test_sites_are_uniform():
    L = 16
    sites = _site_stream(L, 3, 0, 0, 64 * L * L)
    counts = np.zeros((L, L))
    for i, j, _ in sites:
        counts[j, i] += 1
    chi2 = ((counts - 64) ** 2 / 64).sum()     # 255 degrees of freedom
    assert 255 - 5 * np.sqrt(510) < chi2 < 255 + 5 * np.sqrt(510)
