"""Pins of the oracle's height reconstruction and width (arXiv:1204.5072,
Sec. 2.1, eq. Wdef) against independent computations.

* Heights: breadth-first reconstruction over all four bond directions from
  (0,0) must give the oracle's path sum (row 0, then up column i).
* W^2: exact rational arithmetic from explicit heights; and the 128-bit path
  with sums beyond 2^64.
* The packed exchange format round-trips and has the closed-form words of
  the flat start.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import oracle as O
from synth import inputs as I
from tests.test_oracle_rule import _heights_bfs


def _states():
    yield O.State.flat(16)
    for seed in range(3):
        sx, sy = I.separable_surface(32, seed)
        yield O.State(32, sx, sy)
    yield O.State.flat(64).run(20, 16, 16, 1.0, 0.0, seed=3)
    yield O.State.flat(64).run(20, 32, 8, 0.7, 0.45, seed=4, sample=9)
    yield O.State.flat(128).run(10, 128, 128, 0.95, 0.05, seed=5)


def test_heights_match_bfs():
    for st in _states():
        assert np.array_equal(st.heights(), _heights_bfs(st.sx, st.sy))


def test_w2_exact_rational():
    for st in _states():
        h = _heights_bfs(st.sx, st.sy)
        N = h.size
        s1 = int(h.sum())
        s2 = int((h.astype(object) ** 2).sum())
        assert st.sums() == (s1, s2)
        exact = Fraction(s2, N) - Fraction(s1, N) ** 2
        assert st.w2() == float(exact)
        # W^2 does not depend on the gauge (shift of all heights)
        hs = h + 1234
        t1, t2 = int(hs.sum()), int((hs.astype(object) ** 2).sum())
        assert O.w2_from_sums(N, t1, t2) == pytest.approx(float(exact), rel=1e-12, abs=1e-12)


def test_w2_wide_sums():
    # sums of a lattice with N = 2^34 sites and |h| ~ 2^17: S2 exceeds 2^64
    N = 1 << 34
    rng = np.random.default_rng(0)
    for _ in range(20):
        mean = int(rng.integers(1 << 15, 1 << 16)) * (1 if rng.random() < 0.5 else -1)
        var_num = int(rng.integers(0, 1 << 40))
        S1 = mean * N
        S2 = (var_num * N) // (1 << 10) + mean * mean * N   # sum h^2 = N*(var + mean^2)
        exact = Fraction(S2, N) - Fraction(S1, N) ** 2
        assert S2 >= 1 << 64
        assert O.w2_from_sums(N, S1, S2) == float(exact)


def test_pack_roundtrip():
    for st in _states():
        if st.L < 16:
            continue
        w = st.packed()
        back = O.State.from_packed(st.L, w)
        assert np.array_equal(back.sx, st.sx) and np.array_equal(back.sy, st.sy)
        # bit 2(i%16) of word j*L/16 + i/16 is sigma_x(i,j)
        j, i = 5, 21 % st.L
        word = int(w[j * (st.L // 16) + i // 16])
        assert (word >> (2 * (i % 16))) & 1 == st.sx[j, i]
        assert (word >> (2 * (i % 16) + 1)) & 1 == st.sy[j, i]
