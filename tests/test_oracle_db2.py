"""Pins of the oracle's dead border at both layers (the paper's earlier KPZ
scheme, arXiv:1204.5072 Sec. 3.1, with the dead-border rule of Sec. 3 at the
work-group layer): 4 x 4 blocks re-anchored at random inside the tile each
round, one attempt per block at a uniformly random site of its 3 x 3 live
interior.

* Valid surfaces and p = q = 0 identity (eq. rule).
* Blocks of a round and tiles of a sweep touch disjoint slopes, so any
  processing order gives the same lattice; a planted mistake that lets a
  block attempt its own dead border (neighbouring attempts in one round)
  breaks this.
* The tile's dead border never moves (Sec. 3).
* Attempted sites: never on the block's dead border, uniform over the 9
  interior sites, and every site of a tile other than its dead border gets
  one attempt per sweep on average.
"""
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from tests.test_oracle_schedule import _check_valid


@pytest.mark.parametrize("L,B,p,q", [(64, 16, 1.0, 0.0), (64, 32, 0.7, 0.4), (128, 128, 0.95, 0.05),
                                     (256, 128, 0.5, 0.5)])
def test_valid_surfaces(L, B, p, q):
    st = O.State.flat(L)
    for _ in range(6):
        st.sweep_db2(B, B, p, q, seed=3, sample=1)
        _check_valid(st)


def test_zero_rates_identity():
    st = O.State.flat(128).run_db2(3, 32, 32, 1.0, 0.2, seed=2)
    before = st.copy()
    st.run_db2(4, 32, 32, 0.0, 0.0, seed=2)
    assert np.array_equal(st.sx, before.sx) and np.array_equal(st.sy, before.sy) and st.h00 == before.h00


def _orders_agree(lib_sweep, L=128, B=32):
    outs = []
    for order in (0, 1, 7, 123):
        st = O.State.flat(L)
        for _ in range(4):
            lib_sweep(st, B, order)
        outs.append((st.packed(), st.h00))
    return all(np.array_equal(outs[0][0], o[0]) and outs[0][1] == o[1] for o in outs[1:])


def test_order_independence(tmp_path):
    def sweep(st, B, order):
        st.sweep_db2(B, B, 0.9, 0.3, seed=5, sample=0, order=order)
    assert _orders_agree(sweep)
    # planted: the block's own dead column can be attempted
    src = open(O._SRC).read()
    old = "*u = (dx + 4 * kx + 1 + n % 3) & (Bx - 1);"
    assert src.count(old) == 1
    c = os.path.join(tmp_path, "k.c")
    so = os.path.join(tmp_path, "k.so")
    open(c, "w").write(src.replace(old, "*u = (dx + 4 * kx + (n % 4)) & (Bx - 1);"))
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", so, c])
    bad = O.load(so)
    import ctypes

    def bad_sweep(st, B, order):
        h = ctypes.c_int64(st.h00)
        assert bad.orc_sweep_db2(st.L, B, B, O.threshold(0.9), O.threshold(0.3), 5, 0, st.t, st.sx, st.sy,
                                 ctypes.byref(h), order) == 0
        st.h00, st.t = h.value, st.t + 1
    assert not _orders_agree(bad_sweep)


def test_tile_dead_border_never_moves():
    L, B, seed = 128, 32, 9
    st = O.State.flat(L).run_db2(2, B, B, 1.0, 0.3, seed)
    for _ in range(4):
        ox, oy = O.origin(L, seed, 0, st.t)
        h0 = st.heights(absolute=True)
        st.sweep_db2(B, B, 1.0, 0.3, seed)
        d = st.heights(absolute=True) != h0
        jj, ii = np.nonzero(d)
        assert np.all(((ii - ox) % B != 0) & ((jj - oy) % B != 0))


def test_attempted_sites_interior_uniform_and_one_per_sweep():
    L, B, seed = 64, 32, 4
    nb = B // 4
    counts = np.zeros((B, B))
    interior = np.zeros(9)
    S = 48
    for s in range(S):
        S_off = O.philox([9 << 28, 0, s, 0], [seed, 0])
        for r in range(16):
            dx = (int(S_off[r >> 3]) >> (4 * (r & 7))) & 3
            dy = (int(S_off[r >> 3]) >> (4 * (r & 7) + 2)) & 3
            for ky in range(nb):
                for kx in range(nb):
                    u, v, U = O.db2_site(L, B, B, seed, 0, s, 0, r, kx, ky)
                    i, j = (u - dx - 4 * kx) % B, (v - dy - 4 * ky) % B
                    assert 1 <= i <= 3 and 1 <= j <= 3         # never the block's dead border
                    interior[(j - 1) * 3 + (i - 1)] += 1
                    counts[v, u] += 1
    assert stats.chisquare(interior).pvalue > 1e-4
    per_site = counts / S                                      # attempts per site and sweep
    assert abs(per_site.mean() - 1.0) < 1e-12                  # 16 rounds x nb^2 blocks = B^2 attempts
    assert stats.chisquare(counts.ravel()).pvalue > 1e-4       # and spread evenly over the tile
