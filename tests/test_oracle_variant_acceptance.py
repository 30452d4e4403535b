"""Acceptance streams of the oracle's C = 2 work-group layer and colour-class
random-sequential reference (eq. rule: a minimum rises with probability p, a
maximum falls with probability q; both variants draw 16-bit numbers U per
attempted site, bit-sliced, and accept when U < T).

From the flat start (Sec. 2.1, h = (i + j) & 1) every site of even parity is a
local minimum and every odd site a local maximum. In the first C = 2 round a
tile attempts one site of each 2 x 2 cell, all of one parity, and in the
first colour sub-step every selected site of one period-2 sublattice, again
of one parity, so the expected numbers of rises and falls are closed forms:
attempted minima x Tp / 2^16 and attempted maxima x Tq / 2^16. Each check
must also reject a copy of the oracle with a planted mistake (the four
levels of a Philox block read from one word)."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_streams import _planted


def _moves(st_before, st_after):
    d = st_after.heights(absolute=True) - st_before.heights(absolute=True)
    return d


def _c2_expectation(L, B, seed, sample):
    """(attempted minima, attempted maxima, attempted mask) of the first C = 2
    round of sweep 0 from the flat start."""
    ox, oy = O.origin(L, seed, sample, 0)
    ntx = L // B
    att = np.zeros((L, L), bool)
    n_min = n_max = 0
    for T in range(ntx * ntx):
        tx, ty = T % ntx, T // ntx
        k = int(O.philox([1 << 28, T, 0, sample], [seed & 0xFFFFFFFF, seed >> 32])[0]) & 3
        u = np.arange(k & 1, B, 2)
        v = np.arange(k >> 1, B, 2)
        u, v = u[u > 0], v[v > 0]                     # the tile's dead border
        x0, y0 = (ox + tx * B) % L, (oy + ty * B) % L
        n = len(u) * len(v)
        if (x0 + y0 + (k & 1) + (k >> 1)) % 2 == 0:
            n_min += n
        else:
            n_max += n
        att[np.ix_((y0 + v) % L, (x0 + u) % L)] = True
    return n_min, n_max, att


def _c2_counts(lib, L, B, p, q, seeds):
    up = down = e_up = e_down = var = 0.0
    for seed in seeds:
        st = O.State.flat(L)
        before = st.copy()
        h = ctypes.c_int64(0)
        assert lib.orc_sweep_c2_rounds(L, B, B, O.threshold(p), O.threshold(q), seed, 0, 0, st.sx, st.sy,
                                       ctypes.byref(h), 0, 1) == 0
        st.h00 = h.value
        d = _moves(before, st)
        n_min, n_max, att = _c2_expectation(L, B, seed, 0)
        assert not np.any(d[~att])                     # only attempted sites move
        up += (d == 2).sum()
        down += (d == -2).sum()
        tp, tq = O.threshold(p) / 65536, O.threshold(q) / 65536
        e_up += n_min * tp
        e_down += n_max * tq
        var += n_min * tp * (1 - tp) + n_max * tq * (1 - tq)
    return up, down, e_up, e_down, var


def test_c2_first_round_acceptance(tmp_path_factory):
    L, B, p, q, seeds = 256, 128, 0.6, 0.3, (1, 2, 3, 4, 5, 6)
    up, down, e_up, e_down, var = _c2_counts(O.lib(), L, B, p, q, seeds)
    assert abs(up - e_up) < 5 * np.sqrt(var) + 1 and abs(down - e_down) < 5 * np.sqrt(var) + 1, \
        (up, e_up, down, e_down)
    bad = _planted(tmp_path_factory, "U |= ((aw[lev & 3u] >> b) & 1u) << (15 - lev);",
                   "U |= ((aw[0] >> b) & 1u) << (15 - lev);")
    up, down, e_up, e_down, var = _c2_counts(bad, L, B, p, q, seeds)
    assert abs(up - e_up) > 5 * np.sqrt(var) or abs(down - e_down) > 5 * np.sqrt(var)


def _colour_counts(lib, L, p, q, m, seeds):
    up = down = e_up = e_down = var = 0.0
    for seed in seeds:
        st = O.State.flat(L)
        before = st.copy()
        h = ctypes.c_int64(0)
        assert lib.orc_sweep_colour_steps(L, O.threshold(p), O.threshold(q), m, seed, 0, 0, st.sx, st.sy,
                                          ctypes.byref(h), 1) == 0
        st.h00 = h.value
        d = _moves(before, st)
        c = int(O.philox([6 << 28, 0xFFFFFFFF, 0, 0], [seed & 0xFFFFFFFF, seed >> 32])[0]) & 3
        cls = np.zeros((L, L), bool)
        cls[(c >> 1)::2, (c & 1)::2] = True
        assert not np.any(d[~cls])                     # only the drawn sublattice moves
        n = (L * L // 4) / (1 << m)                    # expected attempted sites
        tp, tq = O.threshold(p) / 65536, O.threshold(q) / 65536
        t = tp if ((c & 1) + (c >> 1)) % 2 == 0 else tq
        up += (d == 2).sum()
        down += (d == -2).sum()
        if t is tp:
            e_up += n * tp
        else:
            e_down += n * tq
        var += n * t * (1 - t) + (n * t) ** 2 * (1 - 1 / (1 << m)) / n   # plus the subset draw
    return up, down, e_up, e_down, var


@pytest.mark.parametrize("m", [0, 2])
def test_colour_first_substep_acceptance(tmp_path_factory, m):
    L, p, q, seeds = 256, 0.6, 0.3, (1, 2, 3, 4, 5, 6, 7, 8)
    up, down, e_up, e_down, var = _colour_counts(O.lib(), L, p, q, m, seeds)
    tol = 5 * np.sqrt(var) + 1
    assert abs(up - e_up) < tol and abs(down - e_down) < tol, (up, e_up, down, e_down)
    bad = _planted(tmp_path_factory, "U |= ((A[lev & 3u] >> c4) & 1u) << (15 - lev);",
                   "U |= ((A[0] >> c4) & 1u) << (15 - lev);")
    up, down, e_up, e_down, var = _colour_counts(bad, L, p, q, m, seeds)
    assert abs(up - e_up) > 5 * np.sqrt(var) or abs(down - e_down) > 5 * np.sqrt(var)
