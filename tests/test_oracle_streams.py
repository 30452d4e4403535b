"""Pins of the oracle's random streams (arXiv:1204.5072).

What the method draws, and what fixes each draw:

* Sec. 3, device layer: the origin of each sweep's tile grid is a uniformly
  random site.
* Sec. 3.1, work-group layer: each round one of the four quadrant sets is
  picked at random, with replacement; every cell then attempts one site of
  its active 2 x 2 quadrant, uniformly; neighbouring cells draw independently.
* Eq. (rule): an attempted local minimum flips with probability p, a local
  maximum with probability q. The oracle draws a 16-bit number U per
  candidate and accepts when U < T (T = p quantised to 2^-16): the top four
  bits come bit-sliced per cell row and round, the low twelve only for
  candidates whose top bits tie with T's, from deep blocks taken in cell
  order. U must be uniform, and tied candidates must never share low bits
  (within a row, across the two rounds of a deep block, in overflow blocks).

Every statistic is a chi-square or binomial check on fixed seeds (so the
outcome is reproducible) and, for each, a copy of the oracle is compiled with
one planted mistake and must fail the same check: xi stuck at 0, yi copied
from xi, neighbouring cells sharing a position bit, the origin's y equal to
its x, one set for two rounds, the acceptance levels reusing one word, deep
halves reused within a row, across a round pair or inside an overflow block.
"""
import os
import subprocess

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

P_MIN = 1e-4          # a correct stream passes every check at this level


# --------------------------------------------------------------------------- #
_plants = {}


def _planted(tmp_path_factory, old: str, new: str):
    """The oracle compiled with `old` replaced by `new` (exactly once)."""
    key = (old, new)
    if key not in _plants:
        src = open(O._SRC).read()
        assert src.count(old) == 1, old
        d = tmp_path_factory.mktemp("plant")
        c = os.path.join(d, "kpz_oracle.c")
        so = os.path.join(d, "libplant.so")
        with open(c, "w") as f:
            f.write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", so, c])
        _plants[key] = O.load(so)
    return _plants[key]


def _chi2(counts) -> float:
    """p-value of uniform counts; 1.0 (no evidence) for an empty histogram."""
    c = np.asarray(counts, float).ravel()
    if c.sum() == 0:
        return 1.0
    return float(stats.chisquare(c).pvalue)


# --------------------------------------------------------------------------- #
# Origin of the tile grid (Sec. 3).
def _origin_pvalue(lib=None, n=4096, L=1024):
    lo = np.zeros((16, 16))
    hi = np.zeros((16, 16))
    for s in range(n):
        ox, oy = O.origin(L, 1, 0, s, _lib=lib)
        lo[oy % 16, ox % 16] += 1
        hi[oy >> 6, ox >> 6] += 1
    return min(_chi2(lo), _chi2(hi))


def test_origin_uniform(tmp_path_factory):
    assert _origin_pvalue() > P_MIN
    bad = _planted(tmp_path_factory, "*oy = w[1] & (L - 1);", "*oy = w[0] & (L - 1);")
    assert _origin_pvalue(bad) < P_MIN


# --------------------------------------------------------------------------- #
# Quadrant set per round (Sec. 3.1).
def _set_pvalues(lib=None, L=1024, B=128):
    single = np.zeros(4)
    pairs = np.zeros((4, 4))
    for s in range(24):
        for T in range(64):
            ks = [O.attempt_site(L, B, B, 3, 1, s, T, r, 0, 0, _lib=lib)[2] for r in range(16)]
            for r in range(16):
                single[ks[r]] += 1
                if r:
                    pairs[ks[r - 1], ks[r]] += 1
    return _chi2(single), _chi2(pairs)


def test_quadrant_set_uniform_and_independent_between_rounds(tmp_path_factory):
    p1, p2 = _set_pvalues()
    assert p1 > P_MIN and p2 > P_MIN
    bad = _planted(tmp_path_factory, "return (setw0 >> (2 * r)) & 3u;", "return (setw0 >> (2 * (r >> 1))) & 3u;")
    assert min(_set_pvalues(bad)) < P_MIN


# --------------------------------------------------------------------------- #
# Attempted site inside the active quadrant (Sec. 3.1).
def _position_pvalues(lib=None, L=1024, B=128, n=6000):
    rng = np.random.default_rng(5)
    per_set = np.zeros((4, 2, 2))
    neighbours = np.zeros((2, 2))
    for _ in range(n):
        s, T, r = int(rng.integers(0, 50)), int(rng.integers(0, 64)), int(rng.integers(0, 16))
        cx, cy = int(rng.integers(0, B // 4 - 1)), int(rng.integers(0, B // 4))
        u, v, k = O.attempt_site(L, B, B, 9, 2, s, T, r, cx, cy, _lib=lib)
        u2, v2, _ = O.attempt_site(L, B, B, 9, 2, s, T, r, cx + 1, cy, _lib=lib)
        # the site lies in the active quadrant of its cell
        assert (u // 4, v // 4) == (cx, cy) and ((u % 4) // 2, (v % 4) // 2) == (k & 1, k >> 1)
        per_set[k, v % 2, u % 2] += 1
        neighbours[u % 2, u2 % 2] += 1
    return [_chi2(per_set[k]) for k in range(4)] + [_chi2(neighbours)]


def test_attempted_site_uniform_in_quadrant(tmp_path_factory):
    assert min(_position_pvalues()) > P_MIN
    stuck = _planted(tmp_path_factory, "*xi = (w[2 * (r & 1u)] >> b) & 1u;", "*xi = 0u;")
    assert min(_position_pvalues(stuck)) < P_MIN
    copied = _planted(tmp_path_factory, "*yi = (w[2 * (r & 1u) + 1] >> b) & 1u;",
                      "*yi = (w[2 * (r & 1u)] >> b) & 1u;")
    assert min(_position_pvalues(copied)) < P_MIN
    shared = _planted(tmp_path_factory, "*xi = (w[2 * (r & 1u)] >> b) & 1u;",
                      "*xi = (w[2 * (r & 1u)] >> (b & ~1u)) & 1u;")
    assert min(_position_pvalues(shared)) < P_MIN


# --------------------------------------------------------------------------- #
# Acceptance numbers (eq. rule).
def _rows(lib, Tp, Tq, n, rng, full=False):
    """n row words with random disjoint candidate masks (all 32 cells minima
    when full); yields (r, rw, T, s, cmin, cmax, acc, tied, U)."""
    for i in range(n):
        r, rw, T, s = i % 16, (i // 16) % 64, (i // 1024) % 61, i // (1024 * 61)
        if full:
            cmin, cmax = 0xFFFFFFFF, 0
        else:
            a = int(rng.integers(0, 1 << 32, dtype=np.uint64))
            b = int(rng.integers(0, 1 << 32, dtype=np.uint64))
            cmin, cmax = a & ~b & 0xFFFFFFFF, b & ~a & 0xFFFFFFFF
        acc, tied, U = O.row_acceptance(7, 3, Tp, Tq, T, s, r, rw, cmin, cmax, _lib=lib)
        yield r, rw, T, s, cmin, cmax, acc, tied, U


def _bits(m):
    return [b for b in range(32) if (m >> b) & 1]


def test_acceptance_decision_is_u_below_threshold():
    """accept <=> U < T for every drawn candidate; T = 2^16 accepts and T = 0
    rejects without drawing; cells that are not candidates never move."""
    rng = np.random.default_rng(1)
    for Tp, Tq in [(62259, 3277), (32768, 32768), (1, 65535), (65536, 0), (0, 65536), (40000, 0)]:
        for r, rw, T, s, cmin, cmax, acc, tied, U in _rows(None, Tp, Tq, 400, rng):
            assert acc & ~(cmin | cmax) == 0
            for b in range(32):
                kind = 1 if (cmin >> b) & 1 else 2 if (cmax >> b) & 1 else 0
                if not kind:
                    assert U[b] == 0xFFFFFFFF
                    continue
                thr = Tp if kind == 1 else Tq
                if thr in (0, 65536):
                    assert U[b] == 0xFFFFFFFF and ((acc >> b) & 1) == (thr == 65536)
                else:
                    assert ((acc >> b) & 1) == (U[b] < thr)
                    assert ((tied >> b) & 1) == ((U[b] >> 12) == (thr >> 12))
                    if not (tied >> b) & 1:
                        assert U[b] & 0xFFF == 0


@pytest.mark.parametrize("Tp", [1, 1 << 15, 62259, 65535])
def test_acceptance_frequency_matches_threshold(Tp):
    """P(accept) = T / 2^16 within 5 sigma, over ~10^5 candidates (plus the
    exact count of U below T for T = 1, which must be rare)."""
    rng = np.random.default_rng(Tp)
    n_acc = n = 0
    for *_, cmin, cmax, acc, tied, U in _rows(None, Tp, 0, 3500, rng):
        n += bin(cmin).count("1")
        n_acc += bin(acc & cmin).count("1")
    p = Tp / 65536
    assert abs(n_acc - n * p) <= 5 * np.sqrt(n * p * (1 - p)) + 1, (n_acc, n, p)


def _acceptance_pvalues(lib=None, n=6000):
    """chi-square of the top four bits, of the low twelve bits (two nibbles)
    of tied candidates, separately for the main and the overflow deep blocks;
    and counts of equal low bits between tied candidates that must be
    independent: k = 0 vs k = 1 of a row, k = 0 of rounds 2i and 2i+1 of the
    same row, k = 4 vs k = 5 (one overflow block)."""
    rng = np.random.default_rng(3)
    top = np.zeros(16)
    lo_main = np.zeros((2, 16))
    lo_ovf = np.zeros((2, 16))
    same_row = same_pair = same_ovf = 0
    first_of = {}
    for r, rw, T, s, cmin, cmax, acc, tied, U in _rows(lib, 0x8123, 0, n, rng, full=True):
        for b in range(32):
            top[U[b] >> 12] += 1
        tb = _bits(tied)
        low = [int(U[b]) & 0xFFF for b in tb]
        for k, x in enumerate(low):
            dst = lo_main if k < 4 else lo_ovf
            dst[0, x >> 8] += 1
            dst[1, (x >> 4) & 15] += 1
        if len(low) >= 2 and low[0] == low[1]:
            same_row += 1
        if len(low) >= 6 and low[4] == low[5]:
            same_ovf += 1
        if low:
            key = (rw, T, s, r >> 1)
            if key in first_of and first_of[key] == low[0]:
                same_pair += 1
            first_of[key] = low[0]
    pv = [_chi2(top)] + [_chi2(lo_main[i]) for i in range(2)] + [_chi2(lo_ovf[i]) for i in range(2)]
    return pv, (same_row, same_pair, same_ovf)


def test_acceptance_numbers_uniform_and_independent(tmp_path_factory):
    pv, same = _acceptance_pvalues()
    assert min(pv) > P_MIN, pv
    assert max(same) <= 3, same        # about n / 4096 coincidences expected in each count
    reused = _planted(tmp_path_factory, "top |= ((A[n] >> b) & 1u) << (3 - n);",
                      "top |= ((A[0] >> b) & 1u) << (3 - n);")
    assert min(_acceptance_pvalues(reused, 1500)[0]) < P_MIN
    for old, new in [("H = half16(D, 4u * (r & 1u) + k);", "H = half16(D, 4u * (r & 1u));"),
                     ("H = half16(D, 4u * (r & 1u) + k);", "H = half16(D, k);"),
                     ("H = half16(Dx, (k - 4) % 8);", "H = half16(Dx, 0);")]:
        bad = _planted(tmp_path_factory, old, new)
        assert max(_acceptance_pvalues(bad)[1]) > 20, (old, new)


def test_first_round_general_rates_from_flat_start():
    """One round from the flat start (every even site a minimum, every odd
    site a maximum): the fraction of cells whose minimum rises is
    1/2 (1 - dead share) Tp / 2^16 and of those whose maximum falls
    1/2 (1 - dead share) Tq / 2^16, within 5 sigma."""
    L, B = 512, 128
    cells = 0
    up = down = 0
    for seed in (1, 2, 3, 4):
        st = O.State.flat(L)
        h0 = st.heights(absolute=True)
        st.sweep(B, B, 0.6, 0.3, seed, 0, rounds=1)
        d = st.heights(absolute=True) - h0
        jj, ii = np.nonzero(d)
        assert set(np.unique(d[jj, ii])) <= {-2, 2}
        assert np.all(((ii + jj) % 2 == 0) == (d[jj, ii] == 2))
        up += int((d == 2).sum())
        down += int((d == -2).sum())
        cells += (L // 4) ** 2
    cpt = (B // 4) ** 2
    p_dead = (2 * (B // 4 - 1) * 0.25 + 7 / 16) / cpt
    for got, T in ((up, O.threshold(0.6)), (down, O.threshold(0.3))):
        p = 0.5 * (1 - p_dead) * T / 65536
        assert abs(got - cells * p) < 5 * np.sqrt(cells * p * (1 - p)), (got, cells * p)
