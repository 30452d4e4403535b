"""Pins the oracle's site update (eq. rule of arXiv:1204.5072, Sec. 2.1) by
brute force on the 4x4 torus.

Every valid octahedron surface of the 4x4 periodic lattice (all height
functions with |dh| = 1 on every bond, gauge h(0,0) = 0) is enumerated. For
each surface and each site the slope-level update of the oracle must equal the
height-level statement of the model: a site lower than all four neighbours
rises by 2 (attachment, probability p), a site higher than all four drops by 2
(detachment, probability q), anything else stays. The result must again be a
valid surface. This fixes the orientation of the 2x2 slope patterns, the sign
convention of the slopes and the periodic neighbour indices.
"""
import numpy as np
import pytest

from oracle import oracle as O
from synth import inputs as I


def _slopes_from_heights(h):
    sx = ((np.roll(h, -1, axis=1) - h) == 1).astype(np.uint8)
    sy = ((np.roll(h, -1, axis=0) - h) == 1).astype(np.uint8)
    return sx, sy


def _heights_bfs(sx, sy):
    """Heights by breadth-first search from (0,0) over all four bond directions."""
    L = sx.shape[0]
    h = np.full((L, L), np.iinfo(np.int64).min, np.int64)
    h[0, 0] = 0
    todo = [(0, 0)]
    while todo:
        i, j = todo.pop()
        nb = [((i + 1) % L, j, 1 if sx[j, i] else -1),
              ((i - 1) % L, j, -1 if sx[j, (i - 1) % L] else 1),
              (i, (j + 1) % L, 1 if sy[j, i] else -1),
              (i, (j - 1) % L, -1 if sy[(j - 1) % L, i] else 1)]
        for ii, jj, d in nb:
            want = h[j, i] + d
            if h[jj, ii] == np.iinfo(np.int64).min:
                h[jj, ii] = want
                todo.append((ii, jj))
            else:
                assert h[jj, ii] == want, "inconsistent slopes (curl)"
    return h


@pytest.fixture(scope="module")
def surfaces():
    hs = I.valid_heights_4x4()
    assert len(hs) > 100
    return hs


@pytest.mark.parametrize("acc_min,acc_max", [(1, 0), (0, 1), (1, 1), (0, 0)])
def test_rule_matches_height_minmax_bruteforce(surfaces, acc_min, acc_max):
    L = 4
    n_min = n_max = 0
    for h in surfaces:
        sx, sy = _slopes_from_heights(h)
        for j in range(L):
            for i in range(L):
                st = O.State(L, sx.copy(), sy.copy())
                nbrs = [h[j, (i + 1) % L], h[j, (i - 1) % L], h[(j + 1) % L, i], h[(j - 1) % L, i]]
                want = 0
                if all(h[j, i] < v for v in nbrs):
                    n_min += 1
                    want = 2 if acc_min else 0
                elif all(h[j, i] > v for v in nbrs):
                    n_max += 1
                    want = -2 if acc_max else 0
                got = st.attempt(i, j, acc_min, acc_max)
                assert got == want, (i, j, h)
                h2 = _heights_bfs(st.sx, st.sy)
                expect = h.copy()
                expect[j, i] += want
                expect -= expect[0, 0]
                assert np.array_equal(h2, expect)
    assert n_min > 0 and n_max > 0


def test_rule_on_random_larger_surfaces():
    # Separable random surfaces of L=16; every site, both flips allowed.
    for seed in range(3):
        sx, sy = I.separable_surface(16, seed)
        h = _heights_bfs(sx, sy)
        for j in range(16):
            for i in range(16):
                st = O.State(16, sx.copy(), sy.copy())
                nb = [h[j, (i + 1) % 16], h[j, (i - 1) % 16], h[(j + 1) % 16, i], h[(j - 1) % 16, i]]
                want = 2 if all(h[j, i] < v for v in nb) else (-2 if all(h[j, i] > v for v in nb) else 0)
                assert st.attempt(i, j) == want


def test_thresholds():
    assert O.threshold(1.0) == 65536
    assert O.threshold(0.0) == 0
    assert O.threshold(float("nan")) == 0
    assert O.threshold(0.5) == 32768
    assert O.threshold(0.95) == 62259      # floor(0.95 * 65536 + 0.5)
    assert O.threshold(1.0 - 1e-12) == 65536


def test_threshold_quantisation_bound():
    """p is used as T / 2^16 with T = floor(p 2^16 + 1/2): the acceptance
    probability an attempt actually has differs from p by at most 2^-17
    (7.6e-6), half a quantum, for every p in [0, 1]."""
    import numpy as np
    rng = np.random.default_rng(2)
    for p in np.concatenate([rng.random(20000), np.linspace(0, 1, 4097), [1e-9, 1 - 1e-9, 2.0 ** -17]]):
        T = O.threshold(float(p))
        assert 0 <= T <= 65536 and abs(T / 65536 - p) <= 2.0 ** -17 + 1e-15, (p, T)
