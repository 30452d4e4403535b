"""One single-hit round from the flat start (Sec. 2.1 flat start, Sec. 3.1
rounds): on the checkerboard h = (i + j) & 1 every even site is a local
minimum and every odd site a local maximum, so at p = 1, q = 0 exactly the
attempted live even sites rise by 2; a cell attempts one site of its active
2 x 2 quadrant, which holds two even sites, so about half of the cells move."""
import numpy as np

from oracle import oracle as O


def test_first_round_moves_half_the_cells_each_by_one_minimum():
    L, B = 512, 128
    moved_frac = []
    for seed in (1, 2, 3):
        st = O.State.flat(L)
        h0 = st.heights(absolute=True)
        st.sweep(B, B, 1.0, 0.0, seed, 0, rounds=1)
        d = st.heights(absolute=True) - h0
        assert set(np.unique(d)) <= {0, 2}                     # only rises, by 2
        jj, ii = np.nonzero(d)
        assert np.all((ii + jj) % 2 == 0)                      # only minima of the flat start
        # at most one move per 4 x 4 cell of the tile grid (cells anchored at the origin)
        o = O.philox([0, 0, 0, 0], [seed, 0])
        ox, oy = int(o[0]) & (L - 1), int(o[1]) & (L - 1)
        cells = (((jj - oy) % L) // 4) * (L // 4) + ((ii - ox) % L) // 4
        assert len(np.unique(cells)) == len(cells)
        moved_frac.append(len(cells) / (L // 4) ** 2)
    n = 3 * (L // 4) ** 2
    mean = float(np.mean(moved_frac))
    # An attempt lands on the dead border when its cell is in the tile's first
    # cell column (31 of 1024 cells: active quadrant QX = 0 and xi = 0, 1/4) or
    # first cell row (31 of 1024: 1/4) or both (1 of 1024: 1 - (3/4)^2 = 7/16);
    # a live attempt hits an even site with probability 1/2.
    cpt = (B // 4) ** 2
    p_dead = (2 * (B // 4 - 1) * 0.25 + 7 / 16) / cpt
    expect = 0.5 * (1 - p_dead)
    assert abs(mean - expect) < 5 * 0.5 / np.sqrt(n), (moved_frac, expect)
