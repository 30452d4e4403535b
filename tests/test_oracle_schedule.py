"""Pins of the oracle's decomposed schedule (arXiv:1204.5072, Sec. 3, 3.1)
against what the model and the decomposition fix.

* The flat start has closed-form sums and W^2 = 1/4 (Sec. 2.1).
* Slope flips keep the surface valid: neighbour heights differ by one, every
  row of sigma_x and every column of sigma_y sums to zero, every plaquette is
  curl-free, and h(i,j) = i+j mod 2.
* p = q = 0 leaves every slope unchanged (eq. rule).
* p = 1, q = 0 only raises sites; p = 0, q = 1 only lowers them. Through the
  tracked origin height this also pins the absolute-height bookkeeping.
* Dead border (Sec. 3): no site on the low-x column or the low-y row of a
  tile of the sweep's grid changes height in that sweep.
* Decomposition independence (Sec. 3, 3.1): tiles of one sweep and cells of
  one round touch disjoint slope bits, so processing them in any order gives
  the identical lattice. A missing dead border or overlapping quadrants
  would make the result order dependent.
"""
import numpy as np
import pytest

from oracle import oracle as O


def _check_valid(st):
    L = st.L
    h = st.heights()
    assert h[0, 0] == 0
    dx = np.roll(h, -1, axis=1) - h
    dy = np.roll(h, -1, axis=0) - h
    assert np.all(np.abs(dx) == 1) and np.all(np.abs(dy) == 1)
    # slopes agree with height differences, including the periodic wrap
    assert np.array_equal(dx == 1, st.sx.astype(bool))
    assert np.array_equal(dy == 1, st.sy.astype(bool))
    assert np.all(st.sx.astype(np.int64).sum(axis=1) * 2 == L)   # rows of sigma_x sum to 0
    assert np.all(st.sy.astype(np.int64).sum(axis=0) * 2 == L)   # columns of sigma_y sum to 0
    ii, jj = np.meshgrid(np.arange(L), np.arange(L))
    assert np.all((h - ii - jj) % 2 == 0)


def test_flat_start_closed_form():
    for L in (4, 16, 64, 256):
        st = O.State.flat(L)
        N = L * L
        s1, s2 = st.sums()
        assert (s1, s2) == (N // 2, N // 2)
        assert st.w2() == 0.25
        _check_valid(st)
    w = O.State.flat(64).packed().reshape(64, 4)
    assert np.all(w[0::2] == 0x33333333) and np.all(w[1::2] == 0xCCCCCCCC)


@pytest.mark.parametrize("L,Bx,By,p,q", [(16, 4, 4, 1.0, 0.0), (16, 8, 16, 0.7, 0.4),
                                         (64, 16, 32, 1.0, 0.0), (64, 64, 64, 0.5, 0.5),
                                         (128, 128, 128, 0.95, 0.05), (256, 128, 64, 1.0, 1.0)])
def test_invariants_hold(L, Bx, By, p, q):
    st = O.State.flat(L)
    for _ in range(6):
        st.run(3, Bx, By, p, q, seed=7, sample=3)
        _check_valid(st)


def test_p_q_zero_is_identity():
    st = O.State.flat(64)
    st.run(5, 16, 16, 1.0, 0.0, seed=3)
    before = st.copy()
    st.run(10, 16, 16, 0.0, 0.0, seed=3)
    assert np.array_equal(st.sx, before.sx) and np.array_equal(st.sy, before.sy)
    assert st.h00 == before.h00


@pytest.mark.parametrize("p,q,sign", [(1.0, 0.0, 1), (0.0, 1.0, -1), (0.8, 0.0, 1)])
def test_one_sided_rates_are_monotone(p, q, sign):
    L = 64
    st = O.State.flat(L)
    st.run(4, 32, 32, 1.0, 0.3, seed=11)          # start from a rough surface
    prev = st.heights(absolute=True)
    grew = 0
    for _ in range(8):
        st.sweep(32, 16, p, q, seed=5, sample=1)
        cur = st.heights(absolute=True)
        d = (cur - prev) * sign
        assert np.all(d >= 0) and np.all(d % 2 == 0)
        grew += int(d.sum())
        prev = cur
    assert grew > 0


@pytest.mark.parametrize("L,Bx,By", [(64, 16, 16), (64, 32, 8), (128, 128, 128)])
def test_dead_border_never_moves(L, Bx, By):
    seed, sample = 9, 2
    st = O.State.flat(L)
    st.run(3, Bx, By, 1.0, 0.2, seed=seed, sample=sample)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    ii, jj = np.meshgrid(np.arange(L), np.arange(L))
    for _ in range(5):
        s = st.t
        w = O.philox([0, 0, s, sample], key)        # origin of this sweep's tile grid
        ox, oy = int(w[0]) & (L - 1), int(w[1]) & (L - 1)
        h0 = st.heights(absolute=True)
        st.sweep(Bx, By, 1.0, 0.2, seed=seed, sample=sample)
        moved = st.heights(absolute=True) != h0
        dead = (((ii - ox) % Bx) == 0) | (((jj - oy) % By) == 0)
        assert moved.any()
        assert not (moved & dead).any()


@pytest.mark.parametrize("L,Bx,By,p,q", [(64, 16, 16, 1.0, 0.0), (64, 8, 32, 0.6, 0.3),
                                         (128, 32, 64, 0.95, 0.05)])
def test_tile_and_cell_order_do_not_matter(L, Bx, By, p, q):
    base = O.State.flat(L)
    base.run(2, Bx, By, 1.0, 0.0, seed=1)
    results = []
    for order in (0, 1, 7, 123456789):
        st = base.copy()
        for _ in range(3):
            st.sweep(Bx, By, p, q, seed=4, sample=0, order=order)
        results.append(st)
    for st in results[1:]:
        assert np.array_equal(st.sx, results[0].sx)
        assert np.array_equal(st.sy, results[0].sy)
        assert st.h00 == results[0].h00


def test_samples_and_seeds_give_different_histories():
    a = O.State.flat(64).run(5, 16, 16, 1.0, 0.0, seed=1, sample=0)
    b = O.State.flat(64).run(5, 16, 16, 1.0, 0.0, seed=1, sample=1)
    c = O.State.flat(64).run(5, 16, 16, 1.0, 0.0, seed=2, sample=0)
    assert not np.array_equal(a.sx, b.sx) and not np.array_equal(a.sx, c.sx)


def test_invalid_parameters_rejected():
    st = O.State.flat(16)
    with pytest.raises(ValueError):
        st.sweep(6, 4, 1.0, 0.0, seed=1)          # tile not a power of two
    with pytest.raises(ValueError):
        st.sweep(32, 4, 1.0, 0.0, seed=1)         # tile larger than the lattice


@pytest.mark.parametrize("L,Bx,By", [(64, 16, 16), (128, 128, 32)])
def test_one_round_touches_one_quadrant_per_tile(L, Bx, By):
    """Double tiling (Sec. 3): a cell is bisected in each direction into four
    sets; in one single-hit round every cell of a tile is updated inside the
    same set, a contiguous half in x and in y of the 4x4 cell."""
    seed, sample = 21, 0
    base = O.State.flat(L)
    base.run(2, Bx, By, 1.0, 0.0, seed=seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    ii, jj = np.meshgrid(np.arange(L), np.arange(L))
    for s in range(2, 8):
        st = base.copy()
        w = O.philox([0, 0, s, sample], key)
        ox, oy = int(w[0]) & (L - 1), int(w[1]) & (L - 1)
        h0 = st.heights(absolute=True)
        st.sweep(Bx, By, 1.0, 0.0, seed=seed, sample=sample, s=s, rounds=1)
        moved = st.heights(absolute=True) != h0
        assert moved.any()
        u = (ii - ox) % L
        v = (jj - oy) % L
        tile = (v // By) * (L // Bx) + (u // Bx)
        half_x = (u % 4) // 2
        half_y = (v % 4) // 2
        for T in np.unique(tile[moved]):
            sel = moved & (tile == T)
            assert len(np.unique(half_x[sel])) == 1 and len(np.unique(half_y[sel])) == 1
        # every site is raised at most once in a round and at most one per cell
        cell = ((v // 4) * (L // 4) + (u // 4))
        assert len(np.unique(cell[moved])) == int(moved.sum())


@pytest.mark.parametrize("L,Bx,By,p,q,seed,sample,s", [
    (64, 16, 16, 1.0, 0.0, 3, 0, 0), (128, 32, 64, 0.7, 0.2, 5, 2, 4), (256, 128, 128, 0.95, 0.05, 1, 0, 0),
    (256, 128, 256, 0.6, 0.4, 9, 1, 7)])
def test_flat_tile_windows_assemble_the_full_sweep(L, Bx, By, p, q, seed, sample, s):
    """Tiles of one sweep do not interact (dead border, Sec. 3): computing every
    tile of a sweep from the flat start on its own window and placing the
    windows at their anchors gives the full sweep, slopes and h(0,0)."""
    st = O.State.flat(L)
    st.sweep(Bx, By, p, q, seed, sample, s=s)
    sx = np.zeros((L, L), np.uint8)
    sy = np.zeros((L, L), np.uint8)
    dh = 0
    for T in range((L // Bx) * (L // By)):
        wx, wy, (x0, y0), d = O.flat_tile_sweep(L, Bx, By, p, q, seed, sample, s, T)
        rows = (y0 + np.arange(By)) % L
        cols = (x0 + np.arange(Bx)) % L
        sx[np.ix_(rows, cols)] = wx
        sy[np.ix_(rows, cols)] = wy
        dh += d
    assert np.array_equal(sx, st.sx.reshape(L, L)) and np.array_equal(sy, st.sy.reshape(L, L))
    assert dh == st.h00


@pytest.mark.parametrize("L,Bx,By,p,q", [(256, 32, 32, 1.0, 0.0), (256, 64, 128, 0.8, 0.3), (512, 128, 128, 0.95, 0.05)])
def test_threaded_tiles_give_the_serial_sweep(L, Bx, By, p, q):
    """Tiles of one sweep commute (dead border, Sec. 3): the OpenMP tile loop
    reproduces the serial sweep bit for bit, h(0,0) included."""
    a = O.State.flat(L).run(5, Bx, By, p, q, 3, 1)
    b = O.State.flat(L).run_threads(5, Bx, By, p, q, 3, 1, threads=4)
    assert np.array_equal(a.sx, b.sx) and np.array_equal(a.sy, b.sy)
    assert (a.h00, a.t) == (b.h00, b.t)
