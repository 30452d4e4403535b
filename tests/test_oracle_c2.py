"""Pins of the oracle's C = 2 work-group layer (2 x 2 cells, their four 1 x 1
quadrants as the sets, 4 single-hit rounds per sweep): the limit of the
double tiling the paper discusses (Sec. 3.1), with the dead-border device
layer unchanged."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_schedule import _check_valid


@pytest.mark.parametrize("L,B,p,q", [(64, 16, 1.0, 0.0), (128, 32, 0.7, 0.3), (256, 128, 0.95, 0.05)])
def test_surface_stays_valid(L, B, p, q):
    st = O.State.flat(L)
    for _ in range(6):
        st.sweep_c2(B, B, p, q, 3, 1)
        _check_valid(st)


def test_no_rates_no_change_monotone_rates_and_order_freedom():
    L, B = 128, 32
    assert np.array_equal(O.State.flat(L).run_c2(4, B, B, 0.0, 0.0, 5, 0).packed(), O.State.flat(L).packed())
    up = O.State.flat(L).run_c2(4, B, B, 1.0, 0.0, 5, 0)
    assert np.all(up.heights(absolute=True) >= O.State.flat(L).heights(absolute=True))
    ref = O.State.flat(L)
    for _ in range(3):
        ref.sweep_c2(B, B, 0.8, 0.2, 5, 0)
    for order in (1, 2, 777):
        st = O.State.flat(L)
        for _ in range(3):
            st.sweep_c2(B, B, 0.8, 0.2, 5, 0, order=order)
        assert np.array_equal(st.packed(), ref.packed()) and st.h00 == ref.h00


def test_dead_border_and_sublattice_of_one_round():
    """One C = 2 sweep never moves a tile's low-x column or low-y row; and on
    a 4 x 4 lattice of one 4 x 4 tile the four rounds can only move sites of
    the sublattices their sets name."""
    L, B = 128, 16
    o = O.philox([0, 0, 0, 0], [9, 0])
    ox, oy = int(o[0]) & (L - 1), int(o[1]) & (L - 1)
    border = np.zeros((L, L), bool)
    border[:, (ox + np.arange(0, L, B)) % L] = True
    border[(oy + np.arange(0, L, B)) % L, :] = True
    h0 = O.State.flat(L).heights(absolute=True)
    st = O.State.flat(L).sweep_c2(B, B, 1.0, 0.0, 9, 0)
    assert not np.any((st.heights(absolute=True) != h0) & border)
    moved = st.heights(absolute=True) != h0
    assert moved.any()
    # a site moves only if its class (u mod 2, v mod 2) is one of its tile's four sets
    ntx = L // B
    jj, ii = np.nonzero(moved)
    for i, j in zip(ii, jj):
        x, y = (i - ox) % L, (j - oy) % L
        T = (y // B) * ntx + x // B
        setw = int(O.philox([1 << 28, T, 0, 0], [9, 0])[0])
        drawn = {((setw >> (2 * r)) & 1, (setw >> (2 * r + 1)) & 1) for r in range(4)}
        assert (x % B % 2, y % B % 2) in drawn
