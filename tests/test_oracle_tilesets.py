"""Pins of the oracle's tile-set variant of the device layer (four sets of
tiles swept one after the other in a random order, no dead border; the
double tiling the paper describes for its KMC model, Sec. 3.2)."""
import collections
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_schedule import _check_valid


def test_set_order_is_a_uniform_permutation():
    counts = collections.Counter(tuple(O.tileset_order(s, 0, 7)) for s in range(4800))
    assert set(counts) <= set(itertools.permutations(range(4)))
    assert len(counts) == 24
    # 200 expected per permutation; 4.5 standard deviations either way
    assert all(200 - 64 < c < 200 + 64 for c in counts.values()), counts


@pytest.mark.parametrize("L,Bx,By,p,q", [(64, 16, 16, 1.0, 0.0), (128, 32, 16, 0.7, 0.3), (256, 128, 128, 0.95, 0.05)])
def test_surface_stays_valid(L, Bx, By, p, q):
    st = O.State.flat(L)
    for _ in range(6):
        st.sweep_tilesets(Bx, By, p, q, 3, 1)
        _check_valid(st)


def test_no_rates_no_change_and_order_inside_a_phase_is_free():
    st = O.State.flat(128).run_tilesets(4, 32, 32, 0.0, 0.0, 5, 0)
    assert np.array_equal(st.packed(), O.State.flat(128).packed())
    ref = O.State.flat(128)
    for _ in range(4):
        ref.sweep_tilesets(32, 32, 0.8, 0.2, 5, 0, order=0)
    for order in (1, 2, 12345):
        st = O.State.flat(128)
        for _ in range(4):
            st.sweep_tilesets(32, 32, 0.8, 0.2, 5, 0, order=order)
        assert np.array_equal(st.packed(), ref.packed()) and st.h00 == ref.h00


def test_border_sites_are_live():
    """Without a dead border a sweep can move sites on a tile's low-x column
    and low-y row; the dead-border sweep with the same keys never does."""
    L, B = 128, 16
    o = O.philox([0, 0, 0, 0], [9, 0])
    ox, oy = int(o[0]) & (L - 1), int(o[1]) & (L - 1)
    border = np.zeros((L, L), bool)
    border[:, (ox + np.arange(0, L, B)) % L] = True
    border[(oy + np.arange(0, L, B)) % L, :] = True
    h0 = O.State.flat(L).heights(absolute=True)
    ts = O.State.flat(L).sweep_tilesets(B, B, 1.0, 0.0, 9, 0)
    db = O.State.flat(L).sweep(B, B, 1.0, 0.0, 9, 0)
    assert np.any((ts.heights(absolute=True) != h0) & border)
    assert not np.any((db.heights(absolute=True) != h0) & border)


def test_bad_shapes_are_rejected():
    with pytest.raises(ValueError):
        O.State.flat(64).sweep_tilesets(64, 16, 1.0, 0.0, 1, 0)   # one tile per row: no second set
