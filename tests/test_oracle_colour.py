"""Pins of the oracle's random-sequential reference by colour classes (each
sweep 4 * 2^m sub-steps; a sub-step attempts a random 2^-m subset of one
period-2 sublattice, whose sites are never neighbours): valid surfaces, the
p = q = 0 identity, and agreement with plain random-sequential updates that
improves as the subsets thin out (m = 4) while the synchronous limit (m = 0,
whole sublattices at once) is far from it."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.test_oracle_schedule import _check_valid


def test_valid_surfaces_and_no_rates():
    st = O.State.flat(128)
    for m in (0, 2, 4):
        st.sweep_colour(0.8, 0.3, 5, 1, m=m)
        _check_valid(st)
    z = O.State.flat(128)
    for _ in range(3):
        z.sweep_colour(0.0, 0.0, 5, 0, m=3)
    assert np.array_equal(z.packed(), O.State.flat(128).packed())


def _ens(fn, n, ts):
    out = np.zeros((n, len(ts)))
    for k in range(n):
        st = O.State.flat(128)
        for j, t in enumerate(ts):
            while st.t < t:
                fn(st, k)
            out[k, j] = st.w2()
    return out


def test_thin_subsets_approach_random_sequential_updates():
    ts = [1, 2, 4, 8, 16]
    rsu = _ens(lambda st, k: st.rsu(1, 1.0, 0.0, seed=3, sample=k), 24, ts)
    col = _ens(lambda st, k: st.sweep_colour(1.0, 0.0, 4, k, m=4), 24, ts)
    sync = _ens(lambda st, k: st.sweep_colour(1.0, 0.0, 4, k, m=0), 8, ts)
    mr, mc, ms = rsu.mean(0), col.mean(0), sync.mean(0)
    err = np.sqrt(rsu.var(0, ddof=1) / 24 + col.var(0, ddof=1) / 24)
    assert np.all(np.abs(mc - mr) < 0.03 * mr + 4 * err), (mc / mr - 1)
    # whole sublattices at once: from the flat start at p = 1 a class of minima
    # rises together, which keeps the surface nearly flat
    assert abs(ms[-1] - mr[-1]) > 0.5 * mr[-1], (ms, mr)
