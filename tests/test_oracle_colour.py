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


def _sync_by_heights(h, classes, p, q):
    """Whole sublattices at once, on heights: for each class (cx, cy) in turn,
    every site (x, y) with x = cx, y = cy mod 2 that is a local minimum rises
    by 2 (if p) and every local maximum falls by 2 (if q) (eq. rule, Sec. 2.1),
    all of them simultaneously; heights indexed [y, x], periodic."""
    h = h.copy()
    for c in classes:
        cx, cy = c & 1, c >> 1
        nb = [np.roll(h, 1, 0), np.roll(h, -1, 0), np.roll(h, 1, 1), np.roll(h, -1, 1)]
        lo = np.all([n > h for n in nb], axis=0)
        hi = np.all([n < h for n in nb], axis=0)
        on = np.zeros_like(lo)
        on[cy::2, cx::2] = True
        h = h + 2 * (lo & on & (p == 1.0)) - 2 * (hi & on & (q == 1.0))
    return h


@pytest.mark.parametrize("p,q", [(1.0, 0.0), (0.0, 1.0), (1.0, 1.0)])
def test_synchronous_limit_equals_sublattice_updates_on_heights(p, q):
    """At m = 0 every site of the drawn class is attempted and acceptance is
    certain, so a sweep is four synchronous sublattice updates; the classes
    come from philox(6 << 28 | i, 0xffffffff, s, sample). Checked on absolute
    heights, independently of the oracle's slope representation."""
    L, seed, sample = 128, 11, 2
    st = O.State.flat(L)
    h = st.heights(absolute=True)
    for s in range(5):
        classes = [int(O.philox([(6 << 28) | i, 0xFFFFFFFF, s, sample], [seed, 0])[0]) & 3 for i in range(4)]
        h = _sync_by_heights(h, classes, p, q)
        st.sweep_colour(p, q, seed, sample, m=0)
        assert np.array_equal(st.heights(absolute=True), h), s
