"""The oracle's update against the matrices the paper prints for its rule
(Sec. 2.1, eq. rule; fixture tests/golden/rule_matrices.txt): a site whose
slope matrix is the printed left-hand side becomes the right-hand side on an
accepted attachment, and back on an accepted detachment; sites with any
other matrix do not move."""
import os

import numpy as np

from oracle import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _printed():
    rows = {}
    for line in open(os.path.join(HERE, "golden", "rule_matrices.txt")):
        if line.strip() and not line.startswith("#"):
            name, *vals = line.split()
            rows[name] = np.array([int(v) for v in vals]).reshape(2, 2)
    return rows["before"], rows["after"]


def _matrix(st, i, j):
    L = st.L
    pm = lambda b: 1 if b else -1   # bit 1 = +1
    return np.array([[pm(st.sx[j, (i - 1) % L]), pm(st.sx[j, i])],
                     [pm(st.sy[(j - 1) % L, i]), pm(st.sy[j, i])]])


def test_printed_rule_on_the_flat_start():
    before, after = _printed()
    L = 8
    st = O.State.flat(L)
    h0 = st.heights()
    # flat start h = (i + j) & 1: even sites have the printed left-hand side
    i, j = 2, 4
    assert np.array_equal(_matrix(st, i, j), before)
    assert st.attempt(i, j, acc_min=False, acc_max=True) == 0          # p not accepted
    assert st.attempt(i, j, acc_min=True, acc_max=False) == 2          # attachment: h + 2
    assert np.array_equal(_matrix(st, i, j), after)
    h = st.heights()
    assert h[j, i] - h0[j, i] == 2 and np.count_nonzero(h != h0) == 1
    assert st.attempt(i, j, acc_min=True, acc_max=False) == 0          # q not accepted
    assert st.attempt(i, j, acc_min=False, acc_max=True) == -2         # detachment: back
    assert np.array_equal(_matrix(st, i, j), before)
    assert np.array_equal(st.heights(), h0)


def test_other_matrices_do_not_move():
    before, after = _printed()
    st = O.State.flat(8).run(3, 4, 4, 0.8, 0.3, seed=5)
    L = st.L
    for j in range(L):
        for i in range(L):
            m = _matrix(st, i, j)
            if np.array_equal(m, before) or np.array_equal(m, after):
                continue
            sx, sy = st.sx.copy(), st.sy.copy()
            assert st.attempt(i, j, True, True) == 0
            assert np.array_equal(st.sx, sx) and np.array_equal(st.sy, sy)
