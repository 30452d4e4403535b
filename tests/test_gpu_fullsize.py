"""Properties of the CUDA engine at the benchmark's full size (L = 2^16) and at
the largest accepted size, where the oracle cannot follow every site:
a valid surface (every row of sigma_x and every column of sigma_y sums to
zero, Sec. 2.1) and the exact width computed a second, independent way."""
import numpy as np
import pytest

from tests.gpu_util import engine

pytestmark = pytest.mark.gpu


def _popcount(a):
    if hasattr(np, "bitwise_count"):
        return np.bitwise_count(a)
    a = a.astype(np.uint32)
    a = a - ((a >> 1) & 0x55555555)
    a = (a & 0x33333333) + ((a >> 2) & 0x33333333)
    return (((a + (a >> 4)) & 0x0F0F0F0F) * 0x01010101 & 0xFFFFFFFF) >> 24


@pytest.fixture(scope="module")
def eng():
    return engine()


def _row_col_sums_ok(words, L):
    w = words.reshape(L, L // 16)
    sx_rows = _popcount(w & np.uint32(0x55555555)).sum(axis=1, dtype=np.int64)
    assert np.all(sx_rows == L // 2)
    cols = np.zeros(L, np.int64)
    for b in range(16):
        cols[b::16] = ((w >> np.uint32(2 * b + 1)) & np.uint32(1)).sum(axis=0, dtype=np.int64)
    assert np.all(cols == L // 2)


def _w2_host(words, L):
    """S1, S2 from the packed slopes on the host (gauge h(0,0) = 0)."""
    w = words.reshape(L, L // 16)
    sy0 = ((w[:, 0] >> np.uint32(1)) & np.uint32(1)).astype(np.int64) * 2 - 1
    col0 = np.concatenate([[0], np.cumsum(sy0)[:-1]])
    S1, S2 = 0, 0
    band = max(1, (1 << 24) // L)
    shifts = (2 * np.arange(16, dtype=np.uint32))
    for j0 in range(0, L, band):
        blk = w[j0:j0 + band]
        sx = ((blk[:, :, None] >> shifts) & np.uint32(1)).reshape(blk.shape[0], L).astype(np.int32) * 2 - 1
        h = np.cumsum(sx, axis=1, dtype=np.int64)
        h = np.concatenate([np.zeros((blk.shape[0], 1), np.int64), h[:, :-1]], axis=1)
        h += col0[j0:j0 + band, None]
        S1 += int(h.sum())
        S2 += int((h * h).sum())
    return S1, S2


def test_full_size_valid_and_exact_width(eng):
    L = 1 << 16
    lat = eng.Lattice(L, 1.0, 0.0, seed=1)
    lat.run(20)
    r = lat.roughness()
    words = lat.slopes()
    _row_col_sums_ok(words, L)
    assert r["t"] == 20 and r["w2"] > 0.25


def test_width_matches_host_recomputation(eng):
    L = 1 << 13
    lat = eng.Lattice(L, 0.95, 0.05, seed=2)
    lat.run(30)
    r = lat.roughness()
    words = lat.slopes()
    _row_col_sums_ok(words, L)
    assert (r["S1"], r["S2"]) == _w2_host(words, L)


def test_largest_lattice(eng):
    L = 1 << 17
    lat = eng.Lattice(L, 1.0, 0.0, seed=3)
    lat.run(2)
    r = lat.roughness()
    assert r["n"] == L * L and r["t"] == 2 and r["w2"] > 0.25
    words = lat.slopes()
    w = words.reshape(L, L // 16)
    assert np.all(_popcount(w & np.uint32(0x55555555)).sum(axis=1, dtype=np.int64) == L // 2)
