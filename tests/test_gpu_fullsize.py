"""The CUDA engine at the benchmark's full size (L = 2^16) and at the largest
accepted sizes (2^17, 2^18), where the oracle cannot follow every site: sampled tiles of
the first sweep against the oracle (tiles of one sweep do not interact, so
the oracle computes each from the flat start on its own window), a valid
surface (every row of sigma_x and every column of sigma_y sums to zero,
Sec. 2.1) and the exact width computed a second, independent way."""
import hashlib
import os

import numpy as np
import pytest

from oracle import oracle as O
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
    """L = 2^17: valid surface after two sweeps, and the slopes round-trip
    through an import into a second lattice (128 staging bands each way)."""
    L = 1 << 17
    lat = eng.Lattice(L, 1.0, 0.0, seed=3)
    lat.run(2)
    r = lat.roughness()
    assert r["n"] == L * L and r["t"] == 2 and r["w2"] > 0.25
    words = lat.slopes()
    w = words.reshape(L, L // 16)
    assert np.all(_popcount(w & np.uint32(0x55555555)).sum(axis=1, dtype=np.int64) == L // 2)
    lat.close()
    digest = hashlib.sha256(words.data).hexdigest()
    b = eng.Lattice(L, 1.0, 0.0, seed=3)
    b.set_slopes(words, h00=r["h00"], t=2)
    rb = b.roughness()
    assert (rb["S1"], rb["S2"], rb["h00"], rb["t"]) == (r["S1"], r["S2"], r["h00"], 2)
    words[:] = 0
    b.slopes_into(words)
    assert hashlib.sha256(words.data).hexdigest() == digest
    b.close()


def test_largest_lattice_first_sweep_matches_oracle(eng):
    """L = 2^18 (8 GiB at one bit per site, the largest accepted size): one
    sweep from the flat start, then every row of sigma_x sums to zero (checked
    in bands), and sampled tiles plus the height of site (0,0) equal the
    oracle's window computation of that sweep."""
    L, Bx, seed = 1 << 18, 128, 5
    lat = eng.Lattice(L, 1.0, 0.0, seed=seed)
    lat.run(1)
    r = lat.roughness()
    assert r["n"] == L * L and r["t"] == 1 and r["w2"] > 0.25
    words = lat.slopes()
    lat.close()
    w = words.reshape(L, L // 16)
    for j0 in range(0, L, 8192):
        assert np.all(_popcount(w[j0:j0 + 8192] & np.uint32(0x55555555)).sum(axis=1, dtype=np.int64) == L // 2)
    ntx = L // Bx
    ox, oy = O.origin(L, seed, 0, 0)
    t00 = (((L - oy) % L) // Bx) * ntx + ((L - ox) % L) // Bx
    rng = np.random.default_rng(3)
    dh00 = 0
    for T in sorted({0, ntx - 1, ntx * ntx - 1, t00} | set(rng.integers(0, ntx * ntx, 8).tolist())):
        sx, sy, (x0, y0), d = O.flat_tile_sweep(L, Bx, Bx, 1.0, 0.0, seed, 0, 0, T)
        gx, gy = _window(words, L, x0, y0, Bx, Bx)
        assert np.array_equal(gx, sx) and np.array_equal(gy, sy), T
        if T == t00:
            dh00 = d
    assert r["h00"] == dh00


def _window(words, L, x0, y0, Bx, By):
    """sigma_x, sigma_y bits of the window [v, u] = site ((x0+u) mod L, (y0+v) mod L)
    from the packed exchange format (word j*L/16 + i/16, bits 2(i%16), 2(i%16)+1)."""
    w = words.reshape(L, L // 16)
    rows = (y0 + np.arange(By)) % L
    cols = (x0 + np.arange(Bx)) % L
    sub = w[np.ix_(rows, cols // 16)]
    sh = (2 * (cols % 16)).astype(np.uint32)
    return ((sub >> sh) & 1).astype(np.uint8), ((sub >> (sh + 1)) & 1).astype(np.uint8)


@pytest.mark.parametrize("p,q,ty", [(1.0, 0.0, 128), (0.95, 0.05, 128), (1.0, 0.0, 256)])
def test_L65536_first_sweep_sampled_tiles_match_oracle(eng, p, q, ty):
    """One sweep at L = 2^16 from the flat start in the benchmark's launch
    configuration (default run length and warps per CTA); sampled tiles and the
    height of site (0,0) bit-exact against the oracle's window computation."""
    L, Bx, By, seed, sample = 65536, 128, ty, 1, 0
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, tile_y=ty)
    lat.run(1)
    words = lat.slopes()
    r = lat.roughness()
    lat.close()
    ntx, nty = L // Bx, L // By
    o = O.philox([0, 0, 0, sample], [seed & 0xFFFFFFFF, seed >> 32])
    ox, oy = int(o[0]) & (L - 1), int(o[1]) & (L - 1)
    t00 = (((L - oy) % L) // By) * ntx + ((L - ox) % L) // Bx      # tile holding site (0,0)
    rng = np.random.default_rng(7)
    tiles = {0, ntx - 1, ntx * nty - 1, ntx * (nty - 1), t00} | set(rng.integers(0, ntx * nty, 16).tolist())
    dh00 = 0
    for T in sorted(tiles):
        sx, sy, (x0, y0), d = O.flat_tile_sweep(L, Bx, By, p, q, seed, sample, 0, T)
        gx, gy = _window(words, L, x0, y0, Bx, By)
        assert np.array_equal(gx, sx) and np.array_equal(gy, sy), (p, q, ty, T)
        if T == t00:
            dh00 = d
    assert r["h00"] == dh00 and r["t"] == 1


GOLDEN = {"L4096_P1": "l4096_p1_seed1.txt", "L4096_P095": "l4096_p095_seed1.txt"}


def _golden(name):
    """Records (t, S1, S2, h00, sha256 of the packed slopes) written by
    tests/golden/make_l4096_goldens.py from the CPU oracle alone."""
    path = os.path.join(os.path.dirname(__file__), "golden", GOLDEN[name])
    if not os.path.exists(path):
        pytest.fail(f"missing oracle records {path}")
    out = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t, s1, s2, h00, digest = line.split()
        out.append((int(t), int(s1), int(s2), int(h00), digest))
    return out


@pytest.mark.parametrize("w", ["L4096_P1", "L4096_P095"])
def test_L4096_ten_thousand_sweeps(eng, w):
    """The L = 4096, 10^4-sweep workloads (p = 1 and p = 0.95, seed 1): at
    every one of the run's W^2 sampling times the packed lattice (SHA-256),
    the exact height sums S1, S2 and h(0,0) equal the oracle's records, and
    W^2 equals the value the oracle's sums give."""
    from synth import inputs as I
    W = getattr(I, w)
    L = W.L
    rec = _golden(w)
    assert [r[0] for r in rec] == I.sample_times(W.mcs)
    lat = eng.Lattice(L, W.p, W.q, seed=W.seed, sample=W.sample)
    words = np.empty(L * L // 16, np.uint32)
    for t, s1, s2, h00, digest in rec:
        r = lat.roughness()
        if t > r["t"]:
            lat.run(t - r["t"])
            r = lat.roughness()
        lat.slopes_into(words)
        got = (r["t"], r["S1"], r["S2"], r["h00"], hashlib.sha256(words.data).hexdigest())
        assert got == (t, s1, s2, h00, digest), (w, t)
        assert r["w2"] == O.w2_from_sums(L * L, s1, s2)
    _row_col_sums_ok(words, L)


@pytest.mark.parametrize("p,q,ty", [(1.0, 0.0, 128), (0.95, 0.05, 128), (0.95, 0.05, 256)])
def test_L65536_later_sweeps_sampled_tiles_match_oracle(eng, p, q, ty):
    """Sweeps 2 to 4 at L = 2^16 in the benchmark's launch configuration (runs
    of L/4096 tiles, 4-warp CTAs), each from the rough surface the GPU left:
    for sampled tiles the oracle runs the sweep on the tile's window taken
    from the GPU's lattice before the sweep (tiles of one sweep do not
    interact), and the GPU's window after the sweep and the height change of
    site (0,0) must equal it."""
    L, Bx, By, seed, sample = 65536, 128, ty, 3, 1
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, tile_y=ty)
    lat.run(1)
    ntx, nty = L // Bx, L // By
    rng = np.random.default_rng(11)
    before = lat.slopes()
    h_before = lat.roughness()["h00"]
    after = np.empty_like(before)
    for s in (1, 2, 3):
        lat.run(1)
        lat.slopes_into(after)
        r = lat.roughness()
        assert r["t"] == s + 1
        ox, oy = O.origin(L, seed, sample, s)
        t00 = (((L - oy) % L) // By) * ntx + ((L - ox) % L) // Bx
        tiles = {0, ntx - 1, ntx * nty - 1, t00} | set(rng.integers(0, ntx * nty, 12).tolist())
        dh00 = 0
        for T in sorted(tiles):
            x0, y0 = O.tile_anchor(L, Bx, By, seed, sample, s, T)
            wx, wy = _window(before, L, x0, y0, Bx, By)
            sx, sy, d = O.window_tile_sweep(L, Bx, By, p, q, seed, sample, s, T, wx, wy)
            gx, gy = _window(after, L, x0, y0, Bx, By)
            assert np.array_equal(gx, sx) and np.array_equal(gy, sy), (p, q, ty, s, T)
            if T == t00:
                dh00 = d
        assert r["h00"] - h_before == dh00, (p, q, ty, s)
        before, after = after, before
        h_before = r["h00"]
    lat.close()


def test_full_size_import_export_round_trip(eng):
    """Slopes written back through the banded import (32 bands of 2048 rows at
    L = 2^16, copies overlapping the conversion) give the same lattice: the
    same slopes and exact width, and after more sweeps the same state as the
    original run. With an odd h(0,0) every stored bit differs and the slopes
    still round-trip."""
    L = 1 << 16
    a = eng.Lattice(L, 1.0, 0.0, seed=4)
    a.run(5)
    words, r = a.slopes(), a.roughness()
    b = eng.Lattice(L, 1.0, 0.0, seed=4)
    for h00 in (r["h00"] + 1, r["h00"]):
        b.set_slopes(words, h00=h00, t=5)
        rb = b.roughness()
        assert (rb["S1"], rb["S2"], rb["h00"], rb["t"]) == (r["S1"], r["S2"], h00, 5)
        assert np.array_equal(b.slopes(), words)
    a.run(3)
    b.run(3)
    assert np.array_equal(a.slopes(), b.slopes())
    assert a.roughness()["h00"] == b.roughness()["h00"]
