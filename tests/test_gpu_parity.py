"""Bit-exact parity of the CUDA engine with the CPU oracle, through the C ABI.

The engine and the oracle implement the same decomposed schedule
(arXiv:1204.5072, Sec. 3, 3.1; update rule eq. rule, Sec. 2.1) independently;
integer state must agree bit for bit: the packed slopes, the exact height
sums S1 and S2 of eq. (Wdef), and the tracked height of site (0,0).
"""
import numpy as np
import pytest

from oracle import oracle as O
from synth import inputs as I
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu
TILE = 128


@pytest.fixture(scope="module")
def eng():
    return engine()


def _same(lat, st, where=""):
    got = lat.slopes()
    want = st.packed()
    if not np.array_equal(got, want):
        bad = np.flatnonzero(got != want)
        L = st.L
        j, wi = divmod(int(bad[0]), L // 16)
        raise AssertionError(f"{where}: {bad.size} packed words differ, first at row {j} word {wi}")
    r = lat.roughness()
    s1, s2 = st.sums()
    assert (r["S1"], r["S2"]) == (s1, s2), where
    assert r["h00"] == st.h00, where
    assert r["w2"] == st.w2(), where
    assert r["t"] == st.t, where


def test_flat_start(eng):
    for L in (128, 256, 1024):
        lat = eng.Lattice(L)
        st = O.State.flat(L)
        _same(lat, st, f"L={L}")
        r = lat.roughness()
        assert r["S1"] == L * L // 2 and r["S2"] == L * L // 2 and r["w2"] == 0.25


def test_import_export_heights(eng):
    states = [O.State(256, *I.separable_surface(256, 3)),
              O.State.flat(256).run(15, TILE, TILE, 0.8, 0.3, seed=9),
              O.State.flat(512).run(6, 64, 32, 1.0, 0.0, seed=2)]
    for k, st in enumerate(states):
        st.h00 = 10 * k - 7
        lat = eng.Lattice(st.L)
        lat.set_slopes(st.packed(), h00=st.h00, t=st.t)
        assert np.array_equal(lat.slopes(), st.packed())
        assert np.array_equal(lat.heights(), st.heights())
        assert np.array_equal(lat.heights(absolute=True), st.heights(absolute=True))
        r = lat.roughness()
        assert (r["S1"], r["S2"], r["h00"]) == (*st.sums(), st.h00)


CASES = [
    (128, 1.0, 0.0, 1, 0, 6),       # one tile: the run wraps onto itself
    (256, 1.0, 0.0, 1, 0, 8),
    (256, 0.95, 0.05, 1, 0, 6),
    (512, 0.6, 0.3, 77, 5, 5),
    (256, 0.5, 0.5, 3, 1, 5),       # lambda = 0
    (256, 1.0, 1.0, 4, 0, 4),       # both thresholds 2^16: no acceptance draws
    (256, 0.0, 1.0, 5, 2, 4),
    (256, 0.3, 0.0, 6, 0, 4),
    (256, 0.0, 0.0, 7, 0, 3),       # nothing may flip
    (1024, 1.0, 0.0, (1 << 40) + 3, 9, 4),
]


@pytest.mark.parametrize("L,p,q,seed,sample,n", CASES)
def test_sweeps_bit_exact(eng, L, p, q, seed, sample, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.sweep(TILE, TILE, p, q, seed, sample)
        _same(lat, st, f"L={L} p={p} q={q} after sweep {k + 1}")


def test_L256_1000mcs_every_checkpoint(eng):
    w = I.L256_1000
    lat = eng.Lattice(w.L, w.p, w.q, seed=w.seed, sample=w.sample)
    st = O.State.flat(w.L)
    for t in I.sample_times(w.mcs):
        n = t - st.t
        if n:
            lat.run(n)
            st.run(n, w.bx, w.by, w.p, w.q, w.seed, w.sample)
        _same(lat, st, f"t={t}")


def test_L1024_subrun(eng):
    lat = eng.Lattice(1024, 1.0, 0.0, seed=1)
    st = O.State.flat(1024)
    for n in (1, 4, 15):
        lat.run(n)
        st.run(n, TILE, TILE, 1.0, 0.0, 1, 0)
        _same(lat, st, f"t={st.t}")


def test_L4096_general_rates(eng):
    lat = eng.Lattice(4096, 0.95, 0.05, seed=1)
    st = O.State.flat(4096)
    lat.run(2)
    st.run(2, TILE, TILE, 0.95, 0.05, 1, 0)
    _same(lat, st, "L=4096")


def test_execution_knobs_do_not_change_result(eng):
    ref = None
    for run in (1, 2, 4, 8):
        for wpc in (1, 3, 8):
            lat = eng.Lattice(1024, 0.9, 0.1, seed=12, run=run, warps_per_cta=wpc)
            lat.run(5)
            w = lat.slopes()
            if ref is None:
                ref = (w, lat.roughness())
            else:
                assert np.array_equal(w, ref[0]), (run, wpc)
                assert lat.roughness() == ref[1]


@pytest.mark.parametrize("p,q", [(1.0, 0.0), (0.9, 0.1)])
def test_long_runs_of_tiles_match_oracle(eng, p, q):
    """Runs of 16 and 32 tiles (the lengths the engine picks from L = 2^16
    up) and shorter ones at L = 4096, with 1, 4 and 8 warps per CTA, over
    sweeps 1..4 from the flat start and then 3 more from the rough surface:
    every schedule equals the oracle bit for bit after each sweep."""
    L, seed = 4096, 13
    st = O.State.flat(L)
    want = []
    for _ in range(7):
        st.run_threads(1, TILE, TILE, p, q, seed, 0)
        want.append((st.packed(), st.sums(), st.h00))
    for run in (32, 16, 8, 1):
        for wpc in ((1, 4, 8) if run >= 16 else (4,)):
            lat = eng.Lattice(L, p, q, seed=seed, run=run, warps_per_cta=wpc)
            for k, (words, sums, h00) in enumerate(want):
                lat.run(1)
                r = lat.roughness()
                assert np.array_equal(lat.slopes(), words), (p, run, wpc, k + 1)
                assert ((r["S1"], r["S2"]), r["h00"]) == (sums, h00), (p, run, wpc, k + 1)
            lat.close()


def test_resume_is_bit_exact(eng):
    a = eng.Lattice(512, 0.7, 0.2, seed=4, sample=3)
    a.run(7)
    words, r = a.slopes(), a.roughness()
    b = eng.Lattice(512, 0.7, 0.2, seed=4, sample=3)
    b.set_slopes(words, h00=r["h00"], t=7)
    a.run(5)
    b.run(5)
    assert np.array_equal(a.slopes(), b.slopes())
    assert a.roughness() == b.roughness()


def test_rerun_is_deterministic(eng):
    outs = []
    for _ in range(2):
        lat = eng.Lattice(2048, 1.0, 0.0, seed=5)
        lat.run(10)
        outs.append((lat.slopes(), lat.roughness()))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


# Thresholds at the edges of the acceptance comparison (T = p 2^16): T = 1 and
# 65535; T = 0x8000 (a tie with the top four bits never accepts: the low
# twelve bits of T are 0) and 0x8FFF (a tie accepts unless the low bits are
# 0xFFF); from the flat start every attempted site is a candidate, so many
# rows have five or more ties and take the overflow blocks.
EDGE = [(1 / 65536, 65535 / 65536), (0x8000 / 65536, 0x8FFF / 65536), (0x8FFF / 65536, 0x0001 / 65536),
        (0x1000 / 65536, 0xF000 / 65536)]


@pytest.mark.parametrize("p,q", EDGE)
def test_threshold_edges_bit_exact(eng, p, q):
    assert (O.threshold(p), O.threshold(q)) in [(1, 65535), (0x8000, 0x8FFF), (0x8FFF, 1), (0x1000, 0xF000)]
    for ty in (TILE, 2 * TILE):
        lat = eng.Lattice(512, p, q, seed=19, sample=2, tile_y=ty)
        st = O.State.flat(512)
        for k in range(3):
            lat.run(1)
            st.sweep(TILE, ty, p, q, 19, 2)
            _same(lat, st, f"p={p} q={q} By={ty} after sweep {k + 1}")
        lat.close()


# 128 x 256 tiles (two cell rows per lane): the same schedule with By = 256.
CASES_TALL = [
    (256, 1.0, 0.0, 1, 0, 6),        # one tile row: the tile wraps onto itself in y
    (512, 1.0, 0.0, 2, 0, 6),
    (512, 0.95, 0.05, 3, 1, 5),
    (1024, 0.6, 0.3, 77, 5, 4),
    (512, 0.0, 1.0, 5, 2, 4),
]


@pytest.mark.parametrize("L,p,q,seed,sample,n", CASES_TALL)
def test_tall_tiles_bit_exact(eng, L, p, q, seed, sample, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, tile_y=2 * TILE)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.sweep(TILE, 2 * TILE, p, q, seed, sample)
        _same(lat, st, f"L={L} p={p} q={q} By=256 after sweep {k + 1}")


def test_tall_tiles_knobs_and_resume(eng):
    ref = None
    for run in (1, 4, 8):
        for wpc in (1, 2, 4):
            lat = eng.Lattice(2048, 0.9, 0.1, seed=12, run=run, warps_per_cta=wpc, tile_y=2 * TILE)
            lat.run(3)
            w = lat.slopes()
            if ref is None:
                ref = (w, lat.roughness())
            else:
                assert np.array_equal(w, ref[0]), (run, wpc)
                assert lat.roughness() == ref[1]
    st = O.State.flat(2048).run(3, TILE, 2 * TILE, 0.9, 0.1, 12, 0)
    assert np.array_equal(ref[0], st.packed())
    b = eng.Lattice(2048, 0.9, 0.1, seed=12, tile_y=2 * TILE)
    b.set_slopes(ref[0], h00=ref[1]["h00"], t=3)
    b.run(1)
    st.sweep(TILE, 2 * TILE, 0.9, 0.1, 12, 0)
    _same(b, st, "resume with By=256")


def test_zero_sweeps_change_nothing(eng):
    for L, p, q in [(128, 1.0, 0.0), (256, 0.8, 0.3)]:
        lat = eng.Lattice(L, p, q, seed=5)
        lat.run(0)
        _same(lat, O.State.flat(L), f"L={L} t=0")
        lat.run(3)
        words, r = lat.slopes(), lat.roughness()
        lat.run(0)
        assert np.array_equal(lat.slopes(), words) and lat.roughness() == r
        lat.close()
