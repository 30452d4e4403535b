"""The batched ensemble (one persistent launch for many realisations) gives,
for every realisation, the exact sums a single-lattice run gives at the same
sample times (same decomposition, Sec. 3 of arXiv:1204.5072, same Philox
streams); the scheduling knobs and the autotuner never change results; a
device-side wait that cannot succeed ends in KPZ_ETIMEOUT, not a hang."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu

SPECS = [(256, 1.0, 0.0, 1, 0, 30), (128, 0.9, 0.1, 7, 3, 12), (512, 0.6, 0.4, 2, 1, 9),
         (256, 0.75, 0.25, 1, 5, 20), (128, 1.0, 0.0, 3, 2, 25), (1024, 0.95, 0.05, 4, 0, 5)]


@pytest.fixture(scope="module")
def eng():
    return engine()


def _single(eng, L, p, q, seed, sample, n, times, tile_y=0):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, tile_y=tile_y)
    out, t0 = {}, 0
    for t in times:
        if t > n:
            break
        if t > t0:
            lat.run(t - t0)
        r = lat.roughness()
        out[t] = (r["S1"], r["S2"], r["h00"])
        t0 = t
    lat.close()
    return out


def test_batch_matches_single_lattice_runs(eng):
    b = eng.Batch(SPECS, n_samples=12)
    b.run()
    times = [int(t) for t in b.times()]
    assert times[0] == 0 and max(s[5] for s in SPECS) == times[-1]
    s1, s2, h00 = b.sums()
    w2 = b.w2()
    for i, spec in enumerate(SPECS):
        ref = _single(eng, *spec, times)
        for k, t in enumerate(times):
            if t > spec[5]:
                assert np.isnan(w2[i, k])
                continue
            assert (int(s1[i, k]), s2[i, k]) == ref[t][:2], (spec, t)
        assert h00[i] == ref[spec[5]][2]
    b.close()


def test_batch_member_matches_oracle(eng):
    L, p, q, seed, sample, n = 128, 0.7, 0.2, 9, 4, 6
    b = eng.Batch([(L, p, q, seed, sample, n), (256, 1.0, 0.0, 1, 0, 3)], n_samples=4)
    b.run()
    times = [int(t) for t in b.times()]
    s1, s2, _ = b.sums()
    st = O.State.flat(L).run(n, 128, 128, p, q, seed, sample)
    k = times.index(n)
    assert (int(s1[0, k]), s2[0, k]) == st.sums()
    b.close()


def test_knobs_and_autotune_do_not_change_results(eng):
    ref = None
    for kw in [dict(run=1, warps_per_cta=8), dict(run=4, warps_per_cta=4, ctas_per_sm=1),
               dict(run=8, warps_per_cta=2), dict(autotune=True)]:
        b = eng.Batch(SPECS, n_samples=8, **kw)
        b.run()
        s1, s2, h = b.sums()
        got = (s1.tolist(), s2.tolist(), h.tolist())
        if ref is None:
            ref = got
        assert got == ref, kw
        if kw.get("autotune"):
            info = b.info()
            assert len(info["probe_ms"]) == 8
        b.close()


def test_rerun_is_identical(eng):
    b = eng.Batch(SPECS[:3], n_samples=6)
    b.run()
    first = b.sums()
    b.run()
    second = b.sums()
    assert first[0].tolist() == second[0].tolist() and first[1].tolist() == second[1].tolist()
    b.close()


def test_wait_that_never_succeeds_times_out(eng):
    from paper_1204_5072_gb300 import KpzError
    from paper_1204_5072_gb300._lib import KPZ_ETIMEOUT
    b = eng.Batch(SPECS[:2], n_samples=4, timeout_ms=200, test_block=0)
    with pytest.raises(KpzError) as e:
        b.run()
    assert e.value.status == KPZ_ETIMEOUT
    b.close()
    ok = eng.Batch(SPECS[:2], n_samples=4)      # the device stays usable
    ok.run()
    ok.close()


SPECS_TALL = [(256, 1.0, 0.0, 1, 0, 14), (512, 0.8, 0.2, 7, 3, 9), (1024, 0.95, 0.05, 2, 1, 4),
              (256, 0.5, 0.5, 3, 2, 11)]


def test_tall_tile_batch_matches_single_lattice_runs(eng):
    """128 x 256 tiles in the batch give the single-lattice 128 x 256 schedule."""
    b = eng.Batch(SPECS_TALL, n_samples=6, tile_y=256)
    assert b.info()["tile_y"] == 256
    b.run()
    times = [int(t) for t in b.times()]
    s1, s2, h00 = b.sums()
    for i, spec in enumerate(SPECS_TALL):
        ref = _single(eng, *spec, times, tile_y=256)
        for k, t in enumerate(times):
            if t <= spec[5]:
                assert (int(s1[i, k]), s2[i, k]) == ref[t][:2], (spec, t)
        assert h00[i] == ref[spec[5]][2]
    b.close()


def test_autotuned_tile_shape_is_reported_and_reproducible(eng):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KpzError
    b = eng.Batch(SPECS_TALL, n_samples=6, autotune=True)
    info = b.info()
    assert info["tile_y"] in (128, 256) and len(info["probe_ms"]) == 8
    b.run()
    got = b.sums()
    b.close()
    fixed = eng.Batch(SPECS_TALL, n_samples=6, tile_y=info["tile_y"])
    fixed.run()
    ref = fixed.sums()
    fixed.close()
    assert all(np.array_equal(a, c) for a, c in zip(got, ref))
    with pytest.raises(KpzError) as e:   # 128 x 256 tiles need L >= 256
        eng.Batch([(128, 1.0, 0.0, 1, 0, 3)], tile_y=256)
    assert e.value.status == KPZ_EINVAL


def test_members_without_sweeps(eng):
    """A member with zero sweeps is sampled once, at t = 0 (the flat start,
    W^2 = 1/4 exactly, Sec. 2.1), and is NaN after; the others are unchanged.
    A batch of such members alone has the single time t = 0."""
    specs = [(256, 1.0, 0.0, 1, 0, 0), (128, 0.9, 0.1, 7, 3, 12), (128, 1.0, 0.0, 2, 1, 0)]
    b = eng.Batch(specs, n_samples=6, timeout_ms=2000)
    b.run()
    times = [int(t) for t in b.times()]
    w2 = b.w2()
    s1, s2, h00 = b.sums()
    for i in (0, 2):
        assert w2[i, 0] == 0.25 and np.all(np.isnan(w2[i, 1:])) and h00[i] == 0
    ref = _single(eng, *specs[1], times)
    for k, t in enumerate(times):
        assert (int(s1[1, k]), s2[1, k]) == ref[t][:2], t
    b.close()
    z = eng.Batch([(128, 1.0, 0.0, 1, 0, 0), (512, 0.5, 0.5, 3, 0, 0)], timeout_ms=2000)
    z.run()
    assert [int(t) for t in z.times()] == [0] and np.all(z.w2() == 0.25)
    z.close()
