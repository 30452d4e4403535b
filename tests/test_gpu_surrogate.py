"""The learned surrogate of W^2(t; L, p, q) (not part of the paper): trained by
the engine's own kernels on W^2 curves the batched simulator produces, it
must stay within 5 % of freshly simulated ensemble means at (L, p) it has not
seen, and its saturation times must let the batcher stop runs early while
still reaching the plateau, against the fixed run length 4 L^1.6."""
import math

import numpy as np
import pytest

from tests.gpu_util import engine

pytestmark = pytest.mark.gpu

P_TRAIN = [0.7, 0.8, 0.9, 1.0]
P_TEST = [0.75, 0.95]
LS = [128, 256]


def heuristic(L):
    return int(min(math.ceil(4 * L ** 1.6), 100_000))


def ensemble(eng, pairs, seeds, n_samples=48, run_len=lambda L, p: heuristic(L)):
    specs = [(L, p, 1.0 - p, 100 + s, s, run_len(L, p)) for (L, p) in pairs for s in seeds]
    b = eng.Batch(specs, n_samples=n_samples)
    b.run()
    times, w2 = b.times(), b.w2()
    b.close()
    means = {}
    for (L, p) in pairs:
        rows = [k for k, sp in enumerate(specs) if sp[0] == L and sp[1] == p]
        with np.errstate(invalid="ignore"):
            cols = np.isfinite(w2[rows]).any(axis=0)
            means[(L, p)] = np.full(w2.shape[1], np.nan)
            means[(L, p)][cols] = np.nanmean(w2[rows][:, cols], axis=0)
    return specs, times, w2, means


@pytest.fixture(scope="module")
def trained():
    eng = engine()
    from paper_1204_5072_gb300 import surrogate as S
    pairs = [(L, p) for L in LS for p in P_TRAIN]
    _, times, _, means = ensemble(eng, pairs, range(64))
    # train on ensemble-mean curves: one row per (L, p, t)
    specs = [(L, p, 1.0 - p, 0, 0, heuristic(L)) for (L, p) in pairs]
    w2 = np.stack([means[k] for k in pairs])
    sur = S.Surrogate.fit(specs, times, w2, epochs=400, batch=128, lr=3e-3, seed=1)
    yield eng, S, sur
    sur.close()


def test_held_out_error_within_5_percent(trained):
    eng, S, sur = trained
    pairs = [(L, p) for L in LS for p in P_TEST]
    _, times, _, means = ensemble(eng, pairs, range(200, 328))
    for (L, p), m in means.items():
        sel = (times >= 1) & (times <= heuristic(L)) & np.isfinite(m)
        pred = sur.w2(L, times[sel], p, 1.0 - p)
        rel = np.abs(pred / m[sel] - 1.0)
        assert rel.mean() < 0.05, ((L, p), rel.mean(), rel.max())


def test_planned_run_lengths_reach_saturation_with_fewer_sweeps(trained):
    eng, S, sur = trained
    pairs = [(L, p) for L in LS for p in P_TEST]
    planned = {(L, p): int(min(heuristic(L), math.ceil(2.0 * sur.t_sat(L, p, 1.0 - p, t_max=heuristic(L)))))
               for (L, p) in pairs}
    # long reference runs give the plateau; planned runs must end on it
    _, t_long, _, long_means = ensemble(eng, pairs, range(400, 464))
    _, t_plan, _, plan_means = ensemble(eng, pairs, range(400, 464), run_len=lambda L, p: planned[(L, p)])
    saved = 0.0
    for (L, p) in pairs:
        T = planned[(L, p)]
        plateau = np.nanmean(long_means[(L, p)][(t_long >= 0.5 * heuristic(L))])
        end = plan_means[(L, p)][int(np.searchsorted(t_plan, T))]   # every run is sampled at its end
        assert abs(end / plateau - 1.0) < 0.05, ((L, p), T, end, plateau)
        saved += (heuristic(L) - T) * L * L
    total = sum(heuristic(L) * L * L for (L, p) in pairs)
    assert saved / total > 0.3, saved / total
