"""Random-sequential updates on the GPU (kpz_opts.decomposition = 4): the
undecomposed dynamics, one uniformly random site per attempt and L^2
attempts per sweep (Sec. 2.1, eq. rule), run in rounds of non-neighbouring
sites whose next attempt is the earliest around them. The result must equal
the oracle's one-at-a-time random-sequential run (orc_rsu_run, pinned in
test_oracle_rsu.py) bit for bit: packed lattice, exact height sums and the
height of site (0,0) after every sweep."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_util import engine
from tests.test_gpu_parity import _same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    return engine()


@pytest.mark.parametrize("L,p,q,seed,sample,n", [
    (128, 1.0, 0.0, 1, 0, 5), (256, 0.9, 0.1, 2, 3, 4), (256, 0.5, 0.5, 7, 1, 3),
    (512, 0.6, 0.3, (1 << 40) + 5, 2, 3), (256, 0.0, 1.0, 4, 0, 3), (128, 0.0, 0.0, 5, 0, 2)])
def test_exact_rsu_sweeps_bit_exact(eng, L, p, q, seed, sample, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, decomposition=4)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.rsu(1, p, q, seed, sample)
        _same(lat, st, f"random-sequential L={L} p={p} q={q} after sweep {k + 1}")


def test_exact_rsu_resume_and_options(eng, tmp_path):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KpzError
    a = eng.Lattice(256, 0.8, 0.2, seed=6, decomposition=4)
    a.run(2)
    a.save(tmp_path / "rsu.kpz")
    b = eng.Lattice.load(tmp_path / "rsu.kpz")
    b.run(2)
    st = O.State.flat(256).rsu(4, 0.8, 0.2, 6, 0)
    _same(b, st, "random-sequential after a checkpoint")
    for kw in ({"L": 16384}, {"tile_y": 256}, {"cell": 2}):
        args = {"L": 256, "decomposition": 4}
        args.update(kw)
        with pytest.raises(KpzError) as e:
            eng.Lattice(args.pop("L"), 1.0, 0.0, **args)
        assert e.value.status == KPZ_EINVAL


def test_decomposed_dynamics_against_exact_rsu_at_L512(eng):
    """The paper's decomposed dynamics (dead-border tiles, single-hit double
    tiling) against exact random-sequential updates, both on the GPU, at
    L = 512, p = 1: W^2(t) within the single-hit offset (7 %, the oracle at
    L = 128-256 measures 3-6 %) plus 4 sigma, and the same growth exponent."""
    L, ts, n = 512, [1, 2, 4, 8, 16, 32, 64, 128, 256], 24
    W = {}
    for dec in (0, 4):
        w = np.zeros((n, len(ts)))
        for k in range(n):
            lat = eng.Lattice(L, 1.0, 0.0, seed=31 + dec, sample=k, decomposition=dec)
            t0 = 0
            for j, t in enumerate(ts):
                lat.run(t - t0)
                t0 = t
                w[k, j] = lat.roughness()["w2"]
            lat.close()
        W[dec] = w
    md, mr = W[0].mean(0), W[4].mean(0)
    err = np.sqrt(W[0].var(0, ddof=1) / n + W[4].var(0, ddof=1) / n)
    assert np.all(np.abs(md - mr) < 0.07 * mr + 4 * err), (md / mr - 1, err / mr)
    bd = np.polyfit(np.log(ts[3:]), np.log(md[3:]), 1)[0] / 2
    br = np.polyfit(np.log(ts[3:]), np.log(mr[3:]), 1)[0] / 2
    assert abs(bd - br) < 0.03, (bd, br)
