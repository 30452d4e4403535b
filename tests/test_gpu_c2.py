"""The C = 2 limit of the work-group layer (2 x 2 cells, their 1 x 1 quadrants
as the sets, 4 single-hit rounds per sweep) on the GPU, bit-exact against the
oracle's schedule, with the dead-border device layer."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_util import engine
from tests.test_gpu_parity import _same

pytestmark = pytest.mark.gpu
TILE = 128


@pytest.fixture(scope="module")
def eng():
    return engine()


@pytest.mark.parametrize("L,p,q,seed,sample,n", [
    (128, 1.0, 0.0, 1, 0, 8), (256, 1.0, 0.0, 2, 0, 6), (512, 0.8, 0.2, 3, 2, 5), (256, 0.5, 0.5, 7, 1, 5),
    (1024, 0.95, 0.05, (1 << 40) + 9, 4, 4), (256, 0.0, 1.0, 2, 3, 4), (256, 0.0, 0.0, 5, 0, 3)])
def test_c2_sweeps_bit_exact(eng, L, p, q, seed, sample, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, cell=2)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.sweep_c2(TILE, TILE, p, q, seed, sample)
        _same(lat, st, f"C=2 L={L} p={p} q={q} after sweep {k + 1}")


def test_c2_knobs_checkpoint_and_options(eng, tmp_path):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KpzError
    ref = None
    for run, wpc in ((1, 1), (4, 8), (8, 3)):
        lat = eng.Lattice(1024, 0.9, 0.1, seed=12, run=run, warps_per_cta=wpc, cell=2)
        lat.run(3)
        got = (lat.slopes(), lat.roughness())
        if ref is None:
            ref = got
            lat.save(tmp_path / "c2.kpz")
        else:
            assert np.array_equal(got[0], ref[0]) and got[1] == ref[1], (run, wpc)
    b = eng.Lattice.load(tmp_path / "c2.kpz")
    b.run(2)
    st = O.State.flat(1024).run_c2(5, TILE, TILE, 0.9, 0.1, 12, 0)
    _same(b, st, "C=2 after a checkpoint")
    for kw in ({"cell": 3}, {"cell": 2, "tile_y": 256}, {"cell": 2, "decomposition": 1}):
        with pytest.raises(KpzError) as e:
            eng.Lattice(256, 1.0, 0.0, **kw)
        assert e.value.status == KPZ_EINVAL
