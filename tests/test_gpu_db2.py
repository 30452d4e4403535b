"""Dead borders at both layers (the paper's earlier KPZ scheme, Sec. 3.1;
kpz_opts.decomposition = 3) on the GPU, bit-exact against the oracle's
schedule (orc_sweep_db2): the packed lattice, the exact height sums and the
height of site (0,0) after every sweep."""
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
    (128, 1.0, 0.0, 1, 0, 6),            # one tile: the tile wraps onto itself
    (256, 1.0, 0.0, 2, 0, 8), (512, 0.8, 0.2, 3, 2, 6), (256, 0.5, 0.5, 7, 1, 5),
    (1024, 0.95, 0.05, (1 << 40) + 9, 4, 4), (256, 0.0, 1.0, 2, 3, 4), (512, 0.0, 0.0, 5, 0, 3)])
def test_db2_sweeps_bit_exact(eng, L, p, q, seed, sample, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, decomposition=3)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.sweep_db2(TILE, TILE, p, q, seed, sample)
        _same(lat, st, f"dead borders at both layers L={L} p={p} q={q} after sweep {k + 1}")


def test_db2_checkpoint_and_options(eng, tmp_path):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KpzError
    a = eng.Lattice(512, 0.9, 0.1, seed=3, decomposition=3)
    a.run(4)
    a.save(tmp_path / "db2.kpz")
    b = eng.Lattice.load(tmp_path / "db2.kpz")
    a.run(3)
    b.run(3)
    st = O.State.flat(512).run_db2(7, TILE, TILE, 0.9, 0.1, 3, 0)
    _same(b, st, "dead borders at both layers after a checkpoint")
    assert np.array_equal(a.slopes(), b.slopes())
    for kw in ({"tile_y": 256}, {"cell": 2}, {"colour_sparsity": 2}):
        with pytest.raises(KpzError) as e:
            eng.Lattice(256, 1.0, 0.0, decomposition=3, **kw)
        assert e.value.status == KPZ_EINVAL
