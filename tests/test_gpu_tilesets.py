"""The tile-set variant of the device layer (four tile sets swept in a random
order per sweep, no dead border; the double tiling of the paper's KMC model,
Sec. 3.2) on the GPU, bit-exact against the oracle's schedule."""
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
    (256, 1.0, 0.0, 1, 0, 8), (512, 0.8, 0.2, 3, 2, 6), (256, 0.5, 0.5, 7, 1, 5),
    (1024, 0.95, 0.05, (1 << 40) + 9, 4, 4), (256, 0.0, 1.0, 2, 3, 4), (512, 0.0, 0.0, 5, 0, 3)])
def test_tileset_sweeps_bit_exact(eng, L, p, q, seed, sample, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, decomposition=1)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.sweep_tilesets(TILE, TILE, p, q, seed, sample)
        _same(lat, st, f"tile sets L={L} p={p} q={q} after sweep {k + 1}")


def test_tileset_checkpoint_and_options(eng, tmp_path):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KpzError
    a = eng.Lattice(512, 0.9, 0.1, seed=3, decomposition=1)
    a.run(4)
    a.save(tmp_path / "ts.kpz")
    b = eng.Lattice.load(tmp_path / "ts.kpz")
    a.run(3)
    b.run(3)
    st = O.State.flat(512).run_tilesets(7, TILE, TILE, 0.9, 0.1, 3, 0)
    _same(b, st, "tile sets after a checkpoint")
    assert np.array_equal(a.slopes(), b.slopes())
    for kw in ({"L": 128}, {"tile_y": 256}, {"decomposition": 9}):
        args = {"L": 256, "decomposition": 1}
        args.update(kw)
        with pytest.raises(KpzError) as e:
            eng.Lattice(args.pop("L"), 1.0, 0.0, **args)
        assert e.value.status == KPZ_EINVAL
