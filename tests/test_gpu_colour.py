"""The random-sequential reference by colour classes on the GPU (sub-steps
that attempt random subsets of one period-2 sublattice, no decomposition):
bit-exact against the oracle's definition, and at thin subsets in agreement
with plain random-sequential updates (one attempt at a time)."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_util import engine
from tests.test_gpu_parity import _same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eng():
    return engine()


@pytest.mark.parametrize("L,p,q,seed,sample,m,n", [
    (128, 1.0, 0.0, 1, 0, 3, 5), (256, 0.8, 0.2, 3, 2, 1, 4), (256, 0.5, 0.5, 7, 1, 4, 3),
    (512, 0.95, 0.05, (1 << 40) + 9, 4, 2, 3), (128, 0.0, 0.0, 5, 0, 3, 2)])
def test_colour_reference_bit_exact(eng, L, p, q, seed, sample, m, n):
    lat = eng.Lattice(L, p, q, seed=seed, sample=sample, decomposition=2, colour_sparsity=m)
    st = O.State.flat(L)
    for k in range(n):
        lat.run(1)
        st.sweep_colour(p, q, seed, sample, m=m)
        _same(lat, st, f"colour L={L} p={p} q={q} m={m} after sweep {k + 1}")


def test_colour_reference_checkpoint_and_options(eng, tmp_path):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KpzError
    a = eng.Lattice(256, 0.9, 0.1, seed=3, decomposition=2, colour_sparsity=2)
    a.run(2)
    a.save(tmp_path / "c.kpz")
    b = eng.Lattice.load(tmp_path / "c.kpz")
    b.run(1)
    st = O.State.flat(256)
    for _ in range(3):
        st.sweep_colour(0.9, 0.1, 3, 0, m=2)
    _same(b, st, "colour reference after a checkpoint")
    for kw in ({"colour_sparsity": 5, "decomposition": 2}, {"colour_sparsity": 2},
               {"decomposition": 2, "tile_y": 256}, {"decomposition": 9}):
        with pytest.raises(KpzError) as e:
            eng.Lattice(256, 1.0, 0.0, **kw)
        assert e.value.status == KPZ_EINVAL


def test_thin_subsets_agree_with_random_sequential_updates(eng):
    L, ts = 256, [1, 2, 4, 8, 16, 32]
    rsu = np.zeros((16, len(ts)))
    for k in range(16):
        st = O.State.flat(L)
        for j, t in enumerate(ts):
            st.rsu(t - st.t, 1.0, 0.0, seed=12, sample=k)
            rsu[k, j] = st.w2()
    gpu = np.zeros((64, len(ts)))
    for k in range(64):
        lat = eng.Lattice(L, 1.0, 0.0, seed=21, sample=k, decomposition=2, colour_sparsity=4)
        t0 = 0
        for j, t in enumerate(ts):
            lat.run(t - t0)
            t0 = t
            gpu[k, j] = lat.roughness()["w2"]
        lat.close()
    mr, mg = rsu.mean(0), gpu.mean(0)
    err = np.sqrt(rsu.var(0, ddof=1) / 16 + gpu.var(0, ddof=1) / 64)
    assert np.all(np.abs(mg - mr) < 0.02 * mr + 4 * err), mg / mr - 1
