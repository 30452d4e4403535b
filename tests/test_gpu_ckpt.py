"""Checkpoint save / load through the C ABI (kpz_ckpt_save, kpz_ckpt_load):
a run interrupted by a checkpoint continues bit-exactly, and damaged files
are refused with KPZ_ECKPT."""
import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu
TILE = 128


@pytest.fixture(scope="module")
def eng():
    return engine()


@pytest.mark.parametrize("L,p,q,ty", [(512, 0.7, 0.2, 128), (1024, 1.0, 0.0, 256), (256, 0.5, 0.5, 128)])
def test_resume_from_checkpoint_is_bit_exact(eng, tmp_path, L, p, q, ty):
    a = eng.Lattice(L, p, q, seed=4, sample=3, tile_y=ty)
    a.run(7)
    f = tmp_path / "run.kpz"
    a.save(f)
    b = eng.Lattice.load(f)
    assert (b.L, b.p, b.q, b.seed, b.sample) == (L, p, q, 4, 3)
    assert np.array_equal(a.slopes(), b.slopes()) and a.roughness() == b.roughness()
    a.run(5)
    b.run(5)
    assert np.array_equal(a.slopes(), b.slopes())
    assert a.roughness() == b.roughness()
    # and both equal the oracle's uninterrupted schedule
    st = O.State.flat(L).run(12, TILE, ty, p, q, 4, 3)
    assert np.array_equal(b.slopes(), st.packed())
    r = b.roughness()
    assert (r["S1"], r["S2"], r["h00"], r["t"]) == (*st.sums(), st.h00, 12)


def test_damaged_checkpoints_are_refused(eng, tmp_path):
    from paper_1204_5072_gb300._lib import KPZ_ECKPT, KPZ_EINVAL, KpzError
    a = eng.Lattice(256, 0.9, 0.1, seed=2)
    a.run(3)
    f = tmp_path / "ok.kpz"
    a.save(f)
    raw = f.read_bytes()
    cases = {
        "flipped payload bit": raw[:200] + bytes([raw[200] ^ 4]) + raw[201:],
        "truncated": raw[:-9],
        "trailing byte": raw + b"\0",
        "bad magic": b"X" + raw[1:],
        "threshold mismatch": raw[:32] + (raw[32] ^ 1).to_bytes(1, "little") + raw[33:],
    }
    for name, data in cases.items():
        g = tmp_path / "bad.kpz"
        g.write_bytes(data)
        with pytest.raises(KpzError) as e:
            eng.Lattice.load(g)
        assert e.value.status == KPZ_ECKPT, name
    with pytest.raises(KpzError) as e:
        eng.Lattice.load(tmp_path / "missing.kpz")
    assert e.value.status == KPZ_ECKPT
    # conflicting tile shape in the options
    import ctypes
    from paper_1204_5072_gb300._lib import kpz_opts, load
    o = kpz_opts()
    o.by = 256
    ctx = ctypes.c_void_p()
    assert load().kpz_ckpt_load(ctypes.byref(ctx), str(f).encode(), ctypes.byref(o)) == KPZ_EINVAL
    assert not ctx.value
