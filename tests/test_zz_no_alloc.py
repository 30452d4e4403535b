"""kpz_roughness_static: the exact width of a lattice already on the device,
computed without allocating anything.

It serves callers that cannot call cudaMalloc at the time they need W^2 --
processes whose device memory is held by another framework's allocator, loops
that must not allocate after start-up. Its scratch lives in one static device array; this test checks,
through the C ABI, that it returns exactly what kpz_roughness returns for the
same lattice, on two calls in a row (the shared scratch must not carry a
previous call's sums), that it leaves device memory untouched, and that it
refuses lattices larger than its fixed scratch.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from tests.gpu_util import engine

pytestmark = pytest.mark.gpu


def _static(lib, lat, parity, stream):
    from paper_1204_5072_gb300._lib import kpz_rough
    ptr, _ = lat.device_lattice()
    r = kpz_rough()
    st = lib.kpz_roughness_static(ctypes.c_void_p(ptr), lat.L, parity, ctypes.c_void_p(stream),
                                  ctypes.byref(r))
    assert st == 0, st
    return r


def test_static_scratch_matches_kpz_roughness():
    import torch
    eng = engine()
    from paper_1204_5072_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream

    lats = []
    a = eng.Lattice(1024, 0.9, 0.1, seed=3)
    a.run(12)
    lats.append((a, 0))
    b = eng.Lattice(256, 1.0, 0.0, seed=4)
    b.run(40)
    lats.append((b, 0))
    st = O.State.flat(512).run(5, 128, 128, 0.7, 0.2, seed=5)
    c = eng.Lattice(512, 0.7, 0.2, seed=5)
    c.set_slopes(st.packed(), h00=7, t=st.t)        # odd origin height: parity 1
    lats.append((c, 1))

    # The first call on the device looks up (and, with lazy module loading,
    # materialises) the static scratch; after that no call may take memory.
    _static(lib, lats[0][0], 0, stream)
    for lat, _ in lats:
        lat.roughness()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for lat, parity in lats:
        want = lat.roughness()
        for _ in range(2):
            r = _static(lib, lat, parity, stream)
            S2 = (r.sum_h2_hi << 64) | r.sum_h2_lo
            assert (r.n_sites, r.sum_h, S2) == (want["n"], want["S1"], want["S2"])
            assert r.w2 == want["w2"]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_rejects_sizes():
    eng = engine()
    from paper_1204_5072_gb300 import _lib
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, KPZ_ERANGE, kpz_rough
    lib = _lib.load()
    lat = eng.Lattice(256)
    ptr, _ = lat.device_lattice()
    r = kpz_rough()
    assert lib.kpz_roughness_static(ctypes.c_void_p(ptr), 1 << 18, 0, None, ctypes.byref(r)) == KPZ_ERANGE
    assert lib.kpz_roughness_static(ctypes.c_void_p(ptr), 300, 0, None, ctypes.byref(r)) == KPZ_EINVAL
    assert lib.kpz_roughness_static(None, 256, 0, None, ctypes.byref(r)) == KPZ_EINVAL
