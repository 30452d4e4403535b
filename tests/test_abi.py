"""The C ABI library loads without a GPU, exports every function that
include/kpz.h declares, and rejects invalid arguments before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(kpz_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1204_5072_gb300 import _lib, build
    if not os.path.exists(build.SO):
        build.build()
    return _lib.load()


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "kpz_init" in names and "kpz_run" in names and "kpz_roughness" in names
    for n in names:
        assert hasattr(lib, n), n


def test_invalid_arguments_rejected_without_device(lib):
    from paper_1204_5072_gb300._lib import KPZ_EINVAL, kpz_opts
    c = ctypes.c_void_p()
    bad = [(100, 1.0, 0.0), (64, 1.0, 0.0), (1 << 19, 1.0, 0.0), (256, float("nan"), 0.0),
           (256, 1.5, 0.0), (256, 1.0, -0.1)]
    for L, p, q in bad:
        assert lib.kpz_init(ctypes.byref(c), L, p, q, 1, 0, 0, None) == KPZ_EINVAL
    assert lib.kpz_init(ctypes.byref(c), 256, 1.0, 0.0, 1, 0, 1, None) == KPZ_EINVAL  # init != flat
    for field, val in [("bx", 64), ("bx", 256), ("by", 64), ("by", 512), ("run", 3), ("run", 4),
                       ("warps_per_cta", 9)]:
        o = kpz_opts()
        setattr(o, field, val)
        assert lib.kpz_init(ctypes.byref(c), 256, 1.0, 0.0, 1, 0, 0, ctypes.byref(o)) == KPZ_EINVAL
    o = kpz_opts()
    o.by = 256   # 128 x 256 tiles need L >= 256
    assert lib.kpz_init(ctypes.byref(c), 128, 1.0, 0.0, 1, 0, 0, ctypes.byref(o)) == KPZ_EINVAL
    o = kpz_opts()
    o.decomposition = 4   # the exact random-sequential reference takes L <= 8192
    assert lib.kpz_init(ctypes.byref(c), 16384, 1.0, 0.0, 1, 0, 0, ctypes.byref(o)) == KPZ_EINVAL
    o.decomposition = 5
    assert lib.kpz_init(ctypes.byref(c), 256, 1.0, 0.0, 1, 0, 0, ctypes.byref(o)) == KPZ_EINVAL
    assert lib.kpz_device_bytes(100) == 0 and lib.kpz_device_bytes(1 << 19) == 0
    assert lib.kpz_device_bytes(1 << 18) >= (1 << 36) // 8
    assert lib.kpz_device_bytes(256) >= 256 * 256 // 4
    assert lib.kpz_run(None, 1) == KPZ_EINVAL
    lib.kpz_free(None)
