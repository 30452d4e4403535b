"""ctypes binding of ``libkpz.so`` (include/kpz.h): argument marshalling only.

Every computation runs in the library's CUDA kernels. PyTorch, when present,
only supplies device memory and the stream the work is queued on.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

(KPZ_OK, KPZ_EINVAL, KPZ_ENOMEM, KPZ_ECUDA, KPZ_ETIMEOUT, KPZ_ESTATE, KPZ_ENODEV, KPZ_ERANGE,
 KPZ_ECKPT) = range(9)


class KpzError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class kpz_opts(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_uint32), ("by", ctypes.c_uint32), ("run", ctypes.c_uint32),
                ("warps_per_cta", ctypes.c_uint32), ("stream", ctypes.c_void_p),
                ("dev_buf", ctypes.c_void_p), ("dev_bytes", ctypes.c_size_t),
                ("decomposition", ctypes.c_uint32), ("cell", ctypes.c_uint32),
                ("colour_sparsity", ctypes.c_uint32)]


class kpz_rough(ctypes.Structure):
    _fields_ = [("t_mcs", ctypes.c_uint64), ("n_sites", ctypes.c_uint64), ("sum_h", ctypes.c_int64),
                ("sum_h2_lo", ctypes.c_uint64), ("sum_h2_hi", ctypes.c_uint64),
                ("h00", ctypes.c_int64), ("w2", ctypes.c_double)]


_lib = None


def load(path: str | None = None):
    """Load the in-tree engine; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    so = path or _build.SO
    if not os.path.exists(so):
        raise ImportError(f"CUDA engine not built: {so} missing (run __graft_entry__.build())")
    L = ctypes.CDLL(so)
    c = ctypes
    vp = c.c_void_p
    L.kpz_device_bytes.argtypes = [c.c_uint32]
    L.kpz_device_bytes.restype = c.c_size_t
    L.kpz_init.argtypes = [c.POINTER(vp), c.c_uint32, c.c_double, c.c_double, c.c_uint64,
                           c.c_uint32, c.c_int, c.POINTER(kpz_opts)]
    L.kpz_run.argtypes = [vp, c.c_uint64]
    L.kpz_reset.argtypes = [vp]
    L.kpz_roughness.argtypes = [vp, c.POINTER(kpz_rough)]
    L.kpz_heights.argtypes = [vp, vp, c.c_int]
    L.kpz_slopes.argtypes = [vp, vp]
    L.kpz_set_slopes.argtypes = [vp, vp, c.c_int64, c.c_uint64]
    L.kpz_device_lattice.argtypes = [vp, c.POINTER(vp), c.POINTER(c.c_size_t)]
    L.kpz_ckpt_save.argtypes = [vp, c.c_char_p]
    L.kpz_alu_peak.argtypes = [c.POINTER(c.c_double), c.POINTER(c.c_double)]
    L.kpz_alu_peak.restype = c.c_int
    L.kpz_ckpt_load.argtypes = [c.POINTER(vp), c.c_char_p, c.POINTER(kpz_opts)]
    L.kpz_roughness_static.argtypes = [vp, c.c_uint32, c.c_uint32, vp, c.POINTER(kpz_rough)]
    L.kpz_roughness_static.restype = c.c_int
    L.kpz_launch_count.argtypes = []
    L.kpz_launch_count.restype = c.c_uint64
    L.kpz_free.argtypes = [vp]
    L.kpz_free.restype = None
    L.kpz_strerror.argtypes = [c.c_int]
    L.kpz_strerror.restype = c.c_char_p
    L.kpz_last_error.argtypes = [vp]
    L.kpz_last_error.restype = c.c_char_p
    for fn in ("kpz_init", "kpz_reset", "kpz_run", "kpz_roughness", "kpz_heights", "kpz_slopes",
               "kpz_set_slopes", "kpz_device_lattice", "kpz_ckpt_save", "kpz_ckpt_load"):
        getattr(L, fn).restype = c.c_int
    _lib = L
    return L


def check(st: int, ctx=None):
    if st != KPZ_OK:
        lib = load()
        msg = lib.kpz_strerror(st).decode()
        if ctx:
            detail = lib.kpz_last_error(ctx).decode()
            if detail:
                msg += ": " + detail
        raise KpzError(st, msg)


def launch_count() -> int:
    """Kernels launched by the engine in this process so far."""
    return int(load().kpz_launch_count())


def alu_peak() -> dict:
    """Measured integer-logic (LOP3) lane operations per second (kpz_alu_peak)."""
    rate, ms = ctypes.c_double(), ctypes.c_double()
    check(load().kpz_alu_peak(ctypes.byref(rate), ctypes.byref(ms)))
    return {"lane_ops_per_s": rate.value, "kernel_ms": ms.value}


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Lattice:
    """One L x L octahedron lattice on the GPU (flat start), driven through the C ABI.

    ``stream``: a CUDA stream handle (int) or None for torch's current stream
    when torch is available, else the default stream. ``device_buffer``: a
    torch CUDA tensor of at least ``kpz_device_bytes(L)`` bytes to hold the
    lattice (the caller keeps it alive); None lets the library allocate.
    """

    def __init__(self, L: int, p: float = 1.0, q: float = 0.0, seed: int = 1, sample: int = 0,
                 run: int = 0, warps_per_cta: int = 0, stream=None, device_buffer=None,
                 tile_y: int = 0, decomposition: int = 0, cell: int = 0, colour_sparsity: int = 0):
        lib = load()
        self.L, self.p, self.q, self.seed, self.sample = int(L), float(p), float(q), int(seed), int(sample)
        o = kpz_opts()
        o.run, o.warps_per_cta, o.by = run, warps_per_cta, tile_y
        o.decomposition, o.cell, o.colour_sparsity = decomposition, cell, colour_sparsity
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        o.stream = stream or None
        self._buf = device_buffer
        if device_buffer is not None:
            o.dev_buf = device_buffer.data_ptr()
            o.dev_bytes = device_buffer.numel() * device_buffer.element_size()
        self._ctx = ctypes.c_void_p()
        st = lib.kpz_init(ctypes.byref(self._ctx), self.L, self.p, self.q, self.seed, self.sample, 0,
                          ctypes.byref(o))
        if st != KPZ_OK:
            ctx = self._ctx
            self._ctx = None
            try:
                check(st, ctx)
            finally:
                if ctx:
                    lib.kpz_free(ctx)

    @staticmethod
    def device_bytes(L: int) -> int:
        return int(load().kpz_device_bytes(L))

    def reset(self) -> "Lattice":
        check(load().kpz_reset(self._ctx), self._ctx)
        return self

    @property
    def handle(self):
        return self._ctx

    def run(self, n_mcs: int) -> "Lattice":
        check(load().kpz_run(self._ctx, int(n_mcs)), self._ctx)
        return self

    def roughness(self) -> dict:
        r = kpz_rough()
        check(load().kpz_roughness(self._ctx, ctypes.byref(r)), self._ctx)
        return {"t": r.t_mcs, "n": r.n_sites, "S1": r.sum_h, "S2": (r.sum_h2_hi << 64) | r.sum_h2_lo,
                "h00": r.h00, "w2": r.w2}

    def heights(self, absolute: bool = False) -> np.ndarray:
        out = np.empty((self.L, self.L), np.int64)
        check(load().kpz_heights(self._ctx, _ptr(out), int(bool(absolute))), self._ctx)
        return out

    def slopes(self) -> np.ndarray:
        out = np.empty(self.L * self.L // 16, np.uint32)
        check(load().kpz_slopes(self._ctx, _ptr(out)), self._ctx)
        return out

    def slopes_into(self, out: np.ndarray) -> np.ndarray:
        """Packed slopes into a caller-provided uint32 buffer of L*L/16 words."""
        assert out.dtype == np.uint32 and out.size == self.L * self.L // 16 and out.flags.c_contiguous
        check(load().kpz_slopes(self._ctx, _ptr(out)), self._ctx)
        return out

    def set_slopes(self, words: np.ndarray, h00: int = 0, t: int = 0) -> "Lattice":
        w = np.ascontiguousarray(words, np.uint32)
        assert w.size == self.L * self.L // 16
        check(load().kpz_set_slopes(self._ctx, _ptr(w), int(h00), int(t)), self._ctx)
        return self

    def save(self, path) -> "Lattice":
        """Write a checkpoint (kpz_ckpt_save): header, packed lattice, checksum."""
        check(load().kpz_ckpt_save(self._ctx, os.fsencode(path)), self._ctx)
        return self

    @classmethod
    def load(cls, path, run: int = 0, warps_per_cta: int = 0, stream=None) -> "Lattice":
        """A new lattice from a checkpoint (kpz_ckpt_load); L, p, q, seed,
        sample and tile shape come from the file."""
        lib = load()
        o = kpz_opts()
        o.run, o.warps_per_cta = run, warps_per_cta
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        o.stream = stream or None
        ctx = ctypes.c_void_p()
        check(lib.kpz_ckpt_load(ctypes.byref(ctx), os.fsencode(path), ctypes.byref(o)))
        self = cls.__new__(cls)
        self._buf = None
        self._ctx = ctx
        hd = np.fromfile(path, dtype=np.uint8, count=64)   # header fields of kpz_ckpt_save
        self.L = int(hd[12:16].view(np.uint32)[0])
        self.p, self.q = (float(v) for v in hd[16:32].view(np.float64))
        self.seed = int(hd[40:48].view(np.uint64)[0])
        self.sample = int(hd[48:52].view(np.uint32)[0])
        return self

    def device_lattice(self):
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        check(load().kpz_device_lattice(self._ctx, ctypes.byref(p), ctypes.byref(n)), self._ctx)
        return p.value, n.value

    def close(self):
        if getattr(self, "_ctx", None):
            load().kpz_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# --------------------------------------------------------------------------- #
# Batched ensemble (kpz_batch_* in include/kpz.h)
class kpz_spec(ctypes.Structure):
    _fields_ = [("L", ctypes.c_uint32), ("p", ctypes.c_double), ("q", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("sample", ctypes.c_uint32), ("n_mcs", ctypes.c_uint32)]


class kpz_batch_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("n_samples", ctypes.c_uint32), ("autotune", ctypes.c_int),
                ("run", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("timeout_ms", ctypes.c_uint32),
                ("test_block", ctypes.c_int32), ("tile_y", ctypes.c_uint32)]


class kpz_batch_info(ctypes.Structure):
    _fields_ = [("run", ctypes.c_uint32), ("warps_per_cta", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("grid", ctypes.c_uint32), ("graph", ctypes.c_int),
                ("items", ctypes.c_uint64), ("n_probe", ctypes.c_uint32),
                ("probe_ms", ctypes.c_double * 8), ("tile_y", ctypes.c_uint32)]


def _bind_batch(L):
    c = ctypes
    vp = c.c_void_p
    L.kpz_batch_create.argtypes = [c.POINTER(vp), c.POINTER(kpz_spec), c.c_uint32, c.POINTER(kpz_batch_opts)]
    L.kpz_batch_run.argtypes = [vp]
    L.kpz_batch_times.argtypes = [vp, vp, c.POINTER(c.c_uint32)]
    L.kpz_batch_sums.argtypes = [vp, vp, vp, vp, vp]
    L.kpz_batch_w2.argtypes = [vp, vp]
    L.kpz_batch_get_info.argtypes = [vp, c.POINTER(kpz_batch_info)]
    L.kpz_batch_free.argtypes = [vp]
    L.kpz_batch_free.restype = None
    for fn in ("kpz_batch_create", "kpz_batch_run", "kpz_batch_times", "kpz_batch_sums",
               "kpz_batch_w2", "kpz_batch_get_info"):
        getattr(L, fn).restype = c.c_int


class Batch:
    """Independent realisations (L, p, q, seed, sample, n_mcs) run in one
    persistent launch; results match single Lattice runs bit for bit."""

    def __init__(self, specs, n_samples=0, autotune=False, run=0, warps_per_cta=0, ctas_per_sm=0,
                 timeout_ms=0, test_block=-1, stream=None, tile_y=0):
        lib = load()
        if not hasattr(lib, "_batch_bound"):
            _bind_batch(lib)
            lib._batch_bound = True
        self.specs = [tuple(s) for s in specs]
        arr = (kpz_spec * len(self.specs))()
        for k, (L, p, q, seed, sample, n) in enumerate(self.specs):
            arr[k] = kpz_spec(int(L), float(p), float(q), int(seed), int(sample), int(n))
        o = kpz_batch_opts()
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                pass
        o.stream = stream or None
        o.n_samples, o.autotune, o.run = n_samples, int(bool(autotune)), run
        o.warps_per_cta, o.ctas_per_sm, o.timeout_ms, o.test_block = warps_per_cta, ctas_per_sm, timeout_ms, test_block
        o.tile_y = tile_y
        self._b = ctypes.c_void_p()
        check(lib.kpz_batch_create(ctypes.byref(self._b), arr, len(self.specs), ctypes.byref(o)))

    def run(self) -> "Batch":
        check(load().kpz_batch_run(self._b))
        return self

    def times(self) -> np.ndarray:
        n = ctypes.c_uint32(0)
        check(load().kpz_batch_times(self._b, None, ctypes.byref(n)))
        out = np.zeros(n.value, np.uint64)
        check(load().kpz_batch_times(self._b, _ptr(out), ctypes.byref(n)))
        return out

    def sums(self):
        """(S1, S2 as Python ints) arrays of shape (n_specs, n_times), and h00."""
        n, m = len(self.specs), len(self.times())
        s1 = np.zeros((n, m), np.int64)
        lo = np.zeros((n, m), np.uint64)
        hi = np.zeros((n, m), np.uint64)
        h = np.zeros(n, np.int64)
        check(load().kpz_batch_sums(self._b, _ptr(s1), _ptr(lo), _ptr(hi), _ptr(h)))
        s2 = np.empty((n, m), object)
        for i in range(n):
            for k in range(m):
                s2[i, k] = (int(hi[i, k]) << 64) | int(lo[i, k])
        return s1, s2, h

    def w2(self) -> np.ndarray:
        out = np.zeros((len(self.specs), len(self.times())), np.float64)
        check(load().kpz_batch_w2(self._b, _ptr(out)))
        return out

    def info(self) -> dict:
        i = kpz_batch_info()
        check(load().kpz_batch_get_info(self._b, ctypes.byref(i)))
        return {"run": i.run, "warps_per_cta": i.warps_per_cta, "ctas_per_sm": i.ctas_per_sm,
                "grid": i.grid, "graph": bool(i.graph), "items": i.items,
                "probe_ms": list(i.probe_ms)[:i.n_probe], "tile_y": i.tile_y}

    def close(self):
        if getattr(self, "_b", None):
            load().kpz_batch_free(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
