"""Python handle on the CPU oracle (``kpz_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``. The
product package never imports this module.

Arrays follow the oracle's encoding: ``sx``, ``sy`` are ``uint8`` arrays of
shape ``(L, L)`` indexed ``[j, i]`` (row j = y, column i = x), 1 meaning a
slope of +1 (Sec. 2.1 of arXiv:1204.5072).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kpz_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkpz_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build`` and return the path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC]
        try:   # OpenMP only spreads tiles over threads (orc_sweep_threads); results do not change
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def load(path: str):
    """Load a compiled oracle library and declare its functions' signatures."""
    L = ctypes.CDLL(path)
    u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
    u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
    i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
    c = ctypes
    L.orc_philox.argtypes = [u32p, u32p, u32p]
    L.orc_threshold.argtypes = [c.c_double]
    L.orc_threshold.restype = c.c_uint32
    L.orc_init_flat.argtypes = [c.c_uint32, u8p, u8p]
    L.orc_attempt.argtypes = [c.c_uint32, u8p, u8p, c.c_uint32, c.c_uint32, c.c_int, c.c_int]
    L.orc_attempt.restype = c.c_int
    L.orc_sweep.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                            c.c_uint64, c.c_uint32, c.c_uint32, u8p, u8p,
                            c.POINTER(c.c_int64), c.c_uint64, c.c_uint32]
    L.orc_sweep.restype = c.c_int
    L.orc_run.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                          c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, u8p, u8p,
                          c.POINTER(c.c_int64)]
    L.orc_run.restype = c.c_int
    L.orc_rsu_run.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64, c.c_uint32,
                              c.c_uint32, c.c_uint32, u8p, u8p, c.POINTER(c.c_int64)]
    L.orc_rsu_run.restype = c.c_int
    L.orc_heights.argtypes = [c.c_uint32, u8p, u8p, i64p]
    L.orc_sums.argtypes = [c.c_uint32, i64p, c.POINTER(c.c_int64),
                           c.POINTER(c.c_uint64), c.POINTER(c.c_uint64)]
    L.orc_w2.argtypes = [c.c_uint64, c.c_int64, c.c_uint64, c.c_uint64]
    L.orc_w2.restype = c.c_double
    L.orc_pack.argtypes = [c.c_uint32, u8p, u8p, u32p]
    L.orc_unpack.argtypes = [c.c_uint32, u32p, u8p, u8p]
    L.orc_flat_tile_sweep.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                      c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, u8p, u8p,
                                      c.POINTER(c.c_uint32), c.POINTER(c.c_uint32),
                                      c.POINTER(c.c_int64)]
    L.orc_flat_tile_sweep.restype = c.c_int
    L.orc_window_tile_sweep.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                        c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_int,
                                        u8p, u8p, c.POINTER(c.c_uint32), c.POINTER(c.c_uint32),
                                        c.POINTER(c.c_int64)]
    L.orc_window_tile_sweep.restype = c.c_int
    L.orc_origin.argtypes = [c.c_uint32, c.c_uint64, c.c_uint32, c.c_uint32,
                             c.POINTER(c.c_uint32), c.POINTER(c.c_uint32)]
    L.orc_attempt_site.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64, c.c_uint32,
                                   c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                   c.POINTER(c.c_uint32), c.POINTER(c.c_uint32),
                                   c.POINTER(c.c_uint32)]
    L.orc_attempt_site.restype = c.c_int
    L.orc_row_acceptance.argtypes = [c.c_uint64, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                     c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                     c.POINTER(c.c_uint32), c.POINTER(c.c_uint32), u32p]
    L.orc_row_acceptance.restype = c.c_int
    L.orc_sweep_threads.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                    c.c_uint64, c.c_uint32, c.c_uint32, u8p, u8p,
                                    c.POINTER(c.c_int64), c.c_int]
    L.orc_sweep_threads.restype = c.c_int
    L.orc_sweep_tilesets.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                     c.c_uint64, c.c_uint32, c.c_uint32, u8p, u8p,
                                     c.POINTER(c.c_int64), c.c_uint64]
    L.orc_sweep_tilesets.restype = c.c_int
    L.orc_tileset_order.argtypes = [c.c_uint32, c.c_uint32, c.c_uint64, u32p]
    L.orc_tileset_order.restype = c.c_int
    L.orc_sweep_c2.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                               c.c_uint64, c.c_uint32, c.c_uint32, u8p, u8p,
                               c.POINTER(c.c_int64), c.c_uint64]
    L.orc_sweep_c2.restype = c.c_int
    L.orc_sweep_colour.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64,
                                   c.c_uint32, c.c_uint32, u8p, u8p, c.POINTER(c.c_int64)]
    L.orc_sweep_colour.restype = c.c_int
    L.orc_sweep_c2_rounds.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                      c.c_uint64, c.c_uint32, c.c_uint32, u8p, u8p,
                                      c.POINTER(c.c_int64), c.c_uint64, c.c_uint32]
    L.orc_sweep_c2_rounds.restype = c.c_int
    L.orc_sweep_colour_steps.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64,
                                         c.c_uint32, c.c_uint32, u8p, u8p, c.POINTER(c.c_int64), c.c_uint32]
    L.orc_sweep_colour_steps.restype = c.c_int
    L.orc_sweep_db2.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                                c.c_uint64, c.c_uint32, c.c_uint32, u8p, u8p,
                                c.POINTER(c.c_int64), c.c_uint64]
    L.orc_sweep_db2.restype = c.c_int
    L.orc_db2_site.argtypes = [c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint64, c.c_uint32, c.c_uint32,
                               c.c_uint32, c.c_uint32, c.c_uint32, c.c_uint32,
                               c.POINTER(c.c_uint32), c.POINTER(c.c_uint32), c.POINTER(c.c_uint32)]
    L.orc_db2_site.restype = c.c_int
    return L


# --------------------------------------------------------------------------- #
def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for counter ``ctr`` (4 words) and key ``key`` (2 words)."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def tileset_order(s: int, sample: int, seed: int) -> list:
    """Order in which the four tile sets are swept in sweep s (tile-set variant)."""
    out = np.zeros(4, np.uint32)
    lib().orc_tileset_order(s, sample, seed, out)
    return [int(v) for v in out]


def threshold(p: float) -> int:
    """Acceptance threshold out of 2^16 used for probability ``p``."""
    return int(lib().orc_threshold(float(p)))


def flat_tile_sweep(L, Bx, By, p, q, seed, sample, s, T):
    """Tile T of sweep s from the flat start, computed on its own window (the
    tiles of one sweep do not interact): returns (sx, sy) of shape (By, Bx)
    indexed [v, u] = global site ((x0+u) mod L, (y0+v) mod L), the anchor
    (x0, y0), and the height change of site (0, 0)."""
    sx = np.zeros(By * Bx, np.uint8)
    sy = np.zeros(By * Bx, np.uint8)
    ax, ay, d = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
    rc = lib().orc_flat_tile_sweep(L, Bx, By, threshold(p), threshold(q), seed, sample, s, T, sx, sy,
                                   ctypes.byref(ax), ctypes.byref(ay), ctypes.byref(d))
    if rc:
        raise ValueError("bad arguments")
    return sx.reshape(By, Bx), sy.reshape(By, Bx), (ax.value, ay.value), d.value


def window_tile_sweep(L, Bx, By, p, q, seed, sample, s, T, sx, sy):
    """Tile T of sweep s run on its own window: (sx, sy) of shape (By, Bx)
    indexed [v, u] = global site ((x0+u) mod L, (y0+v) mod L) hold the
    window when sweep s starts; returns the window after the sweep and the
    height change of site (0, 0) (0 unless the tile holds it)."""
    sx = np.ascontiguousarray(sx, np.uint8).reshape(-1).copy()
    sy = np.ascontiguousarray(sy, np.uint8).reshape(-1).copy()
    if sx.size != Bx * By or sy.size != Bx * By:
        raise ValueError("window shape")
    ax, ay, d = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
    rc = lib().orc_window_tile_sweep(L, Bx, By, threshold(p), threshold(q), seed, sample, s, T, 1, sx, sy,
                                     ctypes.byref(ax), ctypes.byref(ay), ctypes.byref(d))
    if rc:
        raise ValueError("bad arguments")
    return sx.reshape(By, Bx), sy.reshape(By, Bx), d.value


def tile_anchor(L, Bx, By, seed, sample, s, T):
    """Global site (x0, y0) of tile T's local (0, 0) in sweep s."""
    dummy = np.zeros(1, np.uint8)
    ax, ay, d = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_int64()
    rc = lib().orc_window_tile_sweep(L, Bx, By, 0, 0, seed, sample, s, T, 0, dummy, dummy,
                                     ctypes.byref(ax), ctypes.byref(ay), ctypes.byref(d))
    if rc:
        raise ValueError("bad arguments")
    return ax.value, ay.value


def origin(L, seed, sample, s, _lib=None):
    """Origin (ox, oy) of sweep s's tile grid (device layer, Sec. 3)."""
    ox, oy = ctypes.c_uint32(), ctypes.c_uint32()
    (_lib or lib()).orc_origin(L, seed, sample, s, ctypes.byref(ox), ctypes.byref(oy))
    return ox.value, oy.value


def attempt_site(L, Bx, By, seed, sample, s, T, r, cx, cy, _lib=None):
    """(u, v, k): tile-local site attempted by cell (cx, cy) of tile T in round
    r of sweep s, and the round's quadrant set k (Sec. 3.1)."""
    u, v, k = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    rc = (_lib or lib()).orc_attempt_site(L, Bx, By, seed, sample, s, T, r, cx, cy,
                                ctypes.byref(u), ctypes.byref(v), ctypes.byref(k))
    if rc:
        raise ValueError("bad arguments")
    return u.value, v.value, k.value


def db2_site(L, Bx, By, seed, sample, s, T, r, kx, ky):
    """(u, v, U): tile-local site attempted by block (kx, ky) of tile T in
    round r of sweep s under dead borders at both layers, and its 16-bit
    acceptance number."""
    u, v, U = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    rc = lib().orc_db2_site(L, Bx, By, seed, sample, s, T, r, kx, ky,
                            ctypes.byref(u), ctypes.byref(v), ctypes.byref(U))
    if rc:
        raise ValueError("bad arguments")
    return u.value, v.value, U.value


def row_acceptance(seed, sample, Tp, Tq, T, s, r, rw, cand_min, cand_max, _lib=None):
    """Acceptance of one round for the 32 cells of row word rw of tile T:
    returns (accepted mask, tied mask, U) with U[b] the 16-bit number of
    candidate b (0xffffffff where no number is drawn). Tp, Tq are thresholds
    out of 2^16."""
    acc, tied = ctypes.c_uint32(), ctypes.c_uint32()
    U = np.zeros(32, np.uint32)
    rc = (_lib or lib()).orc_row_acceptance(seed, sample, Tp, Tq, T, s, r, rw, cand_min, cand_max,
                                  ctypes.byref(acc), ctypes.byref(tied), U)
    if rc:
        raise ValueError("bad arguments")
    return acc.value, tied.value, U


class State:
    """Lattice state of the oracle: slopes plus the absolute height of (0,0)."""

    def __init__(self, L: int, sx: np.ndarray, sy: np.ndarray, h00: int = 0, t: int = 0):
        self.L = int(L)
        self.sx = np.ascontiguousarray(sx, np.uint8)
        self.sy = np.ascontiguousarray(sy, np.uint8)
        self.h00 = int(h00)
        self.t = int(t)

    @classmethod
    def flat(cls, L: int) -> "State":
        sx = np.zeros((L, L), np.uint8)
        sy = np.zeros((L, L), np.uint8)
        lib().orc_init_flat(L, sx, sy)
        return cls(L, sx, sy)

    def copy(self) -> "State":
        return State(self.L, self.sx.copy(), self.sy.copy(), self.h00, self.t)

    # -- dynamics ------------------------------------------------------------
    def sweep(self, Bx, By, p, q, seed, sample=0, order=0, s=None, rounds=16):
        s = self.t if s is None else s
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_sweep(self.L, Bx, By, threshold(p), threshold(q), seed, sample, s,
                             self.sx, self.sy, ctypes.byref(h), order, rounds)
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t = s + 1
        return self

    def sweep_tilesets(self, Bx, By, p, q, seed, sample=0, order=0):
        """One sweep of the tile-set variant of the device layer (four sets of
        tiles swept in a random order, no dead border)."""
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_sweep_tilesets(self.L, Bx, By, threshold(p), threshold(q), seed, sample, self.t,
                                      self.sx, self.sy, ctypes.byref(h), order)
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t += 1
        return self

    def sweep_c2(self, Bx, By, p, q, seed, sample=0, order=0, rounds=4):
        """One sweep with the C = 2 work-group layer (2 x 2 cells, 4 rounds;
        fewer only for tests that look inside a sweep)."""
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_sweep_c2_rounds(self.L, Bx, By, threshold(p), threshold(q), seed, sample, self.t,
                                       self.sx, self.sy, ctypes.byref(h), order, rounds)
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t += 1
        return self

    def sweep_colour(self, p, q, seed, sample=0, m=3, nsub=None):
        """One sweep of random-sequential updates by colour classes (4 * 2^m
        sub-steps, each a random 2^-m subset of one period-2 sublattice; the
        first nsub only, for tests that look inside a sweep)."""
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_sweep_colour_steps(self.L, threshold(p), threshold(q), m, seed, sample, self.t,
                                          self.sx, self.sy, ctypes.byref(h), (4 << m) if nsub is None else nsub)
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t += 1
        return self

    def sweep_db2(self, Bx, By, p, q, seed, sample=0, order=0):
        """One sweep with dead borders at both layers (4 x 4 blocks re-anchored
        at random each round, one attempt per block in its 3 x 3 interior)."""
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_sweep_db2(self.L, Bx, By, threshold(p), threshold(q), seed, sample, self.t,
                                 self.sx, self.sy, ctypes.byref(h), order)
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t += 1
        return self

    def run_db2(self, n, Bx, By, p, q, seed, sample=0):
        for _ in range(n):
            self.sweep_db2(Bx, By, p, q, seed, sample)
        return self

    def run_c2(self, n, Bx, By, p, q, seed, sample=0):
        for _ in range(n):
            self.sweep_c2(Bx, By, p, q, seed, sample)
        return self

    def run_tilesets(self, n, Bx, By, p, q, seed, sample=0):
        for _ in range(n):
            self.sweep_tilesets(Bx, By, p, q, seed, sample)
        return self

    def run_threads(self, n, Bx, By, p, q, seed, sample=0, threads=None):
        """n sweeps with the tiles of each sweep spread over `threads` host
        threads (default: all cores); same result as run()."""
        threads = threads or os.cpu_count() or 1
        h = ctypes.c_int64(self.h00)
        for _ in range(n):
            rc = lib().orc_sweep_threads(self.L, Bx, By, threshold(p), threshold(q), seed, sample, self.t,
                                         self.sx, self.sy, ctypes.byref(h), threads)
            if rc:
                raise ValueError("bad schedule parameters")
            self.t += 1
        self.h00 = h.value
        return self

    def run(self, n, Bx, By, p, q, seed, sample=0):
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_run(self.L, Bx, By, threshold(p), threshold(q), seed, sample,
                           self.t, n, self.sx, self.sy, ctypes.byref(h))
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t += n
        return self

    def rsu(self, n, p, q, seed, sample=0):
        h = ctypes.c_int64(self.h00)
        rc = lib().orc_rsu_run(self.L, threshold(p), threshold(q), seed, sample,
                               self.t, n, self.sx, self.sy, ctypes.byref(h))
        if rc:
            raise ValueError("invalid oracle parameters")
        self.h00 = h.value
        self.t += n
        return self

    def attempt(self, i, j, acc_min=True, acc_max=True) -> int:
        return int(lib().orc_attempt(self.L, self.sx, self.sy, i, j, int(acc_min), int(acc_max)))

    # -- observables ---------------------------------------------------------
    def heights(self, absolute=False) -> np.ndarray:
        h = np.zeros((self.L, self.L), np.int64)
        lib().orc_heights(self.L, self.sx, self.sy, h)
        return h + self.h00 if absolute else h

    def sums(self):
        """(S1, S2) of the relative heights (gauge h(0,0) = 0), exact Python ints."""
        h = self.heights()
        s1 = ctypes.c_int64()
        lo = ctypes.c_uint64()
        hi = ctypes.c_uint64()
        lib().orc_sums(self.L, h, ctypes.byref(s1), ctypes.byref(lo), ctypes.byref(hi))
        return s1.value, (hi.value << 64) | lo.value

    def w2(self) -> float:
        s1, s2 = self.sums()
        return w2_from_sums(self.L * self.L, s1, s2)

    def packed(self) -> np.ndarray:
        """Canonical packed words, shape (L*L/16,), requires L >= 16."""
        w = np.zeros(self.L * self.L // 16, np.uint32)
        lib().orc_pack(self.L, self.sx, self.sy, w)
        return w

    @classmethod
    def from_packed(cls, L: int, words: np.ndarray, h00: int = 0, t: int = 0) -> "State":
        sx = np.zeros((L, L), np.uint8)
        sy = np.zeros((L, L), np.uint8)
        lib().orc_unpack(L, np.ascontiguousarray(words, np.uint32), sx, sy)
        return cls(L, sx, sy, h00, t)


def w2_from_sums(N: int, S1: int, S2: int) -> float:
    mask = (1 << 64) - 1
    return float(lib().orc_w2(N, S1, S2 & mask, S2 >> 64))
