"""CPU oracle for VATE (arXiv 1812.00282) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and nothing here imports the product path.

The arithmetic lives in ``vate_oracle.c`` (plain C, one AT and one pair at a
time, double precision for the estimator); this module compiles it with gcc
and exposes it through ctypes with numpy arrays.  ``exact.py`` holds the
brute-force exact sliding-window distinct counts (Def. 1) used as ground
truth.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vate_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SAT = 1        # flags bit: every VAT of the host is active (V0 replaced by 1)
POOLFULL = 2   # flags bit: no inactive AT in the pool (N0 replaced by 1)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
        u16p = np.ctypeslib.ndpointer(np.uint16, flags="C_CONTIGUOUS")
        u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
        u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
        sig = {
            "vo_mix64": (u64, [u64]),
            "vo_fmix32": (u32, [u32]),
            "vo_create": (vp, [u32, u32, u32, u32, u32, u64]),
            "vo_destroy": (None, [vp]),
            "vo_bh": (u32, [vp, u32]),
            "vo_h": (u64, [vp, u32, u32]),
            "vo_h_of": (u64, [u32, u32, u64, u32, u32]),
            "vo_bh_of": (u32, [u32, u64, u32]),
            "vo_block": (u32, [vp, u64]),
            "vo_bact": (u32, [vp, u32]),
            "vo_act_of": (u32, [vp, u64]),
            "vo_check_at": (C.c_int, [u32, u32, u32, u32]),
            "vo_preserve_general": (u32, [u32, u32, u32]),
            "vo_preserve_fast": (u32, [u32, u32, u32]),
            "vo_pool_size": (u64, [vp]),
            "vo_bact0": (u32, [vp]),
            "vo_slice": (C.c_int64, [vp]),
            "vo_block_a": (u64, [vp]),
            "vo_block_b": (u64, [vp]),
            "vo_copy_pool": (None, [vp, u16p]),
            "vo_copy_dr": (None, [vp, u16p]),
            "vo_load_pool": (None, [vp, u16p]),
            "vo_set_pid": (None, [vp, u64]),
            "vo_set_pids": (None, [vp, u64p, u64]),
            "vo_ingest": (None, [vp, u32p, u64]),
            "vo_pids_of_pairs": (None, [vp, u32p, u64, u64p]),
            "vo_advance": (None, [vp]),
            "vo_advance_general_every_slice": (None, [vp]),
            "vo_check_all": (None, [vp, u32, u8p]),
            "vo_census": (None, [vp, u64p]),
            "vo_set_threads": (None, [C.c_int]),
            "vo_get_threads": (C.c_int, []),
            "vo_pool_inactive": (u64, [vp, u32]),
            "vo_pool_inactive_range": (u64, [vp, u32, u64, u64]),
            "vo_estimate_from_counts": (C.c_double, [u32, u64, u64, u32, C.POINTER(C.c_uint8)]),
            "vo_active_vats": (u32, [vp, u32, u32]),
            "vo_estimate": (None, [vp, u32p, u64, u32, f64p, u32p, u8p]),
            "vo_estimate_hosts": (None, [vp, u32p, u64, u32, u64, f64p, u32p, u8p]),
            "vo_age_counts": (None, [vp, u32p, u64, u32p]),
            "vo_active_vats_dr": (u32, [vp, u32, u32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def set_threads(n: int) -> None:
    """Threads of the oracle's loops over pool ATs and over hosts (1 by
    default); results do not depend on it."""
    _load().vo_set_threads(int(n))


def threads() -> int:
    return int(_load().vo_get_threads())


def h_of(c: int, L: int, seed: int, aip: int, i: int) -> int:
    """H(aip, i) for a pool of 2^c ATs without allocating it."""
    return int(_load().vo_h_of(c, L, seed & 0xFFFFFFFFFFFFFFFF, aip, i))


def bh_of(g: int, seed: int, bip: int) -> int:
    return int(_load().vo_bh_of(g, seed & 0xFFFFFFFFFFFFFFFF, bip))


def fmix32(x: int) -> int:
    return int(_load().vo_fmix32(x & 0xFFFFFFFF))


def mix64(x: int) -> int:
    """SplitMix64 output function (the mixer behind H and BH)."""
    return int(_load().vo_mix64(x & 0xFFFFFFFFFFFFFFFF))


def check_at(v: int, act: int, k: int, kprime: int) -> bool:
    """Algorithm 1 (CheckAT) on one value."""
    return bool(_load().vo_check_at(v, act, k, kprime))


def preserve_fast(v: int, act: int, k: int) -> int:
    """Algorithm 3 (fast PreserveAT) on one value; act must be 0 or k."""
    return int(_load().vo_preserve_fast(v, act, k))


def preserve_general(v: int, act: int, k: int) -> int:
    """Algorithm 2 (general PreserveAT) on one value."""
    return int(_load().vo_preserve_general(v, act, k))


def estimate_from_counts(g: int, P: int, N0: int, A: int):
    """Eq. 11 for one host from (A, N0); returns (estimate, flags)."""
    f = C.c_uint8(0)
    e = _load().vo_estimate_from_counts(g, P, N0, A, C.byref(f))
    return float(e), int(f.value)


def as_pairs(pairs) -> np.ndarray:
    a = np.ascontiguousarray(pairs, dtype=np.uint32)
    if a.ndim != 2 or a.shape[1] != 2:
        raise ValueError("pairs must have shape (n, 2): columns aip, bip")
    return a


class Oracle:
    """One VATE instance on the CPU: the AT pool, BACT^0 and the slice number,
    driven in the order of Algorithm 4 (ingest, estimate, advance)."""

    def __init__(self, c: int, k: int, g: int, seg_len: int = 1, partition: int = 0, seed: int = 0):
        self._lib = _load()
        self._s = self._lib.vo_create(c, k, g, seg_len, partition, seed & 0xFFFFFFFFFFFFFFFF)
        if not self._s:
            raise ValueError("oracle: invalid parameters c=%d k=%d g=%d L=%d partition=%d"
                             % (c, k, g, seg_len, partition))
        self.c, self.k, self.g, self.seg_len, self.partition, self.seed = c, k, g, seg_len, partition, seed
        self.P = 1 << c

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            self._lib.vo_destroy(s)
            self._s = None

    # --- state ---------------------------------------------------------
    @property
    def bact0(self) -> int:
        return int(self._lib.vo_bact0(self._s))

    @property
    def slice(self) -> int:
        return int(self._lib.vo_slice(self._s))

    @property
    def a(self) -> int:
        return int(self._lib.vo_block_a(self._s))

    @property
    def b(self) -> int:
        return int(self._lib.vo_block_b(self._s))

    def pool(self) -> np.ndarray:
        """AT values (uint16; at most 2k)."""
        out = np.empty(self.P, np.uint16)
        self._lib.vo_copy_pool(self._s, out)
        return out

    def dr(self) -> np.ndarray:
        out = np.empty(self.P, np.uint16)
        self._lib.vo_copy_dr(self._s, out)
        return out

    def load_pool(self, pool: np.ndarray) -> None:
        pool = np.ascontiguousarray(pool, np.uint16)
        assert pool.shape == (self.P,)
        self._lib.vo_load_pool(self._s, pool)

    # --- mapping -------------------------------------------------------
    def bh(self, bip: int) -> int:
        return int(self._lib.vo_bh(self._s, bip))

    def h(self, aip: int, i: int) -> int:
        return int(self._lib.vo_h(self._s, aip, i))

    def block(self, pid: int) -> int:
        return int(self._lib.vo_block(self._s, pid))

    def act_of(self, pid: int) -> int:
        return int(self._lib.vo_act_of(self._s, pid))

    def pids_of_pairs(self, pairs) -> np.ndarray:
        p = as_pairs(pairs)
        out = np.empty(p.shape[0], np.uint64)
        self._lib.vo_pids_of_pairs(self._s, p, p.shape[0], out)
        return out

    # --- Algorithm 4 steps ---------------------------------------------
    def set_pid(self, pid: int) -> None:
        self._lib.vo_set_pid(self._s, pid)

    def set_pids(self, pids) -> None:
        p = np.ascontiguousarray(pids, np.uint64)
        self._lib.vo_set_pids(self._s, p, p.shape[0])

    def ingest(self, pairs) -> None:
        p = as_pairs(pairs)
        self._lib.vo_ingest(self._s, p, p.shape[0])

    def advance(self) -> None:
        self._lib.vo_advance(self._s)

    def advance_general_every_slice(self) -> None:
        self._lib.vo_advance_general_every_slice(self._s)

    def check_all(self, kprime: int) -> np.ndarray:
        out = np.empty(self.P, np.uint8)
        self._lib.vo_check_all(self._s, kprime, out)
        return out

    def census(self) -> np.ndarray:
        out = np.empty(2 * self.k + 1, np.uint64)
        self._lib.vo_census(self._s, out)
        return out

    def pool_inactive(self, kprime: int) -> int:
        return int(self._lib.vo_pool_inactive(self._s, kprime))

    def pool_inactive_range(self, kprime: int, start: int, end: int) -> int:
        return int(self._lib.vo_pool_inactive_range(self._s, kprime, start, end))

    def active_vats(self, aip: int, kprime: int) -> int:
        return int(self._lib.vo_active_vats(self._s, aip, kprime))

    def active_vats_dr(self, aip: int, kprime: int) -> int:
        return int(self._lib.vo_active_vats_dr(self._s, aip, kprime))

    def estimate(self, aips, kprime: int):
        """Returns (estimates float64, active counts uint32, flags uint8)."""
        a = np.ascontiguousarray(aips, np.uint32)
        est = np.empty(a.shape[0], np.float64)
        act = np.empty(a.shape[0], np.uint32)
        fl = np.empty(a.shape[0], np.uint8)
        self._lib.vo_estimate(self._s, a, a.shape[0], kprime, est, act, fl)
        return est, act, fl

    def estimate_hosts(self, aips, kprime: int, n0: int):
        """The per-host part of estimate() with the pool's inactive count n0
        given (as pool_inactive(kprime) returns it)."""
        a = np.ascontiguousarray(aips, np.uint32)
        est = np.empty(a.shape[0], np.float64)
        act = np.empty(a.shape[0], np.uint32)
        fl = np.empty(a.shape[0], np.uint8)
        self._lib.vo_estimate_hosts(self._s, a, a.shape[0], kprime, n0, est, act, fl)
        return est, act, fl

    def age_counts(self, aips) -> np.ndarray:
        a = np.ascontiguousarray(aips, np.uint32)
        out = np.empty((a.shape[0], self.k), np.uint32)
        self._lib.vo_age_counts(self._s, a, a.shape[0], out)
        return out
