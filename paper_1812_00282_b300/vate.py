"""Python binding of the VATE C ABI (include/vate.h): argument marshalling only.

Every function carries the C name and forwards to ``libvate.so`` through
ctypes; all work happens in the library's CUDA kernels.  Device arguments are
torch CUDA tensors (their ``data_ptr()`` is passed), host arguments of the
``*_host`` forms are numpy arrays or CPU tensors (page-locked memory gives
copy/compute overlap).  ``stream`` defaults to torch's current stream.

There is no fallback: if the library is missing or fails to load, importing
the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvate.so")
DEBUG_LIB_PATH = os.path.join(_HERE, "libvate_debug.so")   # the checked build (VATE_DEBUG)

VATE_OK, VATE_EINVAL, VATE_ENOMEM, VATE_ESLICE, VATE_ECUDA, VATE_ETIMEOUT, VATE_EDROPPED = 0, 1, 2, 3, 4, 5, 6
VATE_FLAG_SAT, VATE_FLAG_POOLFULL = 1, 2
VATE_DBG_POSITION, VATE_DBG_VALUE, VATE_DBG_BLOCK = 1, 2, 4
VATE_OPT_PERSIST_L2 = 1
ERROR_NAMES = {1: "VATE_EINVAL", 2: "VATE_ENOMEM", 3: "VATE_ESLICE", 4: "VATE_ECUDA", 5: "VATE_ETIMEOUT",
               6: "VATE_EDROPPED"}


class VateError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s: %s" % (ERROR_NAMES.get(code, str(code)), msg))
        self.code = code


class vate_params(C.Structure):
    _fields_ = [("log2_pool", C.c_uint32), ("k", C.c_uint32), ("g", C.c_uint32), ("seg_len", C.c_uint32),
                ("partition", C.c_uint32), ("counter", C.c_uint32), ("at_bits", C.c_uint32),
                ("options", C.c_uint32), ("seed", C.c_uint64)]


class vate_info(C.Structure):
    _fields_ = [("pool_size", C.c_uint64), ("block_a", C.c_uint64), ("block_b", C.c_uint64),
                ("slice", C.c_int64), ("bact0", C.c_uint32), ("closed", C.c_uint32),
                ("pid_lo", C.c_uint64), ("pid_hi", C.c_uint64)]


class vate_group_tuning(C.Structure):
    _fields_ = [("census_tile_chunks", C.c_uint32), ("blocks_per_sm", C.c_uint32),
                ("gather_grab_hosts", C.c_uint32), ("ingest_tile_pairs", C.c_uint32),
                ("preserve_tile_chunks", C.c_uint32), ("wave_pool_mib", C.c_uint32)]

    def as_dict(self):
        return {f: int(getattr(self, f)) for f, _ in self._fields_}


VATE_GROUP_BAD_OFFSETS, VATE_GROUP_BAD_KPRIME, VATE_GROUP_TIMEOUT = 1, 2, 4


class vate_server_config(C.Structure):
    _fields_ = [("memory_budget_bytes", C.c_uint64), ("slots", C.c_uint32), ("slot_records", C.c_uint32)]


class vate_server_stats(C.Structure):
    _fields_ = [("ingests_done", C.c_uint64), ("closes_done", C.c_uint64), ("pairs_done", C.c_uint64),
                ("hosts_done", C.c_uint64), ("merged_ingests", C.c_uint64), ("ingest_p50_ms", C.c_double),
                ("ingest_p99_ms", C.c_double), ("close_p50_ms", C.c_double), ("close_p99_ms", C.c_double),
                ("memory_in_use", C.c_uint64), ("monitors", C.c_uint32), ("max_in_flight", C.c_uint32)]

    def as_dict(self):
        return {f: (round(v, 4) if isinstance(v, float) else int(v)) for f, _ in self._fields_
                for v in [getattr(self, f)]}


VATE_SUBMIT_PINNED = 1
VATE_FAULT_STALL, VATE_FAULT_DROP, VATE_FAULT_HOLD = 1, 2, 3


class vate_server_fault(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("mon", C.c_int32), ("count", C.c_uint32), ("ms", C.c_uint32)]


def _load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError("%s is not built (run `python -m paper_1812_00282_b300.build`): %s"
                          % (os.path.basename(path), path))
    lib = C.CDLL(path)
    vp, u32, u64, i64, i = C.c_void_p, C.c_uint32, C.c_uint64, C.c_int64, C.c_int
    P = C.POINTER
    sig = {
        "vate_create": (i, [P(vate_params), vp, P(vp)]),
        "vate_destroy": (i, [vp]),
        "vate_ingest": (i, [vp, vp, u64, i64, vp]),
        "vate_close_slice": (i, [vp, i64, vp]),
        "vate_estimate": (i, [vp, vp, u64, u32, vp, vp, vp]),
        "vate_active_counts": (i, [vp, vp, u64, u32, vp, vp]),
        "vate_age_counts": (i, [vp, vp, u64, vp, vp]),
        "vate_census": (i, [vp, vp, vp]),
        "vate_copy_pool": (i, [vp, vp, vp]),
        "vate_load_pool": (i, [vp, vp, vp]),
        "vate_ingest_host": (i, [vp, vp, u64, i64, vp]),
        "vate_estimate_host": (i, [vp, vp, u64, u32, vp, vp, vp]),
        "vate_get_info": (i, [vp, P(vate_info)]),
        "vate_host_h": (i, [P(vate_params), u32, u32, P(u64)]),
        "vate_host_bh": (i, [P(vate_params), u32, P(u32)]),
        "vate_host_block": (i, [P(vate_params), u64, P(u32)]),
        "vate_last_error": (C.c_char_p, []),
        "vate_launch_count": (u64, []),
        "vate_census_noalloc": (i, [P(vate_params), vp, u32, vp, vp]),
        "vate_group_create": (i, [vp, u32, vp, P(vp)]),
        "vate_group_destroy": (i, [vp]),
        "vate_group_step": (i, [vp, vp, vp, u64, vp, vp, u64, vp, vp, vp, vp]),
        "vate_group_step_graph": (i, [vp, vp, vp, u64, vp, vp, u64, vp, vp, vp, vp]),
        "vate_group_autotune": (i, [vp, vp, vp, u64, vp, vp, u64, vp, vp, vp, P(vate_group_tuning), vp]),
        "vate_group_set_tuning": (i, [vp, P(vate_group_tuning)]),
        "vate_group_set_wait": (i, [vp, u64, u32]),
        "vate_group_set_trace": (i, [vp, vp, u32]),
        "vate_group_graph_nodes": (i, [vp, P(C.c_uint32)]),
        "vate_group_get_tuning": (i, [vp, P(vate_group_tuning)]),
        "vate_group_status": (i, [vp, P(u32), i, vp]),
        "vate_group_copy_pool": (i, [vp, u32, vp, vp]),
        "vate_group_census": (i, [vp, u32, vp, vp]),
        "vate_group_monitor_info": (i, [vp, u32, P(vate_info), vp]),
        "vate_mlp_param_count": (u64, [u32]),
        "vate_mlp_train_scratch": (u64, [u32, u64]),
        "vate_features": (i, [vp, vp, u64, vp, vp]),
        "vate_mlp_init": (i, [vp, u32, u64, vp]),
        "vate_mlp_forward": (i, [vp, u32, vp, u64, vp, vp]),
        "vate_mlp_apply": (i, [vp, u32, vp, vp, u64, vp, vp, vp]),
        "vate_mlp_train_step": (i, [vp, vp, vp, u32, vp, vp, vp, u32, u64, C.c_float, u32, vp, u64, vp, vp, vp]),
        "vate_estimate_learned": (i, [vp, vp, u64, vp, vp, vp, vp]),
        "vate_server_create": (i, [P(vate_server_config), P(vp)]),
        "vate_server_destroy": (i, [vp]),
        "vate_server_admit": (i, [vp, P(vate_params), P(C.c_int32)]),
        "vate_server_release": (i, [vp, C.c_int32]),
        "vate_server_set_model": (i, [vp, C.c_int32, vp]),
        "vate_server_submit_ingest": (i, [vp, C.c_int32, vp, u64, i64, u32, P(u64)]),
        "vate_server_submit_close": (i, [vp, C.c_int32, i64, vp, u64, u32, vp, vp, u32, P(u64)]),
        "vate_server_wait": (i, [vp, u64, u32]),
        "vate_server_drain": (i, [vp, u32]),
        "vate_server_get_stats": (i, [vp, P(vate_server_stats), i]),
        "vate_server_inject": (i, [vp, P(vate_server_fault)]),
        "vate_create_shard": (i, [P(vate_params), u64, u64, vp, P(vp)]),
        "vate_estimate_from_counts": (i, [P(vate_params), vp, vp, u64, u32, vp, vp, vp]),
        "vate_checkpoint_size": (i, [vp, P(u64)]),
        "vate_checkpoint": (i, [vp, vp, u64, vp]),
        "vate_restore": (i, [vp, u64, vp, P(vp)]),
        "vate_debug_checks": (i, []),
        "vate_debug_status": (i, [vp, P(u32), P(u64), i, vp]),
        "vate_debug_poke": (i, [vp, u64, u32, vp]),
        "vate_hostset_create": (i, [vp, vp, u64, vp, P(vp)]),
        "vate_hostset_destroy": (i, [vp]),
        "vate_hostset_info": (i, [vp, P(u64), P(u64), P(u32)]),
        "vate_estimate_hostset": (i, [vp, vp, u32, vp, vp, vp, vp]),
        "vate_estimate_hostset_host": (i, [vp, vp, u32, vp, vp, vp]),
        "vate_hostset_create_ages": (i, [vp, vp, u64, vp, P(vp)]),
        "vate_estimate_hostset_host_async": (i, [vp, vp, u32, vp, vp, vp]),
        "vate_hostset_wait": (i, [vp]),
        "vate_hostset_time_passes": (i, [vp, u32]),
        "vate_hostset_pass_times": (i, [vp, vp, u32, P(u32)]),
        "vate_age_counts_hostset": (i, [vp, vp, vp, vp]),
        "vate_estimate_learned_hostset": (i, [vp, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


class use_library:
    """Route every function of this binding to another build of the library
    while the block runs -- `with use_library(DEBUG_LIB_PATH): ...` runs the
    same calls on the checked build.  Handles belong to the library that made
    them: create and destroy them inside the block."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self._saved = _lib
        _lib = _load(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def vate_debug_checks() -> bool:
    return bool(_lib.vate_debug_checks())


def vate_debug_status(h, clear: bool = False, stream=None):
    """(VATE_DBG_* bits, first report) of the handle (include/vate.h)."""
    bits, first = C.c_uint32(), C.c_uint64()
    _check(_lib.vate_debug_status(h, C.byref(bits), C.byref(first), 1 if clear else 0, _stream(stream)))
    return int(bits.value), int(first.value)


def vate_debug_poke(h, pid: int, value: int, stream=None) -> None:
    _check(_lib.vate_debug_poke(h, pid, value, _stream(stream)))


def _check(rc: int) -> None:
    if rc != VATE_OK:
        raise VateError(rc, _lib.vate_last_error().decode())


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev(t, dtype, name: str, count: Optional[int] = None) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must have dtype %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if count is not None and t.numel() < count:
        raise ValueError("%s holds %d elements, %d needed" % (name, t.numel(), count))
    return t.data_ptr()


def _host(a, dtype, name: str, output: bool = False):
    """(pointer, keep-alive object, element count) of a host array.  Outputs
    must already have the right dtype and layout (no converting copy)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.is_cuda:
                raise TypeError("%s must be a host array" % name)
            if not a.is_contiguous():
                raise ValueError("%s must be contiguous" % name)
            if a.element_size() != np.dtype(dtype).itemsize:
                raise TypeError("%s must have %d-byte elements" % (name, np.dtype(dtype).itemsize))
            return a.data_ptr(), a, a.numel()
    except ImportError:
        pass
    if output:
        if not isinstance(a, np.ndarray) or a.dtype != np.dtype(dtype) or not a.flags.c_contiguous:
            raise TypeError("%s must be a C-contiguous numpy array of %s" % (name, np.dtype(dtype)))
        return a.ctypes.data, a, a.size
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data, arr, arr.size


VATE_COUNTER_AT, VATE_COUNTER_DR = 0, 1


def make_params(log2_pool: int, k: int, g: int, seg_len: int = 1, partition: int = 0, seed: int = 0,
                counter: int = 0, at_bits: int = 0, options: int = 0) -> vate_params:
    return vate_params(log2_pool, k, g, seg_len, partition, counter, at_bits, options, seed & 0xFFFFFFFFFFFFFFFF)


# ---- the C ABI, one function per entry point --------------------------------

def vate_create(params: vate_params, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.vate_create(C.byref(params), _stream(stream), C.byref(h)))
    _k_of[h.value] = int(params.k)
    return h


def vate_destroy(h) -> None:
    _k_of.pop(h.value if isinstance(h, C.c_void_p) else h, None)
    _check(_lib.vate_destroy(h))


def vate_ingest(h, pairs, slice: int, stream=None) -> None:
    """pairs: CUDA tensor of shape (n, 2), dtype int32/uint32 (aip, bip)."""
    import torch
    n = pairs.shape[0] if pairs.dim() == 2 else pairs.numel() // 2
    ptr = _dev(pairs, pairs.dtype if pairs.dtype in (torch.int32, torch.uint32) else torch.int32, "pairs")
    _check(_lib.vate_ingest(h, ptr if n else None, n, slice, _stream(stream)))


def vate_close_slice(h, slice: int, stream=None) -> None:
    _check(_lib.vate_close_slice(h, slice, _stream(stream)))


def vate_estimate(h, aips, kprime: int, out, flags=None, stream=None) -> None:
    import torch
    n = aips.numel()
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    po = _dev(out, torch.float32, "out", n)
    pf = _dev(flags, torch.uint8, "flags", n) if flags is not None else None
    _check(_lib.vate_estimate(h, pa, n, kprime, po, pf, _stream(stream)))


def vate_active_counts(h, aips, kprime: int, active, stream=None) -> None:
    import torch
    n = aips.numel()
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    pc = _dev(active, active.dtype if active.dtype in (torch.int32, torch.uint32) else torch.int32, "active", n)
    _check(_lib.vate_active_counts(h, pa, n, kprime, pc, _stream(stream)))


def vate_age_counts(h, aips, counts, stream=None) -> None:
    import torch
    n = aips.numel()
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    k = vate_get_info_k(h)
    pc = _dev(counts, counts.dtype if counts.dtype in (torch.int16, torch.uint16) else torch.int16, "counts", n * k)
    _check(_lib.vate_age_counts(h, pa, n, pc, _stream(stream)))


def vate_census(h, hist, stream=None) -> None:
    import torch
    k = vate_get_info_k(h)
    _check(_lib.vate_census(h, _dev(hist, hist.dtype if hist.dtype in (torch.int64, torch.uint64) else torch.int64,
                                    "hist", 2 * k + 1), _stream(stream)))


def pool_dtype(k: int):
    """torch dtype of a pool copy: uint8 ATs for k <= 63, 16-bit ones (int16 in torch) beyond."""
    import torch
    return torch.uint8 if k <= 63 else torch.int16


def vate_copy_pool(h, dst, stream=None) -> None:
    info = vate_get_info(h)
    n = info.pid_hi - info.pid_lo
    _check(_lib.vate_copy_pool(h, _dev(dst, pool_dtype(vate_get_info_k(h)), "dst", n), _stream(stream)))


def vate_load_pool(h, src, stream=None) -> None:
    info = vate_get_info(h)
    n = info.pid_hi - info.pid_lo
    _check(_lib.vate_load_pool(h, _dev(src, pool_dtype(vate_get_info_k(h)), "src", n), _stream(stream)))


def vate_ingest_host(h, pairs, slice: int, stream=None) -> None:
    ptr, keep, cnt = _host(pairs, np.uint32, "pairs")
    n = cnt // 2
    _check(_lib.vate_ingest_host(h, ptr if n else None, n, slice, _stream(stream)))
    return keep


def vate_estimate_host(h, aips, kprime: int, out, flags=None, stream=None) -> None:
    pa, ka, n = _host(aips, np.uint32, "aips")
    po, ko, no = _host(out, np.float32, "out", output=True)
    if no < n:
        raise ValueError("out is too small")
    pf = None
    if flags is not None:
        pf, kf, nf = _host(flags, np.uint8, "flags", output=True)
        if nf < n:
            raise ValueError("flags is too small")
    _check(_lib.vate_estimate_host(h, pa, n, kprime, po, pf, _stream(stream)))


_k_of = {}


def vate_get_info_k(h) -> int:
    """k of a handle (kept by the binding at creation, for buffer-size checks)."""
    return _k_of[h.value if isinstance(h, C.c_void_p) else int(h)]


def vate_get_info(h) -> vate_info:
    info = vate_info()
    _check(_lib.vate_get_info(h, C.byref(info)))
    return info


def vate_host_h(params: vate_params, aip: int, i: int) -> int:
    out = C.c_uint64()
    _check(_lib.vate_host_h(C.byref(params), aip, i, C.byref(out)))
    return int(out.value)


def vate_host_bh(params: vate_params, bip: int) -> int:
    out = C.c_uint32()
    _check(_lib.vate_host_bh(C.byref(params), bip, C.byref(out)))
    return int(out.value)


def vate_host_block(params: vate_params, pid: int) -> int:
    out = C.c_uint32()
    _check(_lib.vate_host_block(C.byref(params), pid, C.byref(out)))
    return int(out.value)


def vate_last_error() -> str:
    return _lib.vate_last_error().decode()


def vate_launch_count() -> int:
    return int(_lib.vate_launch_count())


def vate_census_noalloc(params: vate_params, pool, bact0: int, hist, stream=None) -> None:
    """Census of a caller-owned pool into a caller-owned histogram; the library
    allocates no device memory for it (include/vate.h)."""
    import torch
    pp = _dev(pool, torch.uint8, "pool", 1 << params.log2_pool)
    ph = _dev(hist, hist.dtype if hist.dtype in (torch.int64, torch.uint64) else torch.int64, "hist",
              2 * params.k + 1)
    _check(_lib.vate_census_noalloc(C.byref(params), pp, bact0, ph, _stream(stream)))


# ---- learned estimator (include/vate_learned.h) -------------------------------

VATE_FLAG_FALLBACK, VATE_FLAG_GATED = 4, 8
VATE_MLP_LOSS_SQUARED, VATE_MLP_LOSS_ABSOLUTE = 0, 1


def vate_mlp_param_count(n_in: int) -> int:
    return int(_lib.vate_mlp_param_count(n_in))


def vate_mlp_train_scratch(n_in: int, n: int) -> int:
    return int(_lib.vate_mlp_train_scratch(n_in, n))


def vate_features(h, aips, x, stream=None) -> None:
    import torch
    n = aips.numel()
    k = vate_get_info_k(h)
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    px = _dev(x, torch.float32, "x", n * (2 * k + 2))
    _check(_lib.vate_features(h, pa, n, px, _stream(stream)))


def vate_mlp_init(params, n_in: int, seed: int, stream=None) -> None:
    import torch
    _check(_lib.vate_mlp_init(_dev(params, torch.float32, "params", vate_mlp_param_count(n_in)), n_in,
                              seed & 0xFFFFFFFFFFFFFFFF, _stream(stream)))


def vate_mlp_forward(params, n_in: int, x, y, stream=None) -> None:
    import torch
    n = x.numel() // n_in
    _check(_lib.vate_mlp_forward(_dev(params, torch.float32, "params", vate_mlp_param_count(n_in)), n_in,
                                 _dev(x, torch.float32, "x", n * n_in), n, _dev(y, torch.float32, "y", n),
                                 _stream(stream)))


def vate_mlp_train_step(params, m, v, n_in: int, x, target, lr: float, t: int, scratch, grad=None, loss=None,
                        weight=None, loss_kind: int = VATE_MLP_LOSS_SQUARED, stream=None) -> None:
    import torch
    n = target.numel()
    npar = vate_mlp_param_count(n_in)
    _check(_lib.vate_mlp_train_step(
        _dev(params, torch.float32, "params", npar), _dev(m, torch.float32, "m", npar),
        _dev(v, torch.float32, "v", npar), n_in, _dev(x, torch.float32, "x", n * n_in),
        _dev(target, torch.float32, "target", n),
        _dev(weight, torch.float32, "weight", n) if weight is not None else None, loss_kind, n, float(lr), t,
        _dev(scratch, torch.float32, "scratch"),
        scratch.numel(), _dev(grad, torch.float32, "grad", npar) if grad is not None else None,
        _dev(loss, torch.float32, "loss", 1) if loss is not None else None, _stream(stream)))


def vate_mlp_apply(params, n_in: int, x, plain, out, flags=None, stream=None) -> None:
    """The learned estimator's output rule on feature rows (include/vate_learned.h)."""
    import torch
    n = plain.numel()
    pp = _dev(params, torch.float32, "params", vate_mlp_param_count(n_in))
    px = _dev(x, torch.float32, "x", n * n_in)
    pl = _dev(plain, torch.float32, "plain", n)
    po = _dev(out, torch.float32, "out", n)
    pf = _dev(flags, torch.uint8, "flags", n) if flags is not None else None
    _check(_lib.vate_mlp_apply(pp, n_in, px, pl, n, po, pf, _stream(stream)))


def vate_estimate_learned(h, aips, params, out, flags=None, stream=None) -> None:
    import torch
    n = aips.numel()
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    k = vate_get_info_k(h)
    pp = _dev(params, torch.float32, "params", vate_mlp_param_count(2 * k + 2))
    po = _dev(out, torch.float32, "out", n)
    pf = _dev(flags, torch.uint8, "flags", n) if flags is not None else None
    _check(_lib.vate_estimate_learned(h, pa, n, pp, po, pf, _stream(stream)))


# ---- monitor groups (include/vate_group.h) -----------------------------------

def _group_args(pairs, pair_offsets, hosts, host_offsets, kprime, out, flags):
    import torch
    i32 = lambda t: t.dtype if t.dtype in (torch.int32, torch.uint32) else torch.int32
    i64 = lambda t: t.dtype if t.dtype in (torch.int64, torch.uint64) else torch.int64
    npairs = pairs.shape[0] if pairs.dim() == 2 else pairs.numel() // 2
    pp = _dev(pairs, i32(pairs), "pairs") if npairs else None
    po = _dev(pair_offsets, i64(pair_offsets), "pair_offsets")
    nh = hosts.numel()
    ph = _dev(hosts, i32(hosts), "hosts") if nh else None
    ho = _dev(host_offsets, i64(host_offsets), "host_offsets")
    kp = _dev(kprime, i32(kprime), "kprime")
    pout = _dev(out, torch.float32, "out", nh) if nh else None
    pf = _dev(flags, torch.uint8, "flags", nh) if (flags is not None and nh) else None
    return pp, po, npairs, ph, ho, nh, kp, pout, pf


def vate_group_create(params_list, stream=None) -> C.c_void_p:
    arr = (vate_params * len(params_list))(*params_list)
    g = C.c_void_p()
    _check(_lib.vate_group_create(C.cast(arr, C.c_void_p), len(params_list), _stream(stream), C.byref(g)))
    return g


def vate_group_destroy(g) -> None:
    _check(_lib.vate_group_destroy(g))


def vate_group_step(g, pairs, pair_offsets, hosts, host_offsets, kprime, out, flags=None, stream=None) -> None:
    a = _group_args(pairs, pair_offsets, hosts, host_offsets, kprime, out, flags)
    _check(_lib.vate_group_step(g, *a, _stream(stream)))


def vate_group_step_graph(g, pairs, pair_offsets, hosts, host_offsets, kprime, out, flags=None, stream=None) -> None:
    a = _group_args(pairs, pair_offsets, hosts, host_offsets, kprime, out, flags)
    _check(_lib.vate_group_step_graph(g, *a, _stream(stream)))


def vate_group_autotune(g, pairs, pair_offsets, hosts, host_offsets, kprime, out, flags=None,
                        stream=None) -> vate_group_tuning:
    a = _group_args(pairs, pair_offsets, hosts, host_offsets, kprime, out, flags)
    t = vate_group_tuning()
    _check(_lib.vate_group_autotune(g, *a, C.byref(t), _stream(stream)))
    return t


def vate_group_set_tuning(g, t: vate_group_tuning) -> None:
    _check(_lib.vate_group_set_tuning(g, C.byref(t)))


def vate_group_set_wait(g, spin_limit: int, missing: int = 0) -> None:
    _check(_lib.vate_group_set_wait(g, spin_limit, missing))


def vate_group_set_trace(g, trace=None) -> None:
    """trace: a CUDA int64 tensor of 4 x items, or None to stop tracing."""
    import torch
    if trace is None:
        _check(_lib.vate_group_set_trace(g, None, 0))
    else:
        _check(_lib.vate_group_set_trace(g, _dev(trace, torch.int64, "trace"), trace.numel() // 4))


def vate_group_graph_nodes(g) -> int:
    n = C.c_uint32()
    _check(_lib.vate_group_graph_nodes(g, C.byref(n)))
    return int(n.value)


def vate_group_get_tuning(g) -> vate_group_tuning:
    t = vate_group_tuning()
    _check(_lib.vate_group_get_tuning(g, C.byref(t)))
    return t


def vate_group_status(g, clear: bool = False, stream=None) -> int:
    s = C.c_uint32()
    _check(_lib.vate_group_status(g, C.byref(s), 1 if clear else 0, _stream(stream)))
    return int(s.value)


def vate_group_copy_pool(g, m: int, dst, stream=None) -> None:
    import torch
    _check(_lib.vate_group_copy_pool(g, m, _dev(dst, torch.uint8, "dst"), _stream(stream)))


def vate_group_census(g, m: int, hist, stream=None) -> None:
    import torch
    _check(_lib.vate_group_census(g, m, _dev(hist, hist.dtype if hist.dtype in (torch.int64, torch.uint64)
                                                else torch.int64, "hist"), _stream(stream)))


def vate_group_monitor_info(g, m: int, stream=None) -> vate_info:
    info = vate_info()
    _check(_lib.vate_group_monitor_info(g, m, C.byref(info), _stream(stream)))
    return info


class VateGroup:
    """Owns one monitor group; methods forward to the vate_group_* functions."""

    def __init__(self, params_list, stream=None):
        self.params = list(params_list)
        self.M = len(self.params)
        self.g = vate_group_create(self.params, stream)

    def close(self) -> None:
        if self.g:
            vate_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, *a, graph: bool = False, **kw):
        (vate_group_step_graph if graph else vate_group_step)(self.g, *a, **kw)

    def autotune(self, *a, **kw) -> vate_group_tuning:
        return vate_group_autotune(self.g, *a, **kw)

    def status(self, clear: bool = False) -> int:
        return vate_group_status(self.g, clear)

    def copy_pool(self, m, dst, stream=None):
        vate_group_copy_pool(self.g, m, dst, stream)

    def census(self, m, hist, stream=None):
        vate_group_census(self.g, m, hist, stream)


# ---- serving loop (include/vate_server.h) -------------------------------------

def vate_server_create(memory_budget_bytes: int, slots: int = 8, slot_records: int = 1 << 20) -> C.c_void_p:
    cfg = vate_server_config(memory_budget_bytes, slots, slot_records)
    s = C.c_void_p()
    _check(_lib.vate_server_create(C.byref(cfg), C.byref(s)))
    return s


def vate_server_destroy(s) -> None:
    _check(_lib.vate_server_destroy(s))


def vate_server_admit(s, params: vate_params) -> int:
    i = C.c_int32()
    _check(_lib.vate_server_admit(s, C.byref(params), C.byref(i)))
    return int(i.value)


def vate_server_release(s, mid: int) -> None:
    _check(_lib.vate_server_release(s, mid))


def vate_server_set_model(s, mid: int, params=None) -> None:
    import torch
    _check(_lib.vate_server_set_model(s, mid, _dev(params, torch.float32, "params") if params is not None else None))


def _host_ptr(a, nbytes_per, name):
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous():
            raise TypeError("%s must be a contiguous host tensor" % name)
        return a.data_ptr(), a.numel() * a.element_size() // nbytes_per
    if not isinstance(a, np.ndarray) or not a.flags.c_contiguous:
        raise TypeError("%s must be a C-contiguous numpy array or host tensor" % name)
    return a.ctypes.data, a.nbytes // nbytes_per


def vate_server_submit_ingest(s, mid: int, pairs, slice: int, flags: int = 0) -> int:
    """pairs: host buffer of (aip, bip) uint32 pairs; keep it alive until wait()."""
    ptr, n = _host_ptr(pairs, 8, "pairs")
    t = C.c_uint64()
    _check(_lib.vate_server_submit_ingest(s, mid, ptr if n else None, n, slice, flags, C.byref(t)))
    return int(t.value)


def vate_server_submit_close(s, mid: int, slice: int, hosts, kprime: int, out, flags_out=None, flags: int = 0) -> int:
    ph, n = _host_ptr(hosts, 4, "hosts")
    po, no = _host_ptr(out, 4, "out")
    if no < n:
        raise ValueError("out is too small")
    pf = None
    if flags_out is not None:
        pf, nf = _host_ptr(flags_out, 1, "flags_out")
        if nf < n:
            raise ValueError("flags_out is too small")
    t = C.c_uint64()
    _check(_lib.vate_server_submit_close(s, mid, slice, ph if n else None, n, kprime, po, pf, flags, C.byref(t)))
    return int(t.value)


def vate_server_wait(s, ticket: int, timeout_ms: int = 60000) -> None:
    _check(_lib.vate_server_wait(s, ticket, timeout_ms))


def vate_server_drain(s, timeout_ms: int = 60000) -> None:
    _check(_lib.vate_server_drain(s, timeout_ms))


def vate_server_get_stats(s, reset: bool = False) -> vate_server_stats:
    st = vate_server_stats()
    _check(_lib.vate_server_get_stats(s, C.byref(st), 1 if reset else 0))
    return st


def vate_server_inject(s, kind: int, mon: int = 0, count: int = 0, ms: int = 0) -> None:
    """Host-side fault injection in the serving loop (include/vate_server.h)."""
    _check(_lib.vate_server_inject(s, C.byref(vate_server_fault(kind, mon, count, ms))))


def vate_hostset_create(h, aips, stream=None) -> C.c_void_p:
    """The index of the hosts `aips` for handle h (include/vate_hostset.h)."""
    import torch
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    s = C.c_void_p()
    _check(_lib.vate_hostset_create(h, pa, aips.numel(), _stream(stream), C.byref(s)))
    return s


def vate_hostset_create_ages(h, aips, stream=None) -> C.c_void_p:
    """The age index of the hosts `aips` for handle h (include/vate_hostset.h)."""
    import torch
    pa = _dev(aips, aips.dtype if aips.dtype in (torch.int32, torch.uint32) else torch.int32, "aips")
    s = C.c_void_p()
    _check(_lib.vate_hostset_create_ages(h, pa, aips.numel(), _stream(stream), C.byref(s)))
    return s


def vate_age_counts_hostset(h, s, counts, stream=None) -> None:
    """vate_age_counts for an age index's hosts (include/vate_hostset.h)."""
    import torch
    n = vate_hostset_info(s)[1]
    k = vate_get_info_k(h)
    pc = _dev(counts, counts.dtype if counts.dtype in (torch.int16, torch.uint16) else torch.int16, "counts", n * k)
    _check(_lib.vate_age_counts_hostset(h, s, pc, _stream(stream)))


def vate_estimate_learned_hostset(h, s, params, out, flags=None, stream=None) -> None:
    """vate_estimate_learned for an age index's hosts (include/vate_hostset.h)."""
    import torch
    n = vate_hostset_info(s)[1]
    k = vate_get_info_k(h)
    pp = _dev(params, torch.float32, "params", vate_mlp_param_count(2 * k + 2))
    po = _dev(out, torch.float32, "out", n)
    pf = _dev(flags, torch.uint8, "flags", n) if flags is not None else None
    _check(_lib.vate_estimate_learned_hostset(h, s, pp, po, pf, _stream(stream)))


def vate_hostset_destroy(s) -> None:
    _check(_lib.vate_hostset_destroy(s))


def vate_hostset_info(s):
    """(device bytes, hosts, regions) of a hostset."""
    b, n, r = C.c_uint64(), C.c_uint64(), C.c_uint32()
    _check(_lib.vate_hostset_info(s, C.byref(b), C.byref(n), C.byref(r)))
    return int(b.value), int(n.value), int(r.value)


def vate_estimate_hostset(h, s, kprime: int, out, flags=None, active=None, stream=None) -> None:
    """vate_estimate for the hostset's hosts, through its index (include/vate_hostset.h)."""
    import torch
    n = vate_hostset_info(s)[1]
    po = _dev(out, torch.float32, "out", n)
    pf = _dev(flags, torch.uint8, "flags", n) if flags is not None else None
    pc = _dev(active, active.dtype if active.dtype in (torch.int32, torch.uint32) else torch.int32, "active", n) \
        if active is not None else None
    _check(_lib.vate_estimate_hostset(h, s, kprime, po, pf, pc, _stream(stream)))


def vate_estimate_hostset_host(h, s, kprime: int, out, flags=None, stream=None) -> None:
    """vate_estimate_hostset into host tensors (page-locked for asynchronous copies)."""
    import torch
    n = vate_hostset_info(s)[1]
    for t, dt, name in ((out, torch.float32, "out"), (flags, torch.uint8, "flags")):
        if t is not None and (t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.numel() < n):
            raise ValueError("%s must be a contiguous host %s tensor of at least %d elements" % (name, dt, n))
    _check(_lib.vate_estimate_hostset_host(h, s, kprime, out.data_ptr(),
                                           flags.data_ptr() if flags is not None else None, _stream(stream)))


def vate_estimate_hostset_host_async(h, s, kprime: int, out, flags=None, stream=None) -> None:
    """vate_estimate_hostset_host with its copies on a stream of the hostset;
    the host tensors hold the results after vate_hostset_wait(s)."""
    import torch
    n = vate_hostset_info(s)[1]
    for t, dt, name in ((out, torch.float32, "out"), (flags, torch.uint8, "flags")):
        if t is not None and (t.is_cuda or t.dtype != dt or not t.is_contiguous() or t.numel() < n):
            raise ValueError("%s must be a contiguous host %s tensor of at least %d elements" % (name, dt, n))
    _check(_lib.vate_estimate_hostset_host_async(h, s, kprime, out.data_ptr(),
                                                 flags.data_ptr() if flags is not None else None, _stream(stream)))


def vate_hostset_wait(s) -> None:
    _check(_lib.vate_hostset_wait(s))


def vate_hostset_time_passes(s, n: int) -> None:
    """Time the index pass of the next n closes through hostset s (include/vate_hostset.h)."""
    _check(_lib.vate_hostset_time_passes(s, n))


def vate_hostset_pass_times(s, max_n: int = 4096):
    """The recorded index-pass durations, in ms, in call order."""
    buf = (C.c_float * max(1, max_n))()
    cnt = C.c_uint32()
    _check(_lib.vate_hostset_pass_times(s, C.cast(buf, C.c_void_p), max_n, C.byref(cnt)))
    return [float(buf[i]) for i in range(cnt.value)]


def vate_create_shard(params: vate_params, pid_lo: int, pid_hi: int, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(_lib.vate_create_shard(C.byref(params), pid_lo, pid_hi, _stream(stream), C.byref(h)))
    _k_of[h.value] = int(params.k)
    return h


def vate_estimate_from_counts(params: vate_params, active, hist, kprime: int, out, flags=None, stream=None) -> None:
    import torch
    n = active.numel()
    _check(_lib.vate_estimate_from_counts(
        C.byref(params), _dev(active, torch.int32, "active"), _dev(hist, torch.int64, "hist", 2 * params.k + 1), n,
        kprime, _dev(out, torch.float32, "out", n), _dev(flags, torch.uint8, "flags", n) if flags is not None else None,
        _stream(stream)))


VATE_CHECKPOINT_MAGIC, VATE_CHECKPOINT_VERSION = 0x31544B4345544156, 2


class vate_checkpoint_header(C.Structure):
    _fields_ = [("magic", C.c_uint64), ("version", C.c_uint32), ("header_bytes", C.c_uint32),
                ("params", vate_params), ("slice", C.c_int64), ("bact0", C.c_uint32), ("closed", C.c_uint32),
                ("hist_bytes", C.c_uint64), ("pool_bytes", C.c_uint64), ("checksum", C.c_uint64)]


def vate_checkpoint_size(h) -> int:
    n = C.c_uint64()
    _check(_lib.vate_checkpoint_size(h, C.byref(n)))
    return n.value


def vate_checkpoint(h, buf=None, stream=None) -> np.ndarray:
    """The handle's state as a uint8 host array (written into `buf` if given)."""
    n = vate_checkpoint_size(h)
    if buf is None:
        buf = np.empty(n, np.uint8)
    ptr, keep, cnt = _host(buf, np.uint8, "buf", output=True)
    _check(_lib.vate_checkpoint(h, ptr, cnt, _stream(stream)))
    return buf


def vate_restore(buf, stream=None) -> C.c_void_p:
    ptr, keep, cnt = _host(buf, np.uint8, "buf")
    h = C.c_void_p()
    _check(_lib.vate_restore(ptr, cnt, _stream(stream), C.byref(h)))
    hd = vate_checkpoint_header.from_buffer_copy(C.string_at(ptr, C.sizeof(vate_checkpoint_header)))
    _k_of[h.value] = int(hd.params.k)
    return h


class Vate:
    """Owns one handle; methods forward to the functions above."""

    def __init__(self, log2_pool: int, k: int, g: int, seg_len: int = 1, partition: int = 0, seed: int = 0,
                 stream=None, counter: int = 0, at_bits: int = 0, options: int = 0):
        self.params = make_params(log2_pool, k, g, seg_len, partition, seed, counter, at_bits, options)
        self.k, self.g, self.P = k, g, 1 << log2_pool
        self.h = vate_create(self.params, stream)

    def close(self) -> None:
        if self.h:
            vate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ingest(self, pairs, slice, stream=None):
        vate_ingest(self.h, pairs, slice, stream)

    def close_slice(self, slice, stream=None):
        vate_close_slice(self.h, slice, stream)

    def estimate(self, aips, kprime, out, flags=None, stream=None):
        vate_estimate(self.h, aips, kprime, out, flags, stream)

    def active_counts(self, aips, kprime, active, stream=None):
        vate_active_counts(self.h, aips, kprime, active, stream)

    def age_counts(self, aips, counts, stream=None):
        vate_age_counts(self.h, aips, counts, stream)

    def census(self, hist, stream=None):
        vate_census(self.h, hist, stream)

    def copy_pool(self, dst, stream=None):
        vate_copy_pool(self.h, dst, stream)

    def load_pool(self, src, stream=None):
        vate_load_pool(self.h, src, stream)

    def info(self) -> vate_info:
        return vate_get_info(self.h)

    def checkpoint(self, buf=None, stream=None) -> np.ndarray:
        return vate_checkpoint(self.h, buf, stream)

    @classmethod
    def restore(cls, buf, stream=None) -> "Vate":
        obj = cls.__new__(cls)
        obj.h = None
        obj.h = vate_restore(buf, stream)          # validates the image first
        ptr, keep, _ = _host(buf, np.uint8, "buf")
        hd = vate_checkpoint_header.from_buffer_copy(C.string_at(ptr, C.sizeof(vate_checkpoint_header)))
        obj.params = hd.params
        obj.k, obj.g, obj.P = hd.params.k, hd.params.g, 1 << hd.params.log2_pool
        return obj

    def save(self, path: str, stream=None) -> None:
        self.checkpoint(stream=stream).tofile(path)

    @classmethod
    def load(cls, path: str, stream=None) -> "Vate":
        return cls.restore(np.fromfile(path, dtype=np.uint8), stream)
