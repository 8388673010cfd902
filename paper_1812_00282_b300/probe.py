"""Python binding of the memory-system probes (include/vate_probe.h,
libvate_probe.so): argument marshalling only.  A measurement library for the
benchmark's roofline denominators, separate from libvate.so."""
from __future__ import annotations

import ctypes as C
import os

from .vate import VateError, _dev, _stream

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvate_probe.so")


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError("libvate_probe.so is not built (run `python -m paper_1812_00282_b300.build`): " + LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, u32, u64 = C.c_void_p, C.c_uint32, C.c_uint64
    for name, args in (("vate_probe_sector_read", [vp, u64, u64, vp, u32, u32, vp]),
                       ("vate_probe_byte_write", [vp, u64, u64, u32, u32, vp]),
                       ("vate_probe_stream_read", [vp, u64, vp, u32, u32, vp])):
        f = getattr(lib, name)
        f.restype, f.argtypes = C.c_int, args
    return lib


_lib = _load()


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise VateError(rc, what)


def sector_read(buf, n_sectors: int, sink, loads_in_flight: int = 4, blocks_per_sm: int = 8, stream=None) -> None:
    """Random 32-byte sector reads from a CUDA uint8 buffer, two threads per sector."""
    import torch
    _check(_lib.vate_probe_sector_read(_dev(buf, torch.uint8, "buf"), buf.numel(), n_sectors,
                                       _dev(sink, torch.int32, "sink"), loads_in_flight, blocks_per_sm,
                                       _stream(stream)), "vate_probe_sector_read")


def byte_write(buf, n_writes: int, stores_per_trip: int = 4, blocks_per_sm: int = 8, stream=None) -> None:
    """Random 1-byte stores into a CUDA uint8 buffer."""
    import torch
    _check(_lib.vate_probe_byte_write(_dev(buf, torch.uint8, "buf"), buf.numel(), n_writes, stores_per_trip,
                                      blocks_per_sm, _stream(stream)), "vate_probe_byte_write")


def stream_read(buf, sink, loads_in_flight: int = 4, blocks_per_sm: int = 8, stream=None) -> None:
    """One coalesced read of the whole CUDA uint8 buffer."""
    import torch
    _check(_lib.vate_probe_stream_read(_dev(buf, torch.uint8, "buf"), buf.numel(), _dev(sink, torch.int32, "sink"),
                                       loads_in_flight, blocks_per_sm, _stream(stream)), "vate_probe_stream_read")
