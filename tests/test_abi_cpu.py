"""CPU-side checks of the C-ABI library: it builds, loads, exports every symbol
that include/vate.h declares, validates arguments on the host, and its
host-side mapping (H, BH, block of Eq. 9-10 / low-deviation partition) agrees
with the oracle.  No kernel is launched here."""
import ctypes
import os
import re

import numpy as np
import pytest
import torch

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    from paper_1812_00282_b300 import build
    build.build()
    import paper_1812_00282_b300 as V
    return V


def declared_functions(probe=False):
    """Functions the headers declare: those of include/vate_probe.h (the
    measurement library) or those of every other header (libvate.so)."""
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if not hdr.endswith(".h") or (hdr == "vate_probe.h") != probe:
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(vate_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(V):
    names = declared_functions()
    assert "vate_create" in names and "vate_estimate" in names and len(names) >= 18
    lib = ctypes.CDLL(V.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
        assert hasattr(V, n), "binding lacks " + n
    assert not any(n.startswith("vate_probe") for n in names)


def test_probe_library_exports_its_symbols_and_libvate_does_not(V):
    from paper_1812_00282_b300 import probe
    names = declared_functions(probe=True)
    assert names == ["vate_probe_byte_write", "vate_probe_sector_read", "vate_probe_stream_read"]
    plib = ctypes.CDLL(probe.LIB_PATH)
    main = ctypes.CDLL(V.LIB_PATH)
    for n in names:
        assert hasattr(plib, n), n
        assert not hasattr(main, n), n + " is a measurement helper, not part of libvate.so"
        assert hasattr(probe, n[len("vate_probe_"):]), "binding lacks " + n


@pytest.mark.parametrize("bad", [
    dict(log2_pool=11), dict(log2_pool=33), dict(k=0), dict(k=1024), dict(g=0), dict(g=65537),
    dict(log2_pool=14, k=300),                                   # blocks of fewer than 32 ATs
    dict(k=10, at_bits=4), dict(k=10, at_bits=17), dict(k=300, log2_pool=20, at_bits=9),   # fields too narrow / wide
    dict(seg_len=3), dict(seg_len=128), dict(g=1000, seg_len=32), dict(partition=2),
])
def test_invalid_parameters_rejected_on_host(V, bad):
    p = dict(log2_pool=20, k=5, g=1024, seg_len=32, partition=0, seed=1)
    p.update(bad)
    params = V.make_params(**p)
    with pytest.raises(V.VateError) as ei:
        V.vate_create(params, stream=0)
    assert ei.value.code == V.VATE_EINVAL


def test_unknown_option_bits_are_rejected(V):
    params = V.make_params(20, 5, 1024)
    params.options = 2
    with pytest.raises(V.VateError) as ei:
        V.vate_create(params, stream=0)
    assert ei.value.code == V.VATE_EINVAL


def test_counter_kind_must_be_known(V):
    params = V.make_params(20, 5, 1024)
    params.counter = 2
    with pytest.raises(V.VateError) as ei:
        V.vate_create(params, stream=0)
    assert ei.value.code == V.VATE_EINVAL


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error path")
def test_create_without_gpu_reports_cuda_error(V):
    with pytest.raises(V.VateError) as ei:
        V.vate_create(V.make_params(20, 5, 1024), stream=0)
    assert ei.value.code == V.VATE_ECUDA
    assert "device" in V.vate_last_error().lower() or "driver" in V.vate_last_error().lower()


CASES = [(20, 5, 1024, 1, 0, 1), (20, 5, 1024, 32, 0, 2), (26, 10, 4096, 32, 0, 0xC2), (24, 10, 4096, 32, 1, 3),
         (14, 63, 256, 16, 0, 4), (13, 1, 64, 64, 1, 5), (32, 10, 512, 8, 0, 6), (16, 7, 96, 2, 1, 7)]


@pytest.mark.parametrize("c,k,g,L,part,seed", CASES)
def test_host_mapping_matches_oracle(V, c, k, g, L, part, seed):
    params = V.make_params(c, k, g, L, part, seed)
    o = oracle.Oracle(c=c, k=k, g=g, seg_len=L, partition=part, seed=seed) if c <= 26 else None
    rng = np.random.default_rng(seed)
    if o is None:
        # the oracle allocates the pool; for 2^32 compare the mixer-level spec instead
        key_h, key_bh = oracle.mix64(seed + 1), oracle.mix64(seed + 2)
        for _ in range(200):
            aip, i = int(rng.integers(0, 2**32)), int(rng.integers(0, g))
            j, off = i // L, i % L
            K = oracle.mix64(key_h ^ (aip << 32))
            x = oracle.fmix32((K & 0xFFFFFFFF) ^ ((j * 0x9E3779B9) & 0xFFFFFFFF)) ^ (K >> 32)
            seg = x >> (32 - (c - int(np.log2(L))))
            assert V.vate_host_h(params, aip, i) == seg * L + off
            bip = int(rng.integers(0, 2**32))
            assert V.vate_host_bh(params, bip) == ((oracle.mix64(key_bh ^ bip) >> 32) * g) >> 32
        return
    for _ in range(300):
        aip, i, bip = int(rng.integers(0, 2**32)), int(rng.integers(0, g)), int(rng.integers(0, 2**32))
        assert V.vate_host_h(params, aip, i) == o.h(aip, i)
        assert V.vate_host_bh(params, bip) == o.bh(bip)
    P = 1 << c
    probes = set(int(x) for x in rng.integers(0, P, size=500))
    for i in range(2 * k + 1):          # every block boundary and its neighbours
        for base in (i * o.a, i * (o.a + 1), o.a * (2 * k - o.b) + (i - (2 * k - o.b)) * (o.a + 1)):
            for d in (-1, 0, 1):
                if 0 <= base + d < P:
                    probes.add(base + d)
    probes.add(P - 1)
    for pid in probes:
        assert V.vate_host_block(params, pid) == o.block(pid), pid


def test_block_division_exact_near_2_32(V):
    # c = 32: pool positions up to 2^32 - 1 go through the 64-bit multiply-high
    # division; compare with exact integer division at the extremes.
    for k, part in ((10, 0), (10, 1), (1, 0), (63, 1)):
        params = V.make_params(32, k, 64, 1, part, 0)
        P, twok = 1 << 32, 2 * k
        if part == 0:
            a = P // (twok - 1)
            ref = lambda pid: pid // a
        else:
            a, b = P // twok, P % twok
            first = a * (twok - b)
            ref = lambda pid: pid // a if pid < first else (pid + twok - b) // (a + 1)
        for pid in [0, 1, a - 1, a, a + 1, P - 2, P - 1] + [P - 1 - 7919 * j for j in range(200)]:
            if pid >= P:
                continue
            assert V.vate_host_block(params, pid) == ref(pid), (k, part, pid)


# ---- checkpoint images: every check runs on the host before any device call --
def _fnv1a_words(b: bytes) -> int:
    """FNV-1a, 64-bit (Fowler/Noll/Vo published offset basis and prime), over
    little-endian 8-byte words."""
    h = 0xcbf29ce484222325
    for (w,) in np.frombuffer(b, dtype="<u8").reshape(-1, 1):
        h = ((h ^ int(w)) * 0x100000001b3) & 0xFFFFFFFFFFFFFFFF
    return h


def _image(V, c=12, k=3, slice_=4, bact0=2, closed=1, pool_value=None, counter=0, fix_checksum=True):
    hd = V.vate_checkpoint_header()
    hd.magic, hd.version, hd.header_bytes = V.VATE_CHECKPOINT_MAGIC, V.VATE_CHECKPOINT_VERSION, 96
    hd.params = V.make_params(c, k, 64, 1, 0, 9, counter)
    hd.slice, hd.bact0, hd.closed = slice_, bact0, closed
    hd.hist_bytes, hd.pool_bytes = (2 * k + 1) * 8, 1 << c
    pool = np.full(1 << c, 2 * k if pool_value is None else pool_value, np.uint8)
    pool[:7] = [0, 1, 2, 3, 4, 5, 6][: 7] if pool_value is None else pool_value
    body = bytes(hd) + np.zeros(2 * k + 1, np.uint64).tobytes() + pool.tobytes()
    if fix_checksum:
        hd.checksum = _fnv1a_words(body)
    return np.frombuffer(bytes(hd) + body[96:], np.uint8).copy()


def test_checkpoint_header_layout(V):
    import ctypes as C
    assert C.sizeof(V.vate_checkpoint_header) == 96
    assert V.vate_checkpoint_header.checksum.offset == 88
    assert V.VATE_CHECKPOINT_MAGIC.to_bytes(8, "little") == b"VATECKT1"


def test_valid_checkpoint_passes_every_host_check(V):
    # with no device the image is accepted up to the handle's creation
    if torch.cuda.is_available():
        pytest.skip("checks the no-GPU path")
    with pytest.raises(V.VateError) as ei:
        V.vate_restore(_image(V), stream=0)
    assert ei.value.code == V.VATE_ECUDA


@pytest.mark.parametrize("damage", ["short", "truncated", "magic", "version", "checksum", "value", "dr_value",
                                    "bact0", "closed", "before_first", "sizes", "params"])
def test_damaged_checkpoint_rejected_on_host(V, damage):
    img = _image(V)
    if damage == "short":
        img = img[:40]
    elif damage == "truncated":
        img = img[:-8]
    elif damage == "magic":
        img[0] ^= 0xFF
    elif damage == "version":
        img[8] = 7
    elif damage == "checksum":
        img[200] ^= 1
    elif damage == "value":
        img = _image(V, pool_value=7)                     # 2k + 1
    elif damage == "dr_value":
        img = _image(V, pool_value=4, counter=1)          # k + 1
    elif damage == "bact0":
        img = _image(V, bact0=6)
    elif damage == "closed":
        img = _image(V, closed=2)
    elif damage == "before_first":
        img = _image(V, slice_=-1, bact0=1, closed=0)
    elif damage == "sizes":
        img = _image(V)
        img[72] = 9                                       # hist_bytes
    elif damage == "params":
        img = _image(V, k=0)
    with pytest.raises(V.VateError) as ei:
        V.vate_restore(img, stream=0)
    assert ei.value.code == V.VATE_EINVAL, V.vate_last_error()


def test_hostset_calls_refuse_null_arguments_on_host(V):
    # include/vate_hostset.h: a NULL handle, hostset or output is refused before any device work
    lib = V._lib
    s = ctypes.c_void_p()
    buf = (ctypes.c_uint32 * 4)()
    assert lib.vate_hostset_create(None, ctypes.addressof(buf), 4, None, ctypes.byref(s)) == V.VATE_EINVAL
    assert lib.vate_hostset_create(None, ctypes.addressof(buf), 4, None, None) == V.VATE_EINVAL
    b, n, r = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
    assert lib.vate_hostset_info(None, ctypes.byref(b), ctypes.byref(n), ctypes.byref(r)) == V.VATE_EINVAL
    assert lib.vate_hostset_destroy(None) == V.VATE_OK
    assert lib.vate_estimate_hostset(None, None, 1, None, None, None, None) == V.VATE_EINVAL
    assert lib.vate_estimate_hostset_host(None, None, 1, None, None, None) == V.VATE_EINVAL
