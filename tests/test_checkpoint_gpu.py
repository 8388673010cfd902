"""Checkpoint and resume of a handle (include/vate_checkpoint.h).

A handle restored from a checkpoint must continue exactly as the handle it was
taken from: the same pool byte for byte, the same census, active counts and
estimates after every later slice, and both must still equal the oracle.
Checkpoints are taken at every point of the slice state machine: before the
first call, after an ingest (slice open), after a close, and across a gap of
empty slices; for asynchronous timestamps and for distance recorders.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from traffic import SMALL, Traffic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def state(V, d, hosts, kps):
    """Everything a caller can observe of a closed handle."""
    info = d.info()
    pool = torch.empty(d.P, dtype=V.pool_dtype(d.k), device="cuda")
    d.copy_pool(pool)
    hist = torch.empty(2 * d.k + 1, dtype=torch.int64, device="cuda")
    d.census(hist)
    out = {"slice": info.slice, "bact0": info.bact0, "pool": pool.cpu().numpy(), "hist": hist.cpu().numpy()}
    dh = dev_u32(hosts)
    for kp in kps:
        e = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
        f = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
        a = torch.empty(len(hosts), dtype=torch.int32, device="cuda")
        d.estimate(dh, kp, e, f)
        d.active_counts(dh, kp, a)
        out["est%d" % kp] = e.cpu().numpy()
        out["flags%d" % kp] = f.cpu().numpy()
        out["act%d" % kp] = a.cpu().numpy()
    return out


def assert_same(a, b, where):
    assert a.keys() == b.keys()
    for key in a:
        np.testing.assert_array_equal(a[key], b[key], err_msg="%s: %s" % (where, key))


SCHEDULE = [0, 1, 2, 3, 4, 6, 7, 8, 15, 16, 17, 18]   # gaps of 1 and 6 empty slices


@pytest.mark.parametrize("counter", [0, 1])
@pytest.mark.parametrize("when", ["before_first", "after_ingest", "after_close", "across_gap"])
def test_resume_continues_bit_exactly(V, counter, when, tmp_path):
    c, k, g, L, seed = 17, 5, 1024, 32, 0x5A
    tr = Traffic(SMALL, pkts_per_slice=12_000)
    hosts = tr.aips[:1500]
    kps = (1, 3, k)
    cut = {"before_first": 0, "after_ingest": 4, "after_close": 4, "across_gap": 7}[when]
    ref = V.Vate(c, k, g, L, 0, seed, counter=counter)
    cur = V.Vate(c, k, g, L, 0, seed, counter=counter)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=seed)
    prev = None
    for j, sid in enumerate(SCHEDULE):
        p = tr.slice_pairs(sid)
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        o.ingest(p)
        dp = torch.from_numpy(p.view(np.int32)).cuda()
        if j == cut and when == "before_first":
            cur = V.Vate.restore(cur.checkpoint())
        ref.ingest(dp, sid)
        cur.ingest(dp, sid)
        if j == cut and when == "after_ingest":
            img = cur.checkpoint()
            cur.close()
            cur = V.Vate.restore(img)
        ref.close_slice(sid)
        cur.close_slice(sid)
        if j == cut and when in ("after_close", "across_gap"):
            path = str(tmp_path / "monitor.vckpt")
            cur.save(path)
            cur.close()
            cur = V.Vate.load(path)
        a, b = state(V, ref, hosts, kps), state(V, cur, hosts, kps)
        assert_same(a, b, "slice %d" % sid)
        np.testing.assert_array_equal(b["pool"], o.dr() if counter else o.pool(), err_msg="oracle, slice %d" % sid)
        for kp in kps:
            _, oa, _ = o.estimate(hosts, kp)
            np.testing.assert_array_equal(b["act%d" % kp].view(np.uint32), oa)
    ref.close()
    cur.close()


def test_checkpoint_image_describes_the_handle(V):
    d = V.Vate(16, 4, 512, 32, 1, 7)
    p = Traffic(SMALL, pkts_per_slice=3000).slice_pairs(0)
    d.ingest(torch.from_numpy(p.view(np.int32)).cuda(), 3)
    d.close_slice(3)
    img = d.checkpoint()
    assert img.size == V.vate_checkpoint_size(d.h) == 96 + 9 * 8 + (1 << 16)
    hd = V.vate_checkpoint_header.from_buffer_copy(img[:96].tobytes())
    assert hd.magic == V.VATE_CHECKPOINT_MAGIC and hd.version == V.VATE_CHECKPOINT_VERSION
    assert (hd.slice, hd.bact0, hd.closed, hd.params.partition) == (3, 0, 1, 1)
    pool = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    d.copy_pool(pool)
    np.testing.assert_array_equal(img[96 + 72:], pool.cpu().numpy())
    with pytest.raises(V.VateError) as e:
        V.vate_checkpoint(d.h, np.empty(img.size - 1, np.uint8))
    assert e.value.code == V.VATE_EINVAL
    bad = img.copy()
    bad[96 + 72 + 5] ^= 1                          # one AT flipped: checksum mismatch
    with pytest.raises(V.VateError) as e:
        V.Vate.restore(bad)
    assert e.value.code == V.VATE_EINVAL and "checksum" in V.vate_last_error()
    d.close()


def test_wide_resume_continues_bit_exactly(V):
    c, k, g, L, seed = 18, 150, 512, 32, 0x77
    tr = Traffic(SMALL, pkts_per_slice=4000)
    hosts = tr.aips[:500]
    ref = V.Vate(c, k, g, L, 0, seed)
    cur = V.Vate(c, k, g, L, 0, seed)
    ids = [0, 1, 2, 100, 149, 150, 151, 300, 301, 302, 460]
    for j, sid in enumerate(ids):
        dp = torch.from_numpy(tr.slice_pairs(sid % 64).view(np.int32)).cuda()
        ref.ingest(dp, sid)
        cur.ingest(dp, sid)
        ref.close_slice(sid)
        cur.close_slice(sid)
        if j in (2, 6):
            img = cur.checkpoint()
            assert img.size == 96 + (2 * k + 1) * 8 + 2 * (1 << c)
            cur.close()
            cur = V.Vate.restore(img)
        a, b = state(V, ref, hosts, (1, k)), state(V, cur, hosts, (1, k))
        assert_same(a, b, "slice %d" % sid)
    ref.close()
    cur.close()


def test_packed_resume_continues_bit_exactly(V):
    c, k, g, L, seed = 17, 10, 512, 32, 0x78
    tr = Traffic(SMALL, pkts_per_slice=5000)
    hosts = tr.aips[:500]
    ref = V.Vate(c, k, g, L, 0, seed, at_bits=5)
    cur = V.Vate(c, k, g, L, 0, seed, at_bits=5)
    plain = V.Vate(c, k, g, L, 0, seed)
    for j, sid in enumerate([0, 1, 2, 9, 10, 11, 12, 25, 26]):
        dp = torch.from_numpy(tr.slice_pairs(sid).view(np.int32)).cuda()
        for d in (ref, cur, plain):
            d.ingest(dp, sid)
            d.close_slice(sid)
        if j in (2, 5):
            img = cur.checkpoint()
            assert img.size == 96 + (2 * k + 1) * 8 + (1 << c)      # unpacked: the paper's form
            cur.close()
            cur = V.Vate.restore(img)
        a, b, p = state(V, ref, hosts, (1, k)), state(V, cur, hosts, (1, k)), state(V, plain, hosts, (1, k))
        assert_same(a, b, "slice %d" % sid)
        assert_same(a, p, "packed vs byte, slice %d" % sid)
    for d in (ref, cur, plain):
        d.close()
