"""Parity of the CUDA path with the CPU oracle, element by element.

Every test drives the device through the C ABI (Python binding) and the
oracle through Algorithm 4 on the same seeded inputs and compares:
  - the AT pool, byte for byte, after every slice (bit-exact);
  - the pool census (bit-exact);
  - the active VAT count A of every host and window k' (bit-exact);
  - the per-age VAT counts (bit-exact);
  - the estimates of Eq. 11: |device - oracle| <= 1e-5 * max(|oracle|, 1)
    (FP32 on the device, FP64 in the oracle; the FP32 path evaluates
    g*log1p(x) from exact integers, a few ulp from the FP64 value);
  - the SAT / POOLFULL flags (bit-exact).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import Oracle
from traffic import LINK40G, SMALL, Traffic, mixed_hosts

pytestmark = pytest.mark.gpu
from eq11_tol import RTOL, assert_eq11_close  # noqa: E402


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def dev_pairs(pairs):
    return torch.from_numpy(np.ascontiguousarray(pairs, np.uint32).view(np.int32)).cuda()


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def compare_close(V, d, o, hosts, kps, check_pool=True, check_ages=True, check_estimates=True):
    """Compare device handle d (a Vate) and oracle o at a closed slice."""
    k = o.k
    if check_pool:
        pool = torch.empty(o.P, dtype=V.pool_dtype(k), device="cuda")
        d.copy_pool(pool)
        dp = pool.cpu().numpy().astype(np.int64)
        op = o.pool()
        if not np.array_equal(dp, op):
            bad = np.nonzero(dp != op)[0]
            raise AssertionError("pool differs at %d positions, first %s: dev %s oracle %s"
                                 % (bad.size, bad[:5], dp[bad[:5]], op[bad[:5]]))
    hist = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
    d.census(hist)
    np.testing.assert_array_equal(hist.cpu().numpy().astype(np.uint64), o.census())
    if not check_estimates:
        return
    dh = dev_u32(hosts)
    n = len(hosts)
    for kp in kps:
        est = torch.empty(n, dtype=torch.float32, device="cuda")
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        act = torch.empty(n, dtype=torch.int32, device="cuda")
        d.estimate(dh, kp, est, fl)
        d.active_counts(dh, kp, act)
        oe, oa, of = o.estimate(hosts, kp)
        np.testing.assert_array_equal(act.cpu().numpy().view(np.uint32), oa, err_msg="A, k'=%d" % kp)
        np.testing.assert_array_equal(fl.cpu().numpy(), of, err_msg="flags, k'=%d" % kp)
        de = est.cpu().numpy().astype(np.float64)
        assert_eq11_close(de, oe, o.g, "k'=%d" % kp)
    if check_ages and o.g <= 65535:
        ages = torch.empty(n * k, dtype=torch.int16, device="cuda")
        d.age_counts(dh, ages)
        np.testing.assert_array_equal(ages.cpu().numpy().view(np.uint16).reshape(n, k).astype(np.uint32),
                                      o.age_counts(hosts))


def run_stream(V, params, slices, hosts, kps, slice_ids=None, check_every=1, at_bits=0, pool_every_slice=False,
               **kw):
    c, k, g, L, part, seed = params
    d = V.Vate(c, k, g, L, part, seed, at_bits=at_bits)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=part, seed=seed)
    ids = list(range(len(slices))) if slice_ids is None else slice_ids
    prev = None
    for j, (sid, arr) in enumerate(zip(ids, slices)):
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        d.ingest(dev_pairs(arr), sid)
        o.ingest(arr)
        d.close_slice(sid)
        if j % check_every == 0 or j == len(slices) - 1:
            compare_close(V, d, o, hosts, kps, **kw)
        elif pool_every_slice:
            compare_close(V, d, o, hosts, kps, check_estimates=False, **kw)
    torch.cuda.synchronize()
    d.close()
    return o


@pytest.mark.parametrize("L", [1, 32])
@pytest.mark.parametrize("partition", [0, 1])
def test_small_traffic_parity(V, L, partition):
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    k = 5
    slices = [tr.slice_pairs(s) for s in range(2 * k + 3)]
    run_stream(V, (16, k, 1024, L, partition, 0xC1), slices, tr.aips, kps=(1, 3, k))


@pytest.mark.parametrize("L", [1, 32])
def test_small_workload_exact_shape(V, L):
    # The small workload exactly: 4,096 hosts, 1,000,000 pairs over 20 slices
    # of 50,000, k = 5, a 2^20-AT pool, g = 1,024.  The pool and census at
    # every close, and every host's estimate, active count and per-age counts
    # at k' = 1, 3, 5 at every fourth close and the last, equal the oracle.
    tr = Traffic(SMALL)
    k = 5
    slices = [tr.slice_pairs(s) for s in range(20)]
    assert sum(len(p) for p in slices) == 1_000_000
    run_stream(V, (20, k, 1024, L, 0, 0xC1), slices, tr.aips, kps=(1, 3, k), check_every=4,
               pool_every_slice=True)


@pytest.mark.parametrize("L", [2, 4, 8, 16, 64])
def test_other_segment_lengths(V, L):
    tr = Traffic(SMALL, pkts_per_slice=15_000)
    k = 4
    slices = [tr.slice_pairs(s) for s in range(2 * k + 2)]
    run_stream(V, (15, k, 256, L, 0, 11), slices, tr.aips[:1500], kps=(1, k), check_every=3)


@pytest.mark.parametrize("k,c,g", [(1, 12, 64), (2, 13, 96), (10, 16, 4096), (63, 14, 512)])
def test_window_lengths(V, k, c, g):
    tr = Traffic(SMALL, pkts_per_slice=8_000)
    slices = [tr.slice_pairs(s) for s in range(2 * k + 3 if k < 20 else 20)]
    run_stream(V, (c, k, g, 32 if g % 32 == 0 else 1, 0, k), slices, tr.aips[:800], kps=sorted({1, (k + 1) // 2, k}),
               check_every=2 if k < 20 else 5)


def test_ragged_gaps_and_empty_slices(V):
    # odd batch sizes, an 8-byte aligned (not 16) pointer, empty slices, several
    # ingests per slice, and slice gaps shorter and longer than 2k
    tr = Traffic(SMALL, pkts_per_slice=9_999)
    k = 3
    params = (14, k, 128, 1, 1, 5)
    c, _, g, L, part, seed = params
    d = V.Vate(c, k, g, L, part, seed)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=part, seed=seed)
    ids = [4, 5, 6, 8, 9, 17, 18, 19, 21, 40, 41]
    prev = None
    for j, sid in enumerate(ids):
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        arr = tr.slice_pairs(sid, n=0 if sid in (8, 19) else 9_999 - 2 * j)
        buf = dev_pairs(np.concatenate([np.zeros((1, 2), np.uint32), arr]))   # offset by one pair (8 B)
        half = len(arr) // 3
        d.ingest(buf[1:1 + half], sid)
        d.ingest(buf[1 + half:], sid)
        d.ingest(buf[:0], sid)
        o.ingest(arr)
        d.close_slice(sid)
        compare_close(V, d, o, tr.aips[:700], kps=(1, 2, 3))
    d.close()


def test_constructed_pools_straddling_segments(V):
    # Random AT values everywhere (loaded through the ABI) on a small pool, so
    # that many 32-AT segments straddle a block boundary; census, active counts,
    # estimates and ages must still match the oracle on the same pool.
    rng = np.random.default_rng(3)
    for (c, k, g, L, part) in ((12, 5, 1024, 32, 0), (12, 4, 512, 64, 1), (13, 7, 256, 16, 0), (12, 3, 200, 8, 1)):
        d = V.Vate(c, k, g, L, part, 9)
        o = Oracle(c=c, k=k, g=g, seg_len=L, partition=part, seed=9)
        hosts = rng.integers(0, 2**32, size=600, dtype=np.uint64).astype(np.uint32)
        for t in range(3):
            pool = rng.integers(0, 2 * k + 1, size=1 << c).astype(np.uint8)
            pool[rng.random(1 << c) < 0.3] = 2 * k
            d.ingest(dev_pairs(np.zeros((0, 2), np.uint32)), t)
            if t:
                o.advance()
            d.load_pool(torch.from_numpy(pool).cuda())
            o.load_pool(pool)
            d.close_slice(t)
            compare_close(V, d, o, hosts, kps=range(1, k + 1))
        d.close()


def test_saturation_and_pool_full_flags(V):
    # every pool AT set in the current slice (value = ACT of its block): every
    # VAT of every host is active (SAT) and no pool AT is inactive (POOLFULL)
    c, k, g = 12, 2, 64
    d = V.Vate(c, k, g, 1, 0, 1)
    o = Oracle(c=c, k=k, g=g, seed=1)
    pool = np.array([o.act_of(p) for p in range(1 << c)], np.uint8)
    d.ingest(dev_pairs(np.zeros((0, 2), np.uint32)), 0)
    d.load_pool(torch.from_numpy(pool).cuda())
    o.load_pool(pool)
    d.close_slice(0)
    hosts = np.arange(1, 50, dtype=np.uint32)
    compare_close(V, d, o, hosts, kps=(1, 2), check_ages=False)
    est = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
    fl = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
    d.estimate(dev_u32(hosts), 2, est, fl)
    assert np.all(fl.cpu().numpy() == V.VATE_FLAG_SAT | V.VATE_FLAG_POOLFULL)
    assert np.all(np.isfinite(est.cpu().numpy()))
    d.close()


def test_state_machine_errors(V):
    d = V.Vate(14, 3, 64, 1, 0, 1)
    hosts = dev_u32(np.arange(10, dtype=np.uint32))
    out = torch.empty(10, dtype=torch.float32, device="cuda")
    with pytest.raises(V.VateError) as e:
        d.estimate(hosts, 1, out)                 # no slice closed yet
    assert e.value.code == V.VATE_ESLICE
    d.ingest(dev_pairs(np.array([[1, 2]], np.uint32)), 7)
    with pytest.raises(V.VateError) as e:
        d.ingest(dev_pairs(np.array([[1, 2]], np.uint32)), 6)   # past slice
    assert e.value.code == V.VATE_ESLICE
    d.close_slice(7)
    with pytest.raises(V.VateError) as e:
        d.ingest(dev_pairs(np.array([[1, 2]], np.uint32)), 7)   # closed slice
    assert e.value.code == V.VATE_ESLICE
    with pytest.raises(V.VateError) as e:
        d.close_slice(7)
    assert e.value.code == V.VATE_ESLICE
    for bad_kp in (0, 4):
        with pytest.raises(V.VateError) as e:
            d.estimate(hosts, bad_kp, out)
        assert e.value.code == V.VATE_EINVAL
    d.estimate(hosts, 3, out)                      # repeated estimates are fine
    d.estimate(hosts, 1, out)
    info = d.info()
    assert (info.slice, info.closed, info.bact0) == (7, 1, 0)
    d.ingest(dev_pairs(np.array([[1, 2]], np.uint32)), 9)
    info = d.info()
    assert (info.slice, info.closed, info.bact0) == (9, 0, 2)
    d.close()


def test_host_buffer_entry_points_match_device_ones(V):
    tr = Traffic(SMALL, pkts_per_slice=(1 << 20) + 12345)   # more than one staging chunk
    k = 5
    params = (18, k, 1024, 32, 0, 2)
    d1, d2 = V.Vate(*params), V.Vate(*params)
    # more hosts than one chunk of the estimate pipeline (2^18), ragged tail
    hosts = np.resize(tr.aips, (1 << 19) + 777)
    for s in range(3):
        arr = tr.slice_pairs(s)
        d1.ingest(dev_pairs(arr), s)
        pinned = torch.from_numpy(arr.view(np.int32)).pin_memory()
        V.vate_ingest_host(d2.h, pinned, s)
        d1.close_slice(s)
        d2.close_slice(s)
        p1 = torch.empty(d1.P, dtype=torch.uint8, device="cuda")
        p2 = torch.empty(d2.P, dtype=torch.uint8, device="cuda")
        d1.copy_pool(p1)
        d2.copy_pool(p2)
        assert torch.equal(p1, p2)
        e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
        f1 = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
        d1.estimate(dev_u32(hosts), k, e1, f1)
        if s == 1:                      # page-locked outputs: the copies run asynchronously
            e2 = torch.empty(len(hosts), dtype=torch.float32).pin_memory().numpy()
            f2 = torch.empty(len(hosts), dtype=torch.uint8).pin_memory().numpy()
        else:
            e2 = np.empty(len(hosts), np.float32)
            f2 = np.empty(len(hosts), np.uint8)
        V.vate_estimate_host(d2.h, hosts, k, e2, f2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(e1.cpu().numpy(), e2)
        np.testing.assert_array_equal(f1.cpu().numpy(), f2)
    d1.close()
    d2.close()


def test_host_staging_ring_wraps_and_back_to_back_steps(V):
    """vate_ingest_host with more chunks in one call than the ring has buffers
    (a chunk refills the buffer of an earlier chunk of the same call), then
    slices issued back to back with no synchronisation between them (the
    pairs of slice s+1 are copied while slice s is estimated): pools, estimates
    and flags equal those of the device entry points."""
    k, params = 5, (20, 5, 1024, 32, 0, 7)
    big = Traffic(SMALL, pkts_per_slice=7 * (1 << 20) + 1001).slice_pairs(0)   # 8 chunks, ring of 6
    tr = Traffic(SMALL, pkts_per_slice=(1 << 20) + 4321)
    hosts = np.resize(tr.aips, (1 << 18) + 99)
    d1, d2 = V.Vate(*params), V.Vate(*params)
    slices = [(0, big)] + [(s, tr.slice_pairs(s)) for s in (1, 2, 3)]
    pinned = [torch.from_numpy(arr.view(np.int32)).pin_memory() for _, arr in slices]
    outs = [(torch.empty(len(hosts), dtype=torch.float32).pin_memory(),
             torch.empty(len(hosts), dtype=torch.uint8).pin_memory()) for _ in slices]
    for (s, _), p, (e, f) in zip(slices, pinned, outs):       # issued back to back
        V.vate_ingest_host(d2.h, p, s)
        d2.close_slice(s)
        V.vate_estimate_host(d2.h, hosts, k, e.numpy(), f.numpy())
    torch.cuda.synchronize()
    dh = dev_u32(hosts)
    for (s, arr), (e, f) in zip(slices, outs):
        d1.ingest(dev_pairs(arr), s)
        d1.close_slice(s)
        e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
        f1 = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
        d1.estimate(dh, k, e1, f1)
        np.testing.assert_array_equal(e1.cpu().numpy(), e.numpy())
        np.testing.assert_array_equal(f1.cpu().numpy(), f.numpy())
    p1 = torch.empty(d1.P, dtype=torch.uint8, device="cuda")
    p2 = torch.empty(d2.P, dtype=torch.uint8, device="cuda")
    d1.copy_pool(p1)
    d2.copy_pool(p2)
    assert torch.equal(p1, p2)
    d1.close()
    d2.close()


@pytest.mark.slow
@pytest.mark.parametrize("L", [2, 32])
def test_full_size_40g_shape_sampled(V, L):
    # The 40 Gb/s workload at full size -- 2^26-AT pool, g = 4096, L = 2 (the
    # benchmark's placement) and 32, k = 10, 5M pairs per slice -- through the
    # same entry points and launch configuration as the benchmark.  The whole pool and census are compared
    # every slice; estimates, active counts and per-age counts every fifth
    # slice on a seeded sample of hosts plus every super-spreader (the oracle
    # computes them one by one).
    # 42 slices: two full cycles of every block's ACT (2k = 20 slides each).
    tr = Traffic(LINK40G)
    hosts = mixed_hosts(tr, 2048)
    k = 10
    slices = [tr.slice_pairs(s) for s in range(4 * k + 2)]
    run_stream(V, (26, k, 4096, L, 0, 0xC2), slices, hosts, kps=(1, k), check_every=5, check_ages=True,
               pool_every_slice=True)


@pytest.mark.slow
@pytest.mark.parametrize("L", [2, 32])
def test_full_size_every_host_in_one_launch_sampled(V, L):
    # The benchmark's launch configuration: all 2^20 hosts of the 40 Gb/s
    # workload estimated by one vate_estimate call (so the gather runs on its
    # full grid), in host-table order, with flags, after 5M-pair slices into
    # the 2^26-AT pool, at the benchmark's L = 2 and at L = 32.  The oracle computes a seeded sample of the outputs
    # plus every super-spreader one by one; 2k + 3 slices take every block's
    # ACT through a full cycle.
    tr = Traffic(LINK40G)
    k, n = 10, tr.spec.n_aips
    d = V.Vate(26, k, 4096, L, 0, 0xC2, options=V.VATE_OPT_PERSIST_L2)
    o = Oracle(c=26, k=k, g=4096, seg_len=L, partition=0, seed=0xC2)
    dh = dev_u32(tr.aips)
    rng = np.random.default_rng(11)
    idx = np.union1d(rng.choice(n, 4096, replace=False), tr.super_hosts)
    sample = tr.aips[idx]
    est = torch.empty(n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    act = torch.empty(n, dtype=torch.int32, device="cuda")
    for s in range(2 * k + 3):
        if s:
            o.advance()
        p = tr.slice_pairs(s)
        d.ingest(dev_pairs(p), s)
        o.ingest(p)
        d.close_slice(s)
        if s not in (0, k + 1, 2 * k + 2):
            continue
        for kp in (1, k // 2, k):
            d.estimate(dh, kp, est, fl)
            d.active_counts(dh, kp, act)
            oe, oa, of = o.estimate(sample, kp)
            np.testing.assert_array_equal(act.cpu().numpy().view(np.uint32)[idx], oa, err_msg="A, k'=%d" % kp)
            np.testing.assert_array_equal(fl.cpu().numpy()[idx], of, err_msg="flags, k'=%d" % kp)
            de = est.cpu().numpy()[idx].astype(np.float64)
            assert_eq11_close(de, oe, o.g, "k'=%d" % kp)
    d.close()


@pytest.mark.parametrize("L", [1, 32])
def test_distance_recorders_match_oracle_and_timestamps(V, L):
    # VDRE (distance recorders aged every slide, Sec. 1 / Sec. 5) on the same
    # stream as VATE: the recorder pool equals the oracle's DR pool, and the
    # active counts, censuses and estimates equal those of the timestamps.
    tr = Traffic(SMALL, pkts_per_slice=15_000)
    k, c, g = 4, 16, 512
    dr = V.Vate(c, k, g, L, 0, 21, counter=V.VATE_COUNTER_DR)
    at = V.Vate(c, k, g, L, 0, 21)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=21)
    hosts = tr.aips[:1200]
    dh = dev_u32(hosts)
    ids = [0, 1, 2, 3, 5, 6, 9, 10, 11, 20, 21, 22]
    prev = None
    for sid in ids:
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        p = tr.slice_pairs(sid)
        o.ingest(p)
        for d in (dr, at):
            d.ingest(dev_pairs(p), sid)
            d.close_slice(sid)
        pool = torch.empty(o.P, dtype=torch.uint8, device="cuda")
        dr.copy_pool(pool)
        np.testing.assert_array_equal(pool.cpu().numpy(), o.dr())
        h_dr = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
        h_at = torch.empty_like(h_dr)
        dr.census(h_dr)
        at.census(h_at)
        a, b = h_dr.cpu().numpy(), h_at.cpu().numpy()
        np.testing.assert_array_equal(a[:k], b[:k])
        assert a[k:2 * k].sum() == 0 and a[2 * k] == b[k:].sum()
        for kp in (1, 2, k):
            e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            e2 = torch.empty_like(e1)
            a1 = torch.empty(len(hosts), dtype=torch.int32, device="cuda")
            dr.estimate(dh, kp, e1)
            at.estimate(dh, kp, e2)
            dr.active_counts(dh, kp, a1)
            assert torch.equal(e1, e2)
            _, oa, _ = o.estimate(hosts, kp)
            np.testing.assert_array_equal(a1.cpu().numpy().view(np.uint32), oa)
    dr.close()
    at.close()


# ---- 16-bit ATs (64 <= k <= 1023; the paper's k' = 300 of Sec. 5) ----------
WIDE = [
    (17, 100, 1024, 32, 0, 31),     # 64-byte segments
    (19, 300, 1024, 32, 0, 32),     # the paper's k' = 300
    (17, 64, 512, 8, 1, 33),        # 16-byte segments, low-deviation partition
    (17, 80, 512, 16, 0, 34),       # 32-byte segments
    (18, 70, 1024, 64, 0, 35),      # 128-byte segments
    (17, 100, 256, 1, 0, 36),       # one AT per load
]


@pytest.mark.parametrize("params", WIDE, ids=lambda p: "c%d-k%d-L%d-p%d" % (p[0], p[1], p[3], p[4]))
def test_wide_timestamps_parity(V, params):
    c, k, g, L, part, seed = params
    tr = Traffic(SMALL, pkts_per_slice=4000)
    # runs of consecutive slices with gaps, past 2k so that every block is maintained at ACT 0 and k
    ids = sorted(set(list(range(0, 6)) + list(range(k - 3, k + 4)) + list(range(2 * k - 2, 2 * k + 5))
                     + [3 * k + 1, 5 * k + 7, 5 * k + 8]))
    slices = [tr.slice_pairs(i % 64) for i in ids]
    run_stream(V, params, slices, tr.aips[:700], kps=(1, k // 3, k), slice_ids=ids, check_ages=False)


@pytest.mark.parametrize("L", [1, 32])
def test_wide_distance_recorders_match_oracle(V, L):
    tr = Traffic(SMALL, pkts_per_slice=5000)
    k, c, g = 120, 18, 512
    dr = V.Vate(c, k, g, L, 0, 41, counter=V.VATE_COUNTER_DR)
    at = V.Vate(c, k, g, L, 0, 41)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=41)
    hosts = tr.aips[:600]
    dh = dev_u32(hosts)
    ids = [0, 1, 2, 60, 119, 120, 121, 125, 240, 241]
    prev = None
    for sid in ids:
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        p = tr.slice_pairs(sid % 64)
        o.ingest(p)
        for d in (dr, at):
            d.ingest(dev_pairs(p), sid)
            d.close_slice(sid)
        pool = torch.empty(o.P, dtype=torch.int16, device="cuda")
        dr.copy_pool(pool)
        np.testing.assert_array_equal(pool.cpu().numpy().astype(np.uint16), o.dr())
        h_dr = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
        h_at = torch.empty_like(h_dr)
        dr.census(h_dr)
        at.census(h_at)
        a, b = h_dr.cpu().numpy(), h_at.cpu().numpy()
        np.testing.assert_array_equal(a[:k], b[:k])
        assert a[k:2 * k].sum() == 0 and a[2 * k] == b[k:].sum()
        for kp in (1, 7, k):
            e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            e2 = torch.empty_like(e1)
            a1 = torch.empty(len(hosts), dtype=torch.int32, device="cuda")
            dr.estimate(dh, kp, e1)
            at.estimate(dh, kp, e2)
            dr.active_counts(dh, kp, a1)
            assert torch.equal(e1, e2)
            _, oa, _ = o.estimate(hosts, kp)
            np.testing.assert_array_equal(a1.cpu().numpy().view(np.uint32), oa)
    dr.close()
    at.close()


def test_wide_pool_load_and_age_counts_limits(V):
    d = V.Vate(17, 100, 512, 32, 0, 3)
    tr = Traffic(SMALL, pkts_per_slice=3000)
    d.ingest(dev_pairs(tr.slice_pairs(0)), 0)
    d.close_slice(0)
    pool = torch.empty(d.P, dtype=torch.int16, device="cuda")
    d.copy_pool(pool)
    d2 = V.Vate(17, 100, 512, 32, 0, 3)
    d2.ingest(torch.zeros(0, 2, dtype=torch.int32, device="cuda"), 0)
    d2.load_pool(pool)                              # the paper's form round-trips
    back = torch.empty_like(pool)
    d2.copy_pool(back)
    assert torch.equal(back, pool)
    with pytest.raises(V.VateError) as e:
        d.age_counts(dev_u32(tr.aips[:4]), torch.empty(400, dtype=torch.int16, device="cuda"))
    assert e.value.code == V.VATE_EINVAL
    d.close()
    d2.close()


# ---- packed ATs (the paper's layout: floor(32/b) b-bit fields per word) -------
PACKED = [
    ((17, 10, 1024, 32, 0, 71), 5),      # 6 fields per word, the paper's 5 bits for k = 10
    ((16, 5, 512, 1, 1, 72), 4),         # 8 per word, fully random placement, low-deviation partition
    ((19, 300, 512, 32, 0, 73), 10),     # 3 per word, the paper's 10 bits for k' = 300
    ((15, 1, 256, 8, 0, 74), 2),         # 16 per word
    ((17, 70, 512, 16, 0, 75), 8),       # 4 per word, values up to 140
    ((17, 10, 512, 64, 0, 76), 7),       # 4 per word, 3 bits left over
    ((16, 15, 512, 32, 0, 77), 6),       # 5 per word: an odd count, the odd half's top field absent
    ((18, 200, 512, 16, 1, 78), 9),      # 3 per word, 16-bit values in the paper's form
    ((22, 1000, 256, 32, 0, 79), 11),    # 2 per word, k near the 16-bit limit
]


@pytest.mark.parametrize("params,b", PACKED, ids=lambda x: str(x))
def test_packed_timestamps_parity(V, params, b):
    c, k, g, L, part, seed = params
    tr = Traffic(SMALL, pkts_per_slice=5000)
    ids = sorted(set(list(range(0, 5)) + list(range(k, k + 3)) + list(range(2 * k, 2 * k + 4)) + [4 * k + 3]))
    slices = [tr.slice_pairs(i % 64) for i in ids]
    run_stream(V, params, slices, tr.aips[:700], kps=(1, max(1, k // 2), k), slice_ids=ids, at_bits=b,
               check_ages=False)


def test_packed_recorders_and_pool_round_trip(V):
    k, c, g, L = 10, 17, 512, 32
    tr = Traffic(SMALL, pkts_per_slice=5000)
    dr = V.Vate(c, k, g, L, 0, 81, counter=V.VATE_COUNTER_DR, at_bits=5)
    at = V.Vate(c, k, g, L, 0, 81)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=81)
    hosts = tr.aips[:500]
    dh = dev_u32(hosts)
    prev = None
    for sid in (0, 1, 2, 9, 10, 11, 30):
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        p = tr.slice_pairs(sid)
        o.ingest(p)
        for d in (dr, at):
            d.ingest(dev_pairs(p), sid)
            d.close_slice(sid)
        pool = torch.empty(o.P, dtype=torch.uint8, device="cuda")
        dr.copy_pool(pool)
        np.testing.assert_array_equal(pool.cpu().numpy(), o.dr())
        for kp in (1, k):
            e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            e2 = torch.empty_like(e1)
            dr.estimate(dh, kp, e1)
            at.estimate(dh, kp, e2)
            assert torch.equal(e1, e2)
    # the paper's form loads into a packed pool and copies back unchanged
    d = V.Vate(c, k, g, L, 0, 81, at_bits=5)
    d.ingest(torch.zeros(0, 2, dtype=torch.int32, device="cuda"), 0)
    ref = torch.empty(o.P, dtype=torch.uint8, device="cuda")
    at.copy_pool(ref)
    d.load_pool(ref)
    back = torch.empty_like(ref)
    d.copy_pool(back)
    assert torch.equal(back, ref)
    with pytest.raises(V.VateError) as e:
        V.vate_create_shard(V.make_params(c, k, g, L, 0, 81, 0, 5), 0, 1 << 16)
    assert e.value.code == V.VATE_EINVAL
    for h in (dr, at, d):
        h.close()


@pytest.mark.slow
@pytest.mark.parametrize("L", [1, 32])
def test_maximum_pool_2p32_on_sparse_input(V, L):
    # 2^32 ATs (4 GiB), the largest pool: too large for the oracle's own pool,
    # but on sparse input the exact answer follows from the mapping alone.
    # By Corollary 1 an AT is active for window k' iff its position was last
    # set less than k' slices ago, so the census holds exactly those positions
    # at distances below k', and a host's A counts its VATs among them.
    c, k, g, seed = 32, 4, 512, 0x32
    rng = np.random.default_rng(L)
    hosts = rng.integers(0, 2**32, 40, dtype=np.uint64).astype(np.uint32)
    d = V.Vate(c, k, g, L, 0, seed)
    last = {}                                   # position -> slice of its last SetAT
    vats = {int(a): [oracle.h_of(c, L, seed, int(a), i) for i in range(g)] for a in hosts}
    dh = dev_u32(hosts)
    for s in (0, 1, 2, 5, 6, 7, 13):
        a = hosts[rng.integers(0, len(hosts), 300)]
        b = rng.integers(0, 2**32, 300, dtype=np.uint64).astype(np.uint32)
        pairs = np.stack([a, b], 1)
        d.ingest(dev_pairs(pairs), s)
        d.close_slice(s)
        for x, y in pairs:
            last[oracle.h_of(c, L, seed, int(x), oracle.bh_of(g, seed, int(y)))] = s
        hist = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
        d.census(hist)
        hist = hist.cpu().numpy()
        for kp in (1, 2, k):
            live = {p for p, t in last.items() if s - t < kp}
            assert int(hist[:kp].sum()) == len(live)
            want = np.array([sum(p in live for p in vats[int(h)]) for h in hosts], np.uint32)
            act = torch.empty(len(hosts), dtype=torch.int32, device="cuda")
            d.active_counts(dh, kp, act)
            np.testing.assert_array_equal(act.cpu().numpy().view(np.uint32), want)
            est = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            d.estimate(dh, kp, est)
            n0 = (1 << c) - len(live)
            oe = np.array([oracle.estimate_from_counts(g, 1 << c, n0, int(x))[0] for x in want])
            assert_eq11_close(est.cpu().numpy(), oe, g, "k'=%d" % kp)
    d.close()


def test_empty_host_lists_are_no_ops(V):
    # n = 0 hosts on every per-host entry point: no error, nothing written
    d = V.Vate(16, 4, 512, 32, 0, 5)
    p = Traffic(SMALL, pkts_per_slice=2000).slice_pairs(0)
    d.ingest(dev_pairs(p), 0)
    d.close_slice(0)
    none = torch.zeros(0, dtype=torch.int32, device="cuda")
    sentinel = torch.full((4,), -7.0, device="cuda")
    d.estimate(none, 4, sentinel[:0])
    d.active_counts(none, 4, torch.zeros(0, dtype=torch.int32, device="cuda"))
    d.age_counts(none, torch.zeros(0, dtype=torch.int16, device="cuda"))
    V.vate_estimate_host(d.h, np.zeros(0, np.uint32), 4, np.zeros(0, np.float32))
    V.vate_features(d.h, none, torch.zeros(0, dtype=torch.float32, device="cuda"))
    model = torch.empty(V.vate_mlp_param_count(10), dtype=torch.float32, device="cuda")
    V.vate_mlp_init(model, 10, 1)
    V.vate_estimate_learned(d.h, none, model, sentinel[:0])
    hist = torch.empty(9, dtype=torch.int64, device="cuda")
    d.census(hist)
    V.vate_estimate_from_counts(d.params, none, hist, 4, sentinel[:0])
    torch.cuda.synchronize()
    assert torch.all(sentinel == -7.0)
    d.close()
