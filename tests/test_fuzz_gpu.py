"""Randomised configurations against the oracle.

Each case draws a valid configuration -- pool size, window k (byte ATs up to
63, 16-bit ATs up to 300), vector length g, segment length L, partition,
layout (bytes, 16-bit or b-bit packed fields) -- and a slice sequence with
gaps (some longer than 2k, so that whole windows expire), then compares the
pool, the census, the active counts, the flags and Eq. 11 with the oracle
after every close, as the fixed parity cases do.  Distance recorders (VDRE)
are drawn the same way: their pool equals the oracle's recorder pool, and
their census, active counts, estimates and per-age counts those of the
timestamps.  Monitor
groups of random size and make-up (one segment length per group), stepped
plainly or by graph replay, equal a single handle per monitor bit for bit.
Position shards at random 64-aligned cut points hold the undivided pool
between them and reduce to its census and estimates.  A handle checkpointed
after a random slice and restored continues exactly as the original.  The
close of a random host list through its index equals the per-host gather.
The draws are seeded, so a failing case is reproduced by its id.
"""
import math

import numpy as np
import pytest
import torch

from oracle import Oracle
from test_group_gpu import run_group_vs_single
from test_parity_gpu import dev_pairs, dev_u32, run_stream
from traffic import SMALL, Traffic

pytestmark = pytest.mark.gpu

N_CASES = 64


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def draw(case):
    rng = np.random.default_rng(1000 + case)
    k = int(rng.integers(1, 64)) if rng.random() < 0.7 else int(rng.integers(64, 301))
    cmin = max(12, math.ceil(math.log2((2 * k - 1) * 2 * k)))   # every block of Eq. 9-10 non-empty
    c = int(rng.integers(cmin, max(cmin, 18) + 1))
    L = int(rng.choice([1, 2, 4, 8, 16, 32, 64]))
    g = int(min(L * rng.integers(2, 65), 4096))
    part = int(rng.integers(0, 2))
    bmin = math.ceil(math.log2(2 * k + 1))
    at_bits = int(rng.integers(bmin, 17)) if rng.random() < 0.3 else 0
    ids, s = [], 0
    for _ in range(int(rng.integers(4, 8))):
        ids.append(s)
        s += int(rng.choice([1, 1, 2, 3, k, 2 * k + 1]))
    kps = sorted({1, int(rng.integers(1, k + 1)), k})
    return (c, k, g, L, part, 500 + case), at_bits, ids, kps, int(rng.integers(2_000, 12_000))


@pytest.mark.parametrize("case", range(N_CASES))
def test_random_configuration_matches_oracle(V, case):
    params, at_bits, ids, kps, pkts = draw(case)
    c, k, g, L, part, seed = params
    tr = Traffic(SMALL, pkts_per_slice=pkts)
    slices = [tr.slice_pairs(i % 64) for i in ids]
    hosts = np.concatenate([tr.aips[:300], np.random.default_rng(case).integers(0, 2**32, 50, dtype=np.uint64)
                            .astype(np.uint32)])
    run_stream(V, params, slices, hosts, kps=kps, slice_ids=ids, at_bits=at_bits,
               check_ages=(at_bits == 0 and k <= 63))


@pytest.mark.parametrize("case", range(N_CASES // 2))
def test_random_recorder_configuration_matches_oracle(V, case):
    params, at_bits, ids, kps, pkts = draw(10_000 + case)
    c, k, g, L, part, seed = params
    tr = Traffic(SMALL, pkts_per_slice=pkts)
    hosts = tr.aips[:300]
    dh = dev_u32(hosts)
    dr = V.Vate(c, k, g, L, part, seed, counter=V.VATE_COUNTER_DR, at_bits=at_bits)
    at = V.Vate(c, k, g, L, part, seed, at_bits=at_bits)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=part, seed=seed)
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
        pool = torch.empty(o.P, dtype=V.pool_dtype(k), device="cuda")
        dr.copy_pool(pool)
        np.testing.assert_array_equal(pool.cpu().numpy().astype(np.int64), o.dr().astype(np.int64))
        h_dr = torch.empty(2 * k + 1, dtype=torch.int64, device="cuda")
        h_at = torch.empty_like(h_dr)
        dr.census(h_dr)
        at.census(h_at)
        a, b = h_dr.cpu().numpy(), h_at.cpu().numpy()
        np.testing.assert_array_equal(a[:k], b[:k])
        assert a[k:2 * k].sum() == 0 and a[2 * k] == b[k:].sum()
        for kp in kps:
            e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            e2 = torch.empty_like(e1)
            a1 = torch.empty(len(hosts), dtype=torch.int32, device="cuda")
            dr.estimate(dh, kp, e1)
            at.estimate(dh, kp, e2)
            dr.active_counts(dh, kp, a1)
            assert torch.equal(e1, e2)
            _, oa, _ = o.estimate(hosts, kp)
            np.testing.assert_array_equal(a1.cpu().numpy().view(np.uint32), oa)
        if at_bits == 0 and k <= 63:               # per-age counts: a recorder's value is its age
            g1 = torch.empty(len(hosts) * k, dtype=torch.int16, device="cuda")
            g2 = torch.empty_like(g1)
            dr.age_counts(dh, g1)
            at.age_counts(dh, g2)
            assert torch.equal(g1, g2)
            np.testing.assert_array_equal(g1.cpu().numpy().view(np.uint16).reshape(len(hosts), k).astype(np.uint32),
                                          o.age_counts(hosts))
    dr.close()
    at.close()


@pytest.mark.parametrize("case", range(12))
def test_random_monitor_group_equals_single_handles(V, case):
    rng = np.random.default_rng(20_000 + case)
    L = int(rng.choice([1, 2, 8, 16, 32, 64]))
    monitors = []
    for m in range(int(rng.integers(1, 25))):
        k = int(rng.integers(1, 61))
        cmin = max(12, math.ceil(math.log2((2 * k - 1) * 2 * k)))
        c = int(rng.integers(cmin, max(cmin, 17) + 1))
        g = int(min(L * rng.integers(2, 65), 4096))
        monitors.append((c, k, g, L, int(rng.integers(0, 2)), 30_000 + 100 * case + m))
    run_group_vs_single(V, monitors, nslices=int(rng.integers(4, 10)), graph=bool(rng.integers(0, 2)))


@pytest.mark.parametrize("case", range(12))
def test_random_shards_equal_one_handle(V, case):
    rng = np.random.default_rng(40_000 + case)
    params, _, ids, kps, pkts = draw(50_000 + case)
    c, k, g, L, part, seed = params
    counter = int(rng.integers(0, 2))
    P = 1 << c
    cuts = sorted(set(int(x) * 64 for x in rng.integers(1, P // 64, int(rng.integers(1, 5)))))
    bounds = [0] + cuts + [P]
    ranges = list(zip(bounds[:-1], bounds[1:]))
    vp = V.make_params(c, k, g, L, part, seed, counter)
    full = V.Vate(c, k, g, L, part, seed, counter=counter)
    shards = [V.vate_create_shard(vp, lo, hi) for lo, hi in ranges]
    tr = Traffic(SMALL, pkts_per_slice=pkts)
    hosts = tr.aips[:300]
    dh = dev_u32(hosts)
    dt = V.pool_dtype(k)
    for sid in ids:
        dp = dev_pairs(tr.slice_pairs(sid % 64))
        full.ingest(dp, sid)
        full.close_slice(sid)
        for h in shards:
            V.vate_ingest(h, dp, sid)
            V.vate_close_slice(h, sid)
        whole = torch.empty(P, dtype=dt, device="cuda")
        full.copy_pool(whole)
        parts = []
        for h, (lo, hi) in zip(shards, ranges):
            t = torch.empty(hi - lo, dtype=dt, device="cuda")
            V.vate_copy_pool(h, t)
            parts.append(t)
        assert torch.equal(torch.cat(parts), whole)
        hist = torch.zeros(2 * k + 1, dtype=torch.int64, device="cuda")
        for h in shards:
            t = torch.empty_like(hist)
            V.vate_census(h, t)
            hist += t
        want = torch.empty_like(hist)
        full.census(want)
        assert torch.equal(hist, want)
        for kp in kps:
            act = torch.zeros(len(hosts), dtype=torch.int32, device="cuda")
            for h in shards:
                t = torch.empty_like(act)
                V.vate_active_counts(h, dh, kp, t)
                act += t
            e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            f1 = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
            V.vate_estimate_from_counts(vp, act, hist, kp, e1, f1)
            e2 = torch.empty_like(e1)
            f2 = torch.empty_like(f1)
            full.estimate(dh, kp, e2, f2)
            assert torch.equal(e1, e2) and torch.equal(f1, f2)
    for h in shards:
        V.vate_destroy(h)
    full.close()


@pytest.mark.parametrize("case", range(12))
def test_random_checkpoint_resume_continues_exactly(V, case):
    rng = np.random.default_rng(60_000 + case)
    params, at_bits, ids, kps, pkts = draw(70_000 + case)
    c, k, g, L, part, seed = params
    counter = int(rng.integers(0, 2))
    cut = int(rng.integers(1, len(ids)))             # checkpoint after the close of slice ids[cut - 1]
    tr = Traffic(SMALL, pkts_per_slice=pkts)
    hosts = tr.aips[:300]
    dh = dev_u32(hosts)
    a = V.Vate(c, k, g, L, part, seed, counter=counter, at_bits=at_bits)
    b = None
    for j, sid in enumerate(ids):
        if j == cut:
            b = V.Vate.restore(a.checkpoint())
        p = dev_pairs(tr.slice_pairs(sid % 64))
        for d in (a, b):
            if d is None:
                continue
            d.ingest(p, sid)
            d.close_slice(sid)
        if b is None:
            continue
        pa = torch.empty(1 << c, dtype=V.pool_dtype(k), device="cuda")
        pb = torch.empty_like(pa)
        a.copy_pool(pa)
        b.copy_pool(pb)
        assert torch.equal(pa, pb)
        for kp in kps:
            e1 = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            e2 = torch.empty_like(e1)
            a.estimate(dh, kp, e1)
            b.estimate(dh, kp, e2)
            assert torch.equal(e1, e2)
    a.close()
    b.close()


@pytest.mark.parametrize("case", range(16))
def test_random_hostset_equals_per_host_gather(V, case):
    # the close of a fixed host list through its index (include/vate_hostset.h)
    # equals the per-host gather bit for bit, for random byte-AT configurations
    # with L <= 8 (pools of up to three regions), timestamps or recorders, a
    # random host list (repeats, hosts never seen) and the drawn slice sequence
    rng = np.random.default_rng(70_000 + case)
    params, _, ids, kps, pkts = draw(80_000 + case)
    c, k, g, L, part, seed = params
    k = min(k, 63)
    L = int(rng.choice([1, 2, 4, 8]))
    g = int(min(L * rng.integers(2, 129), 4096))
    c = max(c, int(rng.choice([c, 22])))
    kps = sorted({1, int(rng.integers(1, k + 1)), k})
    counter = int(rng.integers(0, 2))
    d = V.Vate(c, k, g, L, part, seed, counter=counter)
    tr = Traffic(SMALL, pkts_per_slice=pkts)
    n = int(rng.integers(1, 3000))
    hosts = rng.choice(tr.aips, n)
    hosts[: n // 10] = rng.integers(1, 1 << 32, n // 10, dtype=np.uint64).astype(np.uint32)
    dh = dev_u32(hosts)
    s = V.vate_hostset_create(d.h, dh)
    e1 = torch.empty(n, dtype=torch.float32, device="cuda")
    f1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    a1 = torch.empty(n, dtype=torch.int32, device="cuda")
    e2, f2, a2 = torch.empty_like(e1), torch.empty_like(f1), torch.empty_like(a1)
    for sid in ids:
        d.ingest(dev_pairs(tr.slice_pairs(sid % 64)), sid)
        d.close_slice(sid)
        for kp in kps:
            d.estimate(dh, kp, e1, f1)
            V.vate_active_counts(d.h, dh, kp, a1)
            V.vate_estimate_hostset(d.h, s, kp, e2, f2, a2)
            assert torch.equal(a1, a2), (case, sid, kp)
            assert torch.equal(f1, f2), (case, sid, kp)
            assert torch.equal(e1.view(torch.int32), e2.view(torch.int32)), (case, sid, kp)
    V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.parametrize("case", range(12))
def test_random_age_index_equals_per_host_gathers(V, case):
    # the age index (vate_hostset_create_ages): per-age counts and A for several
    # k' equal the per-host gathers bit for bit, for random configurations with
    # k <= 15, L <= 8 (pools of up to eleven 384 K-AT regions), timestamps or
    # recorders, a random host list (repeats, hosts never seen) and the drawn
    # slice sequence
    rng = np.random.default_rng(90_000 + case)
    params, _, ids, kps, pkts = draw(95_000 + case)
    c, k, g, L, part, seed = params
    k = int(rng.integers(1, 16))
    L = int(rng.choice([1, 2, 4, 8]))
    g = int(min(L * rng.integers(2, 129), 4096))
    c = max(c, int(rng.choice([c, 22])))
    kps = sorted({1, int(rng.integers(1, k + 1)), k})
    counter = int(rng.integers(0, 2))
    d = V.Vate(c, k, g, L, part, seed, counter=counter)
    tr = Traffic(SMALL, pkts_per_slice=pkts)
    n = int(rng.integers(1, 3000))
    hosts = rng.choice(tr.aips, n)
    hosts[: n // 10] = rng.integers(1, 1 << 32, n // 10, dtype=np.uint64).astype(np.uint32)
    dh = dev_u32(hosts)
    s = V.vate_hostset_create_ages(d.h, dh)
    c1 = torch.empty(n * k, dtype=torch.int16, device="cuda")
    c2 = torch.empty_like(c1)
    e1 = torch.empty(n, dtype=torch.float32, device="cuda")
    f1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    a1 = torch.empty(n, dtype=torch.int32, device="cuda")
    e2, f2, a2 = torch.empty_like(e1), torch.empty_like(f1), torch.empty_like(a1)
    for sid in ids:
        d.ingest(dev_pairs(tr.slice_pairs(sid % 64)), sid)
        d.close_slice(sid)
        V.vate_age_counts(d.h, dh, c1)
        V.vate_age_counts_hostset(d.h, s, c2)
        assert torch.equal(c1, c2), (case, sid)
        for kp in kps:
            d.estimate(dh, kp, e1, f1)
            V.vate_active_counts(d.h, dh, kp, a1)
            V.vate_estimate_hostset(d.h, s, kp, e2, f2, a2)
            assert torch.equal(a1, a2), (case, sid, kp)
            assert torch.equal(f1, f2), (case, sid, kp)
            assert torch.equal(e1.view(torch.int32), e2.view(torch.int32)), (case, sid, kp)
    V.vate_hostset_destroy(s)
    d.close()
