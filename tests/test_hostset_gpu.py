"""The close of a fixed host list through its index (include/vate_hostset.h):
vate_estimate_hostset must equal vate_estimate (and its counts
vate_active_counts) bit for bit -- the per-host gather is itself checked
against the oracle in test_parity_gpu.py -- and the oracle directly on a
small case.

  - every segment length the index serves (L = 1, 2, 4, 8), both partitions,
    timestamps and distance recorders, several k';
  - pools of one region (2^16 ATs, a partial region), of several (2^22:
    three regions, the last partial) and of many (2^30: 683 regions, most
    of them empty for a single host);
  - host lists with repeats, hosts never seen, and a ragged count;
  - the benchmark's configuration at full size: the 2^26-AT pool, all 2^20
    hosts of the 40 Gb/s traffic, L = 1 and L = 2;
  - the calls it must refuse.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from traffic import LINK40G, SMALL, Traffic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def as_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def host_list(tr, rng, extra=37):
    absent = rng.integers(1, 1 << 32, extra, dtype=np.uint64).astype(np.uint32)
    absent = absent[~np.isin(absent, tr.aips)]
    rep = rng.choice(tr.aips, 50)
    return np.concatenate([tr.aips, absent, rep])


def compare(V, d, s, hosts, kp):
    n = len(hosts)
    dh = as_i32(hosts)
    e1 = torch.empty(n, dtype=torch.float32, device="cuda")
    f1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    a1 = torch.empty(n, dtype=torch.int32, device="cuda")
    e2, f2, a2 = torch.empty_like(e1), torch.empty_like(f1), torch.empty_like(a1)
    d.estimate(dh, kp, e1, f1)
    V.vate_active_counts(d.h, dh, kp, a1)
    V.vate_estimate_hostset(d.h, s, kp, e2, f2, a2)
    torch.cuda.synchronize()
    assert torch.equal(a1, a2), "A, k'=%d" % kp
    assert torch.equal(f1, f2), "flags, k'=%d" % kp
    assert torch.equal(e1.view(torch.int32), e2.view(torch.int32)), "estimates, k'=%d" % kp
    return a2


@pytest.mark.parametrize("L", [1, 2, 4, 8])
@pytest.mark.parametrize("c", [16, 22])
@pytest.mark.parametrize("part", [0, 1])
def test_hostset_equals_per_host_gather(V, L, c, part):
    k, g = 5, 512
    tr = Traffic(SMALL, pkts_per_slice=30_000)
    rng = np.random.default_rng(c * 10 + L)
    hosts = host_list(tr, rng)
    d = V.Vate(c, k, g, L, part, 31 + L)
    s = V.vate_hostset_create(d.h, as_i32(hosts))
    nbytes, nh, nr = V.vate_hostset_info(s)
    assert nh == len(hosts) and nr == (1 if c == 16 else 3)
    assert nbytes >= 16 * len(hosts) * (g // L) // 6          # six 21-bit entries per 16 bytes
    for sl in range(9):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        if sl in (0, 4, 8):
            for kp in (1, 3, k):
                compare(V, d, s, hosts, kp)
    V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.parametrize("L", [1, 2])
def test_hostset_with_distance_recorders(V, L):
    k, c, g = 4, 20, 256
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    hosts = tr.aips
    d = V.Vate(c, k, g, L, 0, 41, counter=V.VATE_COUNTER_DR)
    s = V.vate_hostset_create(d.h, as_i32(hosts))
    for sl in (0, 1, 2, 5, 6):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        for kp in (1, k):
            compare(V, d, s, hosts, kp)
    V.vate_hostset_destroy(s)
    d.close()


def test_hostset_against_the_oracle(V):
    c, k, g, L = 18, 5, 512, 1
    tr = Traffic(SMALL, pkts_per_slice=25_000)
    d = V.Vate(c, k, g, L, 0, 9)
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=9)
    hosts = tr.aips[:1500]
    s = V.vate_hostset_create(d.h, as_i32(hosts))
    n = len(hosts)
    e = torch.empty(n, dtype=torch.float32, device="cuda")
    f = torch.empty(n, dtype=torch.uint8, device="cuda")
    a = torch.empty(n, dtype=torch.int32, device="cuda")
    for sl in range(7):
        p = tr.slice_pairs(sl)
        if sl:
            o.advance()
        o.ingest(p)
        d.ingest(as_i32(p), sl)
        d.close_slice(sl)
        for kp in (2, k):
            V.vate_estimate_hostset(d.h, s, kp, e, f, a)
            oe, oa, of = o.estimate(hosts, kp)
            np.testing.assert_array_equal(a.cpu().numpy().view(np.uint32), oa)
            np.testing.assert_array_equal(f.cpu().numpy(), of)
            de = e.cpu().numpy().astype(np.float64)
            assert np.all(np.abs(de - oe) <= 1e-5 * np.maximum(np.abs(oe), 1.0))
    V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.slow
@pytest.mark.parametrize("L", [1, 2])
def test_hostset_full_size_40g(V, L):
    # the benchmark's configuration: 2^26-AT pool, g = 4096, k = 10, all 2^20
    # hosts of the 40 Gb/s traffic, 5M pairs per slice; every host compared
    # with the per-host gather at three closes and two k'
    tr = Traffic(LINK40G)
    k = 10
    d = V.Vate(26, k, 4096, L, 0, 0xC2, options=V.VATE_OPT_PERSIST_L2)
    s = V.vate_hostset_create(d.h, as_i32(tr.aips))
    assert V.vate_hostset_info(s)[2] == 43
    for sl in range(2 * k + 3):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        if sl in (3, k + 1, 2 * k + 2):
            for kp in (1, k):
                a = compare(V, d, s, tr.aips, kp)
                assert int(a.sum()) > 0
    V.vate_hostset_destroy(s)
    d.close()


def test_hostset_refusals(V):
    tr = Traffic(SMALL, pkts_per_slice=5_000)
    hosts = as_i32(tr.aips[:100])
    d = V.Vate(16, 4, 256, 2, 0, 1)
    other = V.Vate(16, 4, 256, 2, 0, 1)
    wide = V.Vate(16, 4, 256, 16, 0, 1)
    for h, aips in ((wide.h, hosts), (d.h, hosts[:0])):
        with pytest.raises(V.VateError) as e:
            V.vate_hostset_create(h, aips)
        assert e.value.code == V.VATE_EINVAL
    s = V.vate_hostset_create(d.h, hosts)
    out = torch.empty(100, dtype=torch.float32, device="cuda")
    d.ingest(as_i32(tr.slice_pairs(0)), 0)
    with pytest.raises(V.VateError) as e:                     # slice not closed
        V.vate_estimate_hostset(d.h, s, 4, out)
    assert e.value.code == V.VATE_ESLICE
    d.close_slice(0)
    other.ingest(as_i32(tr.slice_pairs(0)), 0)
    other.close_slice(0)
    for h, kp in ((other.h, 4), (d.h, 0), (d.h, 5)):         # another handle; k' outside [1, k]
        with pytest.raises(V.VateError) as e:
            V.vate_estimate_hostset(h, s, kp, out)
        assert e.value.code == V.VATE_EINVAL
    V.vate_estimate_hostset(d.h, s, 4, out)
    V.vate_hostset_destroy(s)
    for x in (d, other, wide):
        x.close()


@pytest.mark.parametrize("L", [1, 8])
def test_hostset_many_regions_and_tiny_lists(V, L):
    # a 2^30-AT pool (683 regions, most of them empty for a short vector), a
    # single host and a list of 300: cells of one or two segments, empty
    # regions between them, against the per-host gather
    c, k, g = 30, 4, 64
    tr = Traffic(SMALL, pkts_per_slice=8_000)
    d = V.Vate(c, k, g, L, 0, 77)
    lists = [tr.aips[:1], tr.aips[:300]]
    sets = [V.vate_hostset_create(d.h, as_i32(h)) for h in lists]
    assert V.vate_hostset_info(sets[0])[2] == 683
    for sl in range(4):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        for h, s in zip(lists, sets):
            compare(V, d, s, h, k)
    for s in sets:
        V.vate_hostset_destroy(s)
    d.close()


@pytest.mark.parametrize("ages", [False, True])
def test_async_host_copies_equal_the_device_results(V, ages):
    # vate_estimate_hostset_host_async: calls back to back, the results of two
    # calls in flight in two host buffers, read after vate_hostset_wait; each
    # equal to vate_estimate_hostset on the device bit for bit
    k, c, g, L = 5, 20, 512, 1
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    hosts = tr.aips
    n = len(hosts)
    d = V.Vate(c, k, g, L, 0, 61)
    s = (V.vate_hostset_create_ages if ages else V.vate_hostset_create)(d.h, as_i32(hosts))
    outs = [(torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.uint8).pin_memory())
            for _ in range(2)]
    refs = []
    for sl in range(7):
        d.ingest(as_i32(tr.slice_pairs(sl)), sl)
        d.close_slice(sl)
        o, f = outs[sl & 1]
        V.vate_estimate_hostset_host_async(d.h, s, k, o, f)
        e = torch.empty(n, dtype=torch.float32, device="cuda")
        fl = torch.empty(n, dtype=torch.uint8, device="cuda")
        V.vate_estimate_hostset(d.h, s, k, e, fl)
        refs.append((e.cpu(), fl.cpu()))
        if sl >= 1:                                  # the call before this one: its copies are done after the wait
            V.vate_hostset_wait(s)
            po, pf = outs[(sl - 1) & 1]
            ro, rf = refs[sl - 1]
            assert torch.equal(po.view(torch.int32), ro.view(torch.int32)) and torch.equal(pf, rf), sl - 1
    V.vate_hostset_wait(s)
    po, pf = outs[6 & 1]
    assert torch.equal(po.view(torch.int32), refs[6][0].view(torch.int32)) and torch.equal(pf, refs[6][1])
    V.vate_hostset_destroy(s)
    d.close()


def test_pass_timings(V):
    # vate_hostset_time_passes: the next n closes record their index pass with
    # CUDA events; later calls are not recorded; a restart starts over
    tr = Traffic(SMALL, pkts_per_slice=10_000)
    d = V.Vate(20, 4, 512, 1, 0, 3)
    for ages in (False, True):
        s = (V.vate_hostset_create_ages if ages else V.vate_hostset_create)(d.h, as_i32(tr.aips))
        out = torch.empty(len(tr.aips), dtype=torch.float32, device="cuda")
        if not ages:
            d.ingest(as_i32(tr.slice_pairs(0)), 0)
            d.close_slice(0)
        assert V.vate_hostset_pass_times(s) == []
        V.vate_hostset_time_passes(s, 3)
        for _ in range(5):
            V.vate_estimate_hostset(d.h, s, 4, out)
        ms = V.vate_hostset_pass_times(s)
        assert len(ms) == 3 and all(0.0 < t < 1000.0 for t in ms)
        V.vate_hostset_time_passes(s, 1)
        V.vate_estimate_hostset(d.h, s, 4, out)
        assert len(V.vate_hostset_pass_times(s)) == 1
        V.vate_hostset_time_passes(s, 0)
        V.vate_estimate_hostset(d.h, s, 4, out)
        assert V.vate_hostset_pass_times(s) == []
        if ages:                                   # the age index's other entry points run the same pass
            V.vate_hostset_time_passes(s, 2)
            V.vate_age_counts_hostset(d.h, s, torch.empty(len(tr.aips) * 4, dtype=torch.int16, device="cuda"))
            V.vate_estimate_hostset(d.h, s, 4, out)
            assert len(V.vate_hostset_pass_times(s)) == 2
        with pytest.raises(V.VateError):
            V.vate_hostset_time_passes(s, 5000)
        V.vate_hostset_destroy(s)
    d.close()
