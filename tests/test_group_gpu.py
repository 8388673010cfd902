"""Monitor groups (include/vate_group.h): many independent VATE monitors
advanced together in one persistent launch per slice.

Every monitor of a group must compute exactly what a single vate_handle with
the same parameters computes on the same pairs and hosts: the pool byte for
byte, the census, and the estimates and flags bit for bit (same device
arithmetic).  One monitor is also checked against the CPU oracle.  The CUDA
graph form must equal the plain form and hold one node, the autotuner must
leave state and outputs unchanged, malformed device-side offsets and k' must
be clamped and reported, never read out of bounds, and a device-side wait
that cannot be satisfied must give up within its limit and report
VATE_GROUP_TIMEOUT (the kernel returns; nothing hangs).  The 64-monitor
configuration is run at full size as the benchmark drives it.
"""
import numpy as np
import pytest
import torch

from oracle import Oracle
from traffic import SMALL, Traffic

pytestmark = pytest.mark.gpu
from eq11_tol import RTOL, assert_eq11_close  # noqa: E402


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def as_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


MONITORS_L32 = [(14, 1, 64, 32, 0, 1), (16, 5, 1024, 32, 0, 2), (15, 3, 96, 32, 1, 3), (17, 10, 512, 32, 0, 4),
                (16, 30, 256, 32, 1, 5), (14, 2, 1024, 32, 0, 6), (18, 10, 4096, 32, 0, 7)]


def make_slice(trs, s, rng, empty_every=3):
    """Per-monitor pairs and hosts of slice s (some monitors idle in some slices)."""
    pairs, hosts = [], []
    for m, tr in enumerate(trs):
        n = 0 if (s + m) % empty_every == 0 else int(rng.integers(200, 6000))
        pairs.append(tr.slice_pairs(s, n=n))
        nh = 0 if (s * 7 + m) % 5 == 0 else int(rng.integers(1, 700))
        hosts.append(tr.aips[:nh])
    return pairs, hosts


def pack(pairs, hosts, kprime):
    po = np.zeros(len(pairs) + 1, np.int64)
    po[1:] = np.cumsum([len(p) for p in pairs])
    ho = np.zeros(len(hosts) + 1, np.int64)
    ho[1:] = np.cumsum([len(h) for h in hosts])
    P = np.concatenate(pairs) if po[-1] else np.zeros((0, 2), np.uint32)
    H = np.concatenate(hosts) if ho[-1] else np.zeros(0, np.uint32)
    return (as_i32(P), torch.from_numpy(po).cuda(), as_i32(H), torch.from_numpy(ho).cuda(),
            torch.tensor(np.asarray(kprime, np.int32)).cuda())


def run_group_vs_single(V, monitors, nslices, graph=False, autotune_at=None, wave_mib=None):
    rng = np.random.default_rng(len(monitors) * 31 + nslices)
    trs = [Traffic(SMALL, pkts_per_slice=5000) for _ in monitors]
    params = [V.make_params(*m) for m in monitors]
    grp = V.VateGroup(params)
    if wave_mib is not None:
        t = V.vate_group_get_tuning(grp.g)
        t.wave_pool_mib = wave_mib
        V.vate_group_set_tuning(grp.g, t)
    singles = [V.Vate(*m) for m in monitors]
    kprime = [max(1, (m[1] + 1) // 2) if i % 2 else m[1] for i, m in enumerate(monitors)]
    cap_p, cap_h = 6000 * len(monitors), 700 * len(monitors)
    bufs = None
    for s in range(nslices):
        pairs, hosts = make_slice(trs, s, rng)
        P, PO, H, HO, KP = pack(pairs, hosts, kprime)
        if graph:
            if bufs is None:
                bufs = (torch.zeros(cap_p, 2, dtype=torch.int32, device="cuda"), torch.zeros_like(PO),
                        torch.zeros(cap_h, dtype=torch.int32, device="cuda"), torch.zeros_like(HO), KP.clone(),
                        torch.zeros(cap_h, dtype=torch.float32, device="cuda"),
                        torch.zeros(cap_h, dtype=torch.uint8, device="cuda"))
            bp, bpo, bh, bho, bkp, out, fl = bufs
            bp[:len(P)].copy_(P)
            bpo.copy_(PO)
            bh[:len(H)].copy_(H)
            bho.copy_(HO)
            grp.step(bp, bpo, bh, bho, bkp, out, fl, graph=True)
        else:
            out = torch.zeros(max(1, len(H)), dtype=torch.float32, device="cuda")
            fl = torch.zeros(max(1, len(H)), dtype=torch.uint8, device="cuda")
            grp.step(P, PO, H, HO, KP, out, fl)
            if autotune_at is not None and s == autotune_at:
                out0, fl0 = out.clone(), fl.clone()
                pools0 = []
                for m, mon in enumerate(monitors):
                    t = torch.empty(1 << mon[0], dtype=torch.uint8, device="cuda")
                    grp.copy_pool(m, t)
                    pools0.append(t)
                tun = grp.autotune(P, PO, H, HO, KP, out, fl)
                assert tun.census_tile_chunks >= 256
                assert torch.equal(out, out0) and torch.equal(fl, fl0)
                for m, mon in enumerate(monitors):
                    t = torch.empty(1 << mon[0], dtype=torch.uint8, device="cuda")
                    grp.copy_pool(m, t)
                    assert torch.equal(t, pools0[m]), "autotune changed monitor %d's pool" % m
        ho = HO.cpu().numpy()
        for m, mon in enumerate(monitors):
            d = singles[m]
            d.ingest(as_i32(pairs[m]).reshape(-1, 2), s)
            d.close_slice(s)
            pa = torch.empty(1 << mon[0], dtype=torch.uint8, device="cuda")
            pb = torch.empty_like(pa)
            grp.copy_pool(m, pa)
            d.copy_pool(pb)
            assert torch.equal(pa, pb), "slice %d monitor %d: pool differs from a single handle" % (s, m)
            ha = torch.empty(2 * mon[1] + 1, dtype=torch.int64, device="cuda")
            hb = torch.empty_like(ha)
            grp.census(m, ha)
            d.census(hb)
            assert torch.equal(ha, hb), "slice %d monitor %d: census differs" % (s, m)
            n = len(hosts[m])
            if n:
                e = torch.empty(n, dtype=torch.float32, device="cuda")
                f = torch.empty(n, dtype=torch.uint8, device="cuda")
                d.estimate(as_i32(hosts[m]), kprime[m], e, f)
                lo = int(ho[m])
                assert torch.equal(out[lo:lo + n], e), "slice %d monitor %d: estimates differ" % (s, m)
                assert torch.equal(fl[lo:lo + n], f)
    assert grp.status() == 0
    grp.close()
    for d in singles:
        d.close()


@pytest.mark.parametrize("wave_mib", [0, 1, 48])
def test_group_equals_single_handles(V, wave_mib):
    # waves of one monitor (1 MiB), of several, and one wave of all
    run_group_vs_single(V, MONITORS_L32, nslices=14, wave_mib=wave_mib)


@pytest.mark.parametrize("L", [1, 2, 4, 8, 16, 64])
def test_group_other_segment_lengths(V, L):
    mons = [(14, 2, 128, L, 0, 11), (15, 5, 256, L, 1, 12), (16, 7, 64 * max(1, L // 16), L, 0, 13)]
    run_group_vs_single(V, mons, nslices=12)


def test_group_graph_replay_equals_single_handles(V):
    run_group_vs_single(V, MONITORS_L32[:5], nslices=12, graph=True)


def test_group_step_graph_is_one_kernel_node(V):
    mons = MONITORS_L32[:3]
    grp = V.VateGroup([V.make_params(*m) for m in mons])
    assert V.vate_group_graph_nodes(grp.g) == 0
    tr = Traffic(SMALL, pkts_per_slice=1000)
    P = as_i32(tr.slice_pairs(0, n=300))
    PO = torch.tensor([0, 100, 200, 300], dtype=torch.int64, device="cuda")
    H = as_i32(tr.aips[:30])
    HO = torch.tensor([0, 10, 20, 30], dtype=torch.int64, device="cuda")
    KP = torch.tensor([m[1] for m in mons], dtype=torch.int32, device="cuda")
    out = torch.zeros(30, dtype=torch.float32, device="cuda")
    grp.step(P, PO, H, HO, KP, out, graph=True)
    grp.step(P, PO, H, HO, KP, out, graph=True)
    assert V.vate_group_graph_nodes(grp.g) == 1
    assert grp.status() == 0
    grp.close()


@pytest.mark.parametrize("spin_limit", [0, 1000])
def test_group_unsatisfiable_wait_times_out_and_returns(V, spin_limit):
    # Every wait of the step is made unsatisfiable (its target raised by one
    # item); with a limit of 0 or 1,000 looks the kernel gives up, sets
    # VATE_GROUP_TIMEOUT and returns.  The timed-out group then does no more
    # work: a later step changes no pool byte.  Then it is destroyed.
    import time
    mons = MONITORS_L32[:3]
    grp = V.VateGroup([V.make_params(*m) for m in mons])
    tr = Traffic(SMALL, pkts_per_slice=1000)
    P = as_i32(tr.slice_pairs(0, n=300))
    PO = torch.tensor([0, 100, 200, 300], dtype=torch.int64, device="cuda")
    H = as_i32(tr.aips[:30])
    HO = torch.tensor([0, 10, 20, 30], dtype=torch.int64, device="cuda")
    KP = torch.tensor([m[1] for m in mons], dtype=torch.int32, device="cuda")
    out = torch.zeros(30, dtype=torch.float32, device="cuda")
    grp.step(P, PO, H, HO, KP, out)                  # a normal step first
    assert grp.status() == 0
    V.vate_group_set_wait(grp.g, spin_limit, 1)
    t0 = time.perf_counter()
    grp.step(P, PO, H, HO, KP, out)
    torch.cuda.synchronize()
    assert time.perf_counter() - t0 < 5.0
    assert grp.status() & V.VATE_GROUP_TIMEOUT
    before = []
    for m, mon in enumerate(mons):
        t = torch.empty(1 << mon[0], dtype=torch.uint8, device="cuda")
        grp.copy_pool(m, t)
        before.append(t)
    V.vate_group_set_wait(grp.g, 1 << 23, 0)
    grp.step(as_i32(tr.slice_pairs(1, n=300)), PO, H, HO, KP, out)
    torch.cuda.synchronize()
    for m, mon in enumerate(mons):
        t = torch.empty(1 << mon[0], dtype=torch.uint8, device="cuda")
        grp.copy_pool(m, t)
        assert torch.equal(t, before[m]), "a timed-out group changed monitor %d's pool" % m
    assert grp.status(clear=True) & V.VATE_GROUP_TIMEOUT
    assert grp.status() & V.VATE_GROUP_TIMEOUT       # not cleared
    grp.close()


def test_group_tuning_is_checked(V):
    grp = V.VateGroup([V.make_params(*m) for m in MONITORS_L32[:2]])
    t = V.vate_group_get_tuning(grp.g)
    assert t.blocks_per_sm >= 1 and t.census_tile_chunks >= 256
    for field, bad in (("blocks_per_sm", 0), ("blocks_per_sm", 99), ("census_tile_chunks", 3000),
                       ("gather_grab_hosts", 33), ("ingest_tile_pairs", 70000), ("preserve_tile_chunks", 0),
                       ("wave_pool_mib", 70000)):
        u = V.vate_group_tuning.from_buffer_copy(t)
        setattr(u, field, bad)
        with pytest.raises(V.VateError) as e:
            V.vate_group_set_tuning(grp.g, u)
        assert e.value.code == V.VATE_EINVAL, field
    V.vate_group_set_tuning(grp.g, t)
    grp.close()


def test_group_autotune_keeps_state_and_outputs(V):
    run_group_vs_single(V, MONITORS_L32[:4], nslices=6, autotune_at=2)


def test_group_monitor_against_oracle(V):
    mons = [(15, 4, 256, 32, 0, 21), (14, 3, 128, 32, 1, 22)]
    trs = [Traffic(SMALL, pkts_per_slice=4000) for _ in mons]
    grp = V.VateGroup([V.make_params(*m) for m in mons])
    oras = [Oracle(c=m[0], k=m[1], g=m[2], seg_len=m[3], partition=m[4], seed=m[5]) for m in mons]
    rng = np.random.default_rng(5)
    for s in range(10):
        pairs, hosts = make_slice(trs, s, rng, empty_every=4)
        P, PO, H, HO, KP = pack(pairs, hosts, [m[1] for m in mons])
        out = torch.zeros(max(1, len(H)), dtype=torch.float32, device="cuda")
        grp.step(P, PO, H, HO, KP, out)
        ho = HO.cpu().numpy()
        for m, o in enumerate(oras):
            if s:
                o.advance()
            o.ingest(pairs[m])
            pool = torch.empty(o.P, dtype=torch.uint8, device="cuda")
            grp.copy_pool(m, pool)
            assert np.array_equal(pool.cpu().numpy(), o.pool())
            if len(hosts[m]):
                oe, _, _ = o.estimate(hosts[m], o.k)
                de = out[int(ho[m]):int(ho[m]) + len(hosts[m])].cpu().numpy().astype(np.float64)
                assert_eq11_close(de, oe, o.g, "monitor %d" % m)
        info = V.vate_group_monitor_info(grp.g, 0)
        assert info.slice == s and info.bact0 == s % (2 * mons[0][1])
    grp.close()


def test_group_bad_device_inputs_are_clamped_and_reported(V):
    mons = [(14, 3, 64, 32, 0, 1), (14, 3, 64, 32, 0, 2), (14, 3, 64, 32, 0, 3)]
    grp = V.VateGroup([V.make_params(*m) for m in mons])
    tr = Traffic(SMALL, pkts_per_slice=100)
    P = as_i32(tr.slice_pairs(0, n=30))
    H = as_i32(tr.aips[:12])
    out = torch.zeros(12, dtype=torch.float32, device="cuda")
    # decreasing pair offsets and a host offset past the buffer
    PO = torch.tensor([0, 20, 10, 30], dtype=torch.int64, device="cuda")
    HO = torch.tensor([0, 4, 8, 99], dtype=torch.int64, device="cuda")
    grp.step(P, PO, H, HO, torch.tensor([3, 3, 3], dtype=torch.int32, device="cuda"), out)
    assert grp.status(clear=True) == V.VATE_GROUP_BAD_OFFSETS
    PO = torch.tensor([0, 10, 20, 30], dtype=torch.int64, device="cuda")
    HO = torch.tensor([0, 4, 8, 12], dtype=torch.int64, device="cuda")
    grp.step(P, PO, H, HO, torch.tensor([0, 3, 7], dtype=torch.int32, device="cuda"), out)
    assert grp.status(clear=True) == V.VATE_GROUP_BAD_KPRIME
    grp.step(P, PO, H, HO, torch.tensor([3, 1, 2], dtype=torch.int32, device="cuda"), out)
    assert grp.status() == 0
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    grp.close()


@pytest.mark.slow
def test_group_full_size_64_monitors(V):
    # The 64-monitor configuration at full size, driven as the benchmark
    # drives it (pools 2^20-2^25, k in {5, 10, 30, 60}, g 512-8192, 44 M pairs
    # and 1.86 M hosts per slice, the tuned tiling, one CUDA graph per slice):
    # every monitor equals a single handle bit for bit (pool, census, every
    # host's estimate and flag) over three slices, and the two busiest equal
    # the oracle (pool, census, a seeded sample of estimates and counts).
    import bench
    from traffic import DeviceTraffic, TrafficSpec
    mons = bench.monitors64_config()
    dts, params, singles = [], [], []
    for m in mons:
        spec = TrafficSpec(n_aips=m["hosts"], pkts_per_slice=m["rate"], zipf_s=1.1, seed=m["seed"])
        dts.append(DeviceTraffic(Traffic(spec)))
        params.append(V.make_params(m["c"], m["k"], m["g"], 32, 0, m["seed"]))
        singles.append(V.Vate(m["c"], m["k"], m["g"], 32, 0, m["seed"]))
    po = np.zeros(65, np.int64)
    po[1:] = np.cumsum([m["rate"] for m in mons])
    ho = np.zeros(65, np.int64)
    ho[1:] = np.cumsum([m["hosts"] for m in mons])
    pairs = torch.empty(int(po[-1]), 2, dtype=torch.int32, device="cuda")
    hosts = torch.cat([d.hosts() for d in dts])
    PO, HO = torch.from_numpy(po).cuda(), torch.from_numpy(ho).cuda()
    KP = torch.tensor([m["k"] for m in mons], dtype=torch.int32, device="cuda")
    out = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
    flags = torch.empty(hosts.numel(), dtype=torch.uint8, device="cuda")

    def fill(s):
        for i, d in enumerate(dts):
            pairs[int(po[i]):int(po[i + 1])].copy_(d.slice_pairs(s))

    fill(0)
    tuner = V.VateGroup(params)
    tuner.step(pairs, PO, hosts, HO, KP, out, flags)
    tun = tuner.autotune(pairs, PO, hosts, HO, KP, out, flags)
    tuner.close()
    grp = V.VateGroup(params)
    V.vate_group_set_tuning(grp.g, tun)
    busiest = [int(i) for i in np.argsort([m["rate"] for m in mons])[-2:]]
    oras = {i: Oracle(c=mons[i]["c"], k=mons[i]["k"], g=mons[i]["g"], seg_len=32, partition=0,
                      seed=mons[i]["seed"]) for i in busiest}
    rng = np.random.default_rng(17)
    for s in range(3):
        fill(s)
        grp.step(pairs, PO, hosts, HO, KP, out, flags, graph=True)
        for i, (m, d) in enumerate(zip(mons, singles)):
            p = pairs[int(po[i]):int(po[i + 1])]
            h = hosts[int(ho[i]):int(ho[i + 1])]
            d.ingest(p, s)
            d.close_slice(s)
            pa = torch.empty(1 << m["c"], dtype=torch.uint8, device="cuda")
            pb = torch.empty_like(pa)
            grp.copy_pool(i, pa)
            d.copy_pool(pb)
            assert torch.equal(pa, pb), "slice %d monitor %d: pool differs from a single handle" % (s, i)
            ha = torch.empty(2 * m["k"] + 1, dtype=torch.int64, device="cuda")
            hb = torch.empty_like(ha)
            grp.census(i, ha)
            d.census(hb)
            assert torch.equal(ha, hb), "slice %d monitor %d: census differs" % (s, i)
            e = torch.empty(h.numel(), dtype=torch.float32, device="cuda")
            f = torch.empty(h.numel(), dtype=torch.uint8, device="cuda")
            d.estimate(h, m["k"], e, f)
            assert torch.equal(out[int(ho[i]):int(ho[i + 1])], e), "slice %d monitor %d: estimates" % (s, i)
            assert torch.equal(flags[int(ho[i]):int(ho[i + 1])], f)
            if i in oras:
                o = oras[i]
                if s:
                    o.advance()
                o.ingest(p.cpu().numpy().view(np.uint32))
                assert np.array_equal(pa.cpu().numpy(), o.pool())
                np.testing.assert_array_equal(hb.cpu().numpy().astype(np.uint64), o.census())
                idx = rng.choice(h.numel(), 512, replace=False)
                hs = h.cpu().numpy().view(np.uint32)[idx]
                oe, oa, of = o.estimate(hs, m["k"])
                act = torch.empty(h.numel(), dtype=torch.int32, device="cuda")
                d.active_counts(h, m["k"], act)
                np.testing.assert_array_equal(act.cpu().numpy().view(np.uint32)[idx], oa)
                np.testing.assert_array_equal(f.cpu().numpy()[idx], of)
                de = e.cpu().numpy()[idx].astype(np.float64)
                assert_eq11_close(de, oe, m["g"], "monitor")
    assert grp.status() == 0
    grp.close()
    for d in singles:
        d.close()
