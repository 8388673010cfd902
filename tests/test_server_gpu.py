"""The serving loop (include/vate_server.h).

Each monitor served must produce exactly what its own vate_handle produces on
the same pairs and hosts, whether it is served alone or mixed with other
monitors whose batches arrive concurrently from other threads, however its
pairs are cut into batches, and whether batches are merged by the scheduler.
Admission respects the memory budget; request errors come back through wait.
"""
import threading

import numpy as np
import pytest
import torch

from traffic import SMALL, Traffic, TrafficSpec

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def as_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def batches(pairs, rng, max_batch):
    out, i = [], 0
    while i < len(pairs):
        n = int(rng.integers(1, max_batch))
        out.append(np.ascontiguousarray(pairs[i:i + n]))
        i += n
    return out


def direct_reference(V, params, slices, hosts, kprime, model=None):
    d = V.Vate(*params)
    res = []
    dh = as_i32(hosts)
    for s, p in enumerate(slices):
        d.ingest(as_i32(p), s)
        d.close_slice(s)
        e = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
        f = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
        if model is None:
            d.estimate(dh, kprime, e, f)
        else:
            V.vate_estimate_learned(d.h, dh, model, e, f)
        res.append((e.cpu().numpy(), f.cpu().numpy()))
    d.close()
    return res


def serve_monitor(V, srv, mid, slices, hosts, kprime, rng, pinned=False):
    res = []
    keep = []
    for s, p in enumerate(slices):
        tickets = []
        for b in batches(p, rng, 3000):
            if pinned:
                b = torch.from_numpy(b.view(np.int32)).pin_memory()
                keep.append(b)
            tickets.append(V.vate_server_submit_ingest(srv, mid, b, s, V.VATE_SUBMIT_PINNED if pinned else 0))
            keep.append(b)
        out = np.empty(len(hosts), np.float32)
        fl = np.empty(len(hosts), np.uint8)
        t = V.vate_server_submit_close(srv, mid, s, hosts, kprime, out, fl)
        for x in tickets:
            V.vate_server_wait(srv, x)
        V.vate_server_wait(srv, t)
        res.append((out, fl))
    return res


MON_A = (18, 5, 1024, 32, 0, 3)


def test_alone_in_mix_and_direct_are_identical(V):
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    slices = [tr.slice_pairs(s) for s in range(8)]
    hosts = tr.aips[:2000]
    ref = direct_reference(V, MON_A, slices, hosts, 5)
    # alone
    srv = V.vate_server_create(1 << 30, slots=4, slot_records=4096)
    a = V.vate_server_admit(srv, V.make_params(*MON_A))
    alone = serve_monitor(V, srv, a, slices, hosts, 5, np.random.default_rng(1))
    V.vate_server_destroy(srv)
    # in a mix: five other monitors fed from other threads at the same time
    srv = V.vate_server_create(1 << 30, slots=6, slot_records=4096)
    others = [(17, 3, 512, 32, 1, 10 + i) for i in range(5)]
    ids = [V.vate_server_admit(srv, V.make_params(*o)) for o in others]
    a = V.vate_server_admit(srv, V.make_params(*MON_A))

    def feed(mid, seed):
        t2 = Traffic(TrafficSpec(n_aips=1024, pkts_per_slice=15_000, zipf_s=1.2, seed=seed))
        serve_monitor(V, srv, mid, [t2.slice_pairs(s) for s in range(8)], t2.aips[:500], 3,
                      np.random.default_rng(seed), pinned=(seed % 2 == 0))

    ths = [threading.Thread(target=feed, args=(m, 100 + m)) for m in ids]
    for t in ths:
        t.start()
    mixed = serve_monitor(V, srv, a, slices, hosts, 5, np.random.default_rng(2), pinned=True)
    for t in ths:
        t.join()
    st = V.vate_server_get_stats(srv)
    assert st.max_in_flight >= 2
    V.vate_server_destroy(srv)
    for s in range(len(slices)):
        np.testing.assert_array_equal(alone[s][0], ref[s][0])
        np.testing.assert_array_equal(alone[s][1], ref[s][1])
        np.testing.assert_array_equal(mixed[s][0], ref[s][0])
        np.testing.assert_array_equal(mixed[s][1], ref[s][1])


def test_small_batches_are_merged_and_exact(V):
    tr = Traffic(SMALL, pkts_per_slice=30_000)
    slices = [tr.slice_pairs(s) for s in range(3)]
    hosts = tr.aips[:1000]
    ref = direct_reference(V, MON_A, slices, hosts, 5)
    srv = V.vate_server_create(1 << 30, slots=2, slot_records=65536)
    a = V.vate_server_admit(srv, V.make_params(*MON_A))
    res = []
    for s, p in enumerate(slices):
        bs = [np.ascontiguousarray(p[i:i + 50]) for i in range(0, len(p), 50)]
        ts = [V.vate_server_submit_ingest(srv, a, b, s) for b in bs]
        out = np.empty(len(hosts), np.float32)
        t = V.vate_server_submit_close(srv, a, s, hosts, 5, out)
        for x in ts + [t]:
            V.vate_server_wait(srv, x)
        res.append(out)
    st = V.vate_server_get_stats(srv)
    assert st.merged_ingests > 0 and st.ingests_done == sum((len(p) + 49) // 50 for p in slices)
    V.vate_server_destroy(srv)
    for s in range(3):
        np.testing.assert_array_equal(res[s], ref[s][0])


def test_admission_follows_the_memory_budget(V):
    slots_bytes = 2 * 1024 * 13
    per = (1 << 20) + 11 * 8 * (1 + 4 * torch.cuda.get_device_properties(0).multi_processor_count) + 256
    srv = V.vate_server_create(slots_bytes + 3 * per + 100, slots=2, slot_records=1024)
    ids = [V.vate_server_admit(srv, V.make_params(20, 5, 64, 1, 0, i)) for i in range(3)]
    with pytest.raises(V.VateError) as e:
        V.vate_server_admit(srv, V.make_params(20, 5, 64, 1, 0, 9))
    assert e.value.code == V.VATE_ENOMEM
    V.vate_server_release(srv, ids[1])
    V.vate_server_admit(srv, V.make_params(20, 5, 64, 1, 0, 9))
    assert V.vate_server_get_stats(srv).monitors == 3
    V.vate_server_destroy(srv)


def test_request_errors_come_back_through_wait(V):
    srv = V.vate_server_create(1 << 28, slots=2, slot_records=1024)
    a = V.vate_server_admit(srv, V.make_params(16, 3, 64, 1, 0, 1))
    p = Traffic(SMALL, pkts_per_slice=500).slice_pairs(0)
    V.vate_server_wait(srv, V.vate_server_submit_ingest(srv, a, p, 5))
    with pytest.raises(V.VateError) as e:
        V.vate_server_wait(srv, V.vate_server_submit_ingest(srv, a, p, 3))   # past slice
    assert e.value.code == V.VATE_ESLICE
    out = np.empty(4, np.float32)
    V.vate_server_wait(srv, V.vate_server_submit_close(srv, a, 5, np.arange(4, dtype=np.uint32), 3, out))
    with pytest.raises(V.VateError) as e:
        V.vate_server_submit_ingest(srv, 42, p, 6)                            # unknown monitor
    assert e.value.code == V.VATE_EINVAL
    V.vate_server_destroy(srv)


def test_learned_close_matches_direct_learned_estimate(V):
    n_in = 12
    model = torch.empty(V.vate_mlp_param_count(n_in), dtype=torch.float32, device="cuda")
    V.vate_mlp_init(model, n_in, 77)
    tr = Traffic(SMALL, pkts_per_slice=20_000)
    slices = [tr.slice_pairs(s) for s in range(6)]
    hosts = tr.aips[:1500]
    ref = direct_reference(V, MON_A, slices, hosts, 5, model=model)
    srv = V.vate_server_create(1 << 30, slots=4, slot_records=4096)
    a = V.vate_server_admit(srv, V.make_params(*MON_A))
    V.vate_server_set_model(srv, a, model)
    res = serve_monitor(V, srv, a, slices, hosts, 5, np.random.default_rng(4))
    V.vate_server_destroy(srv)
    for s in range(len(slices)):
        np.testing.assert_array_equal(res[s][0], ref[s][0])
        np.testing.assert_array_equal(res[s][1], ref[s][1])


def test_wide_and_packed_monitors_are_served_exactly(V):
    # 16-bit ATs (k = 100) and the packed layout (5-bit fields) through the
    # server: the same results as their own handles, and memory counted by layout
    tr = Traffic(SMALL, pkts_per_slice=8_000)
    slices = [tr.slice_pairs(s) for s in range(5)]
    hosts = tr.aips[:800]
    cases = [((17, 100, 512, 32, 0, 21), 0), ((17, 10, 512, 32, 0, 22), 5)]
    srv = V.vate_server_create(1 << 30, slots=4, slot_records=4096)
    for params, bits in cases:
        ref = []
        d = V.Vate(*params, at_bits=bits)
        for s, p in enumerate(slices):
            d.ingest(as_i32(p), s)
            d.close_slice(s)
            e = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
            d.estimate(as_i32(hosts), params[1], e)
            ref.append(e.cpu().numpy())
        d.close()
        before = V.vate_server_get_stats(srv).memory_in_use
        mid = V.vate_server_admit(srv, V.make_params(*params, at_bits=bits))
        pool_bytes = V.vate_server_get_stats(srv).memory_in_use - before
        want = (2 << 17) if params[1] > 63 else (((1 << 17) + 5) // 6 * 4 + 15) // 16 * 16
        assert pool_bytes >= want and pool_bytes < want + (1 << 20)
        got = serve_monitor(V, srv, mid, slices, hosts, params[1], np.random.default_rng(bits))
        for s in range(len(slices)):
            np.testing.assert_array_equal(got[s][0], ref[s])
    V.vate_server_destroy(srv)


@pytest.mark.slow
def test_serving_workload_full_size(V):
    # The serving workload as configured: candidate monitors admitted by an
    # 8 GB AT-memory budget up to 16, Poisson batches of 1k-1M pairs arriving
    # in real time (mean 8 Mpkt/s, bursts to 30 Mpkt/s), 1 s slices, k = 10.
    # Every request completes without error (vate_server_wait raises
    # otherwise), every batch and close is accounted for, the admitted pools
    # fit the budget, and several requests were in flight at once.
    from paper_1812_00282_b300 import serving
    r = serving.run(V, duration=3.0, paced=True)
    st = r["stats"]
    assert 1 <= r["monitors_admitted"] <= 16
    assert sum(1 << c for c in r["log2_pools"]) <= 8 << 30
    assert st["memory_in_use"] <= 8 << 30
    assert st["pairs_done"] == r["pairs"] and st["closes_done"] == 3 * r["monitors_admitted"]
    assert st["max_in_flight"] >= 2
    assert 0 < st["close_p50_ms"] <= st["close_p99_ms"] < 1000.0
    assert 0 < r["offered_mpkts"] < 30.0
