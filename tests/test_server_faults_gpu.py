"""Failure handling of the serving loop, with the faults made on the host
(vate_server_inject and the submitters themselves; no GPU fault).

Four monitors are served at once, each fed by a submitter thread of its own,
while the faults happen:
  - monitor 0: its submitter stalls for 300 ms in the middle of a slice;
  - monitor 1: two of its requests are held back 150 ms each (late batches);
  - monitor 2: one ingest batch is dropped (VATE_FAULT_DROP): its wait
    returns VATE_EDROPPED;
  - monitor 3: it submits an ingest for a slice it has already closed: the
    wait returns VATE_ESLICE;
  - the scheduler itself stalls 200 ms once (VATE_FAULT_STALL).
Every monitor's estimates and flags at every close must equal, bit for bit,
those of a vate_handle fed directly -- with the same pairs for monitors 0, 1
and 3 (the faults do not change them), and without the dropped batch for
monitor 2 -- and the errors must come back through vate_server_wait.
"""
import threading
import time

import numpy as np
import pytest
import torch

from traffic import SMALL, Traffic

pytestmark = pytest.mark.gpu

SLICES = 6
PARAMS = [(16, 5, 512, 2, 0, 41), (17, 4, 1024, 32, 1, 42), (16, 5, 512, 8, 0, 43), (15, 3, 256, 1, 0, 44)]


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def as_i32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def make_batches(m):
    """Per slice, the monitor's pairs cut into batches of 1..2,999 pairs."""
    tr = Traffic(SMALL, pkts_per_slice=9000 + 1000 * m)
    rng = np.random.default_rng(100 + m)
    out = []
    for s in range(SLICES):
        p = tr.slice_pairs(s)
        bs, i = [], 0
        while i < len(p):
            n = int(rng.integers(1, 3000))
            bs.append(np.ascontiguousarray(p[i:i + n]))
            i += n
        out.append(bs)
    return tr.aips[:700], out


def direct(V, params, hosts, slices_batches, skip=None):
    """The same stream through a vate_handle: every batch in order except the
    (slice, batch) given in skip."""
    d = V.Vate(*params)
    dh = as_i32(hosts)
    res = []
    for s, bs in enumerate(slices_batches):
        for j, b in enumerate(bs):
            if skip != (s, j):
                d.ingest(as_i32(b).reshape(-1, 2), s)
        d.close_slice(s)
        e = torch.empty(len(hosts), dtype=torch.float32, device="cuda")
        f = torch.empty(len(hosts), dtype=torch.uint8, device="cuda")
        d.estimate(dh, params[1], e, f)
        res.append((e.cpu().numpy(), f.cpu().numpy()))
    d.close()
    return res


def test_faults_leave_other_monitors_unchanged_and_errors_come_back(V):
    srv = V.vate_server_create(2 << 30, slots=4, slot_records=1 << 14)
    mids = [V.vate_server_admit(srv, V.make_params(*p)) for p in PARAMS]
    data = [make_batches(m) for m in range(len(PARAMS))]
    results = [[] for _ in PARAMS]
    errors = {}
    fails = []
    drop_at = (3, 2)          # monitor 2: slice 3, third batch

    def submitter(m):
        try:
            hosts, sl = data[m]
            mid = mids[m]
            for s, bs in enumerate(sl):
                tickets = []
                for j, b in enumerate(bs):
                    if m == 0 and s == 2 and j == len(bs) // 2:
                        time.sleep(0.3)                      # a stalled submitter
                    if (m == 1 and s == 1 and j == 0) or (m == 2 and (s, j) == drop_at):
                        for t in tickets:                    # nothing of this monitor left in the queue,
                            V.vate_server_wait(srv, t)       # so the fault hits the next request
                        tickets = []
                        if m == 1:
                            V.vate_server_inject(srv, V.VATE_FAULT_HOLD, mid, count=2, ms=150)
                        else:
                            V.vate_server_inject(srv, V.VATE_FAULT_DROP, mid, count=1)
                    t = V.vate_server_submit_ingest(srv, mid, b, s)
                    if m == 2 and (s, j) == drop_at:
                        with pytest.raises(V.VateError) as e:
                            V.vate_server_wait(srv, t)
                        errors["drop"] = e.value.code
                    else:
                        tickets.append(t)
                out = np.empty(len(hosts), np.float32)
                fl = np.empty(len(hosts), np.uint8)
                tc = V.vate_server_submit_close(srv, mid, s, hosts, PARAMS[m][1], out, fl)
                for t in tickets:
                    V.vate_server_wait(srv, t)
                V.vate_server_wait(srv, tc)
                results[m].append((out, fl))
                if m == 3 and s == 3:                        # an ingest into a slice already closed
                    t = V.vate_server_submit_ingest(srv, mid, sl[1][0], 1)
                    with pytest.raises(V.VateError) as e:
                        V.vate_server_wait(srv, t)
                    errors["past"] = e.value.code
        except Exception as ex:                              # reported on the main thread
            fails.append((m, repr(ex)))

    threads = [threading.Thread(target=submitter, args=(m,)) for m in range(len(PARAMS))]
    for t in threads:
        t.start()
    time.sleep(0.05)
    V.vate_server_inject(srv, V.VATE_FAULT_STALL, ms=200)   # the scheduler stalls once
    for t in threads:
        t.join(timeout=300)
    assert not any(t.is_alive() for t in threads), "a submitter did not finish"
    assert not fails, fails
    V.vate_server_drain(srv)
    V.vate_server_destroy(srv)
    assert errors == {"drop": V.VATE_EDROPPED, "past": V.VATE_ESLICE}
    for m, p in enumerate(PARAMS):
        hosts, sl = data[m]
        ref = direct(V, p, hosts, sl, skip=drop_at if m == 2 else None)
        assert len(results[m]) == SLICES
        for s in range(SLICES):
            assert np.array_equal(results[m][s][0], ref[s][0]), "monitor %d slice %d: estimates" % (m, s)
            assert np.array_equal(results[m][s][1], ref[s][1]), "monitor %d slice %d: flags" % (m, s)
    # the dropped batch mattered: with it, monitor 2's estimates differ from slice 3 on
    full = direct(V, PARAMS[2], data[2][0], data[2][1])
    assert not np.array_equal(full[3][0], results[2][3][0])


def test_inject_rejects_unknown_faults_and_monitors(V):
    srv = V.vate_server_create(1 << 28, slots=2, slot_records=1024)
    mid = V.vate_server_admit(srv, V.make_params(14, 2, 64, 1, 0, 1))
    for kind, mon in ((99, mid), (V.VATE_FAULT_DROP, 5), (V.VATE_FAULT_HOLD, -1)):
        with pytest.raises(V.VateError) as e:
            V.vate_server_inject(srv, kind, mon, count=1, ms=1)
        assert e.value.code == V.VATE_EINVAL
    V.vate_server_destroy(srv)
