"""Position shards of one pool (include/vate_shard.h) on the device.

Shards of one pool, driven with the same pairs and slices, must together
hold exactly the undivided pool (their copies, concatenated, equal its copy
and the oracle's), and their summed active counts and censuses must give,
through vate_estimate_from_counts, the estimates and flags of vate_estimate
on one handle bit for bit: for timestamps (byte and 16-bit) and recorders,
both segment layouts, even and uneven splits.  The distributed form
(ShardedVate over gloo) runs as two processes on one GPU whose kernels never
wait on each other; the collectives run on the host.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest
import torch

from oracle import Oracle
from traffic import SMALL, Traffic

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def V():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1812_00282_b300 as V
    return V


def dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.uint32).view(np.int32)).cuda()


def uneven(P):
    return [(0, 64), (64, P // 2 + 192), (P // 2 + 192, P - 128), (P - 128, P)]


CASES = [
    ((17, 5, 1024, 32, 0, 51, 0), "even3"),
    ((17, 5, 1024, 1, 1, 52, 0), "uneven"),
    ((16, 4, 512, 32, 0, 53, 1), "even2"),        # distance recorders
    ((18, 100, 512, 32, 0, 54, 0), "even3"),      # 16-bit ATs
]


@pytest.mark.parametrize("params,split", CASES, ids=["at-even3", "at-L1-uneven", "dr-even2", "wide-even3"])
def test_shards_equal_one_handle(V, params, split):
    from paper_1812_00282_b300.sharded import shard_ranges
    c, k, g, L, part, seed, counter = params
    P = 1 << c
    ranges = {"even3": shard_ranges(P, 3), "even2": shard_ranges(P, 2), "uneven": uneven(P)}[split]
    vp = V.make_params(c, k, g, L, part, seed, counter)
    full = V.Vate(c, k, g, L, part, seed, counter=counter)
    shards = [V.vate_create_shard(vp, lo, hi) for lo, hi in ranges]
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=part, seed=seed)
    tr = Traffic(SMALL, pkts_per_slice=6000)
    hosts = tr.aips[:900]
    dh = dev_u32(hosts)
    dt = V.pool_dtype(k)
    ids = [0, 1, 2, 3, k + 1, k + 2, 2 * k + 5, 2 * k + 6, 4 * k + 9]
    prev = None
    for sid in ids:
        if prev is not None:
            for _ in range(sid - prev):
                o.advance()
        prev = sid
        arr = tr.slice_pairs(sid % 64)
        o.ingest(arr)
        dp = torch.from_numpy(arr.view(np.int32)).cuda()
        full.ingest(dp, sid)
        full.close_slice(sid)
        for h in shards:
            V.vate_ingest(h, dp, sid)
            V.vate_close_slice(h, sid)
        # the shards hold the pool
        whole = torch.empty(P, dtype=dt, device="cuda")
        full.copy_pool(whole)
        parts = []
        for h, (lo, hi) in zip(shards, ranges):
            t = torch.empty(hi - lo, dtype=dt, device="cuda")
            V.vate_copy_pool(h, t)
            parts.append(t)
        joined = torch.cat(parts)
        assert torch.equal(joined, whole)
        np.testing.assert_array_equal(joined.cpu().numpy().astype(np.int64),
                                      (o.dr() if counter else o.pool()).astype(np.int64))
        # summed counts give the same census, A and estimates
        hist = torch.zeros(2 * k + 1, dtype=torch.int64, device="cuda")
        for h in shards:
            t = torch.empty_like(hist)
            V.vate_census(h, t)
            hist += t
        want_hist = torch.empty_like(hist)
        full.census(want_hist)
        assert torch.equal(hist, want_hist)
        for kp in (1, k):
            act = torch.zeros(len(hosts), dtype=torch.int32, device="cuda")
            for h in shards:
                t = torch.empty_like(act)
                V.vate_active_counts(h, dh, kp, t)
                act += t
            want_act = torch.empty_like(act)
            full.active_counts(dh, kp, want_act)
            assert torch.equal(act, want_act)
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


def test_shard_limits(V):
    vp = V.make_params(16, 4, 512, 32, 0, 1)
    for lo, hi in [(0, 0), (32, 1024), (0, 100), (1024, 512), (0, (1 << 16) + 64)]:
        with pytest.raises(V.VateError) as e:
            V.vate_create_shard(vp, lo, hi)
        assert e.value.code == V.VATE_EINVAL
    h = V.vate_create_shard(vp, 1024, 1 << 16)
    info = V.vate_get_info(h)
    assert (info.pid_lo, info.pid_hi, info.pool_size) == (1024, 1 << 16, 1 << 16)
    p = Traffic(SMALL, pkts_per_slice=1000).slice_pairs(0)
    V.vate_ingest(h, torch.from_numpy(p.view(np.int32)).cuda(), 0)
    V.vate_close_slice(h, 0)
    out = torch.empty(4, dtype=torch.float32, device="cuda")
    for call in (lambda: V.vate_estimate(h, dev_u32([1, 2, 3, 4]), 4, out),
                 lambda: V.vate_checkpoint(h)):
        with pytest.raises(V.VateError) as e:
            call()
        assert e.value.code == V.VATE_EINVAL
    V.vate_destroy(h)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("side_stream", [False, True])
def test_two_processes_reduce_to_one_handle(V, tmp_path, side_stream):
    # side_stream: every shard call is queued on a stream other than torch's
    # current one, so the all-reduces and Eq. 11 must be ordered after the
    # counting kernels by the module itself
    c, k, g, L, seed = 17, 5, 1024, 32, 61
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent("""
        import json, os, sys
        sys.path.insert(0, %(root)r)
        import numpy as np, torch, torch.distributed as dist
        from traffic import SMALL, Traffic
        import paper_1812_00282_b300 as V
        from paper_1812_00282_b300.sharded import ShardedVate
        dist.init_process_group("gloo")
        rank = dist.get_rank()
        torch.cuda.set_device(0)
        tr = Traffic(SMALL, pkts_per_slice=6000)
        hosts = torch.from_numpy(np.ascontiguousarray(tr.aips[:800], np.uint32).view(np.int32)).cuda()
        sv = ShardedVate(%(c)d, %(k)d, %(g)d, %(L)d, 0, %(seed)d)
        st = torch.cuda.Stream() if %(side)r else None
        ref = V.Vate(%(c)d, %(k)d, %(g)d, %(L)d, 0, %(seed)d) if rank == 0 else None
        ok = True
        for s in (0, 1, 2, 7, 8, 20):
            p = torch.from_numpy(tr.slice_pairs(s).view(np.int32)).cuda()
            out = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
            fl = torch.empty(hosts.numel(), dtype=torch.uint8, device="cuda")
            if st is not None:
                st.wait_stream(torch.cuda.current_stream())
            sv.ingest(p, s, stream=st)
            sv.close_slice(s, stream=st)
            sv.estimate(hosts, %(k)d, out, fl, stream=st)
            if st is not None:
                torch.cuda.current_stream().wait_stream(st)
            if ref is not None:
                ref.ingest(p, s)
                ref.close_slice(s)
                e = torch.empty_like(out)
                f = torch.empty_like(fl)
                ref.estimate(hosts, %(k)d, e, f)
                ok = ok and torch.equal(e, out) and torch.equal(f, fl)
        sv.close()
        dist.barrier()
        with open(os.path.join(%(tmp)r, "rank%%d.json" %% rank), "w") as fh:
            json.dump({"ok": bool(ok), "range": [sv.lo, sv.hi]}, fh)
        dist.destroy_process_group()
    """ % dict(root=ROOT, tmp=str(tmp_path), c=c, k=k, g=g, L=L, seed=seed, side=side_stream)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % free_port(), str(script)]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    ranks = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert ranks[0]["ok"] and ranks[0]["range"] == [0, 1 << 16] and ranks[1]["range"] == [1 << 16, 1 << 17]
