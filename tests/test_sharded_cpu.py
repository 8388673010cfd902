"""Position sharding of one pool (include/vate_shard.h) on CPU ranks: the
shard ranges tile the pool on 64-position boundaries, and two gloo ranks
running paper_1812_00282_b300.sharded.ShardedVate -- with an oracle-backed
stand-in for the library's shard calls -- reduce their partial counts and
censuses to estimates equal to the oracle's on the undivided pool."""
import json
import os
import socket
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1812_00282_b300.sharded import SHARD_ALIGN, shard_ranges

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("P,world", [(1 << 12, 1), (1 << 12, 2), (1 << 13, 3), (1 << 20, 7), (1 << 32, 8),
                                     (64 * 5, 5)])
def test_shard_ranges_tile_the_pool(P, world):
    r = shard_ranges(P, world)
    assert len(r) == world and r[0][0] == 0 and r[-1][1] == P
    for (a, b), (c, d) in zip(r, r[1:]):
        assert b == c
    for lo, hi in r:
        assert lo < hi and lo % SHARD_ALIGN == 0 and (hi % SHARD_ALIGN == 0 or hi == P)
    sizes = [hi - lo for lo, hi in r]
    assert max(sizes) - min(sizes) <= 2 * SHARD_ALIGN


def test_shard_ranges_reject_too_many_shards():
    with pytest.raises(ValueError):
        shard_ranges(64 * 3, 4)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_reduce_to_the_undivided_pool(tmp_path):
    c, k, g, L, seed = 13, 3, 64, 8, 5
    rng = np.random.default_rng(9)
    hosts = rng.integers(1, 2**32, size=24, dtype=np.uint64).astype(np.uint32)
    slices = {}
    for s in (0, 1, 2, 4, 5, 9, 10):
        h = hosts[rng.integers(0, len(hosts), size=300)]
        b = rng.integers(0, 2**32, size=300, dtype=np.uint64).astype(np.uint32)
        slices[s] = np.stack([h, b], 1)
    np.save(tmp_path / "hosts.npy", hosts)
    np.save(tmp_path / "slices.npy", np.stack([slices[s] for s in sorted(slices)]))
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent("""
        import json, os, sys
        sys.path.insert(0, %(root)r)
        sys.path.insert(0, os.path.join(%(root)r, "tests"))
        import numpy as np, torch, torch.distributed as dist
        from paper_1812_00282_b300.sharded import ShardedVate
        from shard_fake import FakeShardLib
        dist.init_process_group("gloo")
        rank = dist.get_rank()
        hosts = torch.from_numpy(np.load(os.path.join(%(tmp)r, "hosts.npy")).view(np.int32))
        sl = np.load(os.path.join(%(tmp)r, "slices.npy"))
        sv = ShardedVate(%(c)d, %(k)d, %(g)d, %(L)d, 0, %(seed)d, lib=FakeShardLib())
        res = {"range": [sv.lo, sv.hi], "est": []}
        for s, arr in zip(%(ids)r, sl):
            sv.ingest(torch.from_numpy(np.ascontiguousarray(arr).view(np.int32)), s)
            sv.close_slice(s)
            for kp in (1, %(k)d):
                out = torch.empty(hosts.numel(), dtype=torch.float64)
                sv.estimate(hosts, kp, out)
                res["est"].append(out.tolist())
        with open(os.path.join(%(tmp)r, "rank%%d.json" %% rank), "w") as f:
            json.dump(res, f)
        dist.destroy_process_group()
    """ % dict(root=ROOT, tmp=str(tmp_path), c=c, k=k, g=g, L=L, seed=seed, ids=sorted(slices))))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % free_port(), str(script)]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert out.returncode == 0, out.stderr[-3000:]
    ranks = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert ranks[0]["range"] == [0, 1 << 12] and ranks[1]["range"] == [1 << 12, 1 << 13]
    # the undivided pool
    from oracle import Oracle
    o = Oracle(c=c, k=k, g=g, seg_len=L, partition=0, seed=seed)
    want, prev = [], None
    for s in sorted(slices):
        if prev is not None:
            for _ in range(s - prev):
                o.advance()
        prev = s
        o.ingest(slices[s])
        for kp in (1, k):
            want.append(o.estimate(hosts, kp)[0].tolist())
    for r in ranks:
        np.testing.assert_array_equal(np.array(r["est"]), np.array(want))
