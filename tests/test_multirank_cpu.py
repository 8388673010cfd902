"""The benchmark's multi-rank host logic on CPU ranks (gloo, world size 2):
each rank runs an independent replica, the timing is the maximum over ranks
and the packet count the sum, with no data-path collective."""
import os
import socket
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_max_and_sum_over_two_gloo_ranks(tmp_path):
    script = tmp_path / "ranks.py"
    script.write_text(textwrap.dedent("""
        import os, sys, json
        sys.path.insert(0, %r)
        os.environ.setdefault("CUDA_VISIBLE_DEVICES", "")
        import bench
        rank, world, local = bench.dist_setup()
        t = bench.max_over_ranks(1.5 + rank, world)
        p = bench.sum_over_ranks(10.0 * (rank + 1), world)
        bench.barrier(world)
        with open(os.path.join(%r, "rank%%d.json" %% rank), "w") as f:
            json.dump({"rank": rank, "world": world, "max": t, "sum": p}, f)
        import torch.distributed as dist
        dist.destroy_process_group()
    """ % (ROOT, str(tmp_path))))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % free_port(), str(script)]
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=240, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    import json
    lines = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert len(lines) == 2
    for r in lines:
        assert r["world"] == 2 and r["max"] == 2.5 and r["sum"] == 30.0


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "3",
                          "--warmup", "3"], capture_output=True, text=True, timeout=240, env=env, cwd=ROOT)
    assert out.returncode == 0 and out.stdout.strip() == ""
