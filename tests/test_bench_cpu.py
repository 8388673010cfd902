"""Host logic of bench.py that needs no GPU: the checksum that ties the
committed ncu traffic figures to the kernel sources follows their code and
ignores comments and layout; the workload name and the oracle legs follow
the run's arguments."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_code_of_drops_comments_and_layout():
    src = "int a = 1; // one\n/* two\n lines */ int  b =\n 2;\n"
    assert bench.code_of(src) == "int a = 1; int b = 2;"
    assert bench.code_of("x /* a */ y /* b\n c */ z // d") == "x y z"


def test_code_of_keeps_code_changes():
    assert bench.code_of("int a = 1;") != bench.code_of("int a = 2;")
    assert bench.code_of("a // c\nb") == bench.code_of("a b // d")   # only the comments differ
    assert bench.code_of("a /* c */ + b") != bench.code_of("a - b")


def test_traffic_sha_is_the_committed_one_or_the_figure_is_null():
    for kernel in ("hs_tile_kernel@L1", "gather_seg_kernel@L2"):
        sha = bench.traffic_sha(kernel)
        assert len(sha) == 16 and all(c in "0123456789abcdef" for c in sha)
        t = bench.committed_traffic(kernel)
        assert t is None or t > 0
    # each figure depends on its own kernel's sources
    assert bench.traffic_sha("hs_tile_kernel@L1") != bench.traffic_sha("gather_seg_kernel@L2")


def _args(*argv):
    old = sys.argv
    sys.argv = ["bench.py", *argv]
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_workload_name_follows_the_arguments():
    a = _args()
    assert bench.workload_name(a, 1 << 20).startswith(
        "plain VATE at 40 Gb/s shape: 1,048,576 aips, 5,000,000 pkts per 1 s slice, k=10, AT pool 2^26")
    b = _args("--k", "300", "--seg-len", "16", "--pkts", "1000")
    name = bench.workload_name(b, 4096)
    assert "4,096 aips, 1,000 pkts" in name and "k=300" in name and "(16-AT segments)" in name


def test_oracle_step_parts_use_the_given_window():
    # the oracle leg counts with the run's window: the N0 scan and every
    # per-host call of one step get k' = k, for the long window as for the short one
    from oracle import Oracle
    from traffic import SMALL, Traffic

    class Recording(Oracle):
        seen = []

        def pool_inactive(self, kprime):
            self.seen.append(kprime)
            return super().pool_inactive(kprime)

        def estimate_hosts(self, aips, kprime, n0):
            self.seen.append(kprime)
            return super().estimate_hosts(aips, kprime, n0)

    tr = Traffic(SMALL, pkts_per_slice=2000)
    pairs = tr.slice_pairs(0)
    hosts = tr.aips[:8]
    for k in (2, 300):
        o = Recording(c=19, k=k, g=64, seg_len=8, partition=0, seed=3)   # every block of Eq. 9-10 non-empty
        o.seen = []
        parts = bench.oracle_step_parts(o, k, pairs, hosts, 2, advance=True)
        assert o.seen == [k, k]
        assert parts["n_pairs"] == len(pairs) and parts["n_hosts"] == len(hosts)
        assert all(parts[x] >= 0 for x in ("slide", "ingest", "census", "n0", "hosts"))
        full = bench.full_step_s(parts, 10 * len(pairs), 100)
        # the full slice scales SetAT by 10 and the host loop by 100 / 8
        expect = (parts["slide"] + 10 * parts["ingest"] + parts["census"] + parts["n0"] + parts["hosts"] * 100 / 8)
        assert abs(full - expect) <= 1e-12 * max(1.0, expect)


def test_both_arms_print_the_same_config():
    a = _args("--k", "30")
    c1 = bench.make_config(a, 1 << 20, 1)
    c2 = bench.make_config(a, 1 << 20, 1)
    assert c1 == c2 and c1["k"] == 30 and c1["parallelism"] == "single"
    assert bench.make_config(a, 1 << 20, 4)["parallelism"] == "replicas"


def test_host_cpu_reports_threads_and_model():
    cpu = bench.host_cpu()
    assert cpu["nproc"] >= 1 and isinstance(cpu["model"], str) and cpu["model"]
