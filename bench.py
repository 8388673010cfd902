"""Benchmark of the VATE hot path on B300 (one JSON line on stdout).

Workload -- plain VATE at the 40 Gb/s shape: 2^20 hosts, 5,000,000 packets
per 1-second slice (64/576/1500 B mix, ~40 Gb/s), window k = 10, pool of 2^26
ATs, g = 4096 VATs per host in 32-AT segments.  One step is one slice of the
whole hot path through the C ABI:

    vate_ingest(5M pairs, slice s)   slide the window (BACT^0 + 1, PreserveAT on
                                     2 blocks) then SetAT for every pair
    vate_close_slice(s)              pool census (Z_p)
    vate_estimate(2^20 hosts, k'=k)  gather + CheckAT over 4096 VATs per host,
                                     Eq. 11 in FP32

Inputs are synthetic (traffic.DeviceTraffic), generated on the device before
timing, one distinct slice per step.  L2 is flushed (256 MiB write) before
every timed step, outside the step's CUDA-event window.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent monitor on its own GPU (replicas:
a VATE pool is shared by all its hosts, so one monitor does not split without
an exchange step); value = packets of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mpkt/s AT ingest; slice-close p99 ms @1M aips; learned vs plain mean rel. err"

C, K_WIN, G = 26, 10, 4096


def workload_name(args, n_h):
    """The workload as run: the 40 Gb/s traffic shape with this run's hosts,
    packets per slice, window and segment length."""
    return ("plain VATE at 40 Gb/s shape: {:,} aips, {:,} pkts per 1 s slice, k={}, AT pool 2^26, virtual vector "
            "4,096 ({}-AT segments), Zipf(1.05), 0.1% super-spreaders".format(n_h, args.pkts, args.k, args.seg_len))


def use_index(args) -> bool:
    """The close goes through the host list's index (vate_hostset) when asked
    and the pool is one the index serves: byte ATs, segments of 1 to 8 ATs."""
    return args.close == "index" and args.seg_len in (1, 2, 4, 8) and not args.at_bits and args.k <= 63


def make_config(args, n_h, world):
    """The `config` of both arms' JSON lines (the same dict in each)."""
    from traffic import MEAN_PKT_BYTES
    at_width = args.at_bits or (8 if args.k <= 63 else 16)
    pool_mib = ((1 << C) // (32 // args.at_bits) * 4 if args.at_bits else (1 << C) * at_width // 8) / 2**20
    return {"workload": workload_name(args, n_h), "aips": n_h, "pkts_per_slice": args.pkts,
            "k": args.k, "kprime": args.k, "log2_pool": C, "g": G, "seg_len": args.seg_len,
            "partition": args.partition, "at_bits": at_width,
            "link_gbps_equivalent": round(args.pkts * MEAN_PKT_BYTES * 8 / 1e9, 2),
            "l2": "flushed before every timed step (256 MiB write, outside the step events); the %.0f MiB AT pool "
                  "is state kept from slice to slice and its kernels mark it L2-persisting" % pool_mib
            if not args.no_flush else "not flushed",
            "parallelism": "replicas" if world > 1 else "single"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=295)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--close", default="index", choices=["index", "gather"],
                    help="index: the estimates of the fixed host list through its prebuilt index of VAT positions "
                         "(vate_hostset, seg_len 1-8); gather: the per-host gather (vate_estimate)")
    ap.add_argument("--seg-len", type=int, default=1,
                    help="VATs per pool segment: 1 is the paper's random H (the default; with --close index its "
                         "close of 2^20 hosts takes ~4.4 ms); with --close gather 2 is the smallest L that meets the "
                         "10 ms close target (--workload placement)")
    ap.add_argument("--partition", type=int, default=0)
    ap.add_argument("--k", type=int, default=K_WIN,
                    help="window in slices (the 40 Gb/s workload uses 10; the paper's long window is 300)")
    ap.add_argument("--at-bits", type=int, default=0,
                    help="0: one byte per AT; b: the packed layout with b-bit fields (memory against speed)")
    ap.add_argument("--aips", type=int, default=1 << 20, help="hosts estimated per slice")
    ap.add_argument("--pkts", type=int, default=5_000_000, help="packets per slice")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--group-modes", default="plain,graph,graph_tuned",
                    help="monitors64: the step forms to time (plain launch, graph, graph after the autotuner)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-estimator train/evaluate run")
    ap.add_argument("--workload", default="link40g",
                    choices=["link40g", "monitors64", "serving", "pt", "learned-kernels", "probes", "ingest-mix",
                             "placement", "close-kernels"],
                    help="link40g: the headline single-monitor workload; monitors64: 64 independent monitors "
                         "advanced together (vate_group, CUDA graph per slice); learned-kernels: the learned "
                         "estimator's kernels timed one by one at 2^20 hosts; probes: random 32-byte sector "
                         "reads against the working-set size; ingest-mix: vate_ingest of a 40 Gb/s slice "
                         "against uniform random pairs and against the slice's distinct pairs; placement: "
                         "gather time, close latency and accuracy against exact window counts for segment "
                         "lengths L = 1 (the paper's random H) to 64 at the 40 Gb/s shape")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; no data-path collective)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.samples, self.proc, self.t_on, self.t_off = [], None, None, None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", gpu_id], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def mark_on(self):
        self.t_on = time.perf_counter()

    def mark_off(self):
        self.t_off = time.perf_counter()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for t, line in self.samples:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((t, parts))
        inside = [r for t, r in rows if self.t_on is not None and self.t_on - 0.15 <= t <= (self.t_off or t) + 0.15]
        use = inside if inside else rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in use if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(use[0][2]),
                "power_w_max": max((num(r[3]) or 0.0) for r in use), "reasons": reasons,
                "samples": len(use), "samples_in_timed_region": len(inside)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def code_of(text: str) -> str:
    """C/CUDA source without its comments and with whitespace collapsed: what
    the compiler sees, so that a comment edit leaves a kernel's checksum alone.
    (Enough for these sources: no string literal in them holds a comment
    marker.)"""
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


TRAFFIC_SOURCES = {                      # the sources each committed ncu traffic figure depends on
    "hs_tile_kernel": ("vate_hostset_pass.cuh", "vate_device.cuh", "vate_device_ops.cuh"),
}
DEFAULT_TRAFFIC_SOURCES = ("vate_kernels.cu", "vate_device.cuh", "vate_device_ops.cuh")


def traffic_sha(kernel: str = "") -> str:
    """Checksum of the code (comments aside) of the sources a committed ncu
    traffic figure of `kernel` depends on."""
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES.get(kernel.split("@")[0], DEFAULT_TRAFFIC_SOURCES):
        with open(os.path.join(ROOT, "paper_1812_00282_b300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_of(fh.read()).encode())
    return h.hexdigest()[:16]


def committed_traffic(kernel: str):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(kernel)
    if not e or e.get("source_sha") != traffic_sha(kernel):
        return None
    return e.get("dram_bytes_per_launch")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


PROBE_UNROLL = (1, 2, 4, 8)
PROBE_BLOCKS = (2, 4, 8, 16, 32)


def best_of(torch, fn, reps=5, warm=2):
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(warm):
        fn()
    best = float("inf")
    for _ in range(reps):
        ev[0].record()
        fn()
        ev[1].record()
        torch.cuda.synchronize()
        best = min(best, ev[0].elapsed_time(ev[1]))
    return best


def probe_peaks(torch, pool_bytes: int, sweep=True):
    """Ceilings of the three access patterns on a pool-sized buffer (L2-resident
    at 64 MiB), each the fastest over accesses in flight per thread (1, 2, 4, 8)
    x blocks of 256 threads per SM (2..32): random 32-byte sector reads (the
    gather), random byte stores (the ingest) and one coalesced read of the
    buffer (the census).  Rates in GB/s (reads) and G stores/s."""
    from paper_1812_00282_b300 import probe
    buf = torch.zeros(pool_bytes, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    n_sec, n_wr, passes = 1 << 27, 1 << 26, 16
    shapes = [(u, b) for u in PROBE_UNROLL for b in PROBE_BLOCKS] if sweep else [(4, 8)]
    best = {"sector_read": (0.0, None), "byte_store": (0.0, None), "stream_read": (0.0, None)}
    for u, b in shapes:
        r = 32 * n_sec / best_of(torch, lambda: probe.sector_read(buf, n_sec, sink, u, b)) / 1e6
        w = n_wr / best_of(torch, lambda: probe.byte_write(buf, n_wr, u, b)) / 1e6

        def stream():
            for _ in range(passes):
                probe.stream_read(buf, sink, u, b)
        st = passes * pool_bytes / best_of(torch, stream) / 1e6
        for key, val in (("sector_read", r), ("byte_store", w), ("stream_read", st)):
            if val > best[key][0]:
                best[key] = (val, {"in_flight": u, "blocks_per_sm": b})
    del buf
    return {"l2_sector_read_gbs": best["sector_read"][0], "sector_read_shape": best["sector_read"][1],
            "l2_byte_store_gps": best["byte_store"][0], "byte_store_shape": best["byte_store"][1],
            "l2_stream_read_gbs": best["stream_read"][0], "stream_read_shape": best["stream_read"][1],
            "buffer_mib": pool_bytes >> 20, "shapes_tried": len(shapes)}


def accuracy_at_closes(torch, V, dt, hosts, args, first_slice, n_closes=3):
    """Mean relative error |max(est, 0) - n| / n of every host's Eq. 11 estimate
    against its exact window cardinality n (distinct (aip, bip) keys of the
    last k slices, sort-unique on the device), over hosts with n >= 1 and
    n >= 100, pooled over n_closes closes after a full window: for this run's
    segment length and, on the same slices, for L = 1 (the paper's random H)."""
    import collections
    from paper_1812_00282_b300.learned import exact_window_counts
    k = args.k
    lens = [args.seg_len] + ([1] if args.seg_len != 1 else [])
    hs = [V.Vate(C, k, G, L, args.partition, seed=0xACC, at_bits=args.at_bits if L == args.seg_len else 0)
          for L in lens]
    out = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
    hkey = hosts.to(torch.int64) & 0xFFFFFFFF
    err = {L: {1: [0.0, 0], 100: [0.0, 0]} for L in lens}
    window = collections.deque(maxlen=k)
    for i in range(k + n_closes - 1):
        s = first_slice + i
        p = dt.slice_pairs(s)
        window.append(p)
        for h in hs:
            h.ingest(p, s)
        if i < k - 1:
            continue
        uh, cnt = exact_window_counts(window)
        pos = torch.searchsorted(uh, hkey).clamp_(max=uh.numel() - 1)
        n = torch.where(uh[pos] == hkey, cnt[pos], torch.zeros_like(cnt[pos])).to(torch.float64)
        for L, h in zip(lens, hs):
            h.close_slice(s)
            h.estimate(hosts, k, out)
            e = torch.clamp(out.to(torch.float64), min=0.0)
            for lo in (1, 100):
                m = n >= lo
                err[L][lo][0] += float((torch.abs(e[m] - n[m]) / n[m]).sum().item())
                err[L][lo][1] += int(m.sum().item())
    for h in hs:
        h.close()
    res = {"closes": n_closes, "how": "|max(est, 0) - n| / n against exact window counts (sort-unique on the "
                                      "device), every host with n >= 1 (n >= 100), pooled over the closes"}
    for L in lens:
        key = "seg_len_%d" % L + (" (this run)" if L == args.seg_len else " (the paper's random H)")
        res[key] = {"mre_n>=1": round(err[L][1][0] / max(1, err[L][1][1]), 5), "hosts_n>=1": err[L][1][1],
                    "mre_n>=100": round(err[L][100][0] / max(1, err[L][100][1]), 5), "hosts_n>=100": err[L][100][1]}
    return res


def close_latency_loop(torch, mon, dt, estimate, first_slice, n_hosts, flush, no_flush, n=200):
    """Slice-close latency over n closes in a loop of their own (independent of
    --steps): each close follows the ingest of a fresh slice (generated and
    ingested before the close's events, L2 flushed before the ingest) and is
    timed from the vate_close_slice enqueue to the completion of vate_estimate
    for every host (census, gather, Eq. 11)."""
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    for i in range(n):
        s = first_slice + i
        p = dt.slice_pairs(s)
        if not no_flush:
            flush.fill_(s & 0xFF)
        mon.ingest(p, s)
        e0[i].record()
        mon.close_slice(s)
        estimate()
        e1[i].record()
        del p
    torch.cuda.synchronize()
    ms = [e0[i].elapsed_time(e1[i]) for i in range(n)]
    return {"closes": n, "hosts": int(n_hosts), "p50_ms": round(float(np.percentile(ms, 50)), 4),
            "p99_ms": round(float(np.percentile(ms, 99)), 4), "max_ms": round(max(ms), 4),
            "how": "a loop of its own: every close after a fresh slice's ingest, from the vate_close_slice enqueue "
                   "to the completion of the estimates of every host"}


def run_ours(args, rank, world, local):
    import torch
    import paper_1812_00282_b300 as V
    from traffic import LINK40G, MEAN_PKT_BYTES, DeviceTraffic, Traffic
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    props = torch.cuda.get_device_properties(dev)
    K, W = args.steps, args.warmup
    tr = Traffic(LINK40G, pkts_per_slice=args.pkts)
    dt = DeviceTraffic(tr, device=dev)
    pairs = [dt.slice_pairs(s) for s in range(W + K)]
    hosts = dt.hosts()[: args.aips].contiguous()
    n_h = hosts.numel()
    out = torch.empty(n_h, dtype=torch.float32, device=dev)
    flags = torch.empty(n_h, dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()

    peaks = probe_peaks(torch, 1 << C)
    mon = V.Vate(C, args.k, G, args.seg_len, args.partition, seed=0xC2 + rank, at_bits=args.at_bits,
                 options=V.VATE_OPT_PERSIST_L2)
    index = None
    if use_index(args):
        # the host list's index of VAT positions: built once (positions depend only on the
        # monitor's parameters), outside the timed steps
        torch.cuda.synchronize()
        tb = time.perf_counter()
        hs = V.vate_hostset_create(mon.h, hosts)
        torch.cuda.synchronize()
        ib, _, regions = V.vate_hostset_info(hs)
        index = {"build_s": round(time.perf_counter() - tb, 3), "bytes": ib, "regions": regions,
                 "entries_bytes": ib - 4 * (regions + 1) - (1 << C) // 8 - 4 * n_h}

        def estimate():
            V.vate_estimate_hostset(mon.h, hs, args.k, out, flags)
    else:
        def estimate():
            mon.estimate(hosts, args.k, out, flags)

    def step(s):
        mon.ingest(pairs[s], s)
        mon.close_slice(s)
        estimate()

    for s in range(W):
        if not args.no_flush:
            flush.fill_(s & 0xFF)
        step(s)
    torch.cuda.synchronize()

    mk = lambda: [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e0, e1, e2, e3 = mk(), mk(), mk(), mk()
    uuid = "GPU-" + str(props.uuid) if hasattr(props, "uuid") else str(local)
    clocks = ClockSampler(uuid)
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    if index:
        V.vate_hostset_time_passes(hs, K)       # the index pass's own duration in each timed step
    launches0 = V.vate_launch_count()
    clocks.mark_on()
    t0 = time.perf_counter()
    for i in range(K):
        s = W + i
        if not args.no_flush:
            flush.fill_(s & 0xFF)
        e0[i].record()
        mon.ingest(pairs[s], s)
        e1[i].record()
        mon.close_slice(s)
        e2[i].record()
        estimate()
        e3[i].record()
    torch.cuda.synchronize()
    barrier(world)
    t1 = time.perf_counter()
    clocks.mark_off()
    launches = V.vate_launch_count() - launches0
    clock_info = clocks.stop()
    pass_ms = None
    if index:
        pass_ms = V.vate_hostset_pass_times(hs, K)
        V.vate_hostset_time_passes(hs, 0)
    close_loop = close_latency_loop(torch, mon, dt, estimate, W + K, n_h, flush, args.no_flush, n=max(200, K))
    accuracy = accuracy_at_closes(torch, V, dt, hosts, args, W + K + max(200, K)) if rank == 0 else None

    step_ms = [e0[i].elapsed_time(e3[i]) for i in range(K)]
    ingest_ms = [e0[i].elapsed_time(e1[i]) for i in range(K)]
    census_ms = [e1[i].elapsed_time(e2[i]) for i in range(K)]
    gather_ms = [e2[i].elapsed_time(e3[i]) for i in range(K)]
    close_ms = [e1[i].elapsed_time(e3[i]) for i in range(K)]
    dev_ms = sum(step_ms)
    dev_ms_max = max_over_ranks(dev_ms, world)
    total_pkts = sum_over_ranks(float(K * args.pkts), world)
    value = total_pkts / dev_ms_max / 1e3       # packets per ms / 1e3 = Mpkt/s

    # roofline of the dominant kernel: the gather.  Its unit of work is one
    # random segment read, which moves whole 32-byte L2 sectors: g / L segments
    # per host, ceil(L x AT bytes / 32) sectors each (L <= 32 byte ATs: one)
    gather_avg = statistics.mean(gather_ms)
    atb = 1 if args.k <= 63 else 2                            # bytes per AT
    vat_bytes = n_h * G * atb                                 # the VATs themselves
    if args.at_bits:
        vat_bytes = n_h * G * args.at_bits // 8                  # the packed fields the VATs occupy
    seg_sectors = max(1, (args.seg_len * atb + 31) // 32)
    sectors = n_h * (G // args.seg_len) * seg_sectors
    gkernel = ("gather_seg_kernel" if args.seg_len * atb in (2, 4, 8) else
               "gather_vec_kernel" if args.seg_len * atb >= 16 else "gather_scalar_kernel")
    # the committed ncu figures are for the 40 Gb/s workload's shape (any L, either close path)
    default_shape = (args.k == K_WIN and not args.at_bits and args.partition == 0
                     and n_h == 1 << 20 and args.pkts == 5_000_000)
    ekernel = "hs_tile_kernel" if index else gkernel
    traffic = committed_traffic("%s@L%d" % (ekernel, args.seg_len)) if default_shape else None
    ingest_avg = statistics.mean(ingest_ms)
    mp = measured_peaks()
    hbm = mp.get("hbm_gbs", 6400.0)
    at_width = args.at_bits or (8 if args.k <= 63 else 16)                # bits per AT as stored
    pool_mib = ((1 << C) // (32 // args.at_bits) * 4 if args.at_bits else (1 << C) * at_width // 8) / 2**20
    sector_peak = peaks["l2_sector_read_gbs"] / 32.0           # G sectors/s
    achieved_sectors = sectors / gather_avg / 1e6              # G sectors/s
    roofline_note = ("the %.0f MiB pool is state kept in L2 (persisting window); the gather reads it in random "
                     "32-byte sectors, %d per host (g / L segments of %d sector(s)), so its bound is the L2's random-"
                     "sector rate, measured by the same access pattern on a 64 MiB buffer; traffic = DRAM bytes "
                     "of one launch (ncu, profiles/traffic.json) for the default shape, null once the kernel "
                     "sources change" % (pool_mib, (G // args.seg_len) * seg_sectors, seg_sectors))
    if args.at_bits:
        roofline_note += "; packed fields: a segment's words may span more sectors than counted here"

    if index:
        # the index pass streams the index once from HBM (far above L2): its bound is HBM bandwidth.
        # Timed: the pass itself (CUDA events the library records around it in every timed step), and
        # beside it the whole estimate call (the pool's CheckAT bitmap, the index pass, Eq. 11).
        ib = index["entries_bytes"]
        pass_avg = statistics.mean(pass_ms) if pass_ms else gather_avg
        achieved = ib / pass_avg / 1e6                            # GB/s
        call_achieved = ib / gather_avg / 1e6
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(achieved / hbm, 3), "traffic": traffic, "kernel": "hs_tile_kernel",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "algorithmic": "the host list's index streamed once per close: %d bytes (one 21-bit entry per "
                                   "segment of every host, %d segments, six to 16 bytes, in rows of 32-cell "
                                   "tiles whose columns are padded to the tile's largest cell, a 4-byte host "
                                   "per cell and a 4-byte first row per tile), over the pass's mean duration in "
                                   "the timed steps (%d launches, CUDA events on its stream)"
                                   % (ib, n_h * (G // args.seg_len), len(pass_ms or [])),
                    "pass_ms": round(pass_avg, 4),
                    "estimate_call": {"ms": round(gather_avg, 4), "achieved": round(call_achieved, 1),
                                      "frac": round(call_achieved / hbm, 3),
                                      "note": "the whole call, which also writes the pool's CheckAT bitmap (%d "
                                              "bytes) and evaluates Eq. 11" % ((1 << C) // 8)},
                    "vs_gather": {"sectors_equivalent": sectors,
                                  "equivalent_gsector_s": round(achieved_sectors, 1),
                                  "sector_probe": round(sector_peak, 2),
                                  "note": "the per-host gather reads the same VATs as %d random 32-byte sectors, "
                                          "bound by the SMs' sector rate (the probe); the index pass gives the "
                                          "same counts at %.2f times that rate"
                                          % (sectors, achieved_sectors / sector_peak)},
                    "note": "index built once for the fixed host list in %.3f s (%.2f GB, %d pool regions), outside "
                            "the timed steps; traffic = DRAM bytes of one launch of the index pass (ncu, "
                            "profiles/traffic.json), null once the kernel sources change"
                            % (index["build_s"], index["bytes"] / 1e9, index["regions"])}
    else:
        roofline = {"bound": "l2_sector_rate", "achieved": round(achieved_sectors, 2),
                     "peak": round(sector_peak, 2), "unit": "Gsector/s",
                     "frac": round(achieved_sectors / sector_peak, 3), "traffic": traffic, "kernel": gkernel,
                     "peak_source": "random 32-B sector reads from a 64 MiB L2-resident buffer, two threads per "
                                    "sector, measured in this run (vate_probe_sector_read, fastest of %d launch "
                                    "shapes: %s; %.1f GB/s); no L2 figure in MEASURED_PEAKS.json"
                                    % (peaks["shapes_tried"], peaks["sector_read_shape"],
                                       peaks["l2_sector_read_gbs"]),
                     "algorithmic": "aips x g / L segment reads of %d sector(s) per launch (%d sectors); the VATs "
                                    "themselves are %d bytes" % (seg_sectors, sectors, vat_bytes),
                     "vs_hbm": {"achieved_gbs": round(vat_bytes / gather_avg / 1e6, 1), "peak": hbm,
                                "frac": round(vat_bytes / gather_avg / 1e6 / hbm, 3),
                                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured); VAT bytes per launch / "
                                               "launch time"},
                     "note": roofline_note}

    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpkt/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": round(dev_ms_max / K, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u%d" % at_width if not args.at_bits else "%d-bit fields in u32 words" % args.at_bits,
        "data": "synthetic",
        "config": make_config(args, n_h, world),
        "close_p50_ms": close_loop["p50_ms"],
        "close_p99_ms": close_loop["p99_ms"],
        "close_latency": {**close_loop, "in_timed_steps": {"p50_ms": round(float(np.percentile(close_ms, 50)), 4),
                                                           "max_ms": round(max(close_ms), 4), "closes": K}},
        "accuracy": accuracy,
        "ingest_mpkts": round(args.pkts / ingest_avg / 1e3, 1),
        "close_path": ("index (vate_estimate_hostset)" if index else "gather (vate_estimate)"),
        "kernels_ms": {"ingest+preserve": round(ingest_avg, 4), "census": round(statistics.mean(census_ms), 4),
                       "estimate": round(gather_avg, 4)},
        "roofline": roofline,
        "roofline_ingest": {"bound": "l2_random_store", "achieved": round(args.pkts / ingest_avg / 1e6, 2),
                            "peak": round(peaks["l2_byte_store_gps"], 2), "unit": "Gstore/s",
                            "frac": round(args.pkts / ingest_avg / 1e6 / peaks["l2_byte_store_gps"], 3),
                            "note": ("one %s per pair against random 1-byte stores into a 64 MiB buffer (fastest of "
                                     "%d launch shapes: %s); time includes the slide's PreserveAT"
                                     % ("1-byte SetAT store" if at_width == 8 and not args.at_bits else
                                        "2-byte SetAT store" if not args.at_bits else
                                        "SetAT of a %d-bit field (atomicAnd + atomicOr)" % args.at_bits,
                                        peaks["shapes_tried"], peaks["byte_store_shape"]))},
        "roofline_census": {"bound": "l2_stream", "achieved": round(pool_mib * 2**20 / statistics.mean(census_ms)
                                                                     / 1e6, 1),
                            "peak": round(peaks["l2_stream_read_gbs"], 1), "unit": "GB/s",
                            "frac": round(pool_mib * 2**20 / statistics.mean(census_ms) / 1e6
                                          / peaks["l2_stream_read_gbs"], 3),
                            "note": "the pool read once per close against one coalesced read of a 64 MiB buffer "
                                    "(vate_probe_stream_read, fastest of %d launch shapes: %s); time includes the "
                                    "census's launch and its publication of the 2k + 1 counters"
                                    % (peaks["shapes_tried"], peaks["stream_read_shape"])},
        "gpu_launches": int(launches),
        "clocks": clock_info,
        "wall_bracket_s": round(t1 - t0, 4),
        "device": props.name,
    }
    if index:
        V.vate_hostset_destroy(hs)
        result["index"] = index
    mon.close()
    del pairs
    torch.cuda.empty_cache()

    if not args.no_e2e:
        result["e2e"] = run_e2e(args, V, torch, tr, dt, rank, world)
    if not args.no_learned and rank == 0:
        result["learned_vs_plain_mre"] = run_learned(V, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(tr, args, budget_s=20.0)
    return result


def run_learned(V, torch):
    """The learned-estimator workload: the 40 Gb/s traffic on a 2^24-AT pool,
    k = 10, g = 4096; MLP trained on 200 generated slices with exact labels,
    evaluated against the closed form on 100 held-out slices of another seed;
    at 32-AT segments (the configuration of the learned estimator), at 2-AT
    segments and at the paper's placement (L = 1, the 40 Gb/s workload's);
    plus the close-time cost of the learned estimate for 2^20 hosts at each:
    through the per-host gather (vate_estimate_learned) and, for L <= 8,
    through the host list's age index (vate_estimate_learned_hostset, built
    once; checked equal bit for bit here)."""
    from paper_1812_00282_b300 import learned
    from traffic import LINK40G, DeviceTraffic, Traffic
    out = {}
    dt = DeviceTraffic(Traffic(LINK40G))
    hosts = dt.hosts()
    est = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
    for L in (32, 2, 1):
        r = learned.run(V, seg_len=L)
        params = r.pop("params")
        # time both estimators on one closed slice of the same configuration
        mon = V.Vate(24, 10, 4096, L, 0, 0xC4)
        for s in range(11):
            mon.ingest(dt.slice_pairs(s), s)
        mon.close_slice(10)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        times = {}
        calls = [("plain", lambda: mon.estimate(hosts, 10, est)),
                 ("learned", lambda: V.vate_estimate_learned(mon.h, hosts, params, est))]
        ages = None
        if L <= 8:
            torch.cuda.synchronize()
            tb = time.perf_counter()
            ages = V.vate_hostset_create_ages(mon.h, hosts)
            torch.cuda.synchronize()
            r["age_index"] = {"build_s": round(time.perf_counter() - tb, 3), "bytes": V.vate_hostset_info(ages)[0]}
            est2 = torch.empty_like(est)
            V.vate_estimate_learned(mon.h, hosts, params, est)
            V.vate_estimate_learned_hostset(mon.h, ages, params, est2)
            torch.cuda.synchronize()
            r["age_index"]["equal_to_gather"] = bool(torch.equal(est.view(torch.int32), est2.view(torch.int32)))
            calls += [("plain_age_index", lambda: V.vate_estimate_hostset(mon.h, ages, 10, est)),
                      ("learned_age_index", lambda: V.vate_estimate_learned_hostset(mon.h, ages, params, est))]
        mhz = {}
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        uuid = "GPU-" + str(props.uuid) if hasattr(props, "uuid") else "0"
        for name, fn in calls:
            fn()
            # at least 0.3 s of calls, so that the SM clock under them is sampled too
            cs = ClockSampler(uuid)
            cs.mark_on()
            best, spent, reps = 1e9, 0.0, 0
            while reps < 5 or (spent < 300.0 and reps < 200):
                ev[0].record()
                fn()
                ev[1].record()
                torch.cuda.synchronize()
                t = ev[0].elapsed_time(ev[1])
                best, spent, reps = min(best, t), spent + t, reps + 1
            cs.mark_off()
            times[name] = round(best, 4)
            mhz[name] = cs.stop().get("sm_mhz")
        if ages is not None:
            V.vate_hostset_destroy(ages)
        mon.close()
        r["estimate_ms_2p20_hosts"] = times
        r["sm_mhz_during"] = mhz
        r["population"] = "hosts active in the window, sampled per slice; relative error |max(est,0) - n| / n"
        out["seg_len_%d" % L] = r
    return out


def run_e2e(args, V, torch, tr, dt, rank, world):
    """The same steps through the host-buffer entry points: every step copies
    its 5M pairs and 2^20 hosts from pinned memory and reads the estimates
    and flags back.  Reported: the steps issued back to back with one sync
    after the last (wall clock), beside the same steps synchronised one by one
    and the copies alone."""
    E, W = args.e2e_steps, 3
    nbuf = min(E + W, 8)
    host_pairs = [dt.slice_pairs(10_000 + s).cpu().pin_memory() for s in range(nbuf)]
    hosts = dt.hosts()[: args.aips].cpu().pin_memory()
    out = torch.empty(hosts.numel(), dtype=torch.float32).pin_memory()
    fl = torch.empty(hosts.numel(), dtype=torch.uint8).pin_memory()
    mon = V.Vate(C, args.k, G, args.seg_len, args.partition, seed=0xE2E + rank, at_bits=args.at_bits,
                 options=V.VATE_OPT_PERSIST_L2)
    st = torch.cuda.current_stream()
    hs = V.vate_hostset_create(mon.h, dt.hosts()[: args.aips].contiguous()) if use_index(args) else None

    def estimate_host(o, f):
        if hs is not None:                 # the fixed host list is in the index: only the results cross PCIe
            V.vate_estimate_hostset_host(mon.h, hs, args.k, o, f)
        else:
            V.vate_estimate_host(mon.h, hosts, args.k, o.numpy(), f.numpy())

    def step(s):
        V.vate_ingest_host(mon.h, host_pairs[s % nbuf], s)
        mon.close_slice(s)
        estimate_host(out, fl)
        st.synchronize()

    for s in range(W):
        step(s)
    barrier(world)
    t0 = time.perf_counter()
    for s in range(W, W + E):
        step(s)
    t1 = time.perf_counter()
    # the same steps issued back to back (a monitor streaming its slices): the
    # copies of slice s+1 overlap the gather of slice s; every step still reads
    # its estimates back (two host buffers in turn), one synchronisation at the end
    outs = [(out, fl), (torch.empty_like(out).pin_memory(), torch.empty_like(fl).pin_memory())]
    barrier(world)
    t2 = time.perf_counter()
    for s in range(W + E, W + 2 * E):
        o, f = outs[s & 1]
        V.vate_ingest_host(mon.h, host_pairs[s % nbuf], s)
        mon.close_slice(s)
        if hs is not None:                 # the copies out overlap the next slice's kernels
            V.vate_estimate_hostset_host_async(mon.h, hs, args.k, o, f)
        else:
            estimate_host(o, f)
    st.synchronize()
    if hs is not None:
        V.vate_hostset_wait(hs)
    t3 = time.perf_counter()
    if hs is not None:
        V.vate_hostset_destroy(hs)
    mon.close()
    # the ceiling of the back-to-back form: the same steps' input copies alone
    # (pairs in 2^20-pair chunks and the host list, from the same pinned
    # buffers, back to back on one stream) and their estimates and flags back
    # on another, with no kernel
    chunk = 1 << 20
    d_pairs = [torch.empty((chunk, 2), dtype=torch.int32, device="cuda") for _ in range(2)]
    d_hosts = torch.empty(hosts.shape, dtype=hosts.dtype, device="cuda")
    d_out, d_fl = torch.empty(out.shape, device="cuda"), torch.empty(fl.shape, dtype=fl.dtype, device="cuda")
    cs, ds = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    barrier(world)
    t4 = time.perf_counter()
    for s in range(W + E, W + 2 * E):
        hp, o, f = host_pairs[s % nbuf], *outs[s & 1]
        with torch.cuda.stream(cs):
            for j, off in enumerate(range(0, hp.shape[0], chunk)):
                n = min(chunk, hp.shape[0] - off)
                d_pairs[j & 1][:n].copy_(hp[off:off + n], non_blocking=True)
            if hs is None:
                d_hosts.copy_(hosts, non_blocking=True)
        with torch.cuda.stream(ds):
            o.copy_(d_out, non_blocking=True)
            f.copy_(d_fl, non_blocking=True)
    torch.cuda.synchronize()
    t5 = time.perf_counter()
    el = max_over_ranks(t1 - t0, world)
    el_pipe = max_over_ranks(t3 - t2, world)
    el_copy = max_over_ranks(t5 - t4, world)
    pk = sum_over_ranks(float(E * args.pkts), world)
    h2d = args.pkts * 8 + (hosts.numel() * 4 if hs is None else 0)
    return {"value": round(pk / el_pipe / 1e6, 3), "unit": "Mpkt/s", "steps": E,
            "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(hosts.numel() * 5),
            "path": ("vate_ingest_host / vate_close_slice / vate_estimate_hostset_host_async from pinned host "
                     "memory: every step's pairs copied in and its estimates and flags copied out, on a stream of "
                     "the hostset that overlaps the next slice's kernels (the fixed host list lives in the index; "
                     "vate_hostset_wait after the last step)" if hs is not None else
                     "vate_ingest_host / vate_close_slice / vate_estimate_host from pinned host memory, every step's "
                     "pairs and hosts copied in and its estimates and flags copied out") +
                    "; slices issued back to back as a monitor streaming them would, one synchronisation after the "
                    "last step",
            "synchronised": {"value": round(pk / el / 1e6, 3), "unit": "Mpkt/s",
                             "how": "the same steps with the blocking host entry point (vate_estimate_hostset_host "
                                    "with an index) and the stream synchronised after every step"},
            "copy_only": {"value": round(pk / el_copy / 1e6, 3), "unit": "Mpkt/s",
                          "h2d_gbs": round(E * h2d / el_copy / 1e9, 2),
                          "how": "the same steps' host-device copies alone, same pinned buffers, no kernel"},
            "frac_of_copy_only": round(el_copy / el_pipe, 3)}


# ---------------------------------------------------------------------------
# CPU oracle timings (the reference arm and the cpu_baseline field)
# ---------------------------------------------------------------------------
def host_cpu() -> dict:
    """Threads this process may use and the CPU model of the host."""
    try:
        n = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        n = os.cpu_count() or 1
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": n, "model": model}


def oracle_step_parts(o, k, pairs, hosts_sample, threads, advance=True):
    """One oracle step on a bounded sample, timed part by part (seconds): the
    slide and SetAT over `pairs` on one thread (the plain oracle's ingest); the
    census of the whole pool, the inactive count N0 of Z_p and the per-host
    gather + Eq. 11 of `hosts_sample` on `threads` OpenMP threads."""
    import oracle
    oracle.set_threads(1)
    t0 = time.perf_counter()
    if advance:
        o.advance()
    t1 = time.perf_counter()
    o.ingest(pairs)
    t2 = time.perf_counter()
    oracle.set_threads(threads)
    o.census()
    t3 = time.perf_counter()
    n0 = o.pool_inactive(k)
    t4 = time.perf_counter()
    o.estimate_hosts(hosts_sample, k, n0)
    t5 = time.perf_counter()
    oracle.set_threads(1)
    return {"slide": t1 - t0, "ingest": t2 - t1, "census": t3 - t2, "n0": t4 - t3, "hosts": t5 - t4,
            "n_pairs": len(pairs), "n_hosts": len(hosts_sample)}


def full_step_s(parts, pkts_total, n_hosts_total):
    """The measured parts scaled to one full slice: SetAT per pair times the
    slice's pairs, the per-host loop per host times the hosts estimated; the
    slide, census and N0 already cover the whole pool."""
    return (parts["slide"] + parts["ingest"] / max(1, parts["n_pairs"]) * pkts_total + parts["census"]
            + parts["n0"] + parts["hosts"] / max(1, parts["n_hosts"]) * n_hosts_total)


def measured_s(parts):
    return parts["slide"] + parts["ingest"] + parts["census"] + parts["n0"] + parts["hosts"]


def cpu_baseline(tr, args, budget_s=20.0):
    """The oracle as it stands on this host's cores (about budget_s of CPU work):
    three slices of the workload; on the last one SetAT over all the slice's
    pairs (one thread), the whole-pool census and N0, and the per-host loop on a
    seeded host sample, at one thread and at nproc threads, each scaled to a
    full slice of 2^20 hosts."""
    import oracle
    from traffic import mixed_hosts
    cpu = host_cpu()
    nt = cpu["nproc"]
    o = oracle.Oracle(c=C, k=args.k, g=G, seg_len=args.seg_len, partition=args.partition, seed=0xC2)
    n_h = min(args.aips, tr.spec.n_aips)
    for s in range(2):
        if s:
            o.advance()
        o.ingest(tr.slice_pairs(s))
    pairs = tr.slice_pairs(2)
    # per-host cost on one thread, to size the samples
    hs_all = mixed_hosts(tr, 262144)
    t0 = time.perf_counter()
    o.estimate_hosts(hs_all[:64], args.k, 1)
    per_host = max(1e-6, (time.perf_counter() - t0) / 64)
    n1 = int(max(64, min(len(hs_all), 4.0 / per_host)))               # ~4 s on one thread
    nn = int(max(64, min(len(hs_all), 8.0 * nt / per_host)))          # ~8 s on nproc threads
    p_n = oracle_step_parts(o, args.k, pairs, hs_all[:nn], nt, advance=True)
    p_1 = dict(p_n)
    oracle.set_threads(1)
    t0 = time.perf_counter()
    o.census()
    t1 = time.perf_counter()
    n0 = o.pool_inactive(args.k)
    t2 = time.perf_counter()
    o.estimate_hosts(hs_all[:n1], args.k, n0)
    t3 = time.perf_counter()
    p_1.update(census=t1 - t0, n0=t2 - t1, hosts=t3 - t2, n_hosts=n1)
    full_n = full_step_s(p_n, args.pkts, n_h)
    full_1 = full_step_s(p_1, args.pkts, n_h)
    spent = measured_s(p_n) + (t3 - t0)
    return {"value": round(args.pkts / full_n / 1e6, 5), "unit": "Mpkt/s", "cores": nt, "kind": "oracle",
            "cpu_model": cpu["model"], "nproc": nt,
            "value_1_thread": round(args.pkts / full_1 / 1e6, 5),
            "full_slice_s": {"nproc_threads": round(full_n, 3), "1_thread": round(full_1, 3)},
            "parts_s": {"slide_1t": round(p_n["slide"], 4), "setat_all_pairs_1t": round(p_n["ingest"], 3),
                        "census_nt": round(p_n["census"], 4), "census_1t": round(p_1["census"], 4),
                        "n0_nt": round(p_n["n0"], 4), "n0_1t": round(p_1["n0"], 4),
                        "hosts_nt": round(p_n["hosts"], 3), "hosts_1t": round(p_1["hosts"], 3)},
            "sample": "third slice of the workload: the slide and SetAT over all %d pairs on one thread (the plain "
                      "oracle's ingest), the census of the whole 2^26 pool and N0 at %d and at 1 thread(s), and "
                      "the gather + Eq. 11 of %d hosts at %d threads and %d hosts at 1 thread (every "
                      "super-spreader first, then a seeded sample), scaled to %d hosts; %.1f s of CPU work"
                      % (len(pairs), nt, nn, nt, n1, n_h, spent)}


def run_reference(args, rank, world):
    """The oracle as it stands, timed on this host's cores, on the same workload,
    metric and config as the device arm.  Each step is a bounded sample of a
    slice: the slide and SetAT over a contiguous sample of the slice's pairs on
    one thread, the whole-pool census and N0 and the gather + Eq. 11 of a host
    sample on nproc threads.  ms_per_step is the measured time of what ran;
    the value is the throughput of a full slice at the measured per-pair and
    per-host costs, and sample_scale the ratio of the two times."""
    from traffic import LINK40G, Traffic, mixed_hosts
    import oracle
    cpu = host_cpu()
    nt = cpu["nproc"]
    tr = Traffic(LINK40G, pkts_per_slice=args.pkts)
    total = args.steps + args.warmup
    per_step_budget = max(0.2, 100.0 / total)
    o = oracle.Oracle(c=C, k=args.k, g=G, seg_len=args.seg_len, partition=args.partition, seed=0xC2)
    n_h = min(args.aips, tr.spec.n_aips)
    base_pairs = tr.slice_pairs(0)
    hs_all = mixed_hosts(tr, 65536)
    # calibrate the sample so that one step costs about per_step_budget
    cal = oracle_step_parts(o, args.k, base_pairs[:200_000], hs_all[:8 * nt], nt, advance=False)
    per_pair = cal["ingest"] / cal["n_pairs"]
    per_host = cal["hosts"] / cal["n_hosts"]
    fixed = cal["census"] + cal["n0"] + 0.01
    room = max(0.05, per_step_budget - fixed)
    n_pk = int(max(10_000, min(args.pkts, 0.4 * room / per_pair)))
    n_hs = int(max(nt, min(len(hs_all), 0.6 * room / per_host)))
    hs = hs_all[:n_hs]
    full, meas, t_run = [], [], time.perf_counter()
    for s in range(total):
        off = (s * 104_729) % max(1, args.pkts - n_pk)
        parts = oracle_step_parts(o, args.k, base_pairs[off:off + n_pk], hs, nt, advance=True)
        if s >= args.warmup:
            full.append(full_step_s(parts, args.pkts, n_h))
            meas.append(measured_s(parts))
    wall = time.perf_counter() - t_run
    full_s = statistics.median(full)
    ms = 1e3 * statistics.mean(meas)
    value = args.pkts / full_s / 1e6
    return {"metric": METRIC, "impl": "reference", "value": round(value, 5), "unit": "Mpkt/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
            "sample_scale": round(full_s * 1e3 / ms, 3), "ms_per_full_slice": round(full_s * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
            "config": make_config(args, n_h, world),
            "wall_s": round(wall, 2),
            "cpu_baseline": {"value": round(value, 5), "unit": "Mpkt/s", "cores": nt, "kind": "oracle",
                             "cpu_model": cpu["model"], "nproc": nt,
                             "sample": "per step: the slide and SetAT over %d of the slice's %d pairs on one thread, "
                                       "the census of the whole 2^26 pool and N0 and the gather + Eq. 11 of %d "
                                       "hosts on %d threads (one uint16 per AT position, Eq. 11 in float64); "
                                       "ms_per_step is what ran, the value scales SetAT to all pairs and the "
                                       "per-host loop to %d hosts (sample_scale = full slice / sample time)"
                                       % (n_pk, args.pkts, n_hs, nt, n_h)},
            "e2e": {"value": round(value, 5), "unit": "Mpkt/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def monitors64_config(seed=0xC3):
    """64 independent streams: pool 2^U{20..25}, k in {5,10,30,60}, g = 2^U{9..13}
    (32-AT segments), rate log-uniform in [1e4, 5e6] packets per slice, hosts
    in proportion to the rate (1 per 12 packets, 1,024..65,536), Zipf(1.1)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x64]))
    mons = []
    for m in range(64):
        c = int(rng.integers(20, 26))
        k = int(rng.choice([5, 10, 30, 60]))
        g = 1 << int(rng.integers(9, 14))
        rate = int(np.exp(rng.uniform(np.log(1e4), np.log(5e6))))
        hosts = int(min(65536, max(1024, rate // 12)))
        mons.append(dict(c=c, k=k, g=g, rate=rate, hosts=hosts, seed=seed * 1000 + m))
    return mons


def run_monitors64(args):
    """Config 3 as a benchmark: one step = one slice of all 64 monitors (one
    persistent launch, replayed as a one-node CUDA graph).  Each slice's pairs
    are drawn into the same device buffers before the step (outside its CUDA
    events), as a capture card would fill them.  The monitors do not ask for
    persisting L2: the group's 0.58 GiB of pools are far above the L2, and a
    persisting window over them (a random eighth of the arena's lines kept)
    measured slower (2.72 against 2.55 ms per step)."""
    import torch
    import paper_1812_00282_b300 as V
    from traffic import DeviceTraffic, Traffic, TrafficSpec
    torch.cuda.set_device(0)
    K, W = args.steps, args.warmup
    mons = monitors64_config()
    dts, params = [], []
    for m in mons:
        spec = TrafficSpec(n_aips=m["hosts"], pkts_per_slice=m["rate"], zipf_s=1.1, seed=m["seed"])
        dts.append(DeviceTraffic(Traffic(spec)))
        params.append(V.make_params(m["c"], m["k"], m["g"], 32, 0, m["seed"]))
    grp = V.VateGroup(params)
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
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def fill(s):
        for i, d in enumerate(dts):
            pairs[int(po[i]):int(po[i + 1])].copy_(d.slice_pairs(s))
        flush.fill_(s & 0xFF)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    res = {}
    for mode in args.group_modes.split(","):
        grp.close()
        grp = V.VateGroup(params)
        if mode == "graph_tuned":
            fill(0)
            grp.step(pairs, PO, hosts, HO, KP, out, flags)
            tun = grp.autotune(pairs, PO, hosts, HO, KP, out, flags)
            res["tuning"] = tun.as_dict()
            grp.close()
            grp = V.VateGroup(params)
            V.vate_group_set_tuning(grp.g, tun)
        times = []
        for s in range(W + K):
            fill(s)
            a, b = ev(), ev()
            a.record()
            grp.step(pairs, PO, hosts, HO, KP, out, flags, graph=(mode != "plain"))
            b.record()
            torch.cuda.synchronize()
            if s >= W:
                times.append(a.elapsed_time(b))
        assert grp.status() == 0
        res[mode] = {"ms_per_step": round(statistics.mean(times), 4), "p99_ms": round(float(np.percentile(times, 99)), 4),
                     "mpkts": round(int(po[-1]) / statistics.mean(times) / 1e3, 1)}
    grp.close()
    best = min(res[m]["ms_per_step"] for m in args.group_modes.split(","))
    return {"metric": METRIC, "value": round(int(po[-1]) / best / 1e3, 3), "unit": "Mpkt/s", "n_gpus": 1,
            "steps": K, "warmup": W, "ms_per_step": best, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "batched monitors: 64 independent streams, pools 2^20-2^25, k in {5,10,30,60}, "
                                   "g 512-8192, rates log-uniform 1e4-5e6 pkts/slice",
                       "pkts_per_slice": int(po[-1]), "hosts_per_slice": int(ho[-1]),
                       "pool_bytes": int(sum(1 << m["c"] for m in mons)),
                       "l2": "flushed before every step (256 MiB write), outside the step events"},
            "modes": res}


def run_serving(args):
    """Config 5: monitors admitted by an 8 GB AT-memory budget, Poisson batches
    of 1k..1M pairs (mean 8 Mpkt/s, bursts to 30 Mpkt/s), 1 s slices, k = 10,
    learned estimator (trained here on the 2^24-pool configuration) with the
    closed form as fallback; real-time paced and all-at-once runs."""
    import torch
    import paper_1812_00282_b300 as V
    from paper_1812_00282_b300 import learned, serving
    torch.cuda.set_device(0)
    lr = learned.run(V, seg_len=serving.SEG_LEN, train_slices=60, eval_slices=20)   # the served monitors' placement
    model = lr.pop("params") if lr["accepted"] else None   # a model that fails its acceptance is not served
    paced = serving.run(V, duration=5.0, paced=True, model=model)
    flood = serving.run(V, duration=5.0, paced=False, model=model)
    # the same paced workload with the monitors at the 40 Gb/s workload's 2-AT segments (closed form)
    paced2 = serving.run(V, duration=5.0, paced=True, model=None, seg_len=2)
    return {"metric": METRIC, "value": flood["mpkts"], "unit": "Mpkt/s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": round(flood["wall_s"] * 1e3, 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": "serving loop: candidate monitors (pools 2^24..2^31, k=10, g=4096) admitted by an "
                                   "8 GB AT budget up to 16, Poisson batches 1k-1M pairs, mean 8 Mpkt/s, bursts to "
                                   "30 Mpkt/s, 1 s slices, learned estimator with closed-form fallback"},
            "seg_len": serving.SEG_LEN, "paced": paced, "flood": flood, "model_mre": lr["mre"],
            "model_accepted": lr["accepted"],
            "paced_seg_len_2": {kk: paced2[kk] for kk in ("mpkts", "offered_mpkts", "stats")}}


def run_pt(args):
    """Maintenance time per slide (the paper's PT, Sec. 5): asynchronous
    timestamps (PreserveAT on the two blocks whose ACT became 0 or k) against
    distance recorders (every recorder aged each slide), pools of 2^23..2^32
    counters, the 40 Gb/s traffic ingested between slides.  PT of a slide =
    CUDA-event time of vate_ingest with no pairs into the next slice.  The
    timestamps run with both partitions: Eq. 9-10 (2k-1 blocks of a and a
    last block of b < 2k-1) and the low-deviation one (blocks of a' or a'+1),
    whose per-slide PT should spread less (Sec. 4.1)."""
    import torch
    import paper_1812_00282_b300 as V
    from traffic import LINK40G, DeviceTraffic, Traffic
    torch.cuda.set_device(0)
    dt = DeviceTraffic(Traffic(LINK40G))
    empty = torch.zeros(0, 2, dtype=torch.int32, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    hbm = measured_peaks().get("hbm_gbs", 6400.0)
    rows = []
    arms = (("vate", V.VATE_COUNTER_AT, 0), ("vate_lowdev", V.VATE_COUNTER_AT, 1), ("vdre", V.VATE_COUNTER_DR, 0))
    for k in (10, 63, 300):                        # 300: the paper's k' (16-bit counters here)
        for c in range(23, 33):
            res = {"k": k, "log2_counters": c}
            for name, counter, part in arms:
                h = V.Vate(c, k, 1024, 32, part, 0xD7, counter=counter)
                times = []
                for s in range(2 * k + 4):
                    h.ingest(dt.slice_pairs(s % 40), s)
                    ev[0].record()
                    h.ingest(empty, s + 1)          # the slide into slice s+1: maintenance only
                    ev[1].record()
                    torch.cuda.synchronize()
                    if s >= 2:
                        times.append(ev[0].elapsed_time(ev[1]))
                h.close()
                res[name + "_pt_ms"] = round(statistics.mean(times), 4)
                res[name + "_pt_std_ms"] = round(statistics.pstdev(times), 4)
                res[name + "_pt_max_ms"] = round(max(times), 4)
            res["speedup"] = round(res["vdre_pt_ms"] / res["vate_pt_ms"], 1)
            # bytes a slide must read: the whole pool (VDRE) or the two maintained blocks (VATE)
            w = 1 if k <= 63 else 2                    # bytes per counter
            res["counter_bytes"] = w
            res["vdre_read_gbs"] = round(w * (1 << c) / res["vdre_pt_ms"] / 1e6, 1)
            res["vate_read_gbs"] = round(w * 2 * (1 << c) / (2 * k - 1) / res["vate_pt_ms"] / 1e6, 1)
            rows.append(res)
            torch.cuda.empty_cache()
    return {"workload": "maintenance time per slide (PT), VATE (both partitions) vs VDRE, 40 Gb/s traffic "
                        "between slides, g = 1024", "hbm_peak_gbs": hbm, "rows": rows}


def run_learned_kernels(args):
    """The learned estimator's kernels one by one at close, 2^20 hosts (and
    the per-age counts of vate_age_counts, which hold the same numbers): the
    40 Gb/s traffic on a 2^24-AT pool (k = 10, g = 4096, L = 2) after 12
    slices, a model of 2k + 2 = 22 inputs with weights from vate_mlp_init (the
    cost does not depend on them).  CUDA-event mean of 10 calls after 3
    warm-up calls."""
    import torch
    import paper_1812_00282_b300 as V
    from traffic import LINK40G, DeviceTraffic, Traffic
    torch.cuda.set_device(0)
    dt = DeviceTraffic(Traffic(LINK40G))
    k, c, g = 10, 24, 4096
    h = V.Vate(c, k, g, 2, 0, 7)
    for s in range(12):
        h.ingest(dt.slice_pairs(s), s)
    h.close_slice(11)
    hosts = dt.hosts()[: args.aips].contiguous()
    n, n_in = hosts.numel(), 2 * k + 2
    params = torch.empty(V.vate_mlp_param_count(n_in), dtype=torch.float32, device="cuda")
    V.vate_mlp_init(params, n_in, 3)
    x = torch.empty(n * n_in, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    fl = torch.empty(n, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ev[0].record()
        for _ in range(reps):
            fn()
        ev[1].record()
        torch.cuda.synchronize()
        return round(ev[0].elapsed_time(ev[1]) / reps, 4)

    ages = torch.empty(n * k, dtype=torch.int16, device="cuda")
    ms = {"age_counts": timed(lambda: V.vate_age_counts(h.h, hosts, ages)),
          "features": timed(lambda: V.vate_features(h.h, hosts, x)),
          "forward": timed(lambda: V.vate_mlp_forward(params, n_in, x.view(n, n_in), y)),
          "learned_estimate": timed(lambda: V.vate_estimate_learned(h.h, hosts, params, out, fl)),
          "plain_eq11_estimate": timed(lambda: h.estimate(hosts, k, out, fl))}
    h.close()
    # per-age counts with a longer window, k = 30 (shared-memory counters instead of bit planes)
    h30 = V.Vate(c, 30, g, 2, 0, 7)
    for s in range(12):
        h30.ingest(dt.slice_pairs(s), s)
    h30.close_slice(11)
    ages30 = torch.empty(n * 30, dtype=torch.int16, device="cuda")
    ms["age_counts_k30"] = timed(lambda: V.vate_age_counts(h30.h, hosts, ages30))
    h30.close()
    # the same hosts through their age index (vate_hostset_create_ages), at L = 1 and 2: per-age counts, A
    # and the learned close from one pass over the index, beside the per-host gathers
    for L in (1, 2):
        hl = V.Vate(c, k, g, L, 0, 7)
        for s in range(12):
            hl.ingest(dt.slice_pairs(s), s)
        hl.close_slice(11)
        ai = V.vate_hostset_create_ages(hl.h, hosts)
        ms["L%d" % L] = {
            "age_counts_gather": timed(lambda: V.vate_age_counts(hl.h, hosts, ages)),
            "age_counts_age_index": timed(lambda: V.vate_age_counts_hostset(hl.h, ai, ages)),
            "learned_gather": timed(lambda: V.vate_estimate_learned(hl.h, hosts, params, out, fl)),
            "learned_age_index": timed(lambda: V.vate_estimate_learned_hostset(hl.h, ai, params, out, fl)),
            "plain_age_index": timed(lambda: V.vate_estimate_hostset(hl.h, ai, k, out, fl)),
            "age_index_bytes": V.vate_hostset_info(ai)[0]}
        V.vate_hostset_destroy(ai)
        hl.close()
    return {"workload": "learned estimator kernels at close: %d hosts, 2^24-AT pool, k = 10, g = 4096 (L = 2, "
                        "and the age index at L = 1 and 2)" % n, "unit": "ms per call", "ms": ms}


def run_probes(args):
    """The three probe patterns (vate_probe_*) against the working-set size, 8 to
    256 MiB: where the L2 rates give way to the HBM ones.  Each figure is the
    fastest over accesses in flight per thread x blocks per SM (probe_peaks)."""
    import torch
    torch.cuda.set_device(0)
    out = {}
    for mib in (8, 16, 32, 64, 128, 256):
        p = probe_peaks(torch, mib << 20)
        out["%d MiB" % mib] = {"sector_read_gbs": round(p["l2_sector_read_gbs"], 1),
                               "sector_read_shape": p["sector_read_shape"],
                               "byte_store_gps": round(p["l2_byte_store_gps"], 2),
                               "byte_store_shape": p["byte_store_shape"],
                               "stream_read_gbs": round(p["l2_stream_read_gbs"], 1),
                               "stream_read_shape": p["stream_read_shape"]}
    return {"workload": "memory-system probes against the working-set size (best over 1-8 accesses in flight per "
                        "thread x 2-32 blocks of 256 threads per SM)", "rates": out}


def run_ingest_mix(args):
    """vate_ingest alone into a 2^26-AT pool (k = 10, g = 4096, L = 32), L2
    flushed before each launch: one 40 Gb/s slice (5M pairs with the traffic's
    repeats and heavy hosts), the same number of uniform random pairs, and the
    slice's distinct pairs only.  CUDA-event mean of 20 launches after 3."""
    import torch
    import paper_1812_00282_b300 as V
    from traffic import LINK40G, DeviceTraffic, Traffic
    torch.cuda.set_device(0)
    dt = DeviceTraffic(Traffic(LINK40G))
    h = V.Vate(C, 10, G, 32, 0, 7)
    pairs = dt.slice_pairs(5)
    n = pairs.shape[0]
    key = (pairs[:, 0].to(torch.int64) & 0xFFFFFFFF) << 32 | (pairs[:, 1].to(torch.int64) & 0xFFFFFFFF)
    uniq = torch.unique(key)
    distinct = torch.stack([uniq >> 32, uniq & 0xFFFFFFFF], 1)
    distinct = torch.where(distinct >= 2**31, distinct - 2**32, distinct).to(torch.int32).contiguous()
    gen = torch.Generator(device="cuda").manual_seed(1)
    uniform = torch.randint(-2**31, 2**31 - 1, (n, 2), generator=gen, device="cuda", dtype=torch.int32)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    h.ingest(pairs, 0)

    def timed(p, reps=20):
        for _ in range(3):
            V.vate_ingest(h.h, p, 0)
        tot = 0.0
        for r in range(reps):
            flush.fill_(r & 0xFF)
            torch.cuda.synchronize()
            ev[0].record()
            V.vate_ingest(h.h, p, 0)
            ev[1].record()
            torch.cuda.synchronize()
            tot += ev[0].elapsed_time(ev[1])
        return round(1000 * tot / reps, 1)

    res = {"slice_us": timed(pairs), "distinct_only_us": timed(distinct), "uniform_us": timed(uniform)}
    h.close()
    return {"workload": "vate_ingest alone, 2^26-AT pool, k = 10, g = 4096, L = 32, L2 flushed before each launch",
            "pairs": n, "distinct_pairs": int(uniq.numel()), "unit": "us per launch", "times": res}


def run_placement(args, seg_lens=(1, 4, 8, 16, 32, 64), n_slices=40):
    """The placement of a host's virtual ATs at the 40 Gb/s shape (2^26-AT pool,
    g = 4096, k = k' = 10, 5M pairs per slice, all 2^20 hosts estimated per
    close): for each segment length L, the gather + Eq. 11 time, the close
    latency (census + gather + Eq. 11) and the ingest time over the closes of
    slices k..n_slices-1, and the mean relative error |max(est, 0) - n| / n
    against the exact window cardinality n of every host active in the window
    (distinct (aip, bip) keys of the last k slices, sort-unique on the device),
    over n >= 1 and n >= 100, pooled over those closes.  L = 1 is the paper's
    fully random H (Sec. 4.1); larger L place L consecutive VATs of a host in
    one pool segment."""
    import collections
    import torch
    import paper_1812_00282_b300 as V
    from paper_1812_00282_b300.learned import exact_window_counts
    from traffic import LINK40G, DeviceTraffic, Traffic
    torch.cuda.set_device(0)
    k = args.k
    tr = Traffic(LINK40G, pkts_per_slice=args.pkts)
    dt = DeviceTraffic(tr)
    hosts = dt.hosts()
    hkey = hosts.to(torch.int64) & 0xFFFFFFFF
    n_h = hosts.numel()
    out = torch.empty(n_h, dtype=torch.float32, device="cuda")
    fl = torch.empty(n_h, dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    rows = {}
    for L in seg_lens:
        mon = V.Vate(C, k, G, L, 0, seed=0xC2, options=V.VATE_OPT_PERSIST_L2)
        window = collections.deque(maxlen=k)
        ing, cen, gat, clo = [], [], [], []
        err = {1: [0.0, 0], 100: [0.0, 0]}
        sat = 0
        for s in range(n_slices):
            p = dt.slice_pairs(s)
            window.append(p)
            flush.fill_(s & 0xFF)
            ev[0].record()
            mon.ingest(p, s)
            ev[1].record()
            mon.close_slice(s)
            ev[2].record()
            mon.estimate(hosts, k, out, fl)
            ev[3].record()
            torch.cuda.synchronize()
            if s < k:
                continue
            ing.append(ev[0].elapsed_time(ev[1]))
            cen.append(ev[1].elapsed_time(ev[2]))
            gat.append(ev[2].elapsed_time(ev[3]))
            clo.append(ev[1].elapsed_time(ev[3]))
            uh, cnt = exact_window_counts(window)
            pos = torch.searchsorted(uh, hkey).clamp_(max=uh.numel() - 1)
            n = torch.where(uh[pos] == hkey, cnt[pos], torch.zeros_like(cnt[pos])).to(torch.float64)
            e = torch.clamp(out.to(torch.float64), min=0.0)
            for lo in (1, 100):
                m = n >= lo
                err[lo][0] += float((torch.abs(e[m] - n[m]) / n[m]).sum().item())
                err[lo][1] += int(m.sum().item())
            sat += int(((fl & V.VATE_FLAG_SAT) != 0).sum().item())
        mon.close()
        rows["L=%d" % L] = {
            "gather_ms": round(statistics.mean(gat), 4), "census_ms": round(statistics.mean(cen), 4),
            "ingest_ms": round(statistics.mean(ing), 4),
            "close_p50_ms": round(float(np.percentile(clo, 50)), 4),
            "close_p99_ms": round(float(np.percentile(clo, 99)), 4),
            "mre_n>=1": round(err[1][0] / max(1, err[1][1]), 5), "hosts_n>=1": err[1][1],
            "mre_n>=100": round(err[100][0] / max(1, err[100][1]), 5), "hosts_n>=100": err[100][1],
            "saturated_estimates": sat}
    return {"workload": "VAT placement at the 40 Gb/s shape: 2^26-AT pool, g = 4096, k = k' = %d, %d pkts per slice, "
                        "all %d hosts estimated at each of %d closes (slices %d..%d)"
                        % (k, args.pkts, n_h, n_slices - k, k, n_slices - 1),
            "error": "mean of |max(est, 0) - n| / n over hosts active in the window, pooled over the closes; n = "
                     "exact distinct peers in the last k slices", "rows": rows}


def run_close_kernels(args):
    """The slice step's kernels one by one at the 40 Gb/s shape (this run's k,
    L and pool; 2^20 hosts): 12 slices of 5M pairs are ingested and closed,
    then each of 10 more slices is timed piece by piece with CUDA events --
    vate_ingest (slide + SetAT), vate_close_slice (census), vate_estimate
    (gather + Eq. 11) -- with L2 flushed before the ingest.  Small enough to
    run under ncu (about 0.6 GB on the device)."""
    import torch
    import paper_1812_00282_b300 as V
    from traffic import LINK40G, DeviceTraffic, Traffic
    torch.cuda.set_device(0)
    dt = DeviceTraffic(Traffic(LINK40G, pkts_per_slice=args.pkts))
    hosts = dt.hosts()[: args.aips].contiguous()
    mon = V.Vate(C, args.k, G, args.seg_len, args.partition, seed=0xC2, at_bits=args.at_bits,
                 options=V.VATE_OPT_PERSIST_L2)
    out = torch.empty(hosts.numel(), dtype=torch.float32, device="cuda")
    fl = torch.empty(hosts.numel(), dtype=torch.uint8, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    t = {"ingest": [], "census": [], "gather": []}
    for s in range(22):
        p = dt.slice_pairs(s)
        flush.fill_(s & 0xFF)
        ev[0].record()
        mon.ingest(p, s)
        ev[1].record()
        mon.close_slice(s)
        ev[2].record()
        mon.estimate(hosts, args.k, out, fl)
        ev[3].record()
        torch.cuda.synchronize()
        if s >= 12:
            t["ingest"].append(ev[0].elapsed_time(ev[1]))
            t["census"].append(ev[1].elapsed_time(ev[2]))
            t["gather"].append(ev[2].elapsed_time(ev[3]))
    mon.close()
    return {"workload": "slice step kernels at the 40 Gb/s shape: 2^26-AT pool, k = %d, g = 4096, L = %d, %d pairs, "
                        "%d hosts" % (args.k, args.seg_len, args.pkts, hosts.numel()),
            "unit": "ms (CUDA events, mean of 10 slices after 12)",
            "ms": {n: round(statistics.mean(v), 4) for n, v in t.items()}}


def main():
    args = parse()
    if args.workload == "close-kernels":
        print(json.dumps(run_close_kernels(args)), flush=True)
        return
    if args.workload == "placement":
        print(json.dumps(run_placement(args)), flush=True)
        return
    if args.workload == "ingest-mix":
        print(json.dumps(run_ingest_mix(args)), flush=True)
        return
    if args.workload == "probes":
        print(json.dumps(run_probes(args)), flush=True)
        return
    if args.workload == "learned-kernels":
        print(json.dumps(run_learned_kernels(args)), flush=True)
        return
    if args.workload == "pt":
        print(json.dumps(run_pt(args)), flush=True)
        return
    if args.workload == "serving":
        print(json.dumps(run_serving(args)), flush=True)
        return
    if args.workload == "monitors64":
        print(json.dumps(run_monitors64(args)), flush=True)
        return
    if args.impl == "reference":
        # rank 0 alone runs the CPU oracle; the other ranks exit without work
        rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    rank, world, local = dist_setup()
    res = run_ours(args, rank, world, local)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
