"""Serving workload driver for vate_server (include/vate_server.h).

Monitors are offered to the server in turn and admitted while the device
memory budget allows.  Packet batches of uneven size (log-uniform 1k..1M
pairs) arrive as a Poisson process whose rate switches between a normal level
and bursts (a two-state Markov-modulated Poisson process: mean 8 Mpkt/s,
bursts to 30 Mpkt/s), each batch for one monitor; at every 1-second slice
boundary each monitor's slice is closed and its hosts estimated.  Arrivals
are either paced in real time (latency under the offered load) or all
released at once (capacity).  This module only schedules host-side requests;
the server does the work.
"""
from __future__ import annotations

import time
from dataclasses import dataclass
from typing import Dict, List

import numpy as np

# VATs per pool segment of the served monitors.  The monitors' pools (2^24 to
# 2^31 ATs) mostly live in HBM, and every monitor closes at the same slice
# boundary: with 2-AT segments each close of 65,536 hosts reads 2^27 random
# sectors, mostly from HBM, and the sixteen closes of a boundary queue behind
# one another (measured paced, closed form: close p50 12 ms, p99 22 ms); with
# 32-AT segments a close reads 16 times fewer (p50 0.9 ms, p99 1.4 ms).
SEG_LEN = 32


@dataclass
class Arrival:
    t: float          # seconds from the start
    mon: int          # index into the admitted monitors
    n: int            # pairs in the batch


def arrival_schedule(n_mons: int, duration: float, seed: int = 0xC5, mean_rate: float = 8e6,
                     burst_rate: float = 30e6, burst_share: float = 0.1, burst_len: float = 0.05,
                     batch_lo: float = 1e3, batch_hi: float = 1e6) -> List[Arrival]:
    """Batches over `duration` seconds.  The packet rate is `burst_rate` during
    bursts (exponential lengths, mean `burst_len`, a `burst_share` of the time)
    and otherwise the level that makes the mean `mean_rate`."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x5E]))
    normal_rate = (mean_rate - burst_share * burst_rate) / (1.0 - burst_share)
    mean_batch = (batch_hi - batch_lo) / np.log(batch_hi / batch_lo)
    mon_w = 1.0 / np.arange(1, n_mons + 1) ** 0.8
    mon_w /= mon_w.sum()
    out, t = [], 0.0
    burst = False
    switch = rng.exponential(burst_len * (1 - burst_share) / burst_share)
    while t < duration:
        rate = (burst_rate if burst else normal_rate) / mean_batch      # batches per second
        dt = rng.exponential(1.0 / rate)
        if t + dt >= switch:
            t = switch
            burst = not burst
            switch = t + rng.exponential(burst_len if burst else burst_len * (1 - burst_share) / burst_share)
            continue
        t += dt
        if t >= duration:
            break
        n = int(np.exp(rng.uniform(np.log(batch_lo), np.log(batch_hi))))
        out.append(Arrival(t, int(rng.choice(n_mons, p=mon_w)), n))
    return out


def run(V, duration: float = 5.0, budget_bytes: int = 8 << 30, max_monitors: int = 16, candidates: int = 24,
        paced: bool = True, model=None, model_log2_pool: int = 24, hosts_per_close: int = 65536,
        slots: int = 8, seed: int = 0xC5, seg_len: int = SEG_LEN) -> Dict:
    import torch
    from traffic import DeviceTraffic, Traffic, TrafficSpec
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xAD]))
    srv = V.vate_server_create(budget_bytes, slots=slots, slot_records=1 << 20)
    admitted, rejected, cs = [], 0, []
    for i in range(candidates):
        if len(admitted) >= max_monitors:
            break
        # every fourth candidate has the pool the learned model was trained for
        c = model_log2_pool if i % 4 == 0 else int(rng.integers(24, 32))
        try:
            mid = V.vate_server_admit(srv, V.make_params(c, 10, 4096, seg_len, 0, seed * 100 + i, options=V.VATE_OPT_PERSIST_L2))
        except V.VateError as e:
            if e.code != V.VATE_ENOMEM:
                raise
            rejected += 1
            continue
        admitted.append(mid)
        cs.append(c)
        if model is not None and c == model_log2_pool:
            V.vate_server_set_model(srv, mid, model)
    M = len(admitted)
    sched = arrival_schedule(M, duration, seed=seed)
    # each monitor's pairs, drawn on the device and kept in page-locked memory
    need = np.zeros(M, np.int64)
    for a in sched:
        need[a.mon] += a.n
    pools, hosts = [], []
    for m in range(M):
        spec = TrafficSpec(n_aips=1 << 16, pkts_per_slice=int(max(1, need[m])), zipf_s=1.1, seed=seed * 1000 + m)
        dt = DeviceTraffic(Traffic(spec))
        pools.append(dt.slice_pairs(0, n=int(max(1, need[m]))).cpu().pin_memory())
        hosts.append(dt.hosts()[:hosts_per_close].cpu().numpy().view(np.uint32).copy())
    outs = [np.empty(hosts_per_close, np.float32) for _ in range(M)]
    flags = [np.empty(hosts_per_close, np.uint8) for _ in range(M)]
    cursor = np.zeros(M, np.int64)
    tickets = []
    V.vate_server_get_stats(srv, reset=True)
    n_slices = int(np.ceil(duration))
    t0 = time.perf_counter()
    slice_now = 0
    for a in sched:
        s = int(a.t)
        while s > slice_now:                          # slice boundary: close every monitor
            for m in range(M):
                tickets.append(V.vate_server_submit_close(srv, admitted[m], slice_now, hosts[m], 10, outs[m],
                                                          flags[m]))
            slice_now += 1
        if paced:
            wait = a.t - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
        lo = int(cursor[a.mon])
        cursor[a.mon] += a.n
        tickets.append(V.vate_server_submit_ingest(srv, admitted[a.mon], pools[a.mon][lo:lo + a.n], s,
                                                   V.VATE_SUBMIT_PINNED))
    while slice_now < n_slices:
        for m in range(M):
            tickets.append(V.vate_server_submit_close(srv, admitted[m], slice_now, hosts[m], 10, outs[m], flags[m]))
        slice_now += 1
    for t in tickets:
        V.vate_server_wait(srv, t, 600000)
    wall = time.perf_counter() - t0
    st = V.vate_server_get_stats(srv).as_dict()
    V.vate_server_destroy(srv)
    pairs = int(sum(a.n for a in sched))
    return {"mode": "paced" if paced else "flood", "monitors_admitted": M, "monitors_rejected": rejected,
            "log2_pools": cs, "with_model": int(sum(1 for c in cs if model is not None and c == model_log2_pool)),
            "duration_s": duration, "batches": len(sched), "pairs": pairs, "wall_s": round(wall, 3),
            "mpkts": round(pairs / wall / 1e6, 2), "offered_mpkts": round(pairs / duration / 1e6, 2),
            "stats": st}
