"""An oracle-backed stand-in for the library's shard entry points
(include/vate_shard.h), so that the orchestration in
paper_1812_00282_b300.sharded -- shard ranges, the two all-reduces, the call
order -- can run on CPU ranks.  Test infrastructure: every number comes from
the oracle.  Each stand-in shard runs a whole oracle pool and reports only
its own positions, which is what a shard of the library computes."""
import numpy as np
import torch

import oracle
from oracle import Oracle


class _Shard:
    def __init__(self, params, lo, hi):
        self.p = params
        self.lo, self.hi = lo, hi
        self.o = Oracle(c=params["c"], k=params["k"], g=params["g"], seg_len=params["L"],
                        partition=params["partition"], seed=params["seed"])
        self.slice = None

    def to_slice(self, s):
        if self.slice is not None:
            for _ in range(s - self.slice):
                self.o.advance()
        self.slice = s

    def active(self, hosts, kprime):
        o, k = self.o, self.p["k"]
        pool = o.pool()
        out = []
        for aip in hosts:
            n = 0
            for i in range(self.p["g"]):
                pid = o.h(int(aip), i)
                if self.lo <= pid < self.hi and oracle.check_at(int(pool[pid]), o.act_of(pid), k, kprime):
                    n += 1
            out.append(n)
        return out

    def census(self):
        o, twok = self.o, 2 * self.p["k"]
        pool = o.pool()
        hist = np.zeros(twok + 1, np.int64)
        for pid in range(self.lo, self.hi):
            v = int(pool[pid])
            hist[twok if v == twok else (o.act_of(pid) - v) % twok] += 1
        return hist


class FakeShardLib:
    def make_params(self, c, k, g, L=1, partition=0, seed=0, counter=0):
        assert counter == 0
        return {"c": c, "k": k, "g": g, "L": L, "partition": partition, "seed": seed}

    def vate_create_shard(self, params, lo, hi, stream=None):
        return _Shard(params, lo, hi)

    def vate_destroy(self, h):
        pass

    def vate_ingest(self, h, pairs, slice, stream=None):
        h.to_slice(slice)
        h.o.ingest(pairs.numpy().view(np.uint32).reshape(-1, 2))

    def vate_close_slice(self, h, slice, stream=None):
        h.to_slice(slice)

    def vate_active_counts(self, h, hosts, kprime, active, stream=None):
        active.copy_(torch.tensor(h.active(hosts.numpy().view(np.uint32), kprime), dtype=torch.int32))

    def vate_census(self, h, hist, stream=None):
        hist.copy_(torch.from_numpy(h.census()))

    def vate_estimate_from_counts(self, params, active, hist, kprime, out, flags=None, stream=None):
        P = 1 << params["c"]
        n0 = P - int(hist[:kprime].sum())
        for i, a in enumerate(active.tolist()):
            out[i] = oracle.estimate_from_counts(params["g"], P, n0, a)[0]
