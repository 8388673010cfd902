"""Seeded synthetic <aip, bip> traffic shaped like the paper's workloads.

This module only produces inputs.  It contains none of VATE's arithmetic (no
H/BH hashing, no AT values, no estimator) and serves both the CUDA path and
the CPU oracle, which receive the very same arrays.

The paper measures on CAIDA (10 Gb/s, 2015-02-19) and IPtas (40 Gb/s,
2017-10-23) traces (Sec. 5); neither is available here, so seeded synthetic
traffic stands in for them:

* the hosts of ANet are distinct random uint32 addresses;
* host popularity is Zipf(s) over a seeded permutation of the hosts;
* each host owns a pool of opposite hosts (bip) whose size is
  LogNormal(mu, sigma), capped, and a small fraction of "super-spreader"
  hosts -- the most popular ranks -- own log-uniform pools of 1e5..1e6 peers
  (the heavy tail of Sec. 5, where a few hosts exceed 5000 peers);
* every packet picks a host by popularity, then a peer uniformly from that
  host's pool.

Packet sizes (64/576/1500 B with weights 0.25/0.15/0.60, mean 1002.4 B) only
label a packet rate with a link rate; the method reads pairs.
"""
from __future__ import annotations

import dataclasses
from typing import Optional

import numpy as np

PKT_SIZES = (64, 576, 1500)
PKT_WEIGHTS = (0.25, 0.15, 0.60)
MEAN_PKT_BYTES = float(np.dot(PKT_SIZES, PKT_WEIGHTS))  # 1002.4 B


@dataclasses.dataclass(frozen=True)
class TrafficSpec:
    n_aips: int
    pkts_per_slice: int
    zipf_s: float
    lognorm_mu: float = 3.0
    lognorm_sigma: float = 1.5
    pool_cap: int = 50_000
    super_frac: float = 0.0
    super_lo: float = 1e5
    super_hi: float = 1e6
    seed: int = 0


# plain VATE, small: 4096 hosts, 50k packets per slice, Zipf(1.1)
SMALL = TrafficSpec(n_aips=4096, pkts_per_slice=50_000, zipf_s=1.1, seed=0xC1)
# plain VATE at the 40 Gb/s shape: 2^20 hosts, 5M packets per 1 s slice,
# Zipf(1.05), 0.1% super-spreaders with 1e5..1e6 peers
LINK40G = TrafficSpec(n_aips=1 << 20, pkts_per_slice=5_000_000, zipf_s=1.05,
                      super_frac=0.001, seed=0xC2)


class Traffic:
    """Host table plus a per-slice packet generator (counter-based in
    (seed, slice): slice s is the same whatever order slices are drawn in)."""

    def __init__(self, spec: TrafficSpec, pkts_per_slice: Optional[int] = None):
        self.spec = spec
        self.pkts_per_slice = int(pkts_per_slice if pkts_per_slice is not None else spec.pkts_per_slice)
        rng = np.random.Generator(np.random.Philox(key=[spec.seed & 0xFFFFFFFFFFFFFFFF, 0xA1]))
        n = spec.n_aips
        # distinct random host addresses
        aips = np.unique(rng.integers(1, 1 << 32, size=n + n // 8 + 64, dtype=np.uint64).astype(np.uint32))
        while aips.shape[0] < n:
            more = rng.integers(1, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
            aips = np.unique(np.concatenate([aips, more]))
        aips = rng.permutation(aips)[:n]
        self.aips = np.ascontiguousarray(aips, np.uint32)
        # popularity: rank r (0 = most popular) -> host index rank_host[r]
        self.rank_host = rng.permutation(n).astype(np.int64)
        w = np.arange(1, n + 1, dtype=np.float64) ** (-spec.zipf_s)
        self.rank_cdf = np.cumsum(w / w.sum())
        self.rank_cdf[-1] = 1.0
        # peer-pool size per host
        sizes = np.ceil(rng.lognormal(spec.lognorm_mu, spec.lognorm_sigma, size=n))
        sizes = np.clip(sizes, 1, spec.pool_cap)
        n_super = int(round(spec.super_frac * n))
        if n_super:
            lo, hi = np.log(spec.super_lo), np.log(spec.super_hi)
            sup = np.floor(np.exp(rng.uniform(lo, hi, size=n_super)))
            sizes[self.rank_host[:n_super]] = sup
        self.pool_size = sizes.astype(np.int64)
        self.n_super = n_super
        self.super_hosts = np.sort(self.rank_host[:n_super])
        # peer j of host h is base[h] + j * 0x9E3779B1 (mod 2^32): distinct for j < 2^32
        self.peer_base = rng.integers(0, 1 << 32, size=n, dtype=np.uint64)

    def slice_pairs(self, s: int, n: Optional[int] = None) -> np.ndarray:
        """(n, 2) uint32 array of (aip, bip) for slice s."""
        n = self.pkts_per_slice if n is None else int(n)
        rng = np.random.Generator(np.random.Philox(key=[self.spec.seed & 0xFFFFFFFFFFFFFFFF, 0x5100 + int(s)]))
        u = rng.random(n)
        rank = np.searchsorted(self.rank_cdf, u, side="right")
        np.minimum(rank, self.spec.n_aips - 1, out=rank)
        host = self.rank_host[rank]
        j = np.floor(rng.random(n) * self.pool_size[host]).astype(np.uint64)
        bip = (self.peer_base[host] + j * np.uint64(0x9E3779B1)) & np.uint64(0xFFFFFFFF)
        out = np.empty((n, 2), np.uint32)
        out[:, 0] = self.aips[host]
        out[:, 1] = bip.astype(np.uint32)
        return out


def mixed_hosts(tr: Traffic, n: int, seed: int = 7) -> np.ndarray:
    """A seeded sample of n host addresses including every super-spreader."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0xB2]))
    idx = rng.choice(tr.spec.n_aips, size=min(n, tr.spec.n_aips), replace=False)
    idx = np.union1d(idx, tr.super_hosts)
    return tr.aips[idx]


class DeviceTraffic:
    """The same traffic model drawn on a CUDA device with torch's Philox
    generator (a different random stream from ``Traffic.slice_pairs``, the same
    distribution), for benchmarks that need hundreds of 5M-pair slices
    resident in device memory.  Host table = ``tr``'s."""

    def __init__(self, tr: Traffic, device="cuda"):
        import torch
        self.tr, self.device = tr, device
        self.rank_cdf = torch.from_numpy(tr.rank_cdf).to(device)
        self.rank_host = torch.from_numpy(tr.rank_host).to(device)
        self.pool_size = torch.from_numpy(tr.pool_size.astype(np.float64)).to(device)
        self.peer_base = torch.from_numpy(tr.peer_base.astype(np.int64)).to(device)
        self.aips = torch.from_numpy(tr.aips.astype(np.int64)).to(device)
        self.gen = torch.Generator(device=device)

    def slice_pairs(self, s: int, n: Optional[int] = None):
        """(n, 2) int32 CUDA tensor holding the uint32 bit patterns of (aip, bip)."""
        import torch
        n = self.tr.pkts_per_slice if n is None else int(n)
        self.gen.manual_seed((self.tr.spec.seed * 1_000_003 + 7919 * int(s) + 1) & 0x7FFFFFFFFFFFFFFF)
        u = torch.rand(n, generator=self.gen, device=self.device, dtype=torch.float64)
        rank = torch.searchsorted(self.rank_cdf, u, right=True).clamp_(max=self.tr.spec.n_aips - 1)
        host = self.rank_host[rank]
        j = torch.floor(torch.rand(n, generator=self.gen, device=self.device, dtype=torch.float64)
                        * self.pool_size[host]).to(torch.int64)
        bip = (self.peer_base[host] + j * 0x9E3779B1) & 0xFFFFFFFF
        out = torch.stack([self.aips[host], bip], dim=1)
        out = torch.where(out >= 2**31, out - 2**32, out).to(torch.int32).contiguous()
        return out

    def hosts(self):
        """All host addresses as an int32 CUDA tensor (uint32 bit patterns)."""
        import torch
        a = self.aips
        return torch.where(a >= 2**31, a - 2**32, a).to(torch.int32).contiguous()
