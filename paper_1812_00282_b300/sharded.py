"""One VATE pool split by position over the ranks of a process group
(include/vate_shard.h).

Each rank holds the ATs of one range of pool positions and sees every pair.
A close on every rank is followed by two all-reduces -- the per-host active
counts A (uint32, carried as int32; A <= g <= 65536) and the census (int64)
-- after which every rank evaluates Eq. 11 on the summed counts with
vate_estimate_from_counts.  Integer sums do not depend on their order, so the
estimates equal those of one undivided pool bit for bit.

This module only schedules library calls and collectives; the SetAT, slide,
census, gather and Eq. 11 all run in the library's kernels.  The backend
object (`lib`) is the binding module by default; it is a parameter so that
the orchestration can be exercised without a GPU.
"""
from __future__ import annotations

from typing import List, Optional, Tuple

SHARD_ALIGN = 64   # positions; a segment of L <= 64 VATs and a 16-byte chunk lie on one shard


def shard_ranges(P: int, world: int) -> List[Tuple[int, int]]:
    """Contiguous ranges [lo, hi) covering [0, P), boundaries multiples of 64,
    as equal as that allows."""
    if world < 1 or P < SHARD_ALIGN * world:
        raise ValueError("cannot split %d positions into %d shards of at least %d" % (P, world, SHARD_ALIGN))
    cuts = [((P * r) // world) // SHARD_ALIGN * SHARD_ALIGN for r in range(world)] + [P]
    out = [(cuts[r], cuts[r + 1]) for r in range(world)]
    if any(lo >= hi for lo, hi in out):
        raise ValueError("empty shard in %r" % (out,))
    return out


class ShardedVate:
    """The shard of this rank; every rank of `group` must make the same calls
    with the same pairs, hosts and slices."""

    def __init__(self, log2_pool: int, k: int, g: int, seg_len: int = 1, partition: int = 0, seed: int = 0,
                 counter: int = 0, group=None, rank: Optional[int] = None, world: Optional[int] = None, lib=None,
                 stream=None):
        import torch.distributed as dist
        if lib is None:
            import paper_1812_00282_b300 as lib
        self.lib, self.group = lib, group
        self.rank = dist.get_rank(group) if rank is None else rank
        self.world = dist.get_world_size(group) if world is None else world
        self.k, self.g, self.P = k, g, 1 << log2_pool
        self.params = lib.make_params(log2_pool, k, g, seg_len, partition, seed, counter)
        self.lo, self.hi = shard_ranges(self.P, self.world)[self.rank]
        self.h = lib.vate_create_shard(self.params, self.lo, self.hi, stream)
        self._gloo = dist.get_backend(group) == "gloo"

    def close(self) -> None:
        if self.h is not None:
            self.lib.vate_destroy(self.h)
            self.h = None

    def ingest(self, pairs, slice: int, stream=None) -> None:
        self.lib.vate_ingest(self.h, pairs, slice, stream)

    def ingest_host(self, pairs, slice: int, stream=None) -> None:
        self.lib.vate_ingest_host(self.h, pairs, slice, stream)

    def close_slice(self, slice: int, stream=None) -> None:
        self.lib.vate_close_slice(self.h, slice, stream)

    def _all_reduce(self, t) -> None:
        import torch
        import torch.distributed as dist
        if self._gloo and t.is_cuda:          # gloo reduces host tensors
            c = t.cpu()
            dist.all_reduce(c, group=self.group)
            t.copy_(c)
        else:
            dist.all_reduce(t, group=self.group)
        if t.dtype == torch.int32:
            assert int(t.min()) >= 0, "active counts overflowed"

    @staticmethod
    def _torch_stream(stream, dev):
        """The torch stream object for `stream` (None: torch's current stream;
        an int: a raw cudaStream_t)."""
        import torch
        if stream is None:
            return torch.cuda.current_stream(dev)
        if isinstance(stream, int):
            return torch.cuda.ExternalStream(stream, device=dev)
        return stream

    def counts(self, hosts, kprime: int, stream=None):
        """(A, census) summed over the shards.  The counting kernels run on
        `stream`; the all-reduces see their results (gloo: after a
        synchronisation of that stream; NCCL: torch's current stream waits on
        it), and the reduced tensors are ready on torch's current stream."""
        import torch
        dev = hosts.device
        active = torch.empty(hosts.numel(), dtype=torch.int32, device=dev)
        hist = torch.empty(2 * self.k + 1, dtype=torch.int64, device=dev)
        st = self._torch_stream(stream, dev) if dev.type == "cuda" else stream
        if dev.type == "cuda":
            st.wait_stream(torch.cuda.current_stream(dev))   # the buffers were made on the current stream
            active.record_stream(st)
            hist.record_stream(st)
        self.lib.vate_active_counts(self.h, hosts, kprime, active, st)
        self.lib.vate_census(self.h, hist, st)
        if dev.type == "cuda":
            if self._gloo:
                st.synchronize()
            else:
                torch.cuda.current_stream(dev).wait_stream(st)
        self._all_reduce(active)
        self._all_reduce(hist)
        return active, hist

    def estimate(self, hosts, kprime: int, out, flags=None, stream=None) -> None:
        """Eq. 11 on the summed counts, queued on `stream` after the
        all-reduces (which leave their results on torch's current stream)."""
        import torch
        active, hist = self.counts(hosts, kprime, stream)
        st = stream
        if hosts.device.type == "cuda":
            st = self._torch_stream(stream, hosts.device)
            st.wait_stream(torch.cuda.current_stream(hosts.device))
        self.lib.vate_estimate_from_counts(self.params, active, hist, kprime, out, flags, st)

    def copy_pool(self, dst, stream=None) -> None:
        """This shard's positions [lo, hi), in the paper's form."""
        self.lib.vate_copy_pool(self.h, dst, stream)
