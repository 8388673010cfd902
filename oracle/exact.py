"""Brute-force exact sliding-window host cardinalities -- TEST INFRASTRUCTURE ONLY.

|OP(aip, t-k'+1, k')| (Def. 1, Sec. 1): the number of distinct opposite hosts
bip seen with aip in the k' slices ending at slice t.  Computed by sorting the
distinct (aip, bip) keys of the window; no hashing, no counters, no
approximation.  This is the ground truth against which the oracle's and the
device's estimates are scored, and the reference for the no-collision pins.
"""
from __future__ import annotations

from typing import Sequence

import numpy as np


def _keys(pairs: np.ndarray) -> np.ndarray:
    p = np.asarray(pairs, dtype=np.uint32)
    return (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)


def window_cardinality(slices: Sequence[np.ndarray], t: int, kprime: int, aips) -> np.ndarray:
    """Exact |OP(aip, t-k'+1, k')| for each aip in ``aips``.

    ``slices[s]`` holds the (aip, bip) pairs of slice s, shape (n_s, 2).
    The window is truncated at slice 0 when t < k'-1.
    """
    lo = max(0, t - kprime + 1)
    parts = [_keys(slices[s]) for s in range(lo, t + 1) if len(slices[s])]
    aips = np.asarray(aips, dtype=np.uint32)
    if not parts:
        return np.zeros(aips.shape[0], np.int64)
    uniq = np.unique(np.concatenate(parts))
    hosts = (uniq >> np.uint64(32)).astype(np.uint32)
    hv, cnt = np.unique(hosts, return_counts=True)
    idx = np.searchsorted(hv, aips)
    idx_c = np.minimum(idx, len(hv) - 1)
    found = (idx < len(hv)) & (hv[idx_c] == aips)
    return np.where(found, cnt[idx_c], 0).astype(np.int64)


def last_seen(slices: Sequence[np.ndarray], upto: int, aip: int, bip: int) -> int:
    """Slice of the last appearance of one pair up to slice ``upto`` (-1 if none);
    the timestamp counter of Sec. 1 for a single pair, used by small tests."""
    last = -1
    for s in range(0, upto + 1):
        p = np.asarray(slices[s])
        if p.size and np.any((p[:, 0] == aip) & (p[:, 1] == bip)):
            last = s
    return last
