"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks it against a value
printed in the paper, a brute-force ground truth (timestamps, exact distinct
counts), a textbook special case, a published test vector, or a statistical
property of the estimator.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Oracle
from oracle.exact import window_cardinality

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# Hash functions (reading: SplitMix64 output function + Lemire reduction for BH;
# a per-host SplitMix64 key and MurmurHash3's finalizer per segment for H)
# --------------------------------------------------------------------------

def test_mix64_matches_published_splitmix64_sequence():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014; Vigna's reference
    # generator): the n-th output is the output function applied to
    # (n-1) * 0x9E3779B97F4A7C15, whose first three values are published.
    gamma = 0x9E3779B97F4A7C15
    assert oracle.mix64(0) == 0xE220A8397B1DCDAF
    assert oracle.mix64(gamma) == 0x6E789E6AA1B965F4
    assert oracle.mix64((2 * gamma) & (2**64 - 1)) == 0x06C45D188009454F


def test_fmix32_is_murmurhash3_of_the_empty_input():
    # MurmurHash3_x86_32 of a zero-length key with seed s is the finalizer
    # applied to s (no blocks, no tail, length 0 xored in), so the finalizer is
    # pinned by an independent implementation of the whole hash
    # (scikit-learn's) and by the published vector for seed 1.
    from sklearn.utils import murmurhash3_32
    assert oracle.fmix32(1) == 0x514E28B7
    rng = np.random.default_rng(3)
    for s in [0, 1, 2, 0xFFFFFFFF, 0x9E3779B9] + [int(x) for x in rng.integers(0, 2**32, 200)]:
        assert oracle.fmix32(s) == murmurhash3_32(b"", seed=s, positive=True)


@pytest.mark.parametrize("c,L", [(18, 1), (18, 32), (32, 1), (26, 32), (12, 64)])
def test_h_is_the_documented_composition(c, L):
    # H(aip, i) = L * top_{c - log2 L}(fmix32(lo32(K) ^ j * 0x9E3779B9) ^ hi32(K)) + i mod L,
    # K = mix64(mix64(seed + 1) ^ aip << 32), j = i div L; both mixers pinned above
    from sklearn.utils import murmurhash3_32
    seed = 0xC2
    o = Oracle(c=c, k=3, g=256, seg_len=L, seed=seed)
    segbits = c - (L.bit_length() - 1)
    key_h = oracle.mix64(seed + 1)
    for aip in (0, 1, 0xDEADBEEF, 0xFFFFFFFF, 123456):
        K = oracle.mix64(key_h ^ (aip << 32))
        for i in (0, 1, 31, 32, 33, 255):
            j = i // L
            x = murmurhash3_32(b"", seed=(K & 0xFFFFFFFF) ^ ((j * 0x9E3779B9) & 0xFFFFFFFF), positive=True)
            x ^= K >> 32
            assert o.h(aip, i) == L * (x >> (32 - segbits)) + i % L


def test_stateless_mapping_equals_the_pool_state_mapping():
    for c, L, g, seed in [(18, 32, 1024, 5), (16, 1, 256, 9), (20, 64, 4096, 0xC2)]:
        o = Oracle(c=c, k=3, g=g, seg_len=L, seed=seed)
        for aip in (0, 7, 0xDEADBEEF):
            for i in (0, 1, g // 2, g - 1):
                assert oracle.h_of(c, L, seed, aip, i) == o.h(aip, i)
        for bip in (0, 3, 0xFFFFFFFF):
            assert oracle.bh_of(g, seed, bip) == o.bh(bip)


@pytest.mark.parametrize("g", [1, 64, 1000, 4096, 65536])
def test_bh_is_the_documented_composition(g):
    # BH(bip) = ((mix64(mix64(seed + 2) ^ bip) >> 32) * g) >> 32: Lemire's
    # multiply-shift range reduction of the high half of the pinned mixer
    seed = 0xC2
    o = Oracle(c=16, k=3, g=g, seed=seed) if g <= 4096 else None
    key_bh = oracle.mix64(seed + 2)
    for bip in (0, 1, 7, 0x80000000, 0xFFFFFFFF, 123456789):
        want = ((oracle.mix64(key_bh ^ bip) >> 32) * g) >> 32
        assert oracle.bh_of(g, seed, bip) == want
        if o is not None:
            assert o.bh(bip) == want


def test_bh_range_and_uniformity():
    o = Oracle(c=16, k=3, g=64, seed=11)
    vals = np.array([o.bh(b) for b in range(20000)])
    assert vals.min() >= 0 and vals.max() < 64
    counts = np.bincount(vals, minlength=64)
    chi2 = float(((counts - 20000 / 64) ** 2 / (20000 / 64)).sum())
    assert chi2 < 120  # 63 dof: mean 63, sd ~11


@pytest.mark.parametrize("L", [1, 32])
def test_h_range_and_segments(L):
    o = Oracle(c=18, k=3, g=256, seg_len=L, seed=5)
    for aip in (1, 0xDEADBEEF, 123456):
        pids = [o.h(aip, i) for i in range(256)]
        assert all(0 <= p < o.P for p in pids)
        for i in range(256):
            # VAT i sits at offset i mod L of its segment, segments are L-aligned
            assert pids[i] % L == i % L
            assert pids[i] - pids[i - i % L] == i % L
    # different hosts land in different places
    assert [o.h(1, i) for i in range(8)] != [o.h(2, i) for i in range(8)]


# --------------------------------------------------------------------------
# Algorithm 3 against the paper's worked example (k = 9)
# --------------------------------------------------------------------------

def _golden_k9():
    rows = []
    with open(os.path.join(GOLDEN, "alg3_k9.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(tuple(int(x) for x in line.split()))
    return rows


def test_alg3_worked_example_k9():
    rows = _golden_k9()
    assert len(rows) == 19
    for v, at0, at9 in rows:
        assert oracle.preserve_fast(v, 0, 9) == at0, v
        assert oracle.preserve_fast(v, 9, 9) == at9, v


def test_alg3_is_identity_off_maintenance_points():
    for k in (3, 9):
        for act in range(1, 2 * k):
            if act == k:
                continue
            for v in range(2 * k + 1):
                assert oracle.preserve_fast(v, act, k) == v


def test_checkat_distance_definition():
    # Eq. 5: Dist = (ACT + 2k - Value) mod 2k; Algorithm 1 is "Dist <= k'-1".
    # Enumerate, for every last-set slice l and current slice t with t-l < 2k,
    # the value the AT holds (the ACT of slice l) and check the answer.
    for k in (1, 2, 5):
        for act0 in range(2 * k):          # ACT of the AT in slice 0
            for l in range(0, 4 * k):
                for t in range(l, l + 2 * k):
                    v = (act0 + l) % (2 * k)
                    act = (act0 + t) % (2 * k)
                    for kp in range(1, k + 1):
                        assert oracle.check_at(v, act, k, kp) == (t - l < kp)
            for kp in range(1, k + 1):
                assert not oracle.check_at(2 * k, act0, k, kp)


# --------------------------------------------------------------------------
# Exhaustive brute force: every set/no-set pattern of one AT over 4k+2 slices,
# for every block position, against the timestamp shadow (Def. 2 with a TS).
# --------------------------------------------------------------------------

def _closed_form_pool(last, block, t, k):
    """AT value implied by the last-set slice (origin 0, BACT^0 = t mod 2k).

    Inactive (2k) if never set, or if some maintenance point m in (last, t]
    with m = -block (mod k) has m - last >= k; otherwise the ACT of the slice
    of the last set, (last + block) mod 2k."""
    twok = 2 * k
    out = np.full(last.shape, twok, np.int64)
    seen = last >= 0
    # first maintenance point strictly after `last` with m - last >= k:
    # m = smallest value >= last + k with (m + block) % k == 0
    m0 = last + k
    m = m0 + ((-(m0 + block)) % k)
    expired = seen & (m <= t)
    alive = seen & ~expired
    out[alive] = (last[alive] + block[alive]) % twok
    return out


@pytest.mark.parametrize("k", [1, 2, 3, 4])
@pytest.mark.parametrize("partition", [0, 1])
def test_exhaustive_tiny_k(k, partition):
    nslices = 4 * k + 2
    npat = 1 << nslices
    twok = 2 * k
    # pool large enough that every block holds all patterns
    c = max(int(math.ceil(math.log2(npat * twok * 2))), 4)
    o = Oracle(c=c, k=k, g=1, partition=partition, seed=1)
    P = o.P
    pid = np.arange(P, dtype=np.int64)
    block = np.array([o.block(int(p)) for p in range(P)], np.int64) if P <= 1 << 12 else None
    if block is None:
        # block boundaries from the oracle, probed at the range ends
        starts = [0]
        for i in range(1, twok):
            lo, hi = starts[-1], P
            while lo < hi:
                mid = (lo + hi) // 2
                if o.block(mid) >= i:
                    hi = mid
                else:
                    lo = mid + 1
            starts.append(lo)
        block = np.searchsorted(np.array(starts[1:]), pid, side="right").astype(np.int64)
        for s in range(0, P, max(1, P // 4096)):
            assert o.block(s) == block[s]
    starts = np.searchsorted(block, np.arange(twok))
    pattern = pid - starts[block]                   # index inside the block
    used = pattern < npat
    # every block must hold every pattern (eq. 9-10 leaves a tiny last block:
    # there the patterns present are a prefix; others are covered elsewhere)
    last = np.full(P, -1, np.int64)
    for t in range(nslices):
        if t > 0:
            o.advance()
        setmask = used & (((pattern >> t) & 1) == 1)
        o.set_pids(np.nonzero(setmask)[0])
        last[setmask] = t
        pool = o.pool().astype(np.int64)
        expect = _closed_form_pool(last, block, t, k)
        np.testing.assert_array_equal(pool[used], expect[used], err_msg="t=%d" % t)
        for kp in range(1, k + 1):
            act = o.check_all(kp).astype(bool)
            truth = (last >= 0) & (t - last < kp)
            np.testing.assert_array_equal(act[used], truth[used], err_msg="t=%d k'=%d" % (t, kp))


def test_alg2_and_alg3_agree_on_reachable_states():
    # Maintaining every AT with Algorithm 2 in every slice must leave exactly
    # the same pool as Algorithm 3 on the two ACT-0/ACT-k blocks (Corollary 1).
    for k in (1, 2, 3, 4):
        rng = np.random.default_rng(100 + k)
        o3 = Oracle(c=12, k=k, g=1, seed=3)
        o2 = Oracle(c=12, k=k, g=1, seed=3)
        for t in range(8 * k + 3):
            if t > 0:
                o3.advance()
                o2.advance_general_every_slice()
            pids = rng.choice(o3.P, size=300, replace=False)
            o3.set_pids(pids)
            o2.set_pids(pids)
            for kp in range(1, k + 1):
                np.testing.assert_array_equal(o3.check_all(kp), o2.check_all(kp))


def test_alg2_alg3_differ_only_when_value_equals_act():
    for k in (2, 5, 9):
        for act in (0, k):
            for v in range(2 * k + 1):
                f, g_ = oracle.preserve_fast(v, act, k), oracle.preserve_general(v, act, k)
                if v != act:
                    assert f == g_, (k, act, v)


# --------------------------------------------------------------------------
# Block partition (Eq. 9-10 and the low-deviation partition)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("c,k,a,b", [(20, 5, 116508, 4), (26, 10, 3532045, 9), (24, 10, 883011, 7)])
def test_block_sizes_eq9_eq10(c, k, a, b):
    o = Oracle(c=c, k=k, g=1)
    assert (o.a, o.b) == (a, b)
    assert a * (2 * k - 1) + b == 1 << c
    # contiguous blocks of size a, last of size b
    for i in range(2 * k):
        lo = i * a
        assert o.block(lo) == i
        if i < 2 * k - 1:
            assert o.block(lo + a - 1) == i
    assert o.block((1 << c) - 1) == 2 * k - 1


@pytest.mark.parametrize("c,k", [(12, 3), (12, 5), (13, 7), (16, 10)])
def test_low_deviation_partition_both_boundary_forms(c, k):
    o = Oracle(c=c, k=k, g=1, partition=1)
    P, twok = 1 << c, 2 * k
    a2, b2 = P // twok, P % twok
    assert (o.a, o.b) == (a2, b2)
    sizes = [a2] * (twok - b2) + [a2 + 1] * b2
    explicit = np.repeat(np.arange(twok), sizes)
    printed_boundary = a2 * (twok - b2 + 1)      # the form printed in Sec. 4.1
    for i in range(P):
        bi = o.block(i)
        assert bi == explicit[i]
        alt = i // a2 if i < printed_boundary else (i + twok - b2) // (a2 + 1)
        assert alt == bi


# --------------------------------------------------------------------------
# Estimator (Eq. 11 with the sign reading; Eq. 1 as its special case)
# --------------------------------------------------------------------------

def test_estimator_reduces_to_linear_estimator():
    # With Z_p = 1 (no inactive-pool correction), Eq. 11 must equal the linear
    # estimator of Eq. 1: -g ln(g0 / g), g0 = number of zero (inactive) counters.
    g, P = 1024, 1 << 20
    for A in (0, 1, 10, 500, 1000, 1023):
        e, f = oracle.estimate_from_counts(g, P, P, A)
        g0 = g - A
        assert f == 0
        assert e == pytest.approx(-g * math.log(g0 / g), rel=1e-12, abs=1e-12)


def test_estimator_unbiased_under_pool_noise():
    # Throw n distinct peers into g VATs; each VAT is also active with
    # probability q because of other hosts sharing the pool.  The estimator
    # must recover n on average (GSE's bias removal, Eq. 2 / Eq. 11).
    rng = np.random.default_rng(2024)
    g, P = 1024, 1 << 22
    for q in (0.0, 0.2, 0.5):
        N0 = int(round((1 - q) * P))
        for n in (30, 300, 1500):
            ests = []
            for _ in range(400):
                hit = np.zeros(g, bool)
                hit[rng.integers(0, g, size=n)] = True
                hit |= rng.random(g) < q
                e, _ = oracle.estimate_from_counts(g, P, N0, int(hit.sum()))
                ests.append(e)
            ests = np.array(ests)
            se = ests.std(ddof=1) / math.sqrt(len(ests))
            assert abs(ests.mean() - n) < 4 * se + 0.02 * n, (q, n, ests.mean())


def test_estimator_degenerate_cases():
    g, P = 64, 1 << 16
    e, f = oracle.estimate_from_counts(g, P, P // 2, g)
    assert f == oracle.SAT and math.isfinite(e)
    e2, _ = oracle.estimate_from_counts(g, P, P // 2, g - 1)
    assert e == pytest.approx(e2)          # V0 = 0 is read as V0 = 1
    e, f = oracle.estimate_from_counts(g, P, 0, 3)
    assert f == oracle.POOLFULL and math.isfinite(e)
    e, f = oracle.estimate_from_counts(g, P, P, 0)
    assert e == 0.0 and f == 0
    # monotone: more active VATs -> larger estimate; fewer inactive pool ATs -> smaller
    vals = [oracle.estimate_from_counts(g, P, P // 2, A)[0] for A in range(0, g)]
    assert all(b > a for a, b in zip(vals, vals[1:]))


# --------------------------------------------------------------------------
# Whole runs: exact counts when nothing collides; TS shadow; VDRE equality
# --------------------------------------------------------------------------

def _disjoint_hosts(o, g, want, rng):
    taken, hosts = set(), []
    while len(hosts) < want:
        aip = int(rng.integers(1, 2**32))
        pids = {o.h(aip, i) for i in range(g)}
        if len(pids) == g and not (pids & taken):
            hosts.append(aip)
            taken |= pids
    return hosts


@pytest.mark.parametrize("L", [1, 8])
def test_no_collision_active_count_equals_exact_count(L):
    k, g = 3, 64
    o = Oracle(c=20, k=k, g=g, seg_len=L, seed=77)
    rng = np.random.default_rng(9)
    hosts = _disjoint_hosts(o, g, 6, rng)
    peers = {}
    for h in hosts:                       # peers with pairwise distinct BH
        seen, lst = set(), []
        while len(lst) < 40:
            b = int(rng.integers(0, 2**32))
            if o.bh(b) not in seen:
                seen.add(o.bh(b))
                lst.append(b)
        peers[h] = lst
    slices = []
    for t in range(4 * k + 3):
        if t > 0:
            o.advance()
        rows = []
        for h in hosts:
            m = int(rng.integers(0, 12))
            for b in rng.choice(peers[h], size=m, replace=True):
                rows.append((h, int(b)))
        arr = np.array(rows, np.uint32).reshape(-1, 2)
        slices.append(arr)
        o.ingest(arr)
        for kp in range(1, k + 1):
            exact = window_cardinality(slices, t, kp, hosts)
            _, A, _ = o.estimate(hosts, kp)
            np.testing.assert_array_equal(A.astype(np.int64), exact, err_msg="t=%d k'=%d" % (t, kp))
            # the pool census sees exactly the ATs of these hosts
            assert o.P - o.pool_inactive(kp) == int(exact.sum())


def _small_stream(o, nslices, n_per, n_hosts, rng):
    hosts = rng.integers(1, 2**32, size=n_hosts, dtype=np.uint64).astype(np.uint32)
    out = []
    for _ in range(nslices):
        h = hosts[rng.zipf(1.3, size=n_per) % n_hosts]
        b = rng.integers(0, 600, size=n_per).astype(np.uint32) * np.uint32(2654435761 % 2**32)
        out.append(np.stack([h, b], 1).astype(np.uint32))
    return hosts, out


@pytest.mark.parametrize("L,partition", [(1, 0), (32, 0), (1, 1), (32, 1)])
def test_pool_equals_timestamp_closed_form_with_collisions(L, partition):
    k = 4
    o = Oracle(c=14, k=k, g=128, seg_len=L, partition=partition, seed=123)
    rng = np.random.default_rng(L * 10 + partition)
    hosts, slices = _small_stream(o, 5 * k + 1, 3000, 40, rng)
    P = o.P
    block = np.array([o.block(p) for p in range(P)], np.int64)
    last = np.full(P, -1, np.int64)
    for t, arr in enumerate(slices):
        if t > 0:
            o.advance()
        o.ingest(arr)
        last[o.pids_of_pairs(arr).astype(np.int64)] = t
        np.testing.assert_array_equal(o.pool().astype(np.int64), _closed_form_pool(last, block, t, k))
        # census histogram = distances of the shadow timestamps
        hist = o.census()
        expect = np.zeros(2 * k + 1, np.int64)
        alive = _closed_form_pool(last, block, t, k) != 2 * k
        np.add.at(expect, t - last[alive], 1)
        expect[2 * k] = int((~alive).sum())
        np.testing.assert_array_equal(hist.astype(np.int64), expect)


@pytest.mark.slow
@pytest.mark.parametrize("c,k,every", [(16, 100, 5), (19, 300, 17)])
def test_wide_timestamps_equal_closed_form(c, k, every):
    # k beyond one byte (values up to 2k = 600, the paper's k' = 300 of Sec. 5):
    # the pool still equals the closed form of the last-set shadow, through
    # more than one full 2k cycle of every block's ACT.
    o = Oracle(c=c, k=k, g=64, seg_len=1, partition=0, seed=k)
    rng = np.random.default_rng(k)
    hosts, slices = _small_stream(o, 2 * k + 3, 400, 30, rng)
    block = np.array([o.block(p) for p in range(o.P)], np.int64)
    last = np.full(o.P, -1, np.int64)
    for t, arr in enumerate(slices):
        if t > 0:
            o.advance()
        o.ingest(arr)
        last[o.pids_of_pairs(arr).astype(np.int64)] = t
        if t % every == 0 or t >= 2 * k:
            pool = o.pool().astype(np.int64)
            assert pool.max() <= 2 * k
            np.testing.assert_array_equal(pool, _closed_form_pool(last, block, t, k), err_msg="t=%d" % t)
    for kp in (1, k // 2, k):
        for h in hosts[:10]:
            assert o.active_vats(int(h), kp) == o.active_vats_dr(int(h), kp)


def test_vate_equals_vdre():
    # Sec. 5: with the same mapping, VATE (AT pool) and VDRE (DR pool aged every
    # slice) give identical estimates.
    k = 5
    o = Oracle(c=16, k=k, g=256, seed=4)
    rng = np.random.default_rng(5)
    hosts, slices = _small_stream(o, 4 * k, 4000, 60, rng)
    for t, arr in enumerate(slices):
        if t > 0:
            o.advance()
        o.ingest(arr)
        for kp in (1, 2, k):
            for h in hosts[:20]:
                assert o.active_vats(int(h), kp) == o.active_vats_dr(int(h), kp)


def test_age_counts_sum_to_active_counts():
    k = 5
    o = Oracle(c=16, k=k, g=256, seg_len=32, seed=8)
    rng = np.random.default_rng(6)
    hosts, slices = _small_stream(o, 3 * k, 4000, 30, rng)
    for t, arr in enumerate(slices):
        if t > 0:
            o.advance()
        o.ingest(arr)
    ages = o.age_counts(hosts)
    for kp in range(1, k + 1):
        _, A, _ = o.estimate(hosts, kp)
        np.testing.assert_array_equal(ages[:, :kp].sum(1), A)


def test_exact_counts_brute_force():
    rng = np.random.default_rng(1)
    slices = [rng.integers(0, 5, size=(30, 2)).astype(np.uint32) for _ in range(6)]
    for t in range(6):
        for kp in (1, 2, 4):
            lo = max(0, t - kp + 1)
            sets = {}
            for s in range(lo, t + 1):
                for a, b in slices[s]:
                    sets.setdefault(int(a), set()).add(int(b))
            want = [len(sets.get(a, ())) for a in range(5)]
            got = window_cardinality(slices, t, kp, np.arange(5))
            assert list(got) == want


@pytest.mark.slow
def test_error_falls_with_pool_size_and_vector_length():
    # Sec. 5: with g fixed, a larger pool brings the estimates closer to the
    # truth; with the pool fixed, a g too small for the high-cardinality hosts
    # (n near or above g ln g, the saturation point of Eq. 1) estimates them
    # worse than any larger g.  Between two g well above that point the
    # ordering is not fixed: a larger g also takes in more sharing noise from
    # the pool, and on these hosts (n <= 900) g = 512 and g = 2048 are
    # statistically tied.
    from traffic import SMALL, Traffic
    tr = Traffic(SMALL, pkts_per_slice=50_000)
    slices = [tr.slice_pairs(s) for s in range(8)]
    k, t = 5, 7
    exact = window_cardinality(slices, t, k, tr.aips)

    def mre(c, g, sel, L=1):
        o = Oracle(c=c, k=k, g=g, seg_len=L, seed=1)
        for s, arr in enumerate(slices):
            if s > 0:
                o.advance()
            o.ingest(arr)
        est, _, _ = o.estimate(tr.aips[sel], k)
        n = exact[sel].astype(np.float64)
        return float(np.mean(np.abs(np.maximum(est, 0) - n) / n))

    small = exact >= 20
    by_c = [mre(c, 1024, small) for c in (17, 19, 21)]
    assert by_c[0] > by_c[1] > by_c[2], by_c
    # the same trend with 32-VAT segments, which cost some accuracy at equal memory (clustered VATs)
    by_c32 = [mre(c, 1024, small, L=32) for c in (17, 19, 21)]
    assert by_c32[0] > by_c32[1] > by_c32[2], by_c32
    assert by_c32[2] > by_c[2]
    top = np.zeros_like(small)
    top[np.argsort(exact)[-16:]] = True
    by_g = [mre(21, g, top) for g in (128, 512, 2048)]
    assert exact[top].max() > 128 * math.log(128)           # the largest top host saturates g = 128
    assert by_g[0] > by_g[1] and by_g[0] > by_g[2], by_g


def test_error_falls_with_vector_length_where_g_matters():
    # Eq. 1 on a quiet pool: for a host of n distinct peers the relative
    # standard error of the linear-counting estimate over g VATs is
    # sqrt(e^t - t - 1) / (t sqrt(g)) with t = n / g, which falls as g grows,
    # and at n near g ln g the vector saturates (g = 256 here: 256 ln 256 ~
    # 1,420 < n).  Sixteen hosts of 2,000-5,000 peers each, alone on a
    # 2^22-AT pool, one slice: the mean relative error falls strictly over
    # g = 256, 1024, 4096, and for the two unsaturated g it is within a
    # factor of two of sqrt(2 / pi) times the mean standard error (the mean
    # absolute value of a normal error).
    rng = np.random.default_rng(12)
    ns = np.array([2000, 3000, 4000, 5000] * 4)
    aips = (np.arange(1, len(ns) + 1, dtype=np.uint64) * 7919).astype(np.uint32)
    parts = []
    for a, n in zip(aips, ns):
        b = np.unique(rng.integers(1, 2**32, size=2 * n, dtype=np.uint64))[:n]
        rng.shuffle(b)
        parts.append(np.stack([np.full(n, a, np.uint32), b.astype(np.uint32)], 1))
    pairs = np.ascontiguousarray(np.concatenate(parts))
    mre = []
    for g in (256, 1024, 4096):
        o = Oracle(c=22, k=2, g=g, seg_len=1, seed=3)
        o.ingest(pairs)
        est, _, _ = o.estimate(aips, 2)
        mre.append(float(np.mean(np.abs(np.maximum(est, 0) - ns) / ns)))
    assert mre[0] > mre[1] > mre[2], mre
    for g, m in zip((1024, 4096), mre[1:]):
        t = ns / g
        pred = math.sqrt(2 / math.pi) * float(np.mean(np.sqrt(np.exp(t) - t - 1) / (t * math.sqrt(g))))
        assert 0.5 * pred < m < 2 * pred, (g, m, pred)


def test_oracle_results_do_not_depend_on_its_thread_count():
    # the census, the inactive count and the per-host loops may run on
    # several OpenMP threads (for the timed CPU baseline); integer sums and
    # per-host results must be the same for any thread count
    from traffic import SMALL, Traffic
    tr = Traffic(SMALL, pkts_per_slice=30_000)
    o = oracle.Oracle(c=18, k=5, g=512, seg_len=1, partition=0, seed=8)
    for s in range(4):
        if s:
            o.advance()
        o.ingest(tr.slice_pairs(s))
    runs = []
    try:
        for t in (1, 3, 8):
            oracle.set_threads(t)
            assert oracle.threads() == t
            e, a, f = o.estimate(tr.aips, 5)
            n0 = o.pool_inactive(3)
            runs.append((o.census(), e, a, f, o.age_counts(tr.aips), n0, o.estimate_hosts(tr.aips, 3, n0)[0]))
    finally:
        oracle.set_threads(1)
    for r in runs[1:]:
        for x, y in zip(runs[0], r):
            assert np.array_equal(x, y)
