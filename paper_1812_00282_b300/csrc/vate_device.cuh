// vate_device.cuh -- mapping and AT arithmetic shared by the kernels and by the
// host-side checking entry points of the library (all __host__ __device__).
//
//   mix64           SplitMix64 output function (Steele, Lea & Flood 2014), the
//                   mixer behind H and BH (the paper's "random hash functions",
//                   Sec. 4.1).
//   bh / seg_pid    vid = BH(bip) in [0, g) by Lemire's multiply-shift range
//                   reduction; H(aip, i) = L * seg(aip, i / L) + i mod L.
//   block_of        AT -> block for the partition of Eq. 9-10 or the
//                   low-deviation one (Sec. 4.1), divisions done as a 64-bit
//                   multiply-high by ceil(2^64 / d) (Lemire, Kaser & Kurz 2019,
//                   exact for 32-bit numerators).
//   act             ACT of block i: (BACT^0 + i) mod 2k (Eq. 8).
//   frame 0         how a handle's pool stores its ATs: the value v of an AT
//                   of block i (an ACT of that block, Sec. 3) is kept as
//                   u = (v - i) mod 2k, the value it would have in block 0;
//                   the inactive value 2k is kept as 2k.  Since block i's
//                   ACT is (BACT^0 + i) mod 2k, CheckAT, the distance of Eq. 5
//                   and SetAT read the same for every AT with ACT = BACT^0, and
//                   both cases of Algorithm 3 clear the same values.  The map
//                   is a bijection per position; pools leave and enter the
//                   library in the paper's form (to_canonical, from_canonical).
//   swar_*          CheckAT (Algorithm 1) and fast PreserveAT (Algorithm 3) on
//                   four ATs of one 32-bit word at once; every AT value is at
//                   most 2k <= 126, so bit 7 of each byte is free to carry the
//                   result of a per-byte comparison.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

namespace vate {

#define VATE_HD __host__ __device__ __forceinline__

// Geometry of one AT pool, passed by value to every kernel.
struct Geom {
    uint8_t *pool;       // base of pool position 0: pool + pid * atw addresses position pid for lo <= pid < hi
                         // (a shard's allocation starts at position lo; nothing outside [lo, hi) is touched)
    uint64_t P;          // 2^c ATs
    uint64_t key_h;      // key of H
    uint64_t key_bh;     // key of BH
    uint64_t a, b;       // block sizes (Eq. 9-10, or a', b' of the low-deviation partition)
    uint64_t ma;         // ceil(2^64 / a)
    uint64_t ma1;        // ceil(2^64 / (a + 1)) (low-deviation partition)
    uint64_t first;      // low-deviation: ATs below this index are in blocks of size a
    uint32_t c, k, twok, g, L, log2L, segbits, partition;
    uint32_t counter;    // 0: asynchronous timestamps; 1: distance recorders
    uint32_t frame0;     // 1: timestamps stored in the frame of block 0 (every handle and group pool);
                         // 0: the paper's per-block values (pools handed in by a caller)
    uint32_t atw;        // bytes per AT: 1 for k <= 63, 2 (uint16) for 64 <= k <= 1023 (for a packed pool:
                         // the width of its values in the paper's form)
    uint32_t packed;     // 1: b-bit fields, pn of them per 32-bit word (vate_packed.cu)
    uint32_t atb, pn;    // packed: bits per AT and fields per word
    uint64_t mpn;        // packed: ceil(2^64 / pn)
    uint64_t lo, hi;     // pool positions held: [0, P) for a whole pool, a 64-aligned range for a shard
    unsigned long long *dbg;   // checked build (VATE_DEBUG): device status [bits, first report]; may be NULL
    // host side only: L2 access-policy window over the pool for every launch
    // that touches it (l2_window_bytes = 0: none)
    uint64_t l2_window_bytes;
    float l2_hit_ratio;
};

VATE_HD uint64_t mix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

VATE_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// ceil(2^64 / d) for d >= 2
inline uint64_t magic_for(uint64_t d) { return (~0ull) / d + 1ull; }

// vid = BH(bip)
VATE_HD uint32_t bh(const Geom &G, uint32_t bip) {
    uint64_t m = mix64(G.key_bh ^ (uint64_t)bip);
    return (uint32_t)(((m >> 32) * (uint64_t)G.g) >> 32);
}

// MurmurHash3's 32-bit finalizer (Appleby), a bijection on 32-bit words
VATE_HD uint32_t fmix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x;
}

// the 64-bit key of host aip from which all its segments are drawn
VATE_HD uint64_t host_key(const Geom &G, uint32_t aip) { return mix64(G.key_h ^ ((uint64_t)aip << 32)); }

// first pool position of segment j of the host with key hk: seg * L, seg the
// top c - log2 L bits of fmix32(low32(hk) ^ j * 0x9E3779B9) ^ high32(hk)
VATE_HD uint32_t seg_base_k(const Geom &G, uint64_t hk, uint32_t j) {
    uint32_t x = fmix32((uint32_t)hk ^ (j * 0x9E3779B9u)) ^ (uint32_t)(hk >> 32);
    return (x >> (32u - G.segbits)) << G.log2L;
}

VATE_HD uint32_t seg_base(const Geom &G, uint32_t aip, uint32_t j) { return seg_base_k(G, host_key(G, aip), j); }

// pid = H(aip, i), for the host with key hk = host_key(G, aip)
VATE_HD uint32_t vat_pid_k(const Geom &G, uint64_t hk, uint32_t i) {
    return seg_base_k(G, hk, i >> G.log2L) + (i & (G.L - 1));
}

// pid = H(aip, i)
VATE_HD uint32_t vat_pid(const Geom &G, uint32_t aip, uint32_t i) { return vat_pid_k(G, host_key(G, aip), i); }

// block index of pool position pid
VATE_HD uint32_t block_of(const Geom &G, uint32_t pid) {
    if (G.partition == 0 || pid < G.first) return (uint32_t)mulhi64(G.ma, (uint64_t)pid);
    return (uint32_t)mulhi64(G.ma1, (uint64_t)pid + G.twok - G.b);
}

// [start, end) of block i (Eq. 9-10, or the low-deviation partition)
VATE_HD void block_range_of(const Geom &G, uint32_t i, uint64_t *s, uint64_t *e) {
    if (G.partition == 0) {
        *s = (uint64_t)i * G.a;
        *e = (i + 1 < G.twok) ? *s + G.a : G.P;
        return;
    }
    uint64_t nsmall = G.twok - G.b;
    if (i < nsmall) {
        *s = (uint64_t)i * G.a;
        *e = *s + G.a;
    } else {
        *s = nsmall * G.a + (uint64_t)(i - nsmall) * (G.a + 1);
        *e = *s + G.a + 1;
    }
}

// first byte of the memory that holds positions [lo, hi)
VATE_HD uint8_t *pool_mem(const Geom &G) { return G.packed ? G.pool : G.pool + G.lo * G.atw; }

// bytes of a packed pool: whole words, rounded up to 16 bytes
VATE_HD uint64_t packed_bytes(const Geom &G) { return ((G.P + G.pn - 1) / G.pn * 4 + 15) / 16 * 16; }

// device bytes that hold positions [lo, hi)
VATE_HD uint64_t held_bytes(const Geom &G) { return G.packed ? packed_bytes(G) : (G.hi - G.lo) * G.atw; }

// ACT of block blk when BACT^0 = bact0 (Eq. 8)
VATE_HD uint32_t act_of_block(uint32_t bact0, uint32_t blk, uint32_t twok) {
    uint32_t s = bact0 + blk;
    return s >= twok ? s - twok : s;
}

// ---- SWAR helpers (bytes < 128) -------------------------------------------
constexpr uint32_t ONES = 0x01010101u;
constexpr uint32_t HIGH = 0x80808080u;

// ---- checked build ---------------------------------------------------------
// Compiled with VATE_DEBUG, the kernels check what their indexing relies on --
// a computed pool position below P, every AT value read within the counter's
// range, every block index below 2k -- and report a violation into the
// handle's status words (G.dbg[0]: VATE_DBG_* bits, OR-ed; G.dbg[1]: the first
// report, bit 63 set, the position or chunk in the low bits and the bit in
// bits 56-62) instead of trapping: a bad position's access is skipped, a bad
// value is read as it is (every kernel stays in bounds whatever a value
// holds).  Without VATE_DEBUG the checks compile to nothing.
#define VATE_DBG_POSITION 1u
#define VATE_DBG_VALUE 2u
#define VATE_DBG_BLOCK 4u

__device__ __forceinline__ void debug_report(const Geom &G, uint32_t bit, uint64_t where) {
    if (!G.dbg) return;
    atomicOr(G.dbg, (unsigned long long)bit);
    atomicCAS(G.dbg + 1, 0ull, (1ull << 63) | ((unsigned long long)bit << 56) | (where & ((1ull << 56) - 1)));
}

// a word of stored values (bytes, or 16-bit halves for k >= 64) with a value
// above the counter's range (2k for timestamps, k for recorders)
__device__ __forceinline__ bool word_out_of_range(const Geom &G, uint32_t w) {
    const uint32_t top = G.counter == 1u ? G.k : G.twok;
    if (G.atw == 1u) return ((((w & ~HIGH) + (127u - top) * ONES) | w) & HIGH) != 0u;
    return (w & 0xFFFFu) > top || (w >> 16) > top;
}

#ifdef VATE_DEBUG
#define VATE_CHECK_POSITION(G, pid) ((pid) < (G).P ? true : (debug_report((G), VATE_DBG_POSITION, (pid)), false))
#define VATE_CHECK_WORD(G, w, where) \
    do { if (word_out_of_range((G), (w))) debug_report((G), VATE_DBG_VALUE, (where)); } while (0)
#define VATE_CHECK_VALUE(G, v, where) \
    do { if ((v) > ((G).counter == 1u ? (G).k : (G).twok)) debug_report((G), VATE_DBG_VALUE, (where)); } while (0)
#define VATE_CHECK_BLOCK(G, blk, where) \
    do { if ((blk) >= (G).twok) debug_report((G), VATE_DBG_BLOCK, (where)); } while (0)
#else
#define VATE_CHECK_POSITION(G, pid) true
#define VATE_CHECK_WORD(G, w, where) do { } while (0)
#define VATE_CHECK_VALUE(G, v, where) do { } while (0)
#define VATE_CHECK_BLOCK(G, blk, where) do { } while (0)
#endif

// Algorithm 1 on four ATs of one word.  For an AT whose ACT is act, the
// values active in W(t-k'+1, k') are {act, act-1, ..., act-k'+1} mod 2k.
// Either that set is one range [act-k'+1, act], or (when it wraps below 0)
// its complement within [0, 2k-1] is the one range [act+1, act+2k-k'].  So
// one range test per byte suffices: bit 7 of (v + 128 - lo) and not bit 7 of
// (v + 127 - hi) says lo <= v <= hi; f flips the result for the complement
// case, and bit 7 of (v + 128 - 2k) removes the inactive value 2k.
struct RangeConsts {
    uint32_t a1, b1, f, pad;
};

VATE_HD RangeConsts range_consts(uint32_t act, uint32_t kprime, uint32_t twok) {
    RangeConsts rc;
    int lo = (int)act - (int)kprime + 1;
    uint32_t rlo, rhi;
    if (lo >= 0) {
        rlo = (uint32_t)lo;
        rhi = act;
        rc.f = 0u;
    } else {
        rlo = act + 1u;
        rhi = act + twok - kprime;
        rc.f = HIGH;
    }
    rc.a1 = (128u - rlo) * ONES;
    rc.b1 = (127u - rhi) * ONES;
    rc.pad = 0u;
    return rc;
}

// bit 7 set in each byte of w holding an active AT; c2k = (128 - 2k) * ONES
VATE_HD uint32_t swar_active(uint32_t w, const RangeConsts &rc, uint32_t c2k) {
    uint32_t r = ((w + rc.a1) & ~(w + rc.b1)) ^ rc.f;
    return r & ~(w + c2k) & HIGH;
}

// swar_active with its three byte-wise additions written as multiply-adds by
// run-time ones (u1..u3, all 1): the same arithmetic, issued on the
// multiply-add pipe instead of the integer-logic pipe that the two LOP3s
// already load.
__device__ __forceinline__ uint32_t swar_active_fma(uint32_t w, const RangeConsts &rc, uint32_t c2k, uint32_t u1,
                                                    uint32_t u2, uint32_t u3) {
    uint32_t r = ((w * u1 + rc.a1) & ~(w * u2 + rc.b1)) ^ rc.f;
    return r & ~(w * u3 + c2k) & HIGH;
}

// Four byte values with every byte above top (top <= 126) replaced by top.
// The high bit of each byte is tested apart from its low seven bits, so no
// sum crosses into the next byte whatever the bytes hold.
VATE_HD uint32_t swar_clamp(uint32_t w, uint32_t top) {
    const uint32_t lo7 = w & ~HIGH;
    const uint32_t over = ((lo7 + (127u - top) * ONES) | w) & HIGH;   // byte > top
    const uint32_t mask = (over >> 7) * 0xFFu;
    return (w & ~mask) | ((top * ONES) & mask);
}

// Census bin of four ATs whose ACT is act: byte = (act + 2k - v) mod 2k, the
// distance of Eq. 5, or 2k for an inactive AT.  Valid values (v <= 2k) never
// borrow across bytes; a pool that may hold others goes through swar_clamp
// first.
VATE_HD uint32_t swar_bins(uint32_t w, uint32_t act, uint32_t twok) {
    uint32_t t = (act + twok) * ONES - w;
    uint32_t ge = (t + (128u - twok) * ONES) & HIGH;          // t >= 2k
    uint32_t d = t - (ge >> 7) * twok;
    uint32_t e = (w + (128u - twok) * ONES) & HIGH;           // v >= 2k: inactive
    uint32_t E = (e >> 7) * 0xFFu;
    return (d & ~E) | ((twok * ONES) & E);
}

// Distance recorders (VDRE): value 0..k, k = inactive; one slide adds 1 to
// every recorder below k (four recorders per word; values <= 126).
VATE_HD uint32_t swar_dr_age(uint32_t w, uint32_t k) {
    uint32_t t = w + ONES;
    uint32_t over = (t + (127u - k) * ONES) & HIGH;          // t > k
    uint32_t bytes = (over >> 7) * 0xFFu;
    return (t & ~bytes) | ((k * ONES) & bytes);
}

// Range constants of CheckDR for window k': active iff 0 <= v <= k'-1.
VATE_HD RangeConsts dr_range_consts(uint32_t kprime) {
    RangeConsts rc;
    rc.a1 = 128u * ONES;
    rc.b1 = (127u - (kprime - 1u)) * ONES;
    rc.f = 0u;
    rc.pad = 0u;
    return rc;
}

// Scalar forms (boundary bytes, small L)
VATE_HD bool check_dr(uint32_t v, uint32_t kprime) { return v < kprime; }

VATE_HD bool check_at(uint32_t v, uint32_t act, uint32_t kprime, uint32_t twok) {
    if (v == twok) return false;
    uint32_t d = act + twok - v;
    if (d >= twok) d -= twok;
    return d < kprime;
}

VATE_HD uint32_t preserve_at(uint32_t v, uint32_t act, uint32_t k) {
    uint32_t twok = 2u * k;
    if (act == 0u && v <= k) return twok;
    if (act == k && ((v >= k && v <= twok - 1u) || v == 0u)) return twok;
    return v;
}

// ---- 16-bit ATs (k >= 64): two per 32-bit word, bit 15 of each half free ----
constexpr uint32_t ONES16 = 0x00010001u;
constexpr uint32_t HIGH16 = 0x80008000u;

// range_consts for 16-bit lanes (values <= 2k <= 2046)
VATE_HD RangeConsts range_consts16(uint32_t act, uint32_t kprime, uint32_t twok) {
    RangeConsts rc;
    int lo = (int)act - (int)kprime + 1;
    uint32_t rlo, rhi;
    if (lo >= 0) {
        rlo = (uint32_t)lo;
        rhi = act;
        rc.f = 0u;
    } else {
        rlo = act + 1u;
        rhi = act + twok - kprime;
        rc.f = HIGH16;
    }
    rc.a1 = (0x8000u - rlo) * ONES16;
    rc.b1 = (0x7FFFu - rhi) * ONES16;
    rc.pad = 0u;
    return rc;
}

VATE_HD RangeConsts dr_range_consts16(uint32_t kprime) {
    RangeConsts rc;
    rc.a1 = 0x8000u * ONES16;
    rc.b1 = (0x7FFFu - (kprime - 1u)) * ONES16;
    rc.f = 0u;
    rc.pad = 0u;
    return rc;
}

// bit 15 set in each half of w holding an active AT; c2k = (0x8000 - 2k) * ONES16
VATE_HD uint32_t swar16_active(uint32_t w, const RangeConsts &rc, uint32_t c2k) {
    uint32_t r = ((w + rc.a1) & ~(w + rc.b1)) ^ rc.f;
    return r & ~(w + c2k) & HIGH16;
}

// ---- frame 0 ---------------------------------------------------------------
// Algorithm 3 in frame 0.  With B = BACT^0 after the slide, the block whose
// ACT became 0 has index i = -B and the one whose ACT became k has i = k - B
// (mod 2k).  At ACT 0 values 0..k are cleared, i.e. u = v - i in B..B+k; at
// ACT k values k..2k-1 and 0 (= 2k) are cleared, i.e. u = v - i in B..B+k as
// well.  Both blocks clear the cyclic range [B, B + k] (mod 2k).
VATE_HD uint32_t preserve_frame0(uint32_t u, uint32_t B, uint32_t k) {
    uint32_t twok = 2u * k;
    if (u >= twok) return twok;
    uint32_t d = u + twok - B;
    if (d >= twok) d -= twok;
    return d <= k ? twok : u;
}

// Range constants (as for CheckAT) selecting the cyclic range [B, B + k]: one
// range [B, B + k] when it does not wrap, else the complement of
// [B + k - 2k + 1, B - 1] (that complement also takes in 2k, which a clear
// leaves unchanged).
VATE_HD RangeConsts preserve_consts_frame0(uint32_t B, uint32_t k) {
    uint32_t twok = 2u * k, hi = B + k;
    RangeConsts rc;
    if (hi < twok) {
        rc.a1 = (128u - B) * ONES;
        rc.b1 = (127u - hi) * ONES;
        rc.f = 0u;
    } else {
        rc.a1 = (128u - (hi - twok + 1u)) * ONES;
        rc.b1 = (127u - (B - 1u)) * ONES;
        rc.f = HIGH;
    }
    rc.pad = 0u;
    return rc;
}

// preserve_frame0 on four ATs of one word
VATE_HD uint32_t swar_preserve_frame0(uint32_t w, const RangeConsts &pc, uint32_t twok) {
    uint32_t clear = (((w + pc.a1) & ~(w + pc.b1)) ^ pc.f) & HIGH;
    uint32_t bytes = (clear >> 7) * 0xFFu;
    return (w & ~bytes) | ((twok * ONES) & bytes);
}

// The paper's value of a frame-0 AT of block blk, and back.  Values above 2k
// (not produced by the library) are taken as inactive.
VATE_HD uint32_t to_canonical(uint32_t u, uint32_t blk, uint32_t twok) {
    if (u >= twok) return twok;
    uint32_t v = u + blk;
    return v >= twok ? v - twok : v;
}

VATE_HD uint32_t from_canonical(uint32_t v, uint32_t blk, uint32_t twok) {
    if (v >= twok) return twok;
    uint32_t u = v + twok - blk;
    return u >= twok ? u - twok : u;
}

// ---------------------------------------------------------------------------
// SWAR tests on bit-packed ATs: B-bit fields, PN = floor(32 / B) per 32-bit
// word, field f at bits [fB, fB + B).  A word is split into its even fields
// (left in place) and its odd fields (shifted down by B); either half has its
// fields at bits 2iB with B free bits above each, so adding a constant c' <=
// 2^B to the half sets the bit just above a field (its guard, bit 2iB + B) iff
// field + c' >= 2^B, with no carry into the next field.  With c' = 2^B - c the
// guard says "field >= c"; the top field's guard stays inside the word for
// every B in 4..11.
// ---------------------------------------------------------------------------
VATE_HD constexpr uint32_t packed_rep(uint32_t B, uint32_t c) {
    uint32_t r = 0;
    for (uint32_t i = 0; 2u * i < 32u / B; i++) r |= c << (2u * i * B);
    return r;
}

// The constants of one window test: field active iff
// ((field >= a) & !(field >= b)) ^ complement, and field < 2k.
struct PackedRange {
    uint32_t ca, cb, c2k, f;
};

VATE_HD PackedRange packed_range(uint32_t B, uint32_t a, uint32_t b, uint32_t twok, bool complement) {
    PackedRange r;
    r.ca = packed_rep(B, (1u << B) - a);
    r.cb = packed_rep(B, (1u << B) - b);
    r.c2k = packed_rep(B, (1u << B) - twok);
    r.f = complement ? packed_rep(B, 1u << B) : 0u;
    return r;
}

// CheckAT of a frame-0 timestamp (ACT = BACT^0 for every AT): active iff
// v < 2k and (BACT^0 - v) mod 2k < k'.  The window is the cyclic range
// [lo, BACT^0] with lo = (BACT^0 - k' + 1) mod 2k; when it wraps past 0 it is
// the complement of [BACT^0 + 1, lo) in [0, 2k).  Needs 1 <= k' <= k.
VATE_HD PackedRange packed_range_at(uint32_t B, uint32_t bact0, uint32_t kprime, uint32_t twok) {
    const uint32_t lo = bact0 + 1u >= kprime ? bact0 + 1u - kprime : bact0 + 1u + twok - kprime;
    return lo <= bact0 ? packed_range(B, lo, bact0 + 1u, twok, false) : packed_range(B, bact0 + 1u, lo, twok, true);
}

// CheckDR of a recorder: active iff v < k'.
VATE_HD PackedRange packed_range_dr(uint32_t B, uint32_t kprime, uint32_t twok) {
    return packed_range(B, 0u, kprime, twok, false);
}

VATE_HD uint32_t popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return (uint32_t)__popc(x);
#else
    return (uint32_t)__builtin_popcount(x);
#endif
}

// The number of active fields among fields [fa, fb) of word w (0 <= fa <= fb
// <= PN).  An even field's guard sits B bits above its start, an odd field's
// (in the shifted half) at its start; the odd guards are moved up one bit so
// that both halves share one popcount.
template <int B>
VATE_HD uint32_t packed_count_word(uint32_t w, const PackedRange &r, uint32_t fa, uint32_t fb) {
    constexpr uint32_t EVEN = packed_rep(B, (1u << B) - 1u), GUARD = packed_rep(B, 1u << B);
    const uint32_t he = w & EVEN, ho = (w >> B) & EVEN;
    const uint32_t ge = ((((he + r.ca) & ~(he + r.cb)) ^ r.f) & ~(he + r.c2k)) & GUARD;
    const uint32_t go = ((((ho + r.ca) & ~(ho + r.cb)) ^ r.f) & ~(ho + r.c2k)) & GUARD;
    const uint32_t span_e = (uint32_t)((1ull << (fb * B + B)) - (1ull << (fa * B + B)));
    const uint32_t span_o = (uint32_t)((1ull << (fb * B)) - (1ull << (fa * B)));
    return popc32((ge & span_e) | ((go & span_o) << 1));
}

}  // namespace vate
