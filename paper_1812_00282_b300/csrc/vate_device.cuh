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
    uint8_t *pool;
    uint64_t P;          // 2^c ATs
    uint64_t key_h;      // key of H
    uint64_t key_bh;     // key of BH
    uint64_t a, b;       // block sizes (Eq. 9-10, or a', b' of the low-deviation partition)
    uint64_t ma;         // ceil(2^64 / a)
    uint64_t ma1;        // ceil(2^64 / (a + 1)) (low-deviation partition)
    uint64_t first;      // low-deviation: ATs below this index are in blocks of size a
    uint32_t c, k, twok, g, L, log2L, segbits, partition;
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

// first pool position of segment j of host aip: seg(aip, j) * L
VATE_HD uint32_t seg_base(const Geom &G, uint32_t aip, uint32_t j) {
    uint64_t m = mix64(G.key_h ^ ((uint64_t)aip << 32) ^ (uint64_t)j);
    return (uint32_t)(m >> (64 - G.segbits)) << G.log2L;
}

// pid = H(aip, i)
VATE_HD uint32_t vat_pid(const Geom &G, uint32_t aip, uint32_t i) {
    return seg_base(G, aip, i >> G.log2L) + (i & (G.L - 1));
}

// block index of pool position pid
VATE_HD uint32_t block_of(const Geom &G, uint32_t pid) {
    if (G.partition == 0 || pid < G.first) return (uint32_t)mulhi64(G.ma, (uint64_t)pid);
    return (uint32_t)mulhi64(G.ma1, (uint64_t)pid + G.twok - G.b);
}

// ACT of block blk when BACT^0 = bact0 (Eq. 8)
VATE_HD uint32_t act_of_block(uint32_t bact0, uint32_t blk, uint32_t twok) {
    uint32_t s = bact0 + blk;
    return s >= twok ? s - twok : s;
}

// ---- SWAR helpers (bytes < 128) -------------------------------------------
constexpr uint32_t ONES = 0x01010101u;
constexpr uint32_t HIGH = 0x80808080u;

// Constants selecting the ATs active in W(t-k'+1, k') for an AT whose ACT is
// act: the active values are {act, act-1, ..., act-k'+1} mod 2k.  They form
// one range [act-k'+1, act] or, when that wraps below 0, the two ranges
// [0, act] and [act-k'+1+2k, 2k-1].  A range [lo, hi] is tested per byte as
// "bit 7 of (v + 128 - lo)" and not "bit 7 of (v + 127 - hi)"; an empty
// range uses lo = 128.
struct CheckConsts {
    uint32_t ge1, gt1, ge2, gt2;
};

VATE_HD CheckConsts check_consts(uint32_t act, uint32_t kprime, uint32_t twok) {
    CheckConsts cc;
    int lo = (int)act - (int)kprime + 1;
    if (lo >= 0) {
        cc.ge1 = (128u - (uint32_t)lo) * ONES;
        cc.gt1 = (127u - act) * ONES;
        cc.ge2 = 0u;                  // lo = 128: never
        cc.gt2 = 0u;
    } else {
        cc.ge1 = 128u * ONES;         // lo = 0: always
        cc.gt1 = (127u - act) * ONES;
        uint32_t lo2 = (uint32_t)(lo + (int)twok);
        cc.ge2 = (128u - lo2) * ONES;
        cc.gt2 = (127u - (twok - 1u)) * ONES;
    }
    return cc;
}

// bit 7 set in each byte of w holding an active AT (Algorithm 1 on 4 ATs)
VATE_HD uint32_t swar_active(uint32_t w, const CheckConsts &cc) {
    uint32_t r1 = (w + cc.ge1) & ~(w + cc.gt1);
    uint32_t r2 = (w + cc.ge2) & ~(w + cc.gt2);
    return (r1 | r2) & HIGH;
}

// Algorithm 3 on 4 ATs: at ACT 0 values 0..k become 2k; at ACT k values k..2k-1
// and 0 become 2k.  Bytes whose ACT is neither 0 nor k must not be passed here.
VATE_HD uint32_t swar_preserve(uint32_t w, bool act_is_zero, uint32_t k) {
    uint32_t twok = 2u * k;
    uint32_t clear;
    if (act_is_zero) {
        clear = ~(w + (127u - k) * ONES) & HIGH;                          // v <= k
    } else {
        uint32_t in_k_2k1 = (w + (128u - k) * ONES) & ~(w + (127u - (twok - 1u)) * ONES);  // k <= v <= 2k-1
        uint32_t is_zero = ~(w + 127u * ONES);                             // v <= 0
        clear = (in_k_2k1 | is_zero) & HIGH;
    }
    uint32_t bytes = (clear >> 7) * 0xFFu;    // 0xFF in each cleared byte
    return (w & ~bytes) | ((twok * ONES) & bytes);
}

// Scalar forms (boundary bytes, small L)
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

}  // namespace vate
