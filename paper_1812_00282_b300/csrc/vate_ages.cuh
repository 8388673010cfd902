// vate_ages.cuh -- per-age counts of one host's VATs (for d < k, the VATs
// last set d slices ago).  For k <= 15, where every stored value fits a
// 32-bit one-hot mask, as bit-sliced counters in registers (the learned
// estimator's features in vate_learned.cu, and vate_age_counts); for larger k
// as shared-memory counters (age_columns_vec, vate_age_counts).
#pragma once
#include "vate_device.cuh"

namespace vate {

// Per-age counts of one host's VATs seen by this lane, in registers, as
// bit-sliced (vertical) counters over the byte values 0..31 (2k <= 30 here):
// bit u of plane j is bit j of the number of bytes equal to u, planes 1, 2,
// ..., 128.  Sixteen bytes at a time enter as one-hot masks 1 << u through a
// carry-save adder tree (each adder two 3-input logic operations), the
// sixteens rippling into the high planes.  In frame 0 the age of a
// timestamp's value u is (BACT^0 - u) mod 2k; a distance recorder's value is
// its age.  At most 15 chunks (240 bytes) are counted before the planes are
// folded into the warp's totals (lane d holds age d).
__device__ __forceinline__ void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
}

struct AgePlanes {
    uint32_t p[8] = {0, 0, 0, 0, 0, 0, 0, 0};     // planes of weight 1, 2, 4, ..., 128

    __device__ __forceinline__ void add_chunk(uint4 w) {
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        uint32_t m[16];
#pragma unroll
        for (int b = 0; b < 16; b++) m[b] = 1u << ((words[b >> 2] >> (8 * (b & 3))) & 31u);
        uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
        csa(twosA, p[0], p[0], m[0], m[1]);
        csa(twosB, p[0], p[0], m[2], m[3]);
        csa(foursA, p[1], p[1], twosA, twosB);
        csa(twosA, p[0], p[0], m[4], m[5]);
        csa(twosB, p[0], p[0], m[6], m[7]);
        csa(foursB, p[1], p[1], twosA, twosB);
        csa(eightsA, p[2], p[2], foursA, foursB);
        csa(twosA, p[0], p[0], m[8], m[9]);
        csa(twosB, p[0], p[0], m[10], m[11]);
        csa(foursA, p[1], p[1], twosA, twosB);
        csa(twosA, p[0], p[0], m[12], m[13]);
        csa(twosB, p[0], p[0], m[14], m[15]);
        csa(foursB, p[1], p[1], twosA, twosB);
        csa(eightsB, p[2], p[2], foursA, foursB);
        csa(sixteens, p[3], p[3], eightsA, eightsB);
        uint32_t c = sixteens;                 // ripple into 16, 32, 64, 128
#pragma unroll
        for (int j = 4; j < 8; j++) {
            const uint32_t t = p[j] & c;
            p[j] ^= c;
            c = t;
        }
    }
    __device__ __forceinline__ uint32_t count(uint32_t u) const {
        uint32_t c = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) c |= ((p[j] >> u) & 1u) << j;
        return c;
    }
    // add the warp's counts of ages 0..k-1 to the totals (lane d: age d) and restart
    __device__ __forceinline__ void fold(uint32_t bact0, uint32_t k, uint32_t counter, uint32_t lane, uint32_t &cd) {
        const uint32_t twok = 2u * k;
        for (uint32_t d = 0; d < k; d++) {
            uint32_t u = bact0 + twok - d;
            if (u >= twok) u -= twok;
            if (counter == 1u) u = d;
            const uint32_t c = __reduce_add_sync(0xFFFFFFFFu, count(u));
            if (lane == d) cd += c;
        }
#pragma unroll
        for (int j = 0; j < 8; j++) p[j] = 0;
    }
};

// The segments' chunks as in gather_host_vec: the lanes hash 32 segments per
// round, read the round's chunks with the segment base shuffled from the
// hashing lane, all loads of a round issued before any is counted.
template <int CPSL>
__device__ __forceinline__ void age_counts_vec(const Geom &G, uint32_t bact0, uint64_t hk, uint32_t lane,
                                               AgePlanes &ap, uint32_t &cd) {
    constexpr int CPS = 1 << CPSL;
    constexpr uint32_t ROUNDS_PER_FOLD = 15u / CPS;                 // a round gives a lane CPS chunks
    const uint32_t nseg = G.g >> G.log2L;
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    uint32_t since = 0;
    for (uint32_t r0 = 0; r0 < nseg; r0 += 32u) {
        if (since++ == ROUNDS_PER_FOLD) {
            ap.fold(bact0, G.k, G.counter, lane, cd);
            since = 1;
        }
        const uint32_t s = r0 + lane;
        const uint32_t base = s < nseg ? (seg_base_k(G, hk, s) >> 4) : 0u;   // first chunk of the segment
        const uint32_t segs = min(32u, nseg - r0);
        uint4 w[CPS];
        bool valid[CPS];
#pragma unroll
        for (int it = 0; it < CPS; it++) {
            const uint32_t c = it * 32u + lane;
            const uint32_t q = __shfl_sync(0xFFFFFFFFu, base, (c >> CPSL) & 31u) + (c & (CPS - 1u));
            valid[it] = c < (segs << CPSL);
            w[it] = make_uint4(0u, 0u, 0u, 0u);
            if (valid[it]) w[it] = __ldg(pool16 + q);
        }
        const uint32_t none = G.twok * ONES;                          // a missing chunk counts as inactive ATs
#pragma unroll
        for (int it = 0; it < CPS; it++) ap.add_chunk(valid[it] ? w[it] : make_uint4(none, none, none, none));
    }
}

// Segments of SB = 2, 4 or 8 bytes (L = 2, 4, 8 with byte ATs): lane j loads
// segments 32 q + j of a round with one SB-byte load each (hashing each
// segment once, as gather_host_seg), 16 / SB of them filling one 16-byte chunk
// of the planes; missing segments count as inactive ATs.  The rounds are
// warp-uniform, so the fold (a warp reduction) runs in every lane together.
template <int SB>
__device__ __forceinline__ void age_counts_seg(const Geom &G, uint32_t bact0, uint64_t hk, uint32_t lane,
                                               AgePlanes &ap, uint32_t &cd) {
    constexpr int SPC = 16 / SB;                                    // segments per chunk
    const uint32_t nseg = G.g >> G.log2L;
    const uint32_t none = G.twok * ONES;
    uint32_t chunks = 0;
    for (uint32_t r0 = 0; r0 < nseg; r0 += 32u * SPC) {
        uint32_t words[4] = {none, none, none, none};
#pragma unroll
        for (int q = 0; q < SPC; q++) {
            const uint32_t sg = r0 + 32u * q + lane;
            if (sg >= nseg) continue;
            const uint8_t *at = G.pool + seg_base_k(G, hk, sg);     // first AT of the segment (SB-aligned)
            if (SB == 2) {
                const uint32_t v = __ldg(reinterpret_cast<const unsigned short *>(at));
                const int sh = 16 * (q & 1);
                words[q >> 1] = (words[q >> 1] & ~(0xFFFFu << sh)) | (v << sh);
            } else if (SB == 4) {
                words[q] = __ldg(reinterpret_cast<const uint32_t *>(at));
            } else {
                const uint2 v = __ldg(reinterpret_cast<const uint2 *>(at));
                words[2 * q] = v.x;
                words[2 * q + 1] = v.y;
            }
        }
        ap.add_chunk(make_uint4(words[0], words[1], words[2], words[3]));
        if (++chunks == 15u) {                                      // at most 240 ATs per lane per value
            ap.fold(bact0, G.k, G.counter, lane, cd);
            chunks = 0;
        }
    }
}

// The count of age d (d < k) of one host's VATs, in lane d; 0 in other lanes.
__device__ __forceinline__ uint32_t host_age_counts(const Geom &G, uint32_t bact0, uint32_t aip, uint32_t lane) {
    AgePlanes ap;
    uint32_t cd = 0;
    const uint64_t hk = host_key(G, aip);
    if (G.L == 16) age_counts_vec<0>(G, bact0, hk, lane, ap, cd);
    else if (G.L == 32) age_counts_vec<1>(G, bact0, hk, lane, ap, cd);
    else if (G.L == 64) age_counts_vec<2>(G, bact0, hk, lane, ap, cd);
    else if (G.L == 2) age_counts_seg<2>(G, bact0, hk, lane, ap, cd);
    else if (G.L == 4) age_counts_seg<4>(G, bact0, hk, lane, ap, cd);
    else if (G.L == 8) age_counts_seg<8>(G, bact0, hk, lane, ap, cd);
    else {                      // one byte per VAT: sixteen VATs per lane make a chunk
        const uint32_t none = G.twok;
        for (uint32_t i0 = 0; i0 < G.g; i0 += 32u * 16u) {
            uint32_t words[4] = {0, 0, 0, 0};
#pragma unroll
            for (int b = 0; b < 16; b++) {
                const uint32_t i = i0 + 32u * b + lane;
                const uint32_t v = i < G.g ? (uint32_t)__ldg(G.pool + vat_pid_k(G, hk, i)) : none;
                words[b >> 2] |= v << (8 * (b & 3));
            }
            ap.add_chunk(make_uint4(words[0], words[1], words[2], words[3]));
            ap.fold(bact0, G.k, G.counter, lane, cd);
        }
    }
    ap.fold(bact0, G.k, G.counter, lane, cd);
    return cd;
}

// Per-age counts for any k <= 63 into this lane's shared-memory column
// (col[d * 32] for d < k): the host's segments read as 16-byte chunks as in
// age_counts_vec, each word's distances found with SWAR (swar_bins: the
// distance of Eq. 5 with ACT = BACT^0 in frame 0, 2k for an inactive AT; a
// recorder's value is its distance, k when inactive), and every byte with
// d < k added to its counter with a shared-memory atomic.
template <int CPSL>
__device__ __forceinline__ void age_columns_vec(const Geom &G, uint32_t bact0, uint64_t hk, uint32_t lane,
                                                uint32_t *col) {
    constexpr int CPS = 1 << CPSL;
    const uint32_t nseg = G.g >> G.log2L;
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    for (uint32_t r0 = 0; r0 < nseg; r0 += 32u) {
        const uint32_t s = r0 + lane;
        const uint32_t base = s < nseg ? (seg_base_k(G, hk, s) >> 4) : 0u;   // first chunk of the segment
        const uint32_t segs = min(32u, nseg - r0);
        uint4 w[CPS];
        bool valid[CPS];
#pragma unroll
        for (int it = 0; it < CPS; it++) {
            const uint32_t c = it * 32u + lane;
            const uint32_t q = __shfl_sync(0xFFFFFFFFu, base, (c >> CPSL) & 31u) + (c & (CPS - 1u));
            valid[it] = c < (segs << CPSL);
            w[it] = make_uint4(0u, 0u, 0u, 0u);
            if (valid[it]) w[it] = __ldg(pool16 + q);
        }
#pragma unroll
        for (int it = 0; it < CPS; it++) {
            if (!valid[it]) continue;
            const uint32_t words[4] = {w[it].x, w[it].y, w[it].z, w[it].w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint32_t bins = G.counter == 1u ? words[j] : swar_bins(words[j], bact0, G.twok);
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    const uint32_t d = (bins >> (8 * b)) & 0xFFu;
                    if (d < G.k) atomicAdd(&col[d * 32u], 1u);
                }
            }
        }
    }
}

}  // namespace vate
