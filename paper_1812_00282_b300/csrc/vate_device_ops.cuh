// vate_device_ops.cuh -- per-chunk device operations shared by the
// single-pool kernels (vate_kernels.cu) and the monitor-group kernels
// (vate_group.cu), so that both run exactly the same arithmetic.
#pragma once
#include "vate_device.cuh"

namespace vate {

// PreserveAT (Algorithm 3) on the 16-byte chunk at pool offset `base` of a
// frame-0 pool, for the bytes inside [s0, e0) (block with ACT 0) or [s1, e1)
// (block with ACT k): both clear the values selected by pc
// (preserve_consts_frame0 of the new BACT^0).
// CG: the chunk is read with an L2-only load, so that the SM keeps no L1 copy
// of it (the monitor group's single launch later reads the pool through the
// read-only path after other blocks have written it).
template <bool CG = false>
__device__ __forceinline__ void preserve_chunk(uint8_t *pool, uint64_t base, const RangeConsts &pc, uint32_t twok,
                                               uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1) {
    uint4 *p = reinterpret_cast<uint4 *>(pool + base);
    uint4 w = CG ? __ldcg(p) : *p;
    uint4 r;
    r.x = swar_preserve_frame0(w.x, pc, twok);
    r.y = swar_preserve_frame0(w.y, pc, twok);
    r.z = swar_preserve_frame0(w.z, pc, twok);
    r.w = swar_preserve_frame0(w.w, pc, twok);
    bool full = (base >= s0 && base + 16 <= e0) || (base >= s1 && base + 16 <= e1);
    if (!full) {            // keep the bytes outside both blocks
        uint32_t in[4] = {w.x, w.y, w.z, w.w}, out[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int b = 0; b < 16; b++) {
            uint64_t pos = base + b;
            if ((pos >= s0 && pos < e0) || (pos >= s1 && pos < e1)) continue;
            uint32_t m = 0xFFu << (8 * (b & 3));
            out[b >> 2] = (out[b >> 2] & ~m) | (in[b >> 2] & m);
        }
        r.x = out[0]; r.y = out[1]; r.z = out[2]; r.w = out[3];
    }
    if (r.x != w.x || r.y != w.y || r.z != w.z || r.w != w.w) *p = r;
}

// Census of one 16-byte chunk of a timestamp pool in the paper's form (each
// AT read with the ACT of its block) into this lane's column (col[bin * 32]):
// the distance of Eq. 5 for active values, 2k for inactive ones and for any
// byte above 2k (a caller's pool is not checked).
__device__ __forceinline__ void census_chunk(const Geom &G, uint32_t bact0, uint32_t pid0, uint4 w, uint32_t pat,
                                             uint32_t *col, uint32_t &inactive_runs) {
    if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) {
        inactive_runs++;
        return;
    }
    const uint32_t b0 = block_of(G, pid0);
    if (b0 != block_of(G, pid0 + 15u)) {       // the chunk straddles two blocks
        const uint32_t raw[4] = {w.x, w.y, w.z, w.w};
        for (int b = 0; b < 16; b++) {
            const uint32_t v = (raw[b >> 2] >> (8 * (b & 3))) & 0xFFu;
            uint32_t bin = G.twok;
            if (v < G.twok) {
                const uint32_t act = act_of_block(bact0, block_of(G, pid0 + b), G.twok);
                const uint32_t d = act + G.twok - v;
                bin = d >= G.twok ? d - G.twok : d;
            }
            col[bin * 32u] += 1u;
        }
        return;
    }
    const uint32_t act = act_of_block(bact0, b0, G.twok);
    const uint32_t words[4] = {
        swar_bins(swar_clamp(w.x, G.twok), act, G.twok), swar_bins(swar_clamp(w.y, G.twok), act, G.twok),
        swar_bins(swar_clamp(w.z, G.twok), act, G.twok), swar_bins(swar_clamp(w.w, G.twok), act, G.twok)};
    // shared-memory atomics without a return value: consecutive bytes of one
    // bin do not wait for each other's read-modify-write
#pragma unroll
    for (int b = 0; b < 16; b++) atomicAdd(&col[((words[b >> 2] >> (8 * (b & 3))) & 0xFFu) * 32u], 1u);
}

// Census of one 16-byte chunk of a pool whose ATs are all read with the same
// ACT (timestamps in the frame of block 0) or hold their own distance
// (recorders): the stored values themselves go into this lane's column
// (col[value * 32]), each clamped to the inactive value inact -- which is how
// the distance bins count values above it, and keeps every index below
// inact + 1 -- and a chunk of 16 inactive ATs is counted in inactive_runs.
// census_raw_bin turns a value's row into its census bin.
__device__ __forceinline__ void census_chunk_raw(uint4 w, uint32_t pat, uint32_t inact, uint32_t *col,
                                                 uint32_t &inactive_runs) {
    if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) {
        inactive_runs++;
        return;
    }
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int b = 0; b < 16; b++) {
        const uint32_t v = min((words[b >> 2] >> (8 * (b & 3))) & 0xFFu, inact);
        atomicAdd(&col[v * 32u], 1u);
    }
}

// Census bin of stored value r (r <= inact): a frame-0 timestamp at distance
// (BACT^0 - r) mod 2k, 2k inactive; a recorder's value is its distance, k
// inactive (bin 2k).
__device__ __forceinline__ uint32_t census_raw_bin(const Geom &G, uint32_t bact0, uint32_t r) {
    if (G.counter == 1u) return r < G.k ? r : G.twok;
    if (r >= G.twok) return G.twok;
    const uint32_t d = bact0 + G.twok - r;
    return d >= G.twok ? d - G.twok : d;
}

// The end of a census, once a block has added its counts into acc (2k + 1
// counters that are zero between calls) with 64-bit atomics: the last block to
// finish copies acc into hist, zeroes acc and re-arms ticket for the next
// launch.  Called by every thread of the block.
__device__ __forceinline__ void census_publish(uint64_t *__restrict__ acc, uint64_t *__restrict__ hist,
                                               unsigned int *__restrict__ ticket, uint32_t nbins) {
    __threadfence();
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (uint32_t b = threadIdx.x; b < nbins; b += blockDim.x) {
        hist[b] = __ldcg(acc + b);
        acc[b] = 0;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

__device__ __forceinline__ void census_add(uint64_t *acc, uint32_t bin, uint32_t count) {
    if (count) atomicAdd(reinterpret_cast<unsigned long long *>(acc + bin), (unsigned long long)count);
}

// The end of a census whose block counted into nrows shared-memory rows of
// nbins bins (rows[r * nbins + b]): the block's sum of the rows goes into acc,
// then census_publish.  Called by every thread of the block.
__device__ __forceinline__ void census_finish(const uint32_t *rows, uint32_t nrows, uint32_t nbins,
                                              uint64_t *__restrict__ acc, uint64_t *__restrict__ hist,
                                              unsigned int *__restrict__ ticket) {
    __syncthreads();
    for (uint32_t bin = threadIdx.x; bin < nbins; bin += blockDim.x) {
        uint32_t t = 0;
        for (uint32_t r = 0; r < nrows; r++) t += rows[(size_t)r * nbins + bin];
        census_add(acc, bin, t);
    }
    census_publish(acc, hist, ticket, nbins);
}

// Eq. 11 in FP32 from exact integers: g * log1p((N0*g - V0*P) / (V0*P)).
__device__ __forceinline__ float estimate_eq11(uint32_t g, uint64_t P, uint64_t N0, uint32_t A, uint8_t &flags) {
    flags = 0;
    uint64_t V0 = (uint64_t)g - A;
    if (V0 == 0) { V0 = 1; flags |= 1u; }
    if (N0 == 0) { N0 = 1; flags |= 2u; }
    long long num = (long long)(N0 * (uint64_t)g) - (long long)(V0 * P);
    float x = (float)num / (float)(V0 * P);
    return (float)g * log1pf(x);
}

// N0 for window k' from the census of the last close
__device__ __forceinline__ uint64_t pool_inactive(const uint64_t *hist, uint64_t P, uint32_t kprime) {
    uint64_t active = 0;
    for (uint32_t d = 0; d < kprime; d++) active += hist[d];
    return P - active;
}

// Active VATs seen by this lane for one host of a frame-0 pool (warp per
// host; a segment of L ATs of W bytes each spans 16 << CPSL bytes): in each
// round the 32 lanes hash 32 consecutive segments; the segments' 16-byte
// chunks are then read by consecutive lanes (for byte ATs and L = 32, lanes
// 2j and 2j+1 read the two halves of one 32-byte sector), the segment base
// coming from the hashing lane by shuffle.  All RB * CPS loads of a batch are
// issued before any is tested.  FULL: the number of segments is a multiple of
// 32 * RB.  Every AT is tested with the same range constants rc (CheckAT with
// ACT = BACT^0, or CheckDR), so no block is looked up.  Active ATs are counted
// per lane of the SWAR word (4 bytes or 2 halves) in an accumulator folded
// after each batch.  u1..u3 are run-time ones.
// SHARD: the pool holds only the positions [lo, hi) (64-aligned, so a
// segment is wholly inside or outside); segments outside are not read.
template <int CPSL, int RB, bool FULL, int W = 1, bool SHARD = false, bool CG = false>
__device__ __forceinline__ uint32_t gather_host_vec(const Geom &G, const RangeConsts &rc, uint32_t c2k, uint32_t aip,
                                                    uint32_t u1, uint32_t u2, uint32_t u3, uint32_t lane) {
    constexpr int CPS = 1 << CPSL;                      // 16-byte chunks per segment
    constexpr int NL = RB * CPS;                        // loads per lane per batch
    constexpr uint32_t ATS_PER_CHUNK_LOG2 = W == 1 ? 4 : 3;
    const uint32_t nseg = G.g >> G.log2L;              // segments per host
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    uint32_t cnt = 0;
    const uint64_t hk = host_key(G, aip);
    const uint32_t q_lo = (uint32_t)((G.lo * W) >> 4), q_n = (uint32_t)(((G.hi - G.lo) * W) >> 4);
    for (uint32_t r0 = 0; r0 < nseg; r0 += 32u * RB) {
        uint32_t base[RB];                              // first chunk of the segment
#pragma unroll
        for (int rb = 0; rb < RB; rb++) {
            uint32_t s = r0 + 32u * rb + lane;
            base[rb] = (FULL || s < nseg) ? (seg_base_k(G, hk, s) >> ATS_PER_CHUNK_LOG2) : 0u;
        }
        uint4 w[NL];
        bool valid[NL];
#pragma unroll
        for (int rb = 0; rb < RB; rb++) {
            const uint32_t segs_here = FULL ? 32u : ((r0 + 32u * rb < nseg) ? min(32u, nseg - r0 - 32u * rb) : 0u);
#pragma unroll
            for (int it = 0; it < CPS; it++) {
                const int j = rb * CPS + it;
                uint32_t c = it * 32u + lane;
                uint32_t src = (c >> CPSL) & 31u;
                uint32_t q = __shfl_sync(0xFFFFFFFFu, base[rb], src) + (c & (CPS - 1u));
                valid[j] = FULL || c < (segs_here << CPSL);
                if (SHARD) valid[j] = valid[j] && (q - q_lo) < q_n;
                w[j] = make_uint4(0u, 0u, 0u, 0u);
                if (valid[j]) {
                    w[j] = CG ? __ldcg(pool16 + q) : __ldg(pool16 + q);
                    VATE_CHECK_WORD(G, w[j].x, q);
                    VATE_CHECK_WORD(G, w[j].y, q);
                    VATE_CHECK_WORD(G, w[j].z, q);
                    VATE_CHECK_WORD(G, w[j].w, q);
                }
            }
        }
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < NL; j++) {
            if (!valid[j]) continue;
            if (W == 1) {
                // (m >> 7) added as a multiply-high by 2^25 (multiply-add pipe)
                acc = __umulhi(swar_active_fma(w[j].x, rc, c2k, u1, u2, u3), 1u << 25) + acc;
                acc = __umulhi(swar_active_fma(w[j].y, rc, c2k, u1, u2, u3), 1u << 25) + acc;
                acc = __umulhi(swar_active_fma(w[j].z, rc, c2k, u1, u2, u3), 1u << 25) + acc;
                acc = __umulhi(swar_active_fma(w[j].w, rc, c2k, u1, u2, u3), 1u << 25) + acc;
            } else {
                acc = __umulhi(swar16_active(w[j].x, rc, c2k), 1u << 17) + acc;
                acc = __umulhi(swar16_active(w[j].y, rc, c2k), 1u << 17) + acc;
                acc = __umulhi(swar16_active(w[j].z, rc, c2k), 1u << 17) + acc;
                acc = __umulhi(swar16_active(w[j].w, rc, c2k), 1u << 17) + acc;
            }
        }
        if (W == 1) {
            uint32_t t = (acc & 0x00FF00FFu) + ((acc >> 8) & 0x00FF00FFu);
            cnt += (t & 0xFFFFu) + (t >> 16);
        } else {
            cnt += (acc & 0xFFFFu) + (acc >> 16);
        }
    }
    return cnt;
}

// Active VATs seen by this lane for one host of a frame-0 pool, one AT per
// load (any L).  CG: loads cached in L2 only -- for a pool that other blocks
// of the same launch have written (the monitor group's single launch), where
// the read-only path could return a line this SM cached before those writes.
template <bool CG = false>
__device__ __forceinline__ uint32_t load_at(const Geom &G, uint32_t pid) {
    if (CG)
        return G.atw == 1u ? (uint32_t)__ldcg(G.pool + pid)
                           : (uint32_t)__ldcg(reinterpret_cast<const uint16_t *>(G.pool) + pid);
    return G.atw == 1u ? (uint32_t)__ldg(G.pool + pid) : (uint32_t)__ldg(reinterpret_cast<const uint16_t *>(G.pool) + pid);
}

template <bool CG = false>
__device__ __forceinline__ uint32_t gather_host_scalar(const Geom &G, uint32_t bact0, uint32_t kprime, uint32_t aip,
                                                       uint32_t lane) {
    uint32_t cnt = 0;
    const uint64_t hk = host_key(G, aip);
#pragma unroll 4
    for (uint32_t i = lane; i < G.g; i += 32u) {
        uint32_t pid = vat_pid_k(G, hk, i);
        if (pid < G.lo || pid >= G.hi) continue;             // another shard's AT
        uint32_t v = load_at<CG>(G, pid);
        VATE_CHECK_VALUE(G, v, pid);
        if (G.counter == 1u) {
            cnt += check_dr(v, kprime) ? 1u : 0u;
            continue;
        }
        cnt += check_at(v, bact0, kprime, G.twok) ? 1u : 0u;
    }
    return cnt;
}

// Warp per host for segments of SB = L x AT-width bytes with SB in {2, 4, 8}
// (L = 2, 4, 8 with byte ATs; L = 1, 2, 4 with 16-bit ones): lane j of a
// round hashes segment 32 r + j of the host and loads the whole segment with
// one 2-, 4- or 8-byte load (a segment is aligned to its size and never
// crosses a 32-byte sector); RB rounds are loaded before any is tested, so
// RB random sectors are in flight per lane.  CheckAT (ACT = BACT^0 in frame
// 0) is the SWAR range test of the vector gather on the segment's word(s); a
// 2-byte segment is widened to a word with inactive values (2k) in the other
// half.  For these L a host's g VATs span g / L sectors, and the kernel is
// bound by the L2's random-sector rate.
template <int SB, int W, bool SHARD, bool CG = false>
__device__ __forceinline__ uint32_t gather_host_seg(const Geom &G, const RangeConsts &rc, uint32_t c2k, uint32_t pad,
                                                    uint32_t aip, uint32_t lane) {
    constexpr int RB = SB == 8 ? 4 : 8;                  // segments in flight per lane
    constexpr int NW = SB == 8 ? 2 : 1;                  // words per segment
    const uint32_t nseg = G.g >> G.log2L;
    const uint64_t hk = host_key(G, aip);
    uint32_t cnt = 0;
    for (uint32_t r0 = 0; r0 < nseg; r0 += 32u * RB) {
        uint32_t w[RB][NW];
#pragma unroll
        for (int rb = 0; rb < RB; rb++) {
            const uint32_t sg = r0 + 32u * rb + lane;
            bool valid = sg < nseg;
            const uint32_t pos = valid ? seg_base_k(G, hk, sg) : 0u;      // first AT of the segment
            if (SHARD) valid = valid && pos >= G.lo && pos < G.hi;        // another shard's segment
            const uint8_t *at = G.pool + (uint64_t)pos * W;
#pragma unroll
            for (int q = 0; q < NW; q++) w[rb][q] = pad;
            if (valid) {
                if (SB == 2) {
                    const unsigned short *a16 = reinterpret_cast<const unsigned short *>(at);
                    w[rb][0] = (uint32_t)(CG ? __ldcg(a16) : __ldg(a16)) | (pad & 0xFFFF0000u);
                } else if (SB == 4) {
                    const uint32_t *a32 = reinterpret_cast<const uint32_t *>(at);
                    w[rb][0] = CG ? __ldcg(a32) : __ldg(a32);
                } else {
                    const uint2 *a64 = reinterpret_cast<const uint2 *>(at);
                    const uint2 v = CG ? __ldcg(a64) : __ldg(a64);
                    w[rb][0] = v.x;
                    w[rb][NW - 1] = v.y;
                }
            }
        }
#pragma unroll
        for (int rb = 0; rb < RB; rb++) {
#pragma unroll
            for (int q = 0; q < NW; q++) {
                VATE_CHECK_WORD(G, w[rb][q], r0 + 32u * rb + lane);
                cnt += (uint32_t)__popc(W == 1 ? swar_active(w[rb][q], rc, c2k) : swar16_active(w[rb][q], rc, c2k));
            }
        }
    }
    return cnt;
}

}  // namespace vate
