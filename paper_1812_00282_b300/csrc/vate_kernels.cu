// vate_kernels.cu -- the VATE hot path on sm_103a.
//
//   init_pool_kernel      InitAT on the whole pool                      (Algorithm 4, start)
//   ingest_kernel         SetAT for every <aip, bip> pair              (Algorithm 4, scan loop)
//   preserve_kernel       fast PreserveAT on the two blocks whose ACT
//                         became 0 or k                                 (Algorithm 3, Corollary 1)
//   preserve16_kernel     the same for 16-bit ATs (k >= 64)
//   dr_age_kernel         one slide of distance recorders (VDRE),
//   dr_age16_kernel       every recorder below k aged by one            (Sec. 1; the baseline of Sec. 5)
//   census_kernel         histogram of pool distances -> Z_p            (Eq. 11)
//   census16_kernel       the same for 16-bit ATs
//   gather_vec_kernel     per-host CheckAT over g VATs + Eq. 11, for
//                         segment lengths L >= 16 (16-byte loads)       (Algorithm 1, Algorithm 4)
//   gather_scalar_kernel  the same for L < 16 (one byte per VAT)
//   estimate_from_counts_kernel  Eq. 11 from active counts and a census
//                         summed over the shards of one pool            (Eq. 11)
//   age_counts_planes_kernel, age_counts_kernel
//                         per-host counts of VATs by distance d < k
//   frame_convert_kernel  a pool to / from the paper's per-block values
//
// A handle's timestamp pool is kept in the frame of block 0 (each value minus
// its block's index, mod 2k; see vate_device.cuh), so SetAT, CheckAT, the
// census and PreserveAT use constants shared by every AT of a launch and no
// kernel of the slice step looks up a block except to bound the two
// maintained ranges.
//
// Nothing here is a dense contraction: the path is bound by L2/HBM sector
// traffic and integer ALU, so no tensor cores are used.
#include "vate_device.cuh"
#include "vate_internal.h"
#include "vate_device_ops.cuh"
#include "vate_ages.cuh"
#include "vate_launch.cuh"

#include <algorithm>
#include <utility>

namespace vate {

// --------------------------------------------------------------------------
// InitAT: every AT becomes 2k (a distance recorder k).
// --------------------------------------------------------------------------
__global__ void init_pool_kernel(uint8_t *__restrict__ pool, uint64_t nbytes, uint32_t pat) {
    uint4 v;
    v.x = v.y = v.z = v.w = pat;   // the inactive value in every AT of the word
    uint64_t n16 = nbytes >> 4;    // P * AT width, a multiple of 4096
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16;
         i += (uint64_t)gridDim.x * blockDim.x)
        reinterpret_cast<uint4 *>(pool)[i] = v;
}

// --------------------------------------------------------------------------
// Ingest: one thread per two pairs (one 16-byte streaming load).
// --------------------------------------------------------------------------
// SetAT writes the ACT of the AT's block, which in frame 0 is BACT^0 for every
// AT; a distance recorder is reset to 0.
__device__ __forceinline__ void set_at(const Geom &G, uint32_t bact0, uint32_t aip, uint32_t bip) {
    uint32_t vid = bh(G, bip);
    uint32_t pid = vat_pid(G, aip, vid);
    if (!VATE_CHECK_POSITION(G, pid)) return;           // checked build: a position outside the pool
    if (pid < G.lo || pid >= G.hi) return;              // another shard's AT
    uint32_t v = G.counter == 1u ? 0u : bact0;
    if (G.packed) {                  // clear the field, then set it (see vate_packed.cu)
        uint32_t q = (uint32_t)mulhi64(G.mpn, pid), sh = (pid - q * G.pn) * G.atb;
        uint32_t *w = reinterpret_cast<uint32_t *>(G.pool) + q;
        atomicAnd(w, ~(((1u << G.atb) - 1u) << sh));
        atomicOr(w, v << sh);
    } else if (G.atw == 1u) {
        G.pool[pid] = (uint8_t)v;
    } else {
        reinterpret_cast<uint16_t *>(G.pool)[pid] = (uint16_t)v;
    }
}

// U 16-byte loads (2U pairs) in flight per thread before their SetATs, and
// up to VATE_INGEST_BPS blocks per SM.  Measured at the 40 Gb/s shape on B300
// (5M pairs, ingest + slide): U = 1 with 32 blocks/SM 62.5 us, U = 2 with 16
// 62.7 us, U = 1 with 16 65.1 us, U = 4 with 16 65.4 us; the random byte
// stores, not the pair loads, bound it.
#ifndef VATE_INGEST_U
#define VATE_INGEST_U 1
#endif
#ifndef VATE_INGEST_BPS
#define VATE_INGEST_BPS 32
#endif
template <int U>
__global__ void __launch_bounds__(256) ingest_kernel(Geom G, uint32_t bact0, const uint32_t *__restrict__ pairs,
                                                     uint64_t n) {
    // pairs is 16-byte aligned here; n pairs = n/2 uint4 plus an odd tail
    const uint4 *p4 = reinterpret_cast<const uint4 *>(pairs);
    uint64_t n2 = n >> 1;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n2; i += U * stride) {
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t j = i + (uint64_t)u * stride;
            q[u] = j < n2 ? __ldcs(p4 + j) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            if (i + (uint64_t)u * stride >= n2) break;
            set_at(G, bact0, q[u].x, q[u].y);
            set_at(G, bact0, q[u].z, q[u].w);
        }
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        set_at(G, bact0, pairs[2 * (n - 1)], pairs[2 * (n - 1) + 1]);
    }
}

// --------------------------------------------------------------------------
// PreserveAT on blocks i0 (ACT 0) and i1 (ACT k) of a frame-0 pool.  Work is
// enumerated in 16-byte chunks covering [s0, e0) and then [s1, e1); a chunk
// shared by the two ranges (only possible for k = 1) belongs to range 0's
// enumeration and each byte decides by its own position.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) preserve_kernel(uint8_t *__restrict__ pool, RangeConsts pc, uint32_t twok,
                                                       uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1) {
    uint64_t c0s = s0 >> 4, c0e = (e0 + 15) >> 4;
    uint64_t c1s = s1 >> 4, c1e = (e1 + 15) >> 4;
    uint64_t n0 = (e0 > s0) ? c0e - c0s : 0;
    uint64_t n1 = (e1 > s1) ? c1e - c1s : 0;
    uint64_t total = n0 + n1;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t chunk = t < n0 ? c0s + t : c1s + (t - n0);
        if (t >= n0 && n0 && chunk >= c0s && chunk < c0e) continue;   // enumerated by range 0
        preserve_chunk(pool, chunk << 4, pc, twok, s0, e0, s1, e1);
    }
}

// --------------------------------------------------------------------------
// Frame 0 <-> the paper's per-block values, for the n ATs of pool positions
// pid0 .. pid0 + n - 1 (src and dst may be the same buffer; aligned to the AT
// width).  Distance recorders are copied, values above k clamped to k.
// 16 ATs per thread; the block is looked up once unless the 16 straddle a
// block boundary.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) frame_convert_kernel(Geom G, const uint8_t *src, uint8_t *dst, uint64_t pid0,
                                                            uint64_t n, int to_paper) {
    const uint64_t nq = (n + 15) >> 4;
    const uint32_t W = G.atw;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nq; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t o0 = q << 4, o1 = min(o0 + 16, n);
        const uint32_t b0 = block_of(G, (uint32_t)(pid0 + o0));
        const bool one = b0 == block_of(G, (uint32_t)(pid0 + o1 - 1));
        for (uint64_t o = o0; o < o1; o++) {
            const uint32_t blk = one ? b0 : block_of(G, (uint32_t)(pid0 + o));
            VATE_CHECK_BLOCK(G, blk, pid0 + o);
            const uint32_t x = W == 1u ? (uint32_t)src[o] : (uint32_t)reinterpret_cast<const uint16_t *>(src)[o];
            uint32_t y;
            if (G.counter == 1u)          // distance recorders have one frame; out-of-range values become inactive
                y = min(x, G.k);
            else
                y = to_paper ? to_canonical(x, blk, G.twok) : from_canonical(x, blk, G.twok);
            if (W == 1u)
                dst[o] = (uint8_t)y;
            else
                reinterpret_cast<uint16_t *>(dst)[o] = (uint16_t)y;
        }
    }
}

// --------------------------------------------------------------------------
// Distance recorders: one slide ages every recorder of the pool by one
// (saturating at k, the inactive value).  16 bytes per thread.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) dr_age_kernel(uint8_t *__restrict__ pool, uint64_t P, uint32_t k) {
    const uint64_t n16 = P >> 4;
    uint4 *p = reinterpret_cast<uint4 *>(pool);
    const uint32_t pat = k * ONES;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 w = p[i];
        if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) continue;   // all inactive already
        w.x = swar_dr_age(w.x, k);
        w.y = swar_dr_age(w.y, k);
        w.z = swar_dr_age(w.z, k);
        w.w = swar_dr_age(w.w, k);
        p[i] = w;
    }
}

// --------------------------------------------------------------------------
// 16-bit ATs (k >= 64): PreserveAT in frame 0 and the recorders' slide, eight
// ATs per 16-byte chunk, one scalar step per AT (both are bound by memory).
// Chunks cover the AT positions [s0, e0) and [s1, e1); positions outside both
// are left alone.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) preserve16_kernel(uint16_t *__restrict__ pool, uint32_t B, uint32_t k,
                                                         uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1) {
    uint64_t c0s = s0 >> 3, c0e = (e0 + 7) >> 3;
    uint64_t c1s = s1 >> 3, c1e = (e1 + 7) >> 3;
    uint64_t n0 = (e0 > s0) ? c0e - c0s : 0;
    uint64_t n1 = (e1 > s1) ? c1e - c1s : 0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n0 + n1;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t chunk = t < n0 ? c0s + t : c1s + (t - n0);
        if (t >= n0 && n0 && chunk >= c0s && chunk < c0e) continue;   // enumerated by range 0
        uint4 *p = reinterpret_cast<uint4 *>(pool) + chunk;
        uint4 w = *p;
        uint32_t words[4] = {w.x, w.y, w.z, w.w};
        bool changed = false;
#pragma unroll
        for (int e = 0; e < 8; e++) {
            uint64_t pos = (chunk << 3) + e;
            if (!((pos >= s0 && pos < e0) || (pos >= s1 && pos < e1))) continue;
            uint32_t sh = 16 * (e & 1);
            uint32_t u = (words[e >> 1] >> sh) & 0xFFFFu;
            uint32_t nu = preserve_frame0(u, B, k);
            if (nu != u) {
                words[e >> 1] = (words[e >> 1] & ~(0xFFFFu << sh)) | (nu << sh);
                changed = true;
            }
        }
        if (changed) *p = make_uint4(words[0], words[1], words[2], words[3]);
    }
}

__global__ void __launch_bounds__(256) dr_age16_kernel(uint16_t *__restrict__ pool, uint64_t P, uint32_t k) {
    const uint32_t pat = k * ONES16;
    uint4 *p = reinterpret_cast<uint4 *>(pool);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (P >> 3); i += (uint64_t)gridDim.x * blockDim.x) {
        uint4 w = p[i];
        if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) continue;   // all inactive already
        uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int q = 0; q < 4; q++) {
            uint32_t lo = words[q] & 0xFFFFu, hi = words[q] >> 16;
            lo = lo < k ? lo + 1u : k;
            hi = hi < k ? hi + 1u : k;
            words[q] = lo | (hi << 16);
        }
        p[i] = make_uint4(words[0], words[1], words[2], words[3]);
    }
}

// Census of a 16-bit pool (k >= 64): one shared histogram per warp (2k + 1
// bins, shared-memory atomics, so that the warps of a block do not contend
// for the same bins; inactive ATs are counted in a register), two chunks in
// flight per thread, then the block's sums added into acc and published as in
// census_kernel.
__global__ void __launch_bounds__(CENSUS_THREADS) census16_kernel(Geom G, uint32_t bact0, uint64_t *__restrict__ acc,
                                                                  uint64_t *__restrict__ hist,
                                                                  unsigned int *__restrict__ ticket) {
    extern __shared__ uint32_t hsh_all[];   // [warps][nbins]
    const uint32_t nbins = G.twok + 1u;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint32_t *hsh = hsh_all + (size_t)warp * nbins;
    for (uint32_t i = threadIdx.x; i < nwarps * nbins; i += blockDim.x) hsh_all[i] = 0;
    __syncthreads();
    const uint32_t inact = G.counter == 1u ? G.k : G.twok;
    const uint32_t pat = inact * ONES16;
    uint32_t inactive = 0;
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t end = G.hi >> 3;
    // four chunks in flight per thread (a 16-bit pool is usually larger than L2); the per-AT step is
    // branch-free so that the lanes of a warp stay together
    constexpr int U = 4;
    for (uint64_t q = (G.lo >> 3) + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < end; q += U * stride) {
        uint4 ws[U];
#pragma unroll
        for (int c = 0; c < U; c++) {
            const uint64_t qc = q + (uint64_t)c * stride;
            ws[c] = qc < end ? __ldcg(pool16 + qc) : make_uint4(pat, pat, pat, pat);
        }
#pragma unroll
        for (int c = 0; c < U; c++) {
            const uint4 w = ws[c];
            const bool real = q + (uint64_t)c * stride < end;
            if (real) {
                VATE_CHECK_WORD(G, w.x, q + (uint64_t)c * stride);
                VATE_CHECK_WORD(G, w.y, q + (uint64_t)c * stride);
                VATE_CHECK_WORD(G, w.z, q + (uint64_t)c * stride);
                VATE_CHECK_WORD(G, w.w, q + (uint64_t)c * stride);
            }
            if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) {
                inactive += real ? 8u : 0u;
                continue;
            }
            const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 8; e++) {
                const uint32_t v = (words[e >> 1] >> (16 * (e & 1))) & 0xFFFFu;
                const bool act = v < inact;
                uint32_t d = bact0 + G.twok - v;          // frame 0: ACT = BACT^0 for every AT
                d = d >= G.twok ? d - G.twok : d;
                d = G.counter == 1u ? v : d;              // a recorder's value is its distance
                inactive += act ? 0u : 1u;
                if (act) atomicAdd(&hsh[d], 1u);
            }
        }
    }
    inactive = __reduce_add_sync(0xFFFFFFFFu, inactive);
    if (lane == 0) atomicAdd(&hsh[G.twok], inactive);
    census_finish(hsh_all, nwarps, nbins, acc, hist, ticket);
}

// --------------------------------------------------------------------------
// Census: hist[d] = ATs at distance d (d < 2k), hist[2k] = inactive ATs.
// Each lane keeps a private column of the block's shared histogram
// (bin * 32 + lane: no bank conflicts) and counts with shared-memory atomics
// that return nothing, so consecutive ATs of one bin do not wait on each
// other.  A chunk of 16 inactive ATs is counted in a register.
//
// RAW (timestamps in the frame of block 0, or distance recorders): every AT
// of the pool is read with the same ACT, so the census is the histogram of
// the stored values with its bins relabelled once per block
// (census_chunk_raw, census_raw_bin), and an AT costs one byte extract, one
// clamp and one atomic.  Otherwise (the paper's per-block values of a caller's pool) the chunk's
// bins are computed with SWAR, one ACT per chunk when it lies in one block.
//
// Eight 16-byte chunks are in flight per thread; the block's sums go into acc
// with 64-bit atomics and the last block publishes them (census_publish).
// --------------------------------------------------------------------------
template <int RAW>
__global__ void __launch_bounds__(CENSUS_THREADS) census_kernel(Geom G, uint32_t bact0, uint64_t *__restrict__ acc,
                                                                uint64_t *__restrict__ hist,
                                                                unsigned int *__restrict__ ticket) {
    extern __shared__ uint32_t sh[];   // [warps][nbins][32]
    const uint32_t nbins = G.twok + 1u;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    uint32_t *col = sh + (size_t)warp * nbins * 32u + lane;
    for (uint32_t i = threadIdx.x; i < nwarps * nbins * 32u; i += blockDim.x) sh[i] = 0;
    __syncthreads();

    const uint32_t inact = G.counter == 1u ? G.k : G.twok;   // the inactive value, < nbins
    const uint32_t pat = inact * ONES;                        // 16 inactive counters
    uint32_t runs = 0;                                        // chunks of 16 inactive ATs
    const uint64_t n16 = G.hi >> 4;                           // chunks of the positions held, [lo, hi)
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    constexpr int U = 8;
    for (uint64_t q = (G.lo >> 4) + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n16; q += U * stride) {
        uint4 w[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t qu = q + (uint64_t)u * stride;
            w[u] = qu < n16 ? __ldcg(pool16 + qu) : make_uint4(pat, pat, pat, pat);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t qu = q + (uint64_t)u * stride;
            if (qu >= n16) continue;
            VATE_CHECK_WORD(G, w[u].x, qu);
            VATE_CHECK_WORD(G, w[u].y, qu);
            VATE_CHECK_WORD(G, w[u].z, qu);
            VATE_CHECK_WORD(G, w[u].w, qu);
            if (RAW) census_chunk_raw(w[u], pat, inact, col, runs);
            else census_chunk(G, bact0, (uint32_t)(qu << 4), w[u], pat, col, runs);
        }
    }
    col[(RAW ? inact : G.twok) * 32u] += 16u * runs;
    __syncthreads();

    // warp w sums rows w, w + nwarps, ... over every warp's lane columns
    for (uint32_t r = warp; r < nbins; r += nwarps) {
        uint32_t s = 0;
        for (uint32_t wv = 0; wv < nwarps; wv++) s += sh[((size_t)wv * nbins + r) * 32u + lane];
        s = __reduce_add_sync(0xFFFFFFFFu, s);
        if (lane == 0) census_add(acc, RAW ? census_raw_bin(G, bact0, r) : r, s);
    }
    census_publish(acc, hist, ticket, nbins);
}

// --------------------------------------------------------------------------
// Census of a byte pool whose stored values fit a 32-bit one-hot mask (the
// inactive value inact <= 31: frame-0 timestamps and recorders with k <= 15),
// as bit-sliced (vertical) counters in registers: bit u of plane j is bit j of
// the number of bytes equal to u that this thread has read.  Each 16-byte
// chunk enters as sixteen one-hot masks 1 << u (a funnel shift whose amount is
// the byte's low five bits) through a carry-save adder tree into the planes of
// weight 1, 2, 4 and 8 (the tree of AgePlanes::add_chunk, 15 adders of two
// 3-input logic operations); the carries of weight 16 of a batch of eight
// chunks go through a second tree into the planes of weight 16 .. 2048.  An
// AT so costs about two shifts and two logic operations, where
// census_kernel<1> spends a byte extract, a clamp and a shared-memory atomic.
// The planes hold up to 4095 per value; every CP_FOLD_BATCHES batches and at
// the end the warp sums them (warp_fold: each plane transposed over the warp
// as a 32 x 32 bit matrix, so that lane u holds bit u of every lane, then one
// popcount per plane), lane u adds the warp's count of value u to the block's,
// and the block's counts, relabelled as census bins (census_raw_bin), go into
// acc; census_publish ends it.  The loop runs the same number of trips in
// every lane of a warp (lanes past the end count nothing), so that the
// shuffles of warp_fold see the whole warp.
// CLAMP: bytes above inact are counted as inact (a recorder pool may come from
// a caller); a frame-0 timestamp pool of the library never holds them.
// --------------------------------------------------------------------------
constexpr int CP_THREADS = 256;
#ifndef VATE_CENSUS_BATCH
#define VATE_CENSUS_BATCH 8
#endif
#ifndef VATE_CENSUS_PLANES_BPS
#define VATE_CENSUS_PLANES_BPS 2
#endif
constexpr int CP_BATCH = VATE_CENSUS_BATCH;    // chunks loaded per thread per trip (4 or 8, all issued before any use)
constexpr int CP_FOLD_BATCHES = 248 / CP_BATCH; // 248 chunks x 16 ATs = 3968 <= 4095 per value

struct CensusPlanes {
    uint32_t lo[4] = {0, 0, 0, 0};             // weights 1, 2, 4, 8
    uint32_t hi[8] = {0, 0, 0, 0, 0, 0, 0, 0}; // weights 16, 32, ..., 2048

    // the tree of one chunk into lo; returns the chunk's carry of weight 16
    __device__ __forceinline__ uint32_t add_chunk(uint4 w) {
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
        uint32_t m[16];
        // byte b of a word moved down by a multiply-high (w >> 8b = umulhi(w, 2^(32 - 8b)), on the
        // multiply-add pipe), then the funnel shift takes its low five bits as the amount
#pragma unroll
        for (int b = 0; b < 16; b++) {
            const uint32_t w = words[b >> 2];
            const uint32_t x = (b & 3) == 0 ? w : __umulhi(w, 1u << (32 - 8 * (b & 3)));
            m[b] = __funnelshift_l(0u, 1u, x);
        }
        uint32_t twosA, twosB, foursA, foursB, eightsA, eightsB, sixteens;
        csa(twosA, lo[0], lo[0], m[0], m[1]);
        csa(twosB, lo[0], lo[0], m[2], m[3]);
        csa(foursA, lo[1], lo[1], twosA, twosB);
        csa(twosA, lo[0], lo[0], m[4], m[5]);
        csa(twosB, lo[0], lo[0], m[6], m[7]);
        csa(foursB, lo[1], lo[1], twosA, twosB);
        csa(eightsA, lo[2], lo[2], foursA, foursB);
        csa(twosA, lo[0], lo[0], m[8], m[9]);
        csa(twosB, lo[0], lo[0], m[10], m[11]);
        csa(foursA, lo[1], lo[1], twosA, twosB);
        csa(twosA, lo[0], lo[0], m[12], m[13]);
        csa(twosB, lo[0], lo[0], m[14], m[15]);
        csa(foursB, lo[1], lo[1], twosA, twosB);
        csa(eightsB, lo[2], lo[2], foursA, foursB);
        csa(sixteens, lo[3], lo[3], eightsA, eightsB);
        return sixteens;
    }
    // the carries of weight 16 of one batch (4 or 8 chunks) into hi
    __device__ __forceinline__ void add_batch_carries(const uint32_t (&s)[CP_BATCH]) {
        uint32_t t32A, t32B, t64A, t64B, c;
        csa(t32A, hi[0], hi[0], s[0], s[1]);
        csa(t32B, hi[0], hi[0], s[2], s[3]);
        if (CP_BATCH == 8) {
            csa(t64A, hi[1], hi[1], t32A, t32B);
            csa(t32A, hi[0], hi[0], s[CP_BATCH > 4 ? 4 : 0], s[CP_BATCH > 5 ? 5 : 0]);
            csa(t32B, hi[0], hi[0], s[CP_BATCH > 6 ? 6 : 0], s[CP_BATCH > 7 ? 7 : 0]);
            csa(t64B, hi[1], hi[1], t32A, t32B);
            csa(c, hi[2], hi[2], t64A, t64B);            // carry of weight 128
        } else {
            csa(c, hi[1], hi[1], t32A, t32B);            // carry of weight 64
            const uint32_t t = hi[2] & c;                // into 64, carry 128 on
            hi[2] ^= c;
            c = t;
        }
#pragma unroll
        for (int j = 3; j < 8; j++) {                   // ripple into 128 .. 2048
            const uint32_t t = hi[j] & c;
            hi[j] ^= c;
            c = t;
        }
    }
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int j = 0; j < 4; j++) lo[j] = 0;
#pragma unroll
        for (int j = 0; j < 8; j++) hi[j] = 0;
    }
};

// Transpose of a 32 x 32 bit matrix held one row per lane (row i = lane i's
// word): afterwards lane u holds column u, bit i = bit u of row i.  Five
// rounds, each swapping the off-diagonal s x s blocks of lane pairs (lane,
// lane ^ s).  Called by all 32 lanes.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, uint32_t lane) {
    const uint32_t M[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 0; r < 5; r++) {
        const uint32_t sft = 16u >> r;
        const uint32_t y = __shfl_xor_sync(0xFFFFFFFFu, x, sft);
        const bool upper = (lane & sft) != 0u;
        const uint32_t keep = upper ? ~M[r] : M[r];            // the bits this lane keeps
        const uint32_t t = upper ? (y >> sft) : (y << sft);     // the partner's block moved into place
        x = (x & keep) | (t & ~keep);
    }
    return x;
}

// The warp's total count of value u (lane u) in the planes of its 32 lanes.
__device__ __forceinline__ uint32_t warp_fold(const CensusPlanes &cp, uint32_t lane) {
    uint32_t t = 0;
#pragma unroll
    for (int j = 0; j < 4; j++) t += (uint32_t)__popc(warp_transpose32(cp.lo[j], lane)) << j;
#pragma unroll
    for (int j = 0; j < 8; j++) t += (uint32_t)__popc(warp_transpose32(cp.hi[j], lane)) << (4 + j);
    return t;
}

template <bool CLAMP>
__global__ void __launch_bounds__(CP_THREADS, VATE_CENSUS_PLANES_BPS) census_planes_kernel(Geom G, uint32_t bact0, uint64_t *__restrict__ acc,
                                                                   uint64_t *__restrict__ hist,
                                                                   unsigned int *__restrict__ ticket) {
    __shared__ uint32_t blk[32];                                // the block's count of each stored value
    if (threadIdx.x < 32) blk[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t inact = G.counter == 1u ? G.k : G.twok;     // <= 31 here
    const uint32_t pat = inact * ONES;                          // 16 inactive ATs
    const uint64_t n16 = G.hi >> 4;                             // chunks of the positions held, [lo, hi)
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    CensusPlanes cp;
    uint32_t runs = 0;                                          // chunks of 16 inactive ATs
    uint32_t total = 0;                                         // lane u: the warp's folded count of value u
    uint32_t batches = 0;
    // lane 0's chunk bounds the loop, so that every lane of the warp makes the same trips
    for (uint64_t q0 = (G.lo >> 4) + blockIdx.x * (uint64_t)blockDim.x + (threadIdx.x & ~31u); q0 < n16;
         q0 += CP_BATCH * stride) {
        const uint64_t q = q0 + lane;
        uint4 w[CP_BATCH];
#pragma unroll
        for (int b = 0; b < CP_BATCH; b++) {
            const uint64_t qb = q + (uint64_t)b * stride;
            w[b] = qb < n16 ? __ldcg(pool16 + qb) : make_uint4(pat, pat, pat, pat);
        }
        uint32_t s[CP_BATCH];
#pragma unroll
        for (int b = 0; b < CP_BATCH; b++) {
            s[b] = 0u;
            if (q + (uint64_t)b * stride >= n16) continue;      // beyond the pool: not counted
            uint4 c = w[b];
            VATE_CHECK_WORD(G, c.x, q + (uint64_t)b * stride);
            VATE_CHECK_WORD(G, c.y, q + (uint64_t)b * stride);
            VATE_CHECK_WORD(G, c.z, q + (uint64_t)b * stride);
            VATE_CHECK_WORD(G, c.w, q + (uint64_t)b * stride);
            if (CLAMP) {
                c.x = swar_clamp(c.x, inact);
                c.y = swar_clamp(c.y, inact);
                c.z = swar_clamp(c.z, inact);
                c.w = swar_clamp(c.w, inact);
            }
            if (c.x == pat && c.y == pat && c.z == pat && c.w == pat) {
                runs++;
                continue;
            }
            s[b] = cp.add_chunk(c);
        }
        cp.add_batch_carries(s);
        if (++batches == CP_FOLD_BATCHES) {                     // the same trip in every lane
            total += warp_fold(cp, lane);
            cp.clear();
            batches = 0;
        }
    }
    total += warp_fold(cp, lane);
    runs = __reduce_add_sync(0xFFFFFFFFu, runs);
    if (lane == inact) total += 16u * runs;
    if (lane <= inact && total) atomicAdd(&blk[lane], total);
    __syncthreads();
    if (threadIdx.x <= inact) census_add(acc, census_raw_bin(G, bact0, threadIdx.x), blk[threadIdx.x]);
    census_publish(acc, hist, ticket, G.twok + 1u);
}

// --------------------------------------------------------------------------
// Gather + estimate.
// --------------------------------------------------------------------------
template <int MODE>
__device__ __forceinline__ void write_result(const Geom &G, uint64_t N0, uint64_t idx, uint32_t A, float *out,
                                             uint8_t *flags, uint32_t *active) {
    if (MODE == GATHER_ESTIMATE) {
        uint8_t f;
        float e = estimate_eq11(G.g, G.P, N0, A, f);
        out[idx] = e;
        if (flags) flags[idx] = f;
    } else {
        active[idx] = A;
    }
}

// Warp per host; L = 16 << CPSL (16, 32 or 64).  Work goes in batches of RB
// rounds of 32 segments.  In each round the 32 lanes hash 32 consecutive
// segments; the segments' 16-byte chunks are then read by consecutive lanes
// (for L = 32, lanes 2j and 2j+1 read the two halves of one 32-byte sector),
// the segment base coming from the hashing lane by shuffle; one CheckAT
// (ACT = BACT^0 in frame 0) serves every AT of the launch.  All
// RB * CPS loads of a batch are issued before any is tested, so that several
// sectors are in flight per lane.  FULL: every batch is complete (the number
// of segments is a multiple of 32 * RB), so no lane needs a bounds test.
// Active ATs are counted per byte lane in a SWAR accumulator (at most
// RB * CPS * 4 <= 32 per byte lane per batch) and folded after each batch.
// 5 blocks of 256 threads per SM (at most 51 registers a thread): measured
// best for L = 32, g = 4096 on B300 among 2-8 blocks per SM and 1-4 rounds
// per batch (fewer registers spill, more leave too few warps to hide the L2
// latency of the sector loads).
#ifndef VATE_GATHER_MINB
#define VATE_GATHER_MINB 5
#endif
template <int MODE, int CPSL, int RB, bool FULL, int W, bool SHARD>
__global__ void __launch_bounds__(GATHER_THREADS, VATE_GATHER_MINB) gather_vec_kernel(Geom G, uint32_t bact0, uint32_t kprime,
                                                                    const uint64_t *__restrict__ hist,
                                                                    const uint32_t *__restrict__ aips, uint64_t n,
                                                                    float *__restrict__ out,
                                                                    uint8_t *__restrict__ flags,
                                                                    uint32_t *__restrict__ active, uint32_t u1,
                                                                    uint32_t u2, uint32_t u3) {
    __shared__ uint64_t sN0;
    // one CheckAT for every AT of the frame-0 pool (ACT = BACT^0), or CheckDR
    const RangeConsts rc = W == 1 ? (G.counter == 1u ? dr_range_consts(kprime) : range_consts(bact0, kprime, G.twok))
                                  : (G.counter == 1u ? dr_range_consts16(kprime)
                                                     : range_consts16(bact0, kprime, G.twok));
    if (MODE == GATHER_ESTIMATE && threadIdx.x == 0) sN0 = pool_inactive(hist, G.P, kprime);
    __syncthreads();
    const uint64_t N0 = (MODE == GATHER_ESTIMATE) ? sN0 : 0;
    const uint32_t c2k = W == 1 ? (128u - G.twok) * ONES : (0x8000u - G.twok) * ONES16;

    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;

    // The warp takes its hosts 32 at a time (hosts g0 + j * nwarps, j < 32):
    // lane j loads host j's address up front, the warp gathers the hosts one
    // by one, lane j keeps host j's count, and the 32 Eq. 11 epilogues then
    // run side by side, one per lane.
    for (uint64_t g0 = warp0; g0 < n; g0 += 32 * nwarps) {
        const uint64_t mine = g0 + (uint64_t)lane * nwarps;
        const uint32_t my_aip = mine < n ? aips[mine] : 0u;
        uint32_t my_A = 0;
        for (uint32_t j = 0; j < 32u; j++) {
            if (g0 + (uint64_t)j * nwarps >= n) break;
            const uint32_t aip = __shfl_sync(0xFFFFFFFFu, my_aip, j);
            uint32_t cnt = gather_host_vec<CPSL, RB, FULL, W, SHARD>(G, rc, c2k, aip, u1, u2, u3, lane);
            uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
            if (lane == j) my_A = A;
        }
        if (mine < n) write_result<MODE>(G, N0, mine, my_A, out, flags, active);
    }
}

// Warp per host for segments of 2, 4 or 8 bytes (gather_host_seg,
// vate_device_ops.cuh), 32 hosts per warp at a time as in gather_vec_kernel.
template <int MODE, int SB, int W, bool SHARD>
__global__ void __launch_bounds__(GATHER_THREADS) gather_seg_kernel(Geom G, uint32_t bact0, uint32_t kprime,
                                                                    const uint64_t *__restrict__ hist,
                                                                    const uint32_t *__restrict__ aips, uint64_t n,
                                                                    float *__restrict__ out,
                                                                    uint8_t *__restrict__ flags,
                                                                    uint32_t *__restrict__ active) {
    __shared__ uint64_t sN0;
    const RangeConsts rc = W == 1 ? (G.counter == 1u ? dr_range_consts(kprime) : range_consts(bact0, kprime, G.twok))
                                  : (G.counter == 1u ? dr_range_consts16(kprime)
                                                     : range_consts16(bact0, kprime, G.twok));
    if (MODE == GATHER_ESTIMATE && threadIdx.x == 0) sN0 = pool_inactive(hist, G.P, kprime);
    __syncthreads();
    const uint64_t N0 = (MODE == GATHER_ESTIMATE) ? sN0 : 0;
    const uint32_t c2k = W == 1 ? (128u - G.twok) * ONES : (0x8000u - G.twok) * ONES16;
    const uint32_t pad = W == 1 ? G.twok * ONES : G.twok * ONES16;   // never active (2k: inactive; above k' for recorders)
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // 32 hosts per warp at a time, lane j keeping host j's count (as gather_vec_kernel)
    for (uint64_t g0 = warp0; g0 < n; g0 += 32 * nwarps) {
        const uint64_t mine = g0 + (uint64_t)lane * nwarps;
        const uint32_t my_aip = mine < n ? aips[mine] : 0u;
        uint32_t my_A = 0;
        for (uint32_t j = 0; j < 32u; j++) {
            if (g0 + (uint64_t)j * nwarps >= n) break;
            const uint32_t aip = __shfl_sync(0xFFFFFFFFu, my_aip, j);
            const uint32_t A = __reduce_add_sync(0xFFFFFFFFu, gather_host_seg<SB, W, SHARD>(G, rc, c2k, pad, aip, lane));
            if (lane == j) my_A = A;
        }
        if (mine < n) write_result<MODE>(G, N0, mine, my_A, out, flags, active);
    }
}

// Eq. 11 from counts: A per host and the pool census, each summed over the
// shards that hold one pool.
__global__ void __launch_bounds__(256) estimate_from_counts_kernel(uint32_t g, uint64_t P, uint32_t kprime,
                                                                   const uint64_t *__restrict__ hist,
                                                                   const uint32_t *__restrict__ active, uint64_t n,
                                                                   float *__restrict__ out, uint8_t *__restrict__ flags) {
    __shared__ uint64_t sN0;
    if (threadIdx.x == 0) sN0 = pool_inactive(hist, P, kprime);
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        uint8_t f;
        out[i] = estimate_eq11(g, P, sN0, active[i], f);
        if (flags) flags[i] = f;
    }
}

// Warp per host; any L (used for L < 16): lane i reads VATs i, i+32, ...
template <int MODE>
__global__ void __launch_bounds__(GATHER_THREADS) gather_scalar_kernel(Geom G, uint32_t bact0, uint32_t kprime,
                                                                       const uint64_t *__restrict__ hist,
                                                                       const uint32_t *__restrict__ aips, uint64_t n,
                                                                       float *__restrict__ out,
                                                                       uint8_t *__restrict__ flags,
                                                                       uint32_t *__restrict__ active) {
    __shared__ uint64_t sN0;
    if (MODE == GATHER_ESTIMATE && threadIdx.x == 0) sN0 = pool_inactive(hist, G.P, kprime);
    __syncthreads();
    const uint64_t N0 = (MODE == GATHER_ESTIMATE) ? sN0 : 0;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = warp0; h < n; h += nwarps) {
        const uint32_t aip = aips[h];
        uint32_t cnt = gather_host_scalar(G, bact0, kprime, aip, lane);
        uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) write_result<MODE>(G, N0, h, A, out, flags, active);
    }
}

// --------------------------------------------------------------------------
// Per-age counts (vate_age_counts).
// --------------------------------------------------------------------------
// For k <= 15: warp per host, the host's segments read as
// 16-byte chunks (as in the gather) and counted in bit-sliced registers
// (host_age_counts, vate_ages.cuh); lane d < k writes the count of age d.
__global__ void __launch_bounds__(AGE_THREADS) age_counts_planes_kernel(Geom G, uint32_t bact0,
                                                                        const uint32_t *__restrict__ aips, uint64_t n,
                                                                        uint16_t *__restrict__ counts) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = warp0; h < n; h += nwarps) {
        const uint32_t cd = host_age_counts(G, bact0, aips[h], lane);
        if (lane < G.k) counts[h * G.k + lane] = (uint16_t)cd;
    }
}

// Per-age counts for 15 < k <= 63: warp per host, each lane a private column
// of k counters in shared memory ([warp][d][32]); the host's segments read as
// 16-byte chunks for L >= 16 (age_columns_vec, vate_ages.cuh), one VAT per lane
// at a time for shorter segments; d = distance of the VAT, kept when d < k.
__global__ void __launch_bounds__(AGE_THREADS) age_counts_kernel(Geom G, uint32_t bact0,
                                                                 const uint32_t *__restrict__ aips, uint64_t n,
                                                                 uint16_t *__restrict__ counts) {
    extern __shared__ uint32_t sh[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *col = sh + (size_t)warp * G.k * 32u + lane;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = warp0; h < n; h += nwarps) {
        for (uint32_t d = 0; d < G.k; d++) col[d * 32u] = 0;
        __syncwarp();
        const uint64_t hk = host_key(G, aips[h]);
        if (G.L == 16) age_columns_vec<0>(G, bact0, hk, lane, col);
        else if (G.L == 32) age_columns_vec<1>(G, bact0, hk, lane, col);
        else if (G.L == 64) age_columns_vec<2>(G, bact0, hk, lane, col);
        else {                                        // L < 16: one byte per VAT
            for (uint32_t i = lane; i < G.g; i += 32u) {
                uint32_t pid = vat_pid_k(G, hk, i);
                uint32_t v = __ldg(G.pool + pid);
                if (G.counter == 1u) {
                    if (v < G.k) col[v * 32u] += 1u;
                    continue;
                }
                if (v == G.twok) continue;
                uint32_t d = bact0 + G.twok - v;          // frame 0: ACT = BACT^0
                if (d >= G.twok) d -= G.twok;
                if (d < G.k) col[d * 32u] += 1u;
            }
        }
        __syncwarp();
        for (uint32_t d = lane; d < G.k; d += 32u) {
            const uint32_t *row = sh + (size_t)warp * G.k * 32u + d * 32u;
            uint32_t s = 0;
            for (uint32_t l = 0; l < 32u; l++) s += row[l];
            counts[h * G.k + d] = (uint16_t)s;
        }
        __syncwarp();
    }
}

// --------------------------------------------------------------------------
// Launchers (host side).  Each returns cudaGetLastError() of its launch.
// --------------------------------------------------------------------------
static int grid_for(uint64_t work_items, int threads, int max_blocks) {
    uint64_t b = (work_items + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (uint64_t)max_blocks) b = max_blocks;
    return (int)b;
}

cudaError_t launch_init(const Geom &G, cudaStream_t st, int sms) {
    if (G.packed) return launch_packed_init(G, st, sms);
    // InitAT: 2k; a distance recorder starts at k (inactive)
    const uint32_t v = G.counter == 1u ? G.k : G.twok;
    const uint64_t nbytes = (G.hi - G.lo) * G.atw;
    return launch_pool(G, init_pool_kernel, grid_for(nbytes >> 4, 256, sms * 8), 256, 0, st, pool_mem(G), nbytes,
                       G.atw == 1u ? v * ONES : v * ONES16);
}

cudaError_t launch_ingest(const Geom &G, uint32_t bact0, const uint32_t *pairs, uint64_t n, cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(pairs) & 15u) != 0) {
        // 8-byte aligned only: the first pair alone, then the 16-byte aligned rest
        cudaError_t e = launch_pool(G, ingest_kernel<1>, 1, 32, 0, st, G, bact0, pairs, (uint64_t)1);
        if (e != cudaSuccess) return e;
        pairs += 2;
        n -= 1;
        if (n == 0) return cudaSuccess;
    }
    return launch_pool(G, ingest_kernel<VATE_INGEST_U>, grid_for((n + 1) / 2, 256, sms * VATE_INGEST_BPS), 256, 0, st, G,
                       bact0, pairs, n);
}

cudaError_t launch_dr_age(const Geom &G, cudaStream_t st, int sms) {
    if (G.packed) return launch_packed_dr_age(G, st, sms);
    const uint64_t n = G.hi - G.lo;                         // the recorders held
    if (G.atw == 2u)
        return launch_pool(G, dr_age16_kernel, grid_for(n >> 3, 256, sms * 8), 256, 0, st,
                           reinterpret_cast<uint16_t *>(pool_mem(G)), n, G.k);
    return launch_pool(G, dr_age_kernel, grid_for(n >> 4, 256, sms * 8), 256, 0, st, pool_mem(G), n, G.k);
}

cudaError_t launch_preserve(const Geom &G, uint32_t bact0, uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1,
                            cudaStream_t st, int sms) {
    if (G.packed) return launch_packed_preserve(G, bact0, s0, e0, s1, e1, st, sms);
    if (G.atw == 2u) {
        uint64_t chunks = ((e0 - s0) >> 3) + ((e1 - s1) >> 3) + 4;
        return launch_pool(G, preserve16_kernel, grid_for(chunks, 256, sms * 8), 256, 0, st,
                           reinterpret_cast<uint16_t *>(G.pool), bact0, G.k, s0, e0, s1, e1);
    }
    uint64_t chunks = ((e0 - s0) >> 4) + ((e1 - s1) >> 4) + 4;
    return launch_pool(G, preserve_kernel, grid_for(chunks, 256, sms * 8), 256, 0, st, G.pool,
                       preserve_consts_frame0(bact0, G.k), G.twok, s0, e0, s1, e1);
}

cudaError_t launch_frame_convert(const Geom &G, const uint8_t *src, uint8_t *dst, uint64_t pid0, uint64_t n,
                                 bool to_paper, cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    frame_convert_kernel<<<grid_for((n + 15) >> 4, 256, sms * 8), 256, 0, st>>>(G, src, dst, pid0, n, to_paper ? 1 : 0);
    count_launch();
    return cudaGetLastError();
}

size_t census_smem_bytes(uint32_t twok) { return (size_t)(CENSUS_THREADS / 32) * (twok + 1) * 32 * sizeof(uint32_t); }

cudaError_t census_prepare(uint32_t twok) {
    cudaError_t e = cudaFuncSetAttribute(census_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)census_smem_bytes(twok));
    if (e == cudaSuccess) e = packed_census_prepare(twok);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(census_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)census_smem_bytes(twok));
    if (e != cudaSuccess) return e;
    // 16-bit pools: one histogram of up to 2 * 1023 + 1 bins per warp
    return cudaFuncSetAttribute(census16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((CENSUS_THREADS / 32) * (2 * 1023 + 1) * sizeof(uint32_t)));
}

cudaError_t launch_census(const Geom &G, uint32_t bact0, uint64_t *acc, int sms, uint64_t *hist,
                          unsigned int *ticket, cudaStream_t st) {
    if (G.packed) return launch_packed_census(G, bact0, acc, sms, hist, ticket, st);
    if (G.atw == 2u)
        return launch_pool(G, census16_kernel, sms * 4, CENSUS_THREADS,
                           (size_t)(CENSUS_THREADS / 32) * (G.twok + 1) * sizeof(uint32_t), st, G, bact0, acc, hist,
                           ticket);
    // byte pools whose stored values fit a 32-bit one-hot mask (k <= 15):
    // bit-sliced counters, two blocks of 256 threads per SM so that a thread
    // reads enough chunks to pay for reading its planes out
    const uint32_t inact = G.counter == 1u ? G.k : G.twok;
    if ((G.frame0 || G.counter == 1u) && inact <= 31u) {
        if (G.counter == 1u)
            return launch_pool(G, census_planes_kernel<true>, sms * VATE_CENSUS_PLANES_BPS, CP_THREADS, 0, st, G,
                               bact0, acc, hist, ticket);
        return launch_pool(G, census_planes_kernel<false>, sms * VATE_CENSUS_PLANES_BPS, CP_THREADS, 0, st, G, bact0,
                           acc, hist, ticket);
    }
    // other byte pools: up to four blocks per SM, as many as their lane-column
    // histograms fit in about 200 KiB of shared memory (one for k = 63)
    const size_t smem = census_smem_bytes(G.twok);
    const int per_sm = (int)std::min<size_t>(4, std::max<size_t>(1, (size_t)(200u << 10) / smem));
    const int grid = sms * per_sm;
    if (G.frame0 || G.counter == 1u)
        return launch_pool(G, census_kernel<1>, grid, CENSUS_THREADS, smem, st, G, bact0, acc, hist, ticket);
    return launch_pool(G, census_kernel<0>, grid, CENSUS_THREADS, smem, st, G, bact0, acc, hist, ticket);
}

cudaError_t launch_gather(int mode, const Geom &G, uint32_t bact0, uint32_t kprime, const uint64_t *hist,
                          const uint32_t *aips, uint64_t n, float *out, uint8_t *flags, uint32_t *active,
                          cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    if (G.packed) return launch_packed_gather(mode, G, bact0, kprime, hist, aips, n, out, flags, active, st, sms);
    int warps_per_block = GATHER_THREADS / 32;
    int grid = grid_for(n, warps_per_block, sms * 64);
    cudaError_t e = cudaSuccess;
    const uint32_t seg_bytes = G.L * G.atw;
    // a shard only counts active VATs (its estimates come from counts summed over the shards)
    const bool sharded = G.lo != 0 || G.hi != G.P;
    if (sharded && mode == GATHER_ESTIMATE) return cudaErrorInvalidValue;
    if (seg_bytes >= 16) {
        const uint32_t nseg = G.g >> G.log2L;
        const uint32_t rounds = (nseg + 31u) / 32u;
#define VATE_GATHER_LAUNCH(CPSL, RB, FULL, W)                                                                     \
    do {                                                                                                          \
        if (sharded)                                                                                              \
            e = launch_pool(G, gather_vec_kernel<GATHER_ACTIVE, CPSL, RB, FULL, W, true>, grid, GATHER_THREADS, 0, \
                            st, G, bact0, kprime, hist, aips, n, out, flags, active, 1u, 1u, 1u);                 \
        else if (mode == GATHER_ESTIMATE)                                                                         \
            e = launch_pool(G, gather_vec_kernel<GATHER_ESTIMATE, CPSL, RB, FULL, W, false>, grid, GATHER_THREADS, \
                            0, st, G, bact0, kprime, hist, aips, n, out, flags, active, 1u, 1u, 1u);              \
        else                                                                                                      \
            e = launch_pool(G, gather_vec_kernel<GATHER_ACTIVE, CPSL, RB, FULL, W, false>, grid, GATHER_THREADS,   \
                            0, st, G, bact0, kprime, hist, aips, n, out, flags, active, 1u, 1u, 1u);              \
    } while (0)
#define VATE_GATHER_VEC(CPSL, RB, W)                                                                              \
    do {                                                                                                          \
        if (nseg % (32u * RB) == 0) VATE_GATHER_LAUNCH(CPSL, RB, true, W);                                        \
        else VATE_GATHER_LAUNCH(CPSL, RB, false, W);                                                              \
    } while (0)
        // batches of up to 8 loads per lane: RB rounds x 2^CPSL chunks
#ifndef VATE_GATHER_RB
#define VATE_GATHER_RB 2
#endif
        if (G.atw == 1u) {
            if (seg_bytes == 16) {
                if (rounds >= 2) VATE_GATHER_VEC(0, VATE_GATHER_RB, 1);
                else VATE_GATHER_VEC(0, 1, 1);
            } else if (seg_bytes == 32) {
                if (rounds >= 2) VATE_GATHER_VEC(1, VATE_GATHER_RB, 1);
                else VATE_GATHER_VEC(1, 1, 1);
            } else {
                if (rounds >= 2) VATE_GATHER_VEC(2, VATE_GATHER_RB, 1);
                else VATE_GATHER_VEC(2, 1, 1);
            }
        } else {                       // 16-bit ATs: one round per batch (a segment is 16-128 bytes)
            if (seg_bytes == 16) VATE_GATHER_VEC(0, 1, 2);
            else if (seg_bytes == 32) VATE_GATHER_VEC(1, 1, 2);
            else if (seg_bytes == 64) VATE_GATHER_VEC(2, 1, 2);
            else VATE_GATHER_VEC(3, 1, 2);
        }
#undef VATE_GATHER_LAUNCH
#undef VATE_GATHER_VEC
    } else if (seg_bytes == 2 || seg_bytes == 4 || seg_bytes == 8) {
#define VATE_GATHER_SEG(SB, W)                                                                                    \
    do {                                                                                                          \
        if (sharded)                                                                                              \
            e = launch_pool(G, gather_seg_kernel<GATHER_ACTIVE, SB, W, true>, grid, GATHER_THREADS, 0, st, G, bact0,  \
                            kprime, hist, aips, n, out, flags, active);                                           \
        else if (mode == GATHER_ESTIMATE)                                                                         \
            e = launch_pool(G, gather_seg_kernel<GATHER_ESTIMATE, SB, W, false>, grid, GATHER_THREADS, 0, st, G,      \
                            bact0, kprime, hist, aips, n, out, flags, active);                                    \
        else                                                                                                      \
            e = launch_pool(G, gather_seg_kernel<GATHER_ACTIVE, SB, W, false>, grid, GATHER_THREADS, 0, st, G,        \
                            bact0, kprime, hist, aips, n, out, flags, active);                                    \
    } while (0)
        if (G.atw == 1u) {
            if (seg_bytes == 2) VATE_GATHER_SEG(2, 1);
            else if (seg_bytes == 4) VATE_GATHER_SEG(4, 1);
            else VATE_GATHER_SEG(8, 1);
        } else {
            if (seg_bytes == 2) VATE_GATHER_SEG(2, 2);
            else if (seg_bytes == 4) VATE_GATHER_SEG(4, 2);
            else VATE_GATHER_SEG(8, 2);
        }
#undef VATE_GATHER_SEG
    } else {
        if (mode == GATHER_ESTIMATE)
            e = launch_pool(G, gather_scalar_kernel<GATHER_ESTIMATE>, grid, GATHER_THREADS, 0, st, G, bact0, kprime, hist,
                            aips, n, out, flags, active);
        else
            e = launch_pool(G, gather_scalar_kernel<GATHER_ACTIVE>, grid, GATHER_THREADS, 0, st, G, bact0, kprime, hist,
                            aips, n, out, flags, active);
    }
    return e;
}

cudaError_t launch_estimate_from_counts(const Geom &G, uint32_t kprime, const uint64_t *hist, const uint32_t *active,
                                        uint64_t n, float *out, uint8_t *flags, cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    estimate_from_counts_kernel<<<grid_for(n, 256, sms * 8), 256, 0, st>>>(G.g, G.P, kprime, hist, active, n, out, flags);
    count_launch();
    return cudaGetLastError();
}

cudaError_t age_prepare(uint32_t k) {
    return cudaFuncSetAttribute(age_counts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)((size_t)(AGE_THREADS / 32) * k * 32 * sizeof(uint32_t)));
}

cudaError_t launch_age_counts(const Geom &G, uint32_t bact0, const uint32_t *aips, uint64_t n, uint16_t *counts,
                              cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    int grid = grid_for(n, AGE_THREADS / 32, sms * 32);
    if (G.k <= 15u)          // every stored value (at most 2k) fits a 32-bit one-hot mask
        return launch_pool(G, age_counts_planes_kernel, grid, AGE_THREADS, 0, st, G, bact0, aips, n, counts);
    size_t smem = (size_t)(AGE_THREADS / 32) * G.k * 32 * sizeof(uint32_t);
    return launch_pool(G, age_counts_kernel, grid, AGE_THREADS, smem, st, G, bact0, aips, n, counts);
}

}  // namespace vate
