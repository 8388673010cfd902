// vate_packed.cu -- the paper's packed AT layout (Sec. 4.2): b-bit fields,
// floor(32/b) of them per 32-bit word, no field across two words.  Position
// pid lives in word pid / n, field pid mod n (n = G.pn, the division done as a
// multiply-high by ceil(2^64 / n)).  Values are kept in the frame of block 0
// for timestamps (so that every AT is read with ACT = BACT^0), as recorders'
// values for VDRE.
//
//   SetAT              in ingest_kernel (vate_kernels.cu): atomicAnd clears
//                      the field, atomicOr writes BACT^0 (or 0).  Every SetAT
//                      of one launch writes the same value, and each thread's
//                      And precedes its Or, so the last operation on a field
//                      is an Or of that value whatever the interleaving.
//   init / preserve / recorder slide / census / gather / conversion to and
//   from the paper's per-position values: the kernels below.
//
// Every kernel here touches whole words; a word is read-modify-written by one
// thread only (the two maintained ranges share a word only when k = 1, and
// range 1's enumeration then skips the words of range 0).
#include "vate_device.cuh"
#include "vate_internal.h"
#include "vate_device_ops.cuh"
#include "vate_launch.cuh"

#include <algorithm>

namespace vate {

namespace {

__device__ __forceinline__ uint32_t word_of(const Geom &G, uint64_t pid) { return (uint32_t)mulhi64(G.mpn, pid); }

__device__ __forceinline__ uint32_t field(uint32_t w, uint32_t f, uint32_t b) { return (w >> (f * b)) & ((1u << b) - 1u); }

__device__ __forceinline__ uint32_t with_field(uint32_t w, uint32_t f, uint32_t b, uint32_t v) {
    const uint32_t m = ((1u << b) - 1u) << (f * b);
    return (w & ~m) | (v << (f * b));
}

__device__ __forceinline__ uint32_t inactive_value(const Geom &G) { return G.counter == 1u ? G.k : G.twok; }

__global__ void __launch_bounds__(256) init_packed_kernel(uint32_t *__restrict__ words, uint64_t nwords, uint32_t pat) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < nwords; i += (uint64_t)gridDim.x * blockDim.x)
        words[i] = pat;
}

// Algorithm 3 in frame 0 on the fields of [s0, e0) and [s1, e1)
__global__ void __launch_bounds__(256) preserve_packed_kernel(Geom G, uint32_t B, uint64_t s0, uint64_t e0,
                                                              uint64_t s1, uint64_t e1) {
    uint32_t *words = reinterpret_cast<uint32_t *>(G.pool);
    const uint64_t n = G.pn;
    const uint64_t w0s = s0 / n, w0e = (e0 + n - 1) / n, w1s = s1 / n, w1e = (e1 + n - 1) / n;
    const uint64_t n0 = (e0 > s0) ? w0e - w0s : 0;
    const uint64_t n1 = (e1 > s1) ? w1e - w1s : 0;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n0 + n1; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = t < n0 ? w0s + t : w1s + (t - n0);
        if (t >= n0 && n0 && q >= w0s && q < w0e) continue;   // enumerated by range 0
        uint32_t w = words[q], nw = w;
        for (uint32_t f = 0; f < G.pn; f++) {
            const uint64_t pos = q * n + f;
            if (!((pos >= s0 && pos < e0) || (pos >= s1 && pos < e1))) continue;
            nw = with_field(nw, f, G.atb, preserve_frame0(field(w, f, G.atb), B, G.k));
        }
        if (nw != w) words[q] = nw;
    }
}

// Distance recorders: every recorder below k ages by one
__global__ void __launch_bounds__(256) dr_age_packed_kernel(Geom G, uint64_t nwords) {
    uint32_t *words = reinterpret_cast<uint32_t *>(G.pool);
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < nwords; q += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t w = words[q];
        uint32_t nw = w;
        for (uint32_t f = 0; f < G.pn; f++) {
            const uint32_t v = field(w, f, G.atb);
            if (v < G.k) nw = with_field(nw, f, G.atb, v + 1u);
        }
        if (nw != w) words[q] = nw;
    }
}

// Census.  COLS (2k + 1 <= 127): as the byte census, each lane counts the
// stored values (clamped to the inactive one) in its own column of the
// block's shared histogram and the rows are relabelled as distance bins once
// per block (census_raw_bin).  Otherwise one shared histogram of distance bins
// per block.  Four 16-byte chunks (4 words each) in flight per thread; the
// pool is padded to whole chunks, and fields past position P are not counted.
template <bool COLS>
__global__ void __launch_bounds__(CENSUS_THREADS) census_packed_kernel(Geom G, uint32_t bact0, uint32_t pat,
                                                                       uint64_t *__restrict__ acc,
                                                                       uint64_t *__restrict__ hist,
                                                                       unsigned int *__restrict__ ticket) {
    extern __shared__ uint32_t hsh[];   // COLS: [warps][nbins][32]; else [nbins]
    const uint32_t nbins = G.twok + 1u;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t nsh = COLS ? nwarps * nbins * 32u : nbins;
    for (uint32_t i = threadIdx.x; i < nsh; i += blockDim.x) hsh[i] = 0;
    __syncthreads();
    uint32_t *col = hsh + (size_t)warp * nbins * 32u + lane;
    const uint32_t inact = inactive_value(G);
    const uint4 *chunks = reinterpret_cast<const uint4 *>(G.pool);
    const uint64_t nwords = (G.P + G.pn - 1) / G.pn, nchunks = (nwords + 3) / 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t inactive = 0;
    constexpr int U = 4;
    for (uint64_t c0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; c0 < nchunks; c0 += U * stride) {
        uint4 x[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t c = c0 + (uint64_t)u * stride;
            x[u] = c < nchunks ? __ldcg(chunks + c) : make_uint4(pat, pat, pat, pat);
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t c = c0 + (uint64_t)u * stride;
            if (c >= nchunks) continue;
            const uint32_t ws[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const uint64_t q = 4 * c + j;
                const uint64_t first = q * G.pn;                  // position of the word's first field
                const uint32_t nf = first >= G.P ? 0u : (G.P - first < G.pn ? (uint32_t)(G.P - first) : G.pn);
                const uint32_t w = ws[j];
                if (w == pat && nf == G.pn) {
                    inactive += nf;
                    continue;
                }
                for (uint32_t f = 0; f < nf; f++) {
                    const uint32_t v = field(w, f, G.atb);
                    if (COLS) {
                        atomicAdd(&col[min(v, inact) * 32u], 1u);
                        continue;
                    }
                    if (v >= inact) {
                        inactive++;
                        continue;
                    }
                    uint32_t d = v;                               // a recorder's value is its distance
                    if (G.counter != 1u) {                        // frame 0: ACT = BACT^0 for every AT
                        d = bact0 + G.twok - v;
                        if (d >= G.twok) d -= G.twok;
                    }
                    atomicAdd(&hsh[d], 1u);
                }
            }
        }
    }
    if (COLS) {
        col[inact * 32u] += inactive;
        __syncthreads();
        for (uint32_t r = warp; r < nbins; r += nwarps) {
            uint32_t t = 0;
            for (uint32_t wv = 0; wv < nwarps; wv++) t += hsh[((size_t)wv * nbins + r) * 32u + lane];
            t = __reduce_add_sync(0xFFFFFFFFu, t);
            if (lane == 0) census_add(acc, census_raw_bin(G, bact0, r), t);
        }
        census_publish(acc, hist, ticket, nbins);
        return;
    }
    inactive = __reduce_add_sync(0xFFFFFFFFu, inactive);
    if (lane == 0) atomicAdd(&hsh[G.twok], inactive);
    census_finish(hsh, 1, nbins, acc, hist, ticket);
}

// Gather: warp per host.  In each round the lanes hash 32 consecutive
// segments; the round's VATs are then taken 32 at a time, lane l reading VAT
// v + l (the segment base coming from its hashing lane by shuffle), so the
// lanes of one segment read neighbouring words.
template <int MODE>
__global__ void __launch_bounds__(256) gather_packed_kernel(Geom G, uint32_t bact0, uint32_t kprime,
                                                            const uint64_t *__restrict__ hist,
                                                            const uint32_t *__restrict__ aips, uint64_t n,
                                                            float *__restrict__ out, uint8_t *__restrict__ flags,
                                                            uint32_t *__restrict__ active) {
    __shared__ uint64_t sN0;
    if (MODE == GATHER_ESTIMATE && threadIdx.x == 0) sN0 = pool_inactive(hist, G.P, kprime);
    __syncthreads();
    const uint32_t *words = reinterpret_cast<const uint32_t *>(G.pool);
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t nseg = G.g >> G.log2L;
    for (uint64_t h = warp0; h < n; h += nwarps) {
        const uint64_t hk = host_key(G, aips[h]);
        uint32_t cnt = 0;
        for (uint32_t r0 = 0; r0 < nseg; r0 += 32u) {
            const uint32_t s = r0 + lane;
            const uint32_t mybase = s < nseg ? seg_base_k(G, hk, s) : 0u;
            const uint32_t segs = min(32u, nseg - r0);
            const uint32_t vats = segs << G.log2L;
            const uint32_t span = (vats + 31u) & ~31u;      // the same trip count in every lane
            for (uint32_t v = lane; v < span; v += 32u) {
                const uint32_t base = __shfl_sync(0xFFFFFFFFu, mybase, (v >> G.log2L) & 31u);
                if (v < vats) {
                    const uint32_t pid = base + (v & (G.L - 1u));
                    const uint32_t q = word_of(G, pid);
                    const uint32_t val = field(__ldg(words + q), pid - q * G.pn, G.atb);
                    cnt += (G.counter == 1u ? check_dr(val, kprime) : check_at(val, bact0, kprime, G.twok)) ? 1u : 0u;
                }
            }
        }
        const uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) {
            if (MODE == GATHER_ESTIMATE) {
                uint8_t f;
                out[h] = estimate_eq11(G.g, G.P, sN0, A, f);
                if (flags) flags[h] = f;
            } else {
                active[h] = A;
            }
        }
    }
}

// Gather for widths B = 4..11 and segments of L <= 32 ATs: lane per segment.
// In each round the lanes take 32 consecutive segments of the host, one each;
// a lane loads the 16-byte chunks holding the words its segment spans (at
// most NCH, issued together; the pool is padded to whole chunks), moves those
// words into place by their offset in the first chunk (two rounds of selects),
// then counts the active fields of each word that belong to the segment with
// the SWAR test of packed_count_word (the first and last words only in part).
// Chunks rather than words: the loads are scattered, so the L1 cost is per
// request, and a segment of 32 fields takes at most 3 chunk loads against up
// to 7 word loads.
template <int MODE, int B>
__global__ void __launch_bounds__(256) gather_packed_seg_kernel(Geom G, uint32_t bact0, uint32_t kprime,
                                                                const uint64_t *__restrict__ hist,
                                                                const uint32_t *__restrict__ aips, uint64_t n,
                                                                float *__restrict__ out, uint8_t *__restrict__ flags,
                                                                uint32_t *__restrict__ active) {
    constexpr uint32_t PN = 32 / B;                     // fields per word
    constexpr uint32_t MAXW = (PN - 1 + 32 + PN - 1) / PN;   // words a segment of <= 32 fields can span
    constexpr uint32_t NCH = (3 + MAXW + 3) / 4;        // 16-byte chunks they can span
    __shared__ uint64_t sN0;
    if (MODE == GATHER_ESTIMATE && threadIdx.x == 0) sN0 = pool_inactive(hist, G.P, kprime);
    __syncthreads();
    // frame 0: every AT is read with ACT = BACT^0
    const PackedRange r = G.counter == 1u ? packed_range_dr(B, kprime, G.twok) : packed_range_at(B, bact0, kprime, G.twok);
    const uint4 *chunks = reinterpret_cast<const uint4 *>(G.pool);
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t nseg = G.g >> G.log2L;
    for (uint64_t h = warp0; h < n; h += nwarps) {
        const uint64_t hk = host_key(G, aips[h]);
        uint32_t cnt = 0;
        for (uint32_t r0 = 0; r0 < nseg; r0 += 32u) {
            const uint32_t s = r0 + lane;
            if (s >= nseg) continue;
            const uint32_t base = seg_base_k(G, hk, s);
            const uint32_t q0 = base / PN, f0 = base - q0 * PN;
            const uint32_t end = f0 + G.L;                  // the segment: fields [f0, end) from word q0's first
            const uint32_t nw = (end + PN - 1) / PN;        // words holding it
            const uint32_t o = q0 & 3u;                     // q0's place in its chunk
            const uint32_t nch = (o + nw + 3u) >> 2;        // chunks holding words q0 .. q0 + nw - 1
            uint32_t v[4 * NCH];
#pragma unroll
            for (uint32_t c = 0; c < NCH; c++) {
                const uint4 x = c < nch ? __ldg(chunks + (q0 >> 2) + c) : make_uint4(0u, 0u, 0u, 0u);
                v[4 * c] = x.x;
                v[4 * c + 1] = x.y;
                v[4 * c + 2] = x.z;
                v[4 * c + 3] = x.w;
            }
            uint32_t t[4 * NCH - 1], w[MAXW];               // w[j] = v[o + j]
#pragma unroll
            for (uint32_t i = 0; i < 4 * NCH - 1; i++) t[i] = (o & 1u) ? v[i + 1] : v[i];
#pragma unroll
            for (uint32_t j = 0; j < MAXW; j++) w[j] = (o & 2u) ? t[j + 2] : t[j];
#pragma unroll
            for (uint32_t j = 0; j < MAXW; j++)
                if (j < nw) cnt += packed_count_word<B>(w[j], r, j == 0 ? f0 : 0u, min(PN, end - j * PN));
        }
        const uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) {
            if (MODE == GATHER_ESTIMATE) {
                uint8_t f;
                out[h] = estimate_eq11(G.g, G.P, sN0, A, f);
                if (flags) flags[h] = f;
            } else {
                active[h] = A;
            }
        }
    }
}

// The paper's per-position values (uint8 for k <= 63, else uint16) of the n
// positions from pos0, from the packed pool.
__global__ void __launch_bounds__(256) packed_to_paper_kernel(Geom G, uint8_t *dst, uint64_t pos0, uint64_t n) {
    const uint32_t *words = reinterpret_cast<const uint32_t *>(G.pool);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t pos = pos0 + i;
        const uint32_t q = word_of(G, pos);
        uint32_t v = field(words[q], (uint32_t)(pos - (uint64_t)q * G.pn), G.atb);
        if (G.counter != 1u) v = to_canonical(v, block_of(G, (uint32_t)pos), G.twok);
        if (G.atw == 1u)
            dst[i] = (uint8_t)v;
        else
            reinterpret_cast<uint16_t *>(dst)[i] = (uint16_t)v;
    }
}

// The packed words holding positions [pos0, pos0 + n) (pos0 a multiple of the
// fields per word) from the paper's per-position values; fields past P are
// inactive, values above the counter's range are taken as inactive.
__global__ void __launch_bounds__(256) paper_to_packed_kernel(Geom G, const uint8_t *src, uint64_t pos0, uint64_t n) {
    uint32_t *words = reinterpret_cast<uint32_t *>(G.pool);
    const uint64_t q0 = pos0 / G.pn, nq = (n + G.pn - 1) / G.pn;
    const uint32_t inact = inactive_value(G);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < nq; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = q0 + t;
        uint32_t w = 0;
        for (uint32_t f = 0; f < G.pn; f++) {
            const uint64_t pos = q * G.pn + f;
            uint32_t u = inact;
            if (pos < pos0 + n && pos < G.P) {
                const uint64_t i = pos - pos0;
                const uint32_t v = G.atw == 1u ? (uint32_t)src[i] : (uint32_t)reinterpret_cast<const uint16_t *>(src)[i];
                u = G.counter == 1u ? min(v, G.k) : from_canonical(v, block_of(G, (uint32_t)pos), G.twok);
            }
            w |= u << (f * G.atb);
        }
        words[q] = w;
    }
}

int grid_for_packed(uint64_t items, int sms) {
    uint64_t b = (items + 255) / 256;
    if (b < 1) b = 1;
    if (b > (uint64_t)sms * 8) b = (uint64_t)sms * 8;
    return (int)b;
}

}  // namespace

uint32_t packed_pattern(const Geom &G) {
    const uint32_t v = G.counter == 1u ? G.k : G.twok;
    uint32_t w = 0;
    for (uint32_t f = 0; f < G.pn; f++) w |= v << (f * G.atb);
    return w;
}

cudaError_t launch_packed_init(const Geom &G, cudaStream_t st, int sms) {
    const uint64_t nwords = packed_bytes(G) / 4;
    return launch_pool(G, init_packed_kernel, grid_for_packed(nwords, sms), 256, 0, st,
                       reinterpret_cast<uint32_t *>(G.pool), nwords, packed_pattern(G));
}

cudaError_t launch_packed_preserve(const Geom &G, uint32_t bact0, uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1,
                                   cudaStream_t st, int sms) {
    const uint64_t words = (e0 - s0) / G.pn + (e1 - s1) / G.pn + 4;
    return launch_pool(G, preserve_packed_kernel, grid_for_packed(words, sms), 256, 0, st, G, bact0, s0, e0, s1, e1);
}

cudaError_t launch_packed_dr_age(const Geom &G, cudaStream_t st, int sms) {
    const uint64_t nwords = (G.P + G.pn - 1) / G.pn;
    return launch_pool(G, dr_age_packed_kernel, grid_for_packed(nwords, sms), 256, 0, st, G, nwords);
}

cudaError_t packed_census_prepare(uint32_t twok) {
    return cudaFuncSetAttribute(census_packed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)census_smem_bytes(twok));
}

cudaError_t launch_packed_census(const Geom &G, uint32_t bact0, uint64_t *acc, int sms, uint64_t *hist,
                                 unsigned int *ticket, cudaStream_t st) {
    if (G.twok + 1u <= 127u) {      // lane columns, as many blocks per SM as fit in about 200 KiB (up to four)
        const size_t smem = census_smem_bytes(G.twok);
        const int per_sm = (int)std::min<size_t>(4, std::max<size_t>(1, (size_t)(200u << 10) / smem));
        return launch_pool(G, census_packed_kernel<true>, sms * per_sm, CENSUS_THREADS, smem, st, G, bact0,
                           packed_pattern(G), acc, hist, ticket);
    }
    return launch_pool(G, census_packed_kernel<false>, sms * 4, CENSUS_THREADS, (size_t)(G.twok + 1) * sizeof(uint32_t),
                       st, G, bact0, packed_pattern(G), acc, hist, ticket);
}

cudaError_t launch_packed_gather(int mode, const Geom &G, uint32_t bact0, uint32_t kprime, const uint64_t *hist,
                                 const uint32_t *aips, uint64_t n, float *out, uint8_t *flags, uint32_t *active,
                                 cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 7) / 8;
    int grid = (int)(blocks < (uint64_t)sms * 64 ? blocks : (uint64_t)sms * 64);
    if (G.L <= 32) {
#define VATE_PACKED_SEG(B)                                                                                        \
    case B:                                                                                                       \
        return mode == GATHER_ESTIMATE                                                                            \
                   ? launch_pool(G, gather_packed_seg_kernel<GATHER_ESTIMATE, B>, grid, 256, 0, st, G, bact0,     \
                                 kprime, hist, aips, n, out, flags, active)                                       \
                   : launch_pool(G, gather_packed_seg_kernel<GATHER_ACTIVE, B>, grid, 256, 0, st, G, bact0,       \
                                 kprime, hist, aips, n, out, flags, active);
        switch (G.atb) {
            VATE_PACKED_SEG(4)
            VATE_PACKED_SEG(5)
            VATE_PACKED_SEG(6)
            VATE_PACKED_SEG(7)
            VATE_PACKED_SEG(8)
            VATE_PACKED_SEG(9)
            VATE_PACKED_SEG(10)
            VATE_PACKED_SEG(11)
            default: break;
        }
#undef VATE_PACKED_SEG
    }
    if (mode == GATHER_ESTIMATE)
        return launch_pool(G, gather_packed_kernel<GATHER_ESTIMATE>, grid, 256, 0, st, G, bact0, kprime, hist, aips, n,
                           out, flags, active);
    return launch_pool(G, gather_packed_kernel<GATHER_ACTIVE>, grid, 256, 0, st, G, bact0, kprime, hist, aips, n, out,
                       flags, active);
}

cudaError_t launch_packed_to_paper(const Geom &G, uint8_t *dst, uint64_t pos0, uint64_t n, cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    packed_to_paper_kernel<<<grid_for_packed(n, sms), 256, 0, st>>>(G, dst, pos0, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_paper_to_packed(const Geom &G, const uint8_t *src, uint64_t pos0, uint64_t n, cudaStream_t st,
                                   int sms) {
    if (n == 0) return cudaSuccess;
    paper_to_packed_kernel<<<grid_for_packed((n + G.pn - 1) / G.pn, sms), 256, 0, st>>>(G, src, pos0, n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vate
