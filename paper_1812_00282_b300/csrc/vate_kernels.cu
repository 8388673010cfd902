// vate_kernels.cu -- the VATE hot path on sm_103a.
//
//   init_pool_kernel      InitAT on the whole pool                      (Algorithm 4, start)
//   ingest_kernel         SetAT for every <aip, bip> pair              (Algorithm 4, scan loop)
//   preserve_kernel       fast PreserveAT on the two blocks whose ACT
//                         became 0 or k                                 (Algorithm 3, Corollary 1)
//   census_kernel         histogram of pool distances -> Z_p            (Eq. 11)
//   gather_vec_kernel     per-host CheckAT over g VATs + Eq. 11, for
//                         segment lengths L >= 16 (16-byte loads)       (Algorithm 1, Algorithm 4)
//   gather_scalar_kernel  the same for L < 16 (one byte per VAT)
//   age_counts_kernel     per-host counts of VATs by distance d < k
//
// Nothing here is a dense contraction: the path is bound by L2/HBM sector
// traffic and integer ALU, so no tensor cores are used.
#include "vate_device.cuh"
#include "vate_internal.h"

namespace vate {

// --------------------------------------------------------------------------
// InitAT: every AT becomes 2k.
// --------------------------------------------------------------------------
__global__ void init_pool_kernel(uint8_t *__restrict__ pool, uint64_t P, uint32_t twok) {
    uint4 v;
    v.x = v.y = v.z = v.w = twok * ONES;
    uint64_t n16 = P >> 4;   // P is a power of two >= 4096
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16;
         i += (uint64_t)gridDim.x * blockDim.x)
        reinterpret_cast<uint4 *>(pool)[i] = v;
}

// --------------------------------------------------------------------------
// Ingest: one thread per two pairs (one 16-byte streaming load).
// --------------------------------------------------------------------------
__device__ __forceinline__ void set_at(const Geom &G, uint32_t bact0, uint32_t aip, uint32_t bip) {
    uint32_t vid = bh(G, bip);
    uint32_t pid = vat_pid(G, aip, vid);
    uint32_t act = act_of_block(bact0, block_of(G, pid), G.twok);
    G.pool[pid] = (uint8_t)act;
}

__global__ void __launch_bounds__(256) ingest_kernel(Geom G, uint32_t bact0, const uint32_t *__restrict__ pairs,
                                                     uint64_t n) {
    // pairs is 16-byte aligned here; n pairs = n/2 uint4 plus an odd tail
    const uint4 *p4 = reinterpret_cast<const uint4 *>(pairs);
    uint64_t n2 = n >> 1;
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n2; i += stride) {
        uint4 q = __ldcs(p4 + i);
        set_at(G, bact0, q.x, q.y);
        set_at(G, bact0, q.z, q.w);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        set_at(G, bact0, pairs[2 * (n - 1)], pairs[2 * (n - 1) + 1]);
    }
}

// --------------------------------------------------------------------------
// PreserveAT on blocks i0 (ACT 0) and i1 (ACT k).  Work is enumerated in
// 16-byte chunks covering [s0, e0) and then [s1, e1); a chunk shared by the
// two ranges (only possible for k = 1) belongs to range 0's enumeration and
// each byte decides by its own position.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) preserve_kernel(uint8_t *__restrict__ pool, uint32_t k, uint64_t s0,
                                                       uint64_t e0, uint64_t s1, uint64_t e1) {
    uint64_t c0s = s0 >> 4, c0e = (e0 + 15) >> 4;
    uint64_t c1s = s1 >> 4, c1e = (e1 + 15) >> 4;
    uint64_t n0 = (e0 > s0) ? c0e - c0s : 0;
    uint64_t n1 = (e1 > s1) ? c1e - c1s : 0;
    uint64_t total = n0 + n1;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t chunk = t < n0 ? c0s + t : c1s + (t - n0);
        if (t >= n0 && n0 && chunk >= c0s && chunk < c0e) continue;   // enumerated by range 0
        uint64_t base = chunk << 4;
        uint4 *p = reinterpret_cast<uint4 *>(pool + base);
        uint4 w = *p;
        uint4 r = w;
        bool full0 = base >= s0 && base + 16 <= e0;
        bool full1 = base >= s1 && base + 16 <= e1;
        if (full0 || full1) {
            r.x = swar_preserve(w.x, full0, k);
            r.y = swar_preserve(w.y, full0, k);
            r.z = swar_preserve(w.z, full0, k);
            r.w = swar_preserve(w.w, full0, k);
        } else {
            uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int b = 0; b < 16; b++) {
                uint64_t pos = base + b;
                uint32_t v = (words[b >> 2] >> (8 * (b & 3))) & 0xFFu;
                uint32_t nv = v;
                if (pos >= s0 && pos < e0) nv = preserve_at(v, 0u, k);
                else if (pos >= s1 && pos < e1) nv = preserve_at(v, k, k);
                words[b >> 2] = (words[b >> 2] & ~(0xFFu << (8 * (b & 3)))) | (nv << (8 * (b & 3)));
            }
            r.x = words[0]; r.y = words[1]; r.z = words[2]; r.w = words[3];
        }
        if (r.x != w.x || r.y != w.y || r.z != w.z || r.w != w.w) *p = r;
    }
}

// --------------------------------------------------------------------------
// Census: hist[d] = ATs at distance d (d < 2k), hist[2k] = inactive ATs.
// Each lane keeps a private column of the block's shared histogram
// (bin * 32 + lane: no bank conflicts, no atomics); runs of 16 inactive ATs
// are counted in a register.  Block rows go to `partial`; the last block to
// finish adds the rows up into `hist` and re-arms `ticket` for the next call.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(CENSUS_THREADS) census_kernel(Geom G, uint32_t bact0, uint64_t *__restrict__ partial,
                                                                uint64_t *__restrict__ hist,
                                                                unsigned int *__restrict__ ticket) {
    extern __shared__ uint32_t sh[];   // [warps][nbins][32]
    const uint32_t nbins = G.twok + 1u;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nwarps = blockDim.x >> 5;
    uint32_t *col = sh + (size_t)warp * nbins * 32u + lane;
    for (uint32_t i = threadIdx.x; i < nwarps * nbins * 32u; i += blockDim.x) sh[i] = 0;
    __syncthreads();

    const uint32_t pat = G.twok * ONES;
    uint32_t inactive_runs = 0;   // chunks of 16 inactive ATs
    const uint64_t n16 = G.P >> 4;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n16;
         q += (uint64_t)gridDim.x * blockDim.x) {
        uint4 w = __ldcg(reinterpret_cast<const uint4 *>(G.pool) + q);
        if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) {
            inactive_runs++;
            continue;
        }
        uint32_t pid0 = (uint32_t)(q << 4);
        uint32_t b0 = block_of(G, pid0), b15 = block_of(G, pid0 + 15u);
        uint32_t act0 = act_of_block(bact0, b0, G.twok);
        uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int b = 0; b < 16; b++) {
            uint32_t v = (words[b >> 2] >> (8 * (b & 3))) & 0xFFu;
            uint32_t bin;
            if (v >= G.twok) {   // 2k = inactive (larger values never arise from the ABI)
                bin = G.twok;
            } else {
                uint32_t act = (b0 == b15) ? act0 : act_of_block(bact0, block_of(G, pid0 + b), G.twok);
                uint32_t d = act + G.twok - v;
                bin = d >= G.twok ? d - G.twok : d;
            }
            col[bin * 32u] += 1u;
        }
    }
    col[G.twok * 32u] += 16u * inactive_runs;
    __syncthreads();

    // block row: sum every lane column of every warp
    for (uint32_t bin = threadIdx.x; bin < nbins; bin += blockDim.x) {
        uint64_t s = 0;
        for (uint32_t wv = 0; wv < nwarps; wv++) {
            const uint32_t *c = sh + ((size_t)wv * nbins + bin) * 32u;
            for (uint32_t l = 0; l < 32u; l++) s += c[l];
        }
        partial[(uint64_t)blockIdx.x * nbins + bin] = s;
    }
    __threadfence();
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1u);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (uint32_t bin = threadIdx.x; bin < nbins; bin += blockDim.x) {
        uint64_t s = 0;
        for (uint32_t blk = 0; blk < gridDim.x; blk++) s += __ldcg(partial + (uint64_t)blk * nbins + bin);
        hist[bin] = s;
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// --------------------------------------------------------------------------
// Gather + estimate.
// --------------------------------------------------------------------------
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

// Per-byte CheckAT of one 16-byte chunk whose bytes may lie in two blocks.
__device__ __forceinline__ uint32_t count_chunk_bytes(const Geom &G, uint32_t bact0, uint32_t kprime, uint32_t pid,
                                                   uint4 w) {
    uint32_t words[4] = {w.x, w.y, w.z, w.w};
    uint32_t n = 0;
    for (int b = 0; b < 16; b++) {
        uint32_t v = (words[b >> 2] >> (8 * (b & 3))) & 0xFFu;
        uint32_t act = act_of_block(bact0, block_of(G, pid + b), G.twok);
        n += check_at(v, act, kprime, G.twok) ? 1u : 0u;
    }
    return n;
}

// Warp per host; L >= 16.  In each round the 32 lanes hash 32 consecutive
// segments; the segments' 16-byte chunks are then read by consecutive lanes
// (for L = 32, lanes 2j and 2j+1 read the two halves of one 32-byte sector),
// the segment base and ACT coming from the hashing lane by shuffle.
template <int MODE>
__global__ void __launch_bounds__(GATHER_THREADS) gather_vec_kernel(Geom G, uint32_t bact0, uint32_t kprime,
                                                                    const uint64_t *__restrict__ hist,
                                                                    const uint32_t *__restrict__ aips, uint64_t n,
                                                                    float *__restrict__ out,
                                                                    uint8_t *__restrict__ flags,
                                                                    uint32_t *__restrict__ active) {
    __shared__ CheckConsts tbl[128];
    __shared__ uint64_t sN0;
    for (uint32_t a = threadIdx.x; a < G.twok; a += blockDim.x) tbl[a] = check_consts(a, kprime, G.twok);
    if (MODE == GATHER_ESTIMATE && threadIdx.x == 0) sN0 = pool_inactive(hist, G.P, kprime);
    __syncthreads();
    const uint64_t N0 = (MODE == GATHER_ESTIMATE) ? sN0 : 0;

    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t nseg = G.g >> G.log2L;              // segments per host
    const uint32_t cps_log2 = G.log2L - 4u;             // log2(16-byte chunks per segment)
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);

    for (uint64_t h = warp0; h < n; h += nwarps) {
        const uint32_t aip = aips[h];
        uint32_t cnt = 0;
        for (uint32_t r0 = 0; r0 < nseg; r0 += 32u) {
            // hash one segment per lane
            uint32_t s = r0 + lane;
            uint32_t base = 0, act = 0;
            bool straddle = false;
            if (s < nseg) {
                base = seg_base(G, aip, s);
                uint32_t b0 = block_of(G, base), b1 = block_of(G, base + G.L - 1u);
                act = act_of_block(bact0, b0, G.twok);
                straddle = (b0 != b1);
            }
            uint32_t segs_here = min(32u, nseg - r0);
            uint32_t chunks = segs_here << cps_log2;
            unsigned straddle_mask = __ballot_sync(0xFFFFFFFFu, straddle);
            for (uint32_t c0 = 0; c0 < chunks; c0 += 32u) {
                uint32_t c = c0 + lane;
                uint32_t src = c >> cps_log2;            // lane that hashed this chunk's segment
                uint32_t sbase = __shfl_sync(0xFFFFFFFFu, base, src & 31u);
                uint32_t sact = __shfl_sync(0xFFFFFFFFu, act, src & 31u);
                if (c < chunks) {
                    uint32_t pid = sbase + ((c & ((1u << cps_log2) - 1u)) << 4);
                    uint4 w = __ldg(pool16 + (pid >> 4));
                    if (straddle_mask & (1u << src)) {
                        cnt += count_chunk_bytes(G, bact0, kprime, pid, w);
                    } else {
                        CheckConsts cc = tbl[sact];
                        cnt += __popc(swar_active(w.x, cc)) + __popc(swar_active(w.y, cc)) +
                               __popc(swar_active(w.z, cc)) + __popc(swar_active(w.w, cc));
                    }
                }
            }
        }
        uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) write_result<MODE>(G, N0, h, A, out, flags, active);
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
        uint32_t cnt = 0;
#pragma unroll 4
        for (uint32_t i = lane; i < G.g; i += 32u) {
            uint32_t pid = vat_pid(G, aip, i);
            uint32_t v = __ldg(G.pool + pid);
            uint32_t act = act_of_block(bact0, block_of(G, pid), G.twok);
            cnt += check_at(v, act, kprime, G.twok) ? 1u : 0u;
        }
        uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
        if (lane == 0) write_result<MODE>(G, N0, h, A, out, flags, active);
    }
}

// --------------------------------------------------------------------------
// Per-age counts: warp per host, each lane a private column of k counters in
// shared memory ([warp][d][32]); d = distance of the VAT, kept when d < k.
// --------------------------------------------------------------------------
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
        const uint32_t aip = aips[h];
        for (uint32_t i = lane; i < G.g; i += 32u) {
            uint32_t pid = vat_pid(G, aip, i);
            uint32_t v = __ldg(G.pool + pid);
            if (v == G.twok) continue;
            uint32_t act = act_of_block(bact0, block_of(G, pid), G.twok);
            uint32_t d = act + G.twok - v;
            if (d >= G.twok) d -= G.twok;
            if (d < G.k) col[d * 32u] += 1u;
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
    init_pool_kernel<<<grid_for(G.P >> 4, 256, sms * 8), 256, 0, st>>>(G.pool, G.P, G.twok);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_ingest(const Geom &G, uint32_t bact0, const uint32_t *pairs, uint64_t n, cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(pairs) & 15u) != 0) {
        // 8-byte aligned only: the first pair alone, then the 16-byte aligned rest
        ingest_kernel<<<1, 32, 0, st>>>(G, bact0, pairs, 1);
        count_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        pairs += 2;
        n -= 1;
        if (n == 0) return cudaSuccess;
    }
    ingest_kernel<<<grid_for((n + 1) / 2, 256, sms * 16), 256, 0, st>>>(G, bact0, pairs, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_preserve(uint8_t *pool, uint32_t k, uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1,
                            cudaStream_t st, int sms) {
    uint64_t chunks = ((e0 - s0) >> 4) + ((e1 - s1) >> 4) + 4;
    preserve_kernel<<<grid_for(chunks, 256, sms * 8), 256, 0, st>>>(pool, k, s0, e0, s1, e1);
    count_launch();
    return cudaGetLastError();
}

size_t census_smem_bytes(uint32_t twok) { return (size_t)(CENSUS_THREADS / 32) * (twok + 1) * 32 * sizeof(uint32_t); }

cudaError_t census_prepare(uint32_t twok) {
    return cudaFuncSetAttribute(census_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)census_smem_bytes(twok));
}

cudaError_t launch_census(const Geom &G, uint32_t bact0, uint64_t *partial, int grid, uint64_t *hist,
                          unsigned int *ticket, cudaStream_t st) {
    census_kernel<<<grid, CENSUS_THREADS, census_smem_bytes(G.twok), st>>>(G, bact0, partial, hist, ticket);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_gather(int mode, const Geom &G, uint32_t bact0, uint32_t kprime, const uint64_t *hist,
                          const uint32_t *aips, uint64_t n, float *out, uint8_t *flags, uint32_t *active,
                          cudaStream_t st, int sms) {
    if (n == 0) return cudaSuccess;
    int warps_per_block = GATHER_THREADS / 32;
    int grid = grid_for(n, warps_per_block, sms * 64);
    if (G.L >= 16) {
        if (mode == GATHER_ESTIMATE)
            gather_vec_kernel<GATHER_ESTIMATE><<<grid, GATHER_THREADS, 0, st>>>(G, bact0, kprime, hist, aips, n, out, flags, active);
        else
            gather_vec_kernel<GATHER_ACTIVE><<<grid, GATHER_THREADS, 0, st>>>(G, bact0, kprime, hist, aips, n, out, flags, active);
    } else {
        if (mode == GATHER_ESTIMATE)
            gather_scalar_kernel<GATHER_ESTIMATE><<<grid, GATHER_THREADS, 0, st>>>(G, bact0, kprime, hist, aips, n, out, flags, active);
        else
            gather_scalar_kernel<GATHER_ACTIVE><<<grid, GATHER_THREADS, 0, st>>>(G, bact0, kprime, hist, aips, n, out, flags, active);
    }
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
    size_t smem = (size_t)(AGE_THREADS / 32) * G.k * 32 * sizeof(uint32_t);
    int grid = grid_for(n, AGE_THREADS / 32, sms * 32);
    age_counts_kernel<<<grid, AGE_THREADS, smem, st>>>(G, bact0, aips, n, counts);
    count_launch();
    return cudaGetLastError();
}

}  // namespace vate
