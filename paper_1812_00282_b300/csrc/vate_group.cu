// vate_group.cu -- many independent monitors advanced together (include/vate_group.h).
//
// One slice of every monitor is five launches, each a persistent grid over a
// work table that spans all monitors:
//   group_begin_kernel     slice number + 1 (device-resident), clear the census
//                          histograms and the work-queue counters
//   group_preserve_kernel  PreserveAT (Algorithm 3) on each monitor's two blocks
//                          whose ACT became 0 or k, as (monitor, 16-byte chunk) items
//   group_ingest_kernel    SetAT for every pair, each pair's monitor found from
//                          the CSR offsets of the batch
//   group_census_kernel    census tiles (monitor, chunk range) from a work queue,
//                          histograms accumulated per monitor
//   group_gather_kernel    warp per host from a work queue, CheckAT gather and Eq. 11
// The per-chunk and per-host arithmetic is the one of the single-pool kernels
// (vate_device_ops.cuh).  Because the slice number, the batch offsets and k'
// are read on the device, the five launches can be captured once as a CUDA
// graph and replayed every slice.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "vate.h"
#include "vate_group.h"
#include "vate_device_ops.cuh"
#include "vate_launch.cuh"

using namespace vate;

namespace vate {
int make_geom_checked(const vate_params *p, Geom *G);   // vate_api.cu
int set_error(int code, const char *msg);               // vate_api.cu
}  // namespace vate

namespace {

constexpr uint32_t MAX_MONITORS = 256;
constexpr int G_THREADS = 256;

struct GroupState {                 // device-resident
    unsigned long long step;        // slides since slice 0
    unsigned int started;           // set by the first step
    unsigned int status;            // VATE_GROUP_* bits
    unsigned int q_census;          // census tiles handed out
    unsigned int q_gather;          // hosts handed out
};

struct CensusTile {
    uint32_t mon;
    uint32_t nchunks;
    uint64_t chunk0;
};

// census_chunk_raw (vate_device_ops.cuh) into columns of counter pairs:
// values 2j and 2j + 1 share the 32-bit word col[j * 32] as its low and high
// 16 bits, halving the shared memory.  The caller keeps every count below
// 2^16 (at most 4,096 ATs per lane between two clearings).
__device__ __forceinline__ void census_chunk_raw_pairs(uint4 w, uint32_t pat, uint32_t inact, uint32_t *col,
                                                       uint32_t &inactive_runs) {
    if (w.x == pat && w.y == pat && w.z == pat && w.w == pat) {
        inactive_runs++;
        return;
    }
    const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int b = 0; b < 16; b++) {
        const uint32_t v = min((words[b >> 2] >> (8 * (b & 3))) & 0xFFu, inact);
        atomicAdd(&col[(v >> 1) * 32u], 1u << ((v & 1u) << 4));
    }
}

__device__ __forceinline__ uint32_t bact0_of(unsigned long long step, uint32_t twok) {
    return (uint32_t)(step % twok);
}

// index of the monitor whose [off[m], off[m+1]) holds i (off non-decreasing, off[0] <= i < off[M])
__device__ __forceinline__ uint32_t find_monitor(const uint64_t *off, uint32_t M, uint64_t i) {
    uint32_t lo = 0, hi = M;            // invariant: off[lo] <= i < off[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Load M+1 offsets into shared memory, clamped to [0, cap] and made
// non-decreasing; a repair sets `bad` in the status word.
__device__ void load_offsets(const uint64_t *__restrict__ off, uint32_t M, uint64_t cap, uint64_t *s,
                             GroupState *st, unsigned bad) {
    for (uint32_t t = threadIdx.x; t <= M; t += blockDim.x) s[t] = off[t];
    __syncthreads();
    if (threadIdx.x == 0) {
        bool repaired = false;
        uint64_t prev = 0;
        for (uint32_t t = 0; t <= M; t++) {
            uint64_t v = s[t];
            if (v > cap) { v = cap; repaired = true; }
            if (t && v < prev) { v = prev; repaired = true; }
            s[t] = v;
            prev = v;
        }
        if (repaired && blockIdx.x == 0) atomicOr(&st->status, bad);
    }
    __syncthreads();
}

__global__ void group_begin_kernel(GroupState *st, uint64_t *__restrict__ hist_all, uint32_t hist_words) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (st->started) st->step += 1ull;
        else st->started = 1u;
        st->q_census = 0u;
        st->q_gather = 0u;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < hist_words; i += gridDim.x * blockDim.x)
        hist_all[i] = 0ull;
}

// Clears the queue counters (and optionally the histograms) without moving
// the slice: used when the autotuner repeats a phase of the same slice.
__global__ void group_reset_kernel(GroupState *st, uint64_t *__restrict__ hist_all, uint32_t hist_words) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->q_census = 0u;
        st->q_gather = 0u;
    }
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < hist_words; i += gridDim.x * blockDim.x)
        hist_all[i] = 0ull;
}

__global__ void __launch_bounds__(G_THREADS) group_preserve_kernel(const Geom *__restrict__ descs, uint32_t M,
                                                                   const GroupState *__restrict__ st) {
    __shared__ uint64_t r[MAX_MONITORS][4];      // s0, e0, s1, e1
    __shared__ uint64_t pre[MAX_MONITORS + 1];   // prefix of chunk counts
    __shared__ uint64_t n0s[MAX_MONITORS];
    const unsigned long long step = st->step;
    if (step == 0ull) return;                    // slice 0: nothing to maintain
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) {
        const Geom &G = descs[m];
        uint32_t b0 = bact0_of(step, G.twok);
        uint32_t i0 = (G.twok - b0) % G.twok, i1 = (G.k + G.twok - b0) % G.twok;
        uint64_t s0, e0, s1, e1;
        block_range_of(G, i0, &s0, &e0);
        block_range_of(G, i1, &s1, &e1);
        r[m][0] = s0; r[m][1] = e0; r[m][2] = s1; r[m][3] = e1;
        uint64_t c0s = s0 >> 4, c0e = (e0 + 15) >> 4, c1s = s1 >> 4, c1e = (e1 + 15) >> 4;
        n0s[m] = (e0 > s0) ? c0e - c0s : 0;
        pre[m + 1] = n0s[m] + ((e1 > s1) ? c1e - c1s : 0);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        pre[0] = 0;
        for (uint32_t m = 0; m < M; m++) pre[m + 1] += pre[m];
    }
    __syncthreads();
    const uint64_t total = pre[M];
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t m = find_monitor(pre, M, t);
        uint64_t local = t - pre[m];
        const uint64_t s0 = r[m][0], e0 = r[m][1], s1 = r[m][2], e1 = r[m][3];
        uint64_t c0s = s0 >> 4, c0e = (e0 + 15) >> 4, c1s = s1 >> 4;
        uint64_t n0 = n0s[m];
        uint64_t chunk = local < n0 ? c0s + local : c1s + (local - n0);
        if (local >= n0 && n0 && chunk >= c0s && chunk < c0e) continue;   // enumerated with range 0
        const uint32_t k = descs[m].k;
        preserve_chunk(descs[m].pool, chunk << 4, preserve_consts_frame0(bact0_of(step, 2u * k), k), 2u * k, s0, e0,
                       s1, e1);
    }
}

__global__ void __launch_bounds__(G_THREADS) group_ingest_kernel(const Geom *__restrict__ descs, uint32_t M,
                                                                 GroupState *st,
                                                                 const uint32_t *__restrict__ pairs,
                                                                 const uint64_t *__restrict__ off, uint64_t cap) {
    extern __shared__ uint64_t dyn[];
    uint64_t *so = dyn;                                          // M + 1 offsets
    Geom *sd = reinterpret_cast<Geom *>(so + ((M + 2) & ~1u));   // M descriptors
    load_offsets(off, M, cap, so, st, VATE_GROUP_BAD_OFFSETS);
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) sd[m] = descs[m];
    __syncthreads();
    const unsigned long long step = st->step;
    const uint64_t lo = so[0], hi = so[M];
    const uint2 *p2 = reinterpret_cast<const uint2 *>(pairs);          // 8-byte aligned (checked on the host)
    __shared__ uint32_t tile_mon[2];
    // Tiles of INGEST_TILE consecutive pairs, in order across the grid, so the
    // pools being written at any time are those of the few monitors whose
    // pairs are in flight.  A tile inside one monitor runs with that monitor's
    // descriptor in registers; only a tile that straddles monitors looks up
    // the monitor of each pair.
    constexpr uint32_t INGEST_TILE = G_THREADS * 8;
    const uint64_t ntiles = (hi - lo + INGEST_TILE - 1) / INGEST_TILE;
    for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const uint64_t t0 = lo + tile * INGEST_TILE, t1 = min(t0 + INGEST_TILE, hi);
        __syncthreads();                        // the previous tile's tile_mon has been read
        if (threadIdx.x == 0) {
            tile_mon[0] = find_monitor(so, M, t0);
            tile_mon[1] = find_monitor(so, M, t1 - 1);
        }
        __syncthreads();
        const uint32_t m0 = tile_mon[0];
        if (m0 == tile_mon[1]) {
            const Geom G = sd[m0];
            const uint8_t v = (uint8_t)bact0_of(step, G.twok);        // SetAT in frame 0
#pragma unroll 4
            for (uint64_t i = t0 + threadIdx.x; i < t1; i += G_THREADS) {
                const uint2 q = __ldcs(p2 + i);
                G.pool[vat_pid(G, q.x, bh(G, q.y))] = v;
            }
        } else {
            for (uint64_t i = t0 + threadIdx.x; i < t1; i += G_THREADS) {
                const uint32_t m = find_monitor(so, M, i);
                const Geom &G = sd[m];
                const uint2 q = __ldcs(p2 + i);
                G.pool[vat_pid(G, q.x, bh(G, q.y))] = (uint8_t)bact0_of(step, G.twok);
            }
        }
    }
}

__global__ void __launch_bounds__(G_THREADS) group_census_kernel(const Geom *__restrict__ descs, GroupState *st,
                                                                 const CensusTile *__restrict__ tiles, uint32_t ntiles,
                                                                 uint64_t *__restrict__ hist_all, uint32_t maxbins) {
    extern __shared__ uint32_t sh[];             // [warps][maxpairs][32]: lane columns of 16-bit counter pairs
    __shared__ Geom G;
    __shared__ CensusTile tile;
    __shared__ unsigned int ticket;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t maxpairs = (maxbins + 1u) / 2u;
    uint32_t *col = sh + (size_t)warp * maxpairs * 32u + lane;
    const unsigned long long step = st->step;
    for (;;) {
        if (threadIdx.x == 0) ticket = atomicAdd(&st->q_census, 1u);
        __syncthreads();
        if (ticket >= ntiles) break;
        if (threadIdx.x == 0) {
            tile = tiles[ticket];
            G = descs[tile.mon];
        }
        __syncthreads();
        const uint32_t nbins = G.twok + 1u, npairs = (nbins + 1u) / 2u;
        for (uint32_t b = 0; b < npairs; b++) col[b * 32u] = 0u;
        const uint32_t pat = G.twok * ONES;
        const uint32_t bact0 = bact0_of(step, G.twok);
        uint32_t inactive_runs = 0;
        const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
        // eight chunks in flight per thread: the pools of a group exceed L2, so the loads wait on memory;
        // frame-0 pools: the stored values are counted and relabelled as bins below.  A tile holds at
        // most 65,536 chunks, so a lane counts at most 4,096 ATs and every 16-bit counter stays exact.
        constexpr int U = 8;
        const uint64_t qend = tile.chunk0 + tile.nchunks;
        for (uint64_t q = tile.chunk0 + threadIdx.x; q < qend; q += (uint64_t)U * blockDim.x) {
            uint4 w[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint64_t qu = q + (uint64_t)u * blockDim.x;
                w[u] = qu < qend ? __ldcg(pool16 + qu) : make_uint4(pat, pat, pat, pat);
            }
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint64_t qu = q + (uint64_t)u * blockDim.x;
                if (qu < qend) census_chunk_raw_pairs(w[u], pat, G.twok, col, inactive_runs);
            }
        }
        col[(G.twok >> 1) * 32u] += 16u * inactive_runs;     // 2k is even: the low half of pair k
        __syncthreads();
        for (uint32_t r = warp; r < npairs; r += nwarps) {
            uint32_t lo = 0, hi = 0;
            for (uint32_t wv = 0; wv < nwarps; wv++) {
                const uint32_t x = sh[((size_t)wv * maxpairs + r) * 32u + lane];
                lo += x & 0xFFFFu;
                hi += x >> 16;
            }
            lo = __reduce_add_sync(0xFFFFFFFFu, lo);
            hi = __reduce_add_sync(0xFFFFFFFFu, hi);
            unsigned long long *h = reinterpret_cast<unsigned long long *>(hist_all) + (size_t)tile.mon * maxbins;
            if (lane == 0 && lo) atomicAdd(h + census_raw_bin(G, bact0, 2u * r), (unsigned long long)lo);
            if (lane == 0 && hi && 2u * r + 1u < nbins)
                atomicAdd(h + census_raw_bin(G, bact0, 2u * r + 1u), (unsigned long long)hi);
        }
        __syncthreads();
    }
}

template <int CPSL, int RB>
__global__ void __launch_bounds__(G_THREADS) group_gather_kernel(const Geom *__restrict__ descs, uint32_t M,
                                                                 GroupState *st, const uint32_t *__restrict__ hosts,
                                                                 const uint64_t *__restrict__ off, uint64_t cap,
                                                                 const uint32_t *__restrict__ kprimes,
                                                                 const uint64_t *__restrict__ hist_all,
                                                                 uint32_t maxbins, float *__restrict__ out,
                                                                 uint8_t *__restrict__ flags, uint32_t grab,
                                                                 uint32_t u1, uint32_t u2, uint32_t u3) {
    extern __shared__ uint64_t dyn[];
    uint64_t *so = dyn;                                          // M + 1 host offsets
    uint64_t *n0 = so + M + 1;                                   // N0 per monitor
    uint32_t *kp = reinterpret_cast<uint32_t *>(n0 + M);         // k' per monitor
    Geom *sd = reinterpret_cast<Geom *>(so + ((2 * M + 1 + (M + 1) / 2 + 1) & ~1u));
    load_offsets(off, M, cap, so, st, VATE_GROUP_BAD_OFFSETS);
    for (uint32_t m = threadIdx.x; m < M; m += blockDim.x) {
        sd[m] = descs[m];
        uint32_t k = descs[m].k, x = kprimes[m];
        if (x < 1u || x > k) {
            if (blockIdx.x == 0) atomicOr(&st->status, VATE_GROUP_BAD_KPRIME);
            x = k;
        }
        kp[m] = x;
        n0[m] = pool_inactive(hist_all + (size_t)m * maxbins, descs[m].P, x);
    }
    __syncthreads();
    const unsigned long long step = st->step;
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t lo = so[0], hi = so[M];
    // the monitor of the last host and its host range [cur_lo, cur_hi): hosts
    // come in runs of one monitor, so the binary search runs once per run
    uint32_t cur = 0;
    uint64_t cur_lo = 1, cur_hi = 0;
    RangeConsts rc = {};
    for (;;) {
        uint64_t base = 0;
        if (lane == 0) base = lo + (uint64_t)atomicAdd(&st->q_gather, grab);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= hi) break;
        const uint64_t end = min(base + grab, hi);
        // up to 32 hosts at a time: lane j keeps host b0 + j's count and
        // monitor, and the warp's lanes evaluate their Eq. 11 side by side
        for (uint64_t b0 = base; b0 < end; b0 += 32) {
            const uint64_t b1 = min(b0 + 32, end);
            uint32_t myA = 0, mym = 0;
            for (uint64_t h = b0; h < b1; h++) {
                if (h < cur_lo || h >= cur_hi) {   // CheckAT of monitor m: ACT = BACT^0 for every AT in frame 0
                    cur = find_monitor(so, M, h);
                    cur_lo = so[cur];
                    cur_hi = so[cur + 1];
                    rc = range_consts(bact0_of(step, sd[cur].twok), kp[cur], sd[cur].twok);
                }
                const Geom &G = sd[cur];
                const uint32_t aip = hosts[h];
                uint32_t cnt;
                if (CPSL >= 0) {
                    const uint32_t nseg = G.g >> G.log2L;
                    const uint32_t c2k = (128u - G.twok) * ONES;
                    if (nseg % (32u * RB) == 0)
                        cnt = gather_host_vec<(CPSL < 0 ? 0 : CPSL), RB, true>(G, rc, c2k, aip, u1, u2, u3, lane);
                    else
                        cnt = gather_host_vec<(CPSL < 0 ? 0 : CPSL), RB, false>(G, rc, c2k, aip, u1, u2, u3, lane);
                } else {
                    cnt = gather_host_scalar(G, bact0_of(step, G.twok), kp[cur], aip, lane);
                }
                const uint32_t A = __reduce_add_sync(0xFFFFFFFFu, cnt);
                if (lane == (uint32_t)(h - b0)) {
                    myA = A;
                    mym = cur;
                }
            }
            if (b0 + lane < b1) {
                const Geom &G = sd[mym];
                uint8_t f;
                out[b0 + lane] = estimate_eq11(G.g, G.P, n0[mym], myA, f);
                if (flags) flags[b0 + lane] = f;
            }
        }
    }
}

int sm_count_current() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

struct vate_group {
    uint32_t M = 0;
    std::vector<vate_params> prm;
    std::vector<Geom> geoms;         // host copies (pool pointers into the arena)
    Geom arena_geom;                 // carries the L2 window over the whole arena
    uint8_t *arena = nullptr;
    uint64_t arena_bytes = 0;
    Geom *d_descs = nullptr;
    GroupState *d_state = nullptr;
    uint64_t *d_hist = nullptr;      // M x maxbins
    uint32_t maxbins = 0;
    CensusTile *d_tiles = nullptr;
    uint32_t ntiles = 0, tiles_capacity = 0;
    uint32_t L = 1, log2L = 0;
    int sms = 148;
    uint32_t steps = 0;              // steps queued so far (host count)
    vate_group_tuning tuning;
    bool persist_l2 = false;         // VATE_OPT_PERSIST_L2 in some monitor's options
    // CUDA graph of one step
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t graph_key[12] = {};
};

namespace {

int rebuild_tiles(vate_group *g, cudaStream_t st) {
    std::vector<CensusTile> t;
    const uint64_t per = g->tuning.census_tile_chunks;
    for (uint32_t m = 0; m < g->M; m++) {
        uint64_t nch = g->geoms[m].P >> 4;          // chunks of monitor m's own pool
        for (uint64_t c = 0; c < nch; c += per) {
            CensusTile x;
            x.mon = m;
            x.nchunks = (uint32_t)std::min(per, nch - c);
            x.chunk0 = c;                           // relative to monitor m's pool
            t.push_back(x);
        }
    }
    if (t.size() > g->tiles_capacity) return vate::set_error(VATE_EINVAL, "census tile table overflow");
    g->ntiles = (uint32_t)t.size();
    cudaError_t e = cudaMemcpyAsync(g->d_tiles, t.data(), t.size() * sizeof(CensusTile), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

int check_tuning(const vate_group_tuning *t) {
    if (!t) return vate::set_error(VATE_EINVAL, "tuning is NULL");
    uint32_t c = t->census_tile_chunks;
    if (c < 256 || c > 65536 || (c & (c - 1))) return vate::set_error(VATE_EINVAL, "census_tile_chunks: power of two in [256, 65536]");
    for (uint32_t v : {t->gather_blocks_per_sm, t->ingest_blocks_per_sm, t->preserve_blocks_per_sm})
        if (v < 1 || v > 32) return vate::set_error(VATE_EINVAL, "blocks per SM must be in [1, 32]");
    if (t->gather_hosts_per_grab < 1 || t->gather_hosts_per_grab > 64) return vate::set_error(VATE_EINVAL, "gather_hosts_per_grab in [1, 64]");
    return VATE_OK;
}

size_t ingest_smem(uint32_t M) { return (size_t)((M + 2) & ~1u) * 8 + (size_t)M * sizeof(Geom); }
size_t gather_smem(uint32_t M) { return (size_t)((2 * M + 1 + (M + 1) / 2 + 1) & ~1u) * 8 + (size_t)M * sizeof(Geom); }
size_t census_smem(uint32_t maxbins) { return (size_t)(G_THREADS / 32) * ((maxbins + 1) / 2) * 32 * sizeof(uint32_t); }

template <int CPSL, int RB>
cudaError_t launch_group_gather(vate_group *g, const uint32_t *hosts, const uint64_t *hoff, uint64_t hcap,
                                const uint32_t *kprime, float *out, uint8_t *flags, cudaStream_t st) {
    auto kern = group_gather_kernel<CPSL, RB>;
    size_t smem = gather_smem(g->M);
    if (cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return e;
    return vate::launch_pool(g->arena_geom, kern, g->sms * g->tuning.gather_blocks_per_sm, G_THREADS, smem, st,
                             (const Geom *)g->d_descs, g->M, g->d_state, hosts, hoff, hcap, kprime,
                             (const uint64_t *)g->d_hist, g->maxbins, out, flags, g->tuning.gather_hosts_per_grab, 1u,
                             1u, 1u);
}

cudaError_t enqueue_gather(vate_group *g, const uint32_t *hosts, const uint64_t *hoff, uint64_t hcap,
                           const uint32_t *kprime, float *out, uint8_t *flags, cudaStream_t st) {
    if (g->L == 16) return launch_group_gather<0, 2>(g, hosts, hoff, hcap, kprime, out, flags, st);
    if (g->L == 32) return launch_group_gather<1, 2>(g, hosts, hoff, hcap, kprime, out, flags, st);
    if (g->L == 64) return launch_group_gather<2, 2>(g, hosts, hoff, hcap, kprime, out, flags, st);
    return launch_group_gather<-1, 1>(g, hosts, hoff, hcap, kprime, out, flags, st);
}

cudaError_t enqueue_ingest(vate_group *g, const vate_pair *pairs, const uint64_t *poff, uint64_t pcap,
                           cudaStream_t st) {
    size_t smem = ingest_smem(g->M);
    if (cudaError_t e = cudaFuncSetAttribute(group_ingest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return e;
    return vate::launch_pool(g->arena_geom, group_ingest_kernel, g->sms * g->tuning.ingest_blocks_per_sm, G_THREADS,
                             smem, st, (const Geom *)g->d_descs, g->M, g->d_state,
                             reinterpret_cast<const uint32_t *>(pairs), poff, pcap);
}

cudaError_t enqueue_census(vate_group *g, cudaStream_t st) {
    size_t smem = census_smem(g->maxbins);
    if (cudaError_t e = cudaFuncSetAttribute(group_census_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return e;
    // as many blocks per SM as their columns fit in about 200 KiB, up to four
    const int per_sm = (int)std::min<size_t>(4, std::max<size_t>(1, (size_t)(200u << 10) / smem));
    return vate::launch_pool(g->arena_geom, group_census_kernel, g->sms * per_sm, G_THREADS, smem, st,
                             (const Geom *)g->d_descs, g->d_state, (const CensusTile *)g->d_tiles, g->ntiles, g->d_hist,
                             g->maxbins);
}

cudaError_t enqueue_step(vate_group *g, const vate_pair *pairs, const uint64_t *poff, uint64_t pcap,
                         const uint32_t *hosts, const uint64_t *hoff, uint64_t hcap, const uint32_t *kprime,
                         float *out, uint8_t *flags, cudaStream_t st) {
    const uint32_t hist_words = g->M * g->maxbins;
    cudaError_t e = vate::launch_pool(g->arena_geom, group_begin_kernel, 8, G_THREADS, 0, st, g->d_state, g->d_hist,
                                      hist_words);
    if (e == cudaSuccess)
        e = vate::launch_pool(g->arena_geom, group_preserve_kernel, g->sms * g->tuning.preserve_blocks_per_sm,
                              G_THREADS, 0, st, (const Geom *)g->d_descs, g->M, (const GroupState *)g->d_state);
    if (e == cudaSuccess) e = enqueue_ingest(g, pairs, poff, pcap, st);
    if (e == cudaSuccess) e = enqueue_census(g, st);
    if (e == cudaSuccess) e = enqueue_gather(g, hosts, hoff, hcap, kprime, out, flags, st);
    return e;
}

int check_step_args(vate_group *g, const vate_pair *pairs, const uint64_t *poff, uint64_t pcap, const uint32_t *hosts,
                    const uint64_t *hoff, uint64_t hcap, const uint32_t *kprime, float *out) {
    if (!g) return vate::set_error(VATE_EINVAL, "group is NULL");
    if (!poff || !hoff || !kprime) return vate::set_error(VATE_EINVAL, "offsets and k' must not be NULL");
    if ((pcap && !pairs) || (hcap && (!hosts || !out))) return vate::set_error(VATE_EINVAL, "NULL buffer with a nonzero capacity");
    if ((reinterpret_cast<uintptr_t>(pairs) & 7u) != 0) return vate::set_error(VATE_EINVAL, "d_pairs must be 8-byte aligned");
    return VATE_OK;
}

}  // namespace

extern "C" {

int vate_group_create(const vate_params *params, uint32_t n_monitors, void *stream, vate_group **out) {
    if (!out || !params) return vate::set_error(VATE_EINVAL, "params and out must not be NULL");
    if (n_monitors < 1 || n_monitors > MAX_MONITORS) return vate::set_error(VATE_EINVAL, "n_monitors must be in [1, 256]");
    cudaStream_t st = (cudaStream_t)stream;
    vate_group *g = new (std::nothrow) vate_group();
    if (!g) return vate::set_error(VATE_ENOMEM, "host allocation failed");
    g->M = n_monitors;
    g->prm.assign(params, params + n_monitors);
    for (uint32_t m = 0; m < n_monitors; m++)
        if (params[m].options & VATE_OPT_PERSIST_L2) g->persist_l2 = true;
    g->geoms.resize(n_monitors);
    uint64_t off = 0;
    for (uint32_t m = 0; m < n_monitors; m++) {
        int rc = vate::make_geom_checked(&params[m], &g->geoms[m]);
        if (rc) { delete g; return rc; }
        if (params[m].counter != VATE_COUNTER_AT) {
            delete g;
            return vate::set_error(VATE_EINVAL, "groups run asynchronous timestamps (counter 0)");
        }
        if (g->geoms[m].atw != 1u || g->geoms[m].packed) {
            delete g;
            return vate::set_error(VATE_EINVAL, "groups hold byte ATs (k <= 63)");
        }
        if (m && params[m].seg_len != params[0].seg_len) {
            delete g;
            return vate::set_error(VATE_EINVAL, "all monitors of a group must use the same seg_len");
        }
        g->geoms[m].frame0 = 1u;                 // pools keep timestamps in the frame of block 0
        g->maxbins = std::max(g->maxbins, g->geoms[m].twok + 1);
        off = (off + 255) & ~255ull;
        off += g->geoms[m].P;
    }
    g->L = params[0].seg_len;
    g->arena_bytes = (off + 255) & ~255ull;
    g->sms = sm_count_current();
    g->tuning.census_tile_chunks = 4096;
    g->tuning.gather_blocks_per_sm = 5;
    g->tuning.gather_hosts_per_grab = 4;
    g->tuning.ingest_blocks_per_sm = 16;
    g->tuning.preserve_blocks_per_sm = 8;
    g->tuning.reserved = 0;
    for (uint32_t m = 0; m < n_monitors; m++) g->tiles_capacity += (uint32_t)(((g->geoms[m].P >> 4) + 255) / 256);
    bool ok = cudaMalloc(&g->arena, g->arena_bytes) == cudaSuccess &&
              cudaMalloc(&g->d_descs, n_monitors * sizeof(Geom)) == cudaSuccess &&
              cudaMalloc(&g->d_state, sizeof(GroupState)) == cudaSuccess &&
              cudaMalloc(&g->d_hist, (size_t)n_monitors * g->maxbins * sizeof(uint64_t)) == cudaSuccess &&
              cudaMalloc(&g->d_tiles, (size_t)g->tiles_capacity * sizeof(CensusTile)) == cudaSuccess &&
              cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        vate_group_destroy(g);
        return vate::set_error(VATE_ENOMEM, "out of device memory for the group");
    }
    off = 0;
    for (uint32_t m = 0; m < n_monitors; m++) {
        off = (off + 255) & ~255ull;
        g->geoms[m].pool = g->arena + off;
        off += g->geoms[m].P;
    }
    // L2 window over the whole arena for every group launch
    memset(&g->arena_geom, 0, sizeof g->arena_geom);
    g->arena_geom.pool = g->arena;
    {
        int dev = 0, persist_max = 0, window_max = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&persist_max, cudaDevAttrMaxPersistingL2CacheSize, dev);
        cudaDeviceGetAttribute(&window_max, cudaDevAttrMaxAccessPolicyWindowSize, dev);
        size_t cur = 0;
        if (persist_max > 0 && window_max > 0 && cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) == cudaSuccess) {
            // the process-wide limit only on request (VATE_OPT_PERSIST_L2 in any monitor's options)
            if (g->persist_l2 && cur < (size_t)persist_max)
                cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, (size_t)persist_max);
            cudaGetLastError();
            g->arena_geom.l2_window_bytes = std::min<uint64_t>(g->arena_bytes, (uint64_t)window_max);
            double ratio = (double)persist_max / (double)g->arena_geom.l2_window_bytes;
            g->arena_geom.l2_hit_ratio = ratio >= 1.0 ? 1.0f : (float)ratio;
        }
    }
    GroupState s0;
    memset(&s0, 0, sizeof s0);
    cudaError_t e = cudaMemcpyAsync(g->d_descs, g->geoms.data(), n_monitors * sizeof(Geom), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, st);
    for (uint32_t m = 0; m < n_monitors && e == cudaSuccess; m++) {
        Geom G = g->geoms[m];
        G.l2_window_bytes = 0;
        e = vate::launch_init(G, st, g->sms);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        vate_group_destroy(g);
        return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    }
    int rc = rebuild_tiles(g, st);
    if (rc) {
        vate_group_destroy(g);
        return rc;
    }
    *out = g;
    return VATE_OK;
}

int vate_group_destroy(vate_group *g) {
    if (!g) return VATE_OK;
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->arena_geom.l2_window_bytes && g->persist_l2) cudaCtxResetPersistingL2Cache();
    cudaFree(g->arena);
    cudaFree(g->d_descs);
    cudaFree(g->d_state);
    cudaFree(g->d_hist);
    cudaFree(g->d_tiles);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    cudaGetLastError();
    delete g;
    return VATE_OK;
}

int vate_group_step(vate_group *g, const vate_pair *d_pairs, const uint64_t *d_pair_offsets, uint64_t pair_capacity,
                    const uint32_t *d_hosts, const uint64_t *d_host_offsets, uint64_t host_capacity,
                    const uint32_t *d_kprime, float *d_out, uint8_t *d_flags, void *stream) {
    if (int rc = check_step_args(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets, host_capacity,
                                 d_kprime, d_out))
        return rc;
    cudaError_t e = enqueue_step(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets, host_capacity,
                                 d_kprime, d_out, d_flags, (cudaStream_t)stream);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    g->steps++;
    return VATE_OK;
}

int vate_group_step_graph(vate_group *g, const vate_pair *d_pairs, const uint64_t *d_pair_offsets,
                          uint64_t pair_capacity, const uint32_t *d_hosts, const uint64_t *d_host_offsets,
                          uint64_t host_capacity, const uint32_t *d_kprime, float *d_out, uint8_t *d_flags,
                          void *stream) {
    if (int rc = check_step_args(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets, host_capacity,
                                 d_kprime, d_out))
        return rc;
    const vate_group_tuning &t = g->tuning;
    uint64_t key[12] = {(uint64_t)d_pairs, (uint64_t)d_pair_offsets, pair_capacity, (uint64_t)d_hosts,
                        (uint64_t)d_host_offsets, host_capacity, (uint64_t)d_kprime, (uint64_t)d_out,
                        (uint64_t)d_flags,
                        ((uint64_t)t.census_tile_chunks << 32) | t.gather_blocks_per_sm,
                        ((uint64_t)t.gather_hosts_per_grab << 32) | t.ingest_blocks_per_sm, t.preserve_blocks_per_sm};
    if (!g->exec || memcmp(key, g->graph_key, sizeof key) != 0) {
        if (g->exec) {
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = enqueue_step(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets,
                                          host_capacity, d_kprime, d_out, d_flags, g->cap_stream);
            e = cudaStreamEndCapture(g->cap_stream, &graph);
            if (e == cudaSuccess) e = le;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g->exec = nullptr;
            return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
        }
        memcpy(g->graph_key, key, sizeof key);
    }
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    g->steps++;
    return VATE_OK;
}

int vate_group_set_tuning(vate_group *g, const vate_group_tuning *t) {
    if (!g) return vate::set_error(VATE_EINVAL, "group is NULL");
    if (int rc = check_tuning(t)) return rc;
    bool tiles = t->census_tile_chunks != g->tuning.census_tile_chunks;
    g->tuning = *t;
    g->tuning.reserved = 0;
    if (tiles) return rebuild_tiles(g, g->cap_stream);
    return VATE_OK;
}

int vate_group_get_tuning(const vate_group *g, vate_group_tuning *t) {
    if (!g || !t) return vate::set_error(VATE_EINVAL, "NULL argument");
    *t = g->tuning;
    return VATE_OK;
}

int vate_group_autotune(vate_group *g, const vate_pair *d_pairs, const uint64_t *d_pair_offsets,
                        uint64_t pair_capacity, const uint32_t *d_hosts, const uint64_t *d_host_offsets,
                        uint64_t host_capacity, const uint32_t *d_kprime, float *d_out, uint8_t *d_flags,
                        vate_group_tuning *chosen, void *stream) {
    if (int rc = check_step_args(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets, host_capacity,
                                 d_kprime, d_out))
        return rc;
    if (g->steps == 0) return vate::set_error(VATE_ESLICE, "autotune needs one step of the slice to repeat");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return vate::set_error(VATE_ECUDA, "autotune: cudaEventCreate failed");
    }
    const vate_group_tuning entry = g->tuning;
    // every return after this point destroys the events; an error restores the
    // tiling the group had on entry
    auto fail = [&](int rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        g->tuning = entry;
        rebuild_tiles(g, st);
        return rc;
    };
    const uint32_t hist_words = g->M * g->maxbins;
    auto reset = [&](bool hist) {
        return vate::launch_pool(g->arena_geom, group_reset_kernel, 8, G_THREADS, 0, st, g->d_state, g->d_hist,
                                 hist ? hist_words : 0u);
    };
    auto timed = [&](auto &&fn) -> float {
        float best = 1e30f;
        for (int r = 0; r < 3; r++) {
            cudaEventRecord(e0, st);
            fn();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            best = std::min(best, ms);
        }
        return best;
    };
    vate_group_tuning best = g->tuning;
    // ingest: repeating the last step's SetATs rewrites the values they wrote
    // (d_pairs and d_pair_offsets must be that step's inputs, see the header)
    float bt = 1e30f;
    for (uint32_t b : {4u, 8u, 16u, 24u}) {
        g->tuning.ingest_blocks_per_sm = b;
        float ms = timed([&] { enqueue_ingest(g, d_pairs, d_pair_offsets, pair_capacity, st); });
        if (ms < bt) { bt = ms; best.ingest_blocks_per_sm = b; }
    }
    g->tuning.ingest_blocks_per_sm = best.ingest_blocks_per_sm;
    // census (histograms cleared before each run)
    bt = 1e30f;
    for (uint32_t c : {1024u, 4096u, 16384u, 65536u}) {
        g->tuning.census_tile_chunks = c;
        if (int rc = rebuild_tiles(g, st)) return fail(rc);
        float ms = timed([&] { reset(true); enqueue_census(g, st); });
        if (ms < bt) { bt = ms; best.census_tile_chunks = c; }
    }
    g->tuning.census_tile_chunks = best.census_tile_chunks;
    if (int rc = rebuild_tiles(g, st)) return fail(rc);
    reset(true);
    enqueue_census(g, st);                       // leave the slice's census in place
    // gather (queue counter cleared before each run)
    bt = 1e30f;
    for (uint32_t b : {3u, 4u, 5u, 6u}) {
        for (uint32_t grab : {1u, 4u, 16u}) {
            g->tuning.gather_blocks_per_sm = b;
            g->tuning.gather_hosts_per_grab = grab;
            float ms = timed([&] {
                reset(false);
                enqueue_gather(g, d_hosts, d_host_offsets, host_capacity, d_kprime, d_out, d_flags, st);
            });
            if (ms < bt) { bt = ms; best.gather_blocks_per_sm = b; best.gather_hosts_per_grab = grab; }
        }
    }
    g->tuning = best;
    reset(false);
    cudaError_t e = enqueue_gather(g, d_hosts, d_host_offsets, host_capacity, d_kprime, d_out, d_flags, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(vate::set_error(VATE_ECUDA, cudaGetErrorString(e)));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (chosen) *chosen = best;
    return VATE_OK;
}

int vate_group_status(vate_group *g, uint32_t *status, int clear, void *stream) {
    if (!g || !status) return vate::set_error(VATE_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    GroupState s;
    cudaError_t e = cudaMemcpyAsync(&s, g->d_state, sizeof s, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && clear) {
        unsigned int z = 0;
        e = cudaMemcpyAsync(&g->d_state->status, &z, sizeof z, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    *status = s.status;
    return VATE_OK;
}

int vate_group_copy_pool(vate_group *g, uint32_t m, uint8_t *d_dst, void *stream) {
    if (!g || m >= g->M || !d_dst) return vate::set_error(VATE_EINVAL, "bad group, monitor or destination");
    cudaStream_t st = (cudaStream_t)stream;
    const Geom &G = g->geoms[m];
    cudaError_t e = cudaMemcpyAsync(d_dst, G.pool, G.P, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = vate::launch_frame_convert(G, d_dst, d_dst, 0, G.P, true, st, g->sms);   // paper's form
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

int vate_group_census(vate_group *g, uint32_t m, uint64_t *d_hist, void *stream) {
    if (!g || m >= g->M || !d_hist) return vate::set_error(VATE_EINVAL, "bad group, monitor or destination");
    if (g->steps == 0) return vate::set_error(VATE_ESLICE, "no step has run yet");
    cudaError_t e = cudaMemcpyAsync(d_hist, g->d_hist + (size_t)m * g->maxbins, (g->geoms[m].twok + 1) * sizeof(uint64_t),
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

int vate_group_monitor_info(vate_group *g, uint32_t m, vate_info *out, void *stream) {
    if (!g || m >= g->M || !out) return vate::set_error(VATE_EINVAL, "bad group, monitor or output");
    cudaStream_t st = (cudaStream_t)stream;
    GroupState s;
    cudaError_t e = cudaMemcpyAsync(&s, g->d_state, sizeof s, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    const Geom &G = g->geoms[m];
    out->pool_size = G.P;
    out->block_a = G.a;
    out->block_b = G.b;
    out->slice = s.started ? (int64_t)s.step : -1;
    out->bact0 = (uint32_t)(s.step % G.twok);
    out->closed = s.started ? 1u : 0u;
    out->pid_lo = 0;
    out->pid_hi = G.P;
    return VATE_OK;
}

}  // extern "C"
