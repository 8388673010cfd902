// vate_group.cu -- many independent monitors advanced together (include/vate_group.h).
//
// One slice of every monitor is ONE persistent launch, group_step_kernel.  Its
// blocks take work items in order from a device queue.  Each monitor's items
// follow Algorithm 4's per-slice pipeline:
//   B  begin: clear the monitor's census histogram                  (1 item)
//   P  PreserveAT (Algorithm 3) on the two blocks whose ACT became
//      0 or k, in tiles of 16-byte chunks                          (none at slice 0)
//   I  SetAT for the monitor's pairs, in tiles of pairs
//   C  pool census, in tiles of 16-byte chunks
// An item of one phase of monitor m starts once every item of the earlier
// phases of m has finished: a per-monitor count of finished items, waited on
// by the block's first thread with a bounded spin.  Every item waits only on
// items earlier in the list, and an item is handed out only to a running
// block, so the smallest unfinished item can always proceed: no wait can
// depend on a block that is not running, and the launch needs no
// co-residency guarantee.  A wait that runs past its spin limit marks the
// step as timed out in the group's status word (VATE_GROUP_TIMEOUT) and every
// later wait of the launch gives up at once, so the kernel always returns.
//
// The list is cut into waves of consecutive monitors whose pools together fit a
// byte budget (the tuning's wave_pool_mib; 0: one wave of all monitors), and
// the waves are software-pipelined: step s lists the B, P and I items of wave
// s, then the C items of wave s - 1, each phase monitor after monitor.  With
// one wave the order is phase-major: every B, P and I item, then every C.
//
//   G  CheckAT gather + Eq. 11 is not an item: a block that finds the list
//      exhausted turns its warps loose on the hosts, monitor after monitor,
//      each warp taking a few hosts at a time from the monitor's host
//      counter (the tuning's gather_grab_hosts, scaled by g).  A warp's first
//      batch of a monitor waits (its first lane, bounded as above) until
//      every item of the monitor has finished.  Warps never wait for one
//      another, and the hosts in flight at any time are those of one or two
//      monitors, whose pools then stay in L2 (blocks of whole tiles of hosts
//      would spread the reads over many pools).  The waits depend only on
//      items, all of which are held by running blocks by then.
//
// Loads: PreserveAT reads its chunks L2-only, SetAT only stores and the
// census reads L2-only, so no SM holds an L1 copy of a pool line when the
// gather reads it through the read-only path after the writes of other
// blocks (L1 starts empty at every launch).  The per-chunk and per-host
// arithmetic is the one of the single-pool kernels (vate_device_ops.cuh), so
// every monitor is bit-identical to a vate_handle run alone.  The slice
// number, the batch offsets and k' are read on the device, so the one launch
// is captured once as a CUDA graph and replayed every slice.
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
constexpr int G_WARPS = G_THREADS / 32;
constexpr int NPHASE = 5;                 // B, P, I, C, G
// Compile-time shape of the step kernel, measured on the 64-monitor workload
// (44.2 M pairs, 1.86 M hosts, 0.58 GiB of pools, no persisting L2): at most
// 64 registers (4 blocks per SM) and six census warps 3.50 ms; 80 registers
// (3 blocks per SM) 2.56 ms with six census warps, 2.55 with four, 2.68 with
// two (the gather phase 1.96 -> 1.19 ms: its loads in flight); 96 registers
// (2 blocks per SM) 2.90 ms.
#ifndef VATE_GROUP_CWARPS
#define VATE_GROUP_CWARPS 4
#endif
#ifndef VATE_GROUP_MINB
#define VATE_GROUP_MINB 3
#endif
#ifndef VATE_GROUP_INGEST_U
#define VATE_GROUP_INGEST_U 8
#endif
#ifndef VATE_GROUP_GATHER_CG
#define VATE_GROUP_GATHER_CG 0
#endif
constexpr int C_WARPS = VATE_GROUP_CWARPS;      // warps that count a census item (lane columns in shared memory)
constexpr int G_MIN_BLOCKS = VATE_GROUP_MINB;   // blocks per SM the step kernel is built for (3: at most 80 registers)
constexpr int I_BATCH = VATE_GROUP_INGEST_U;    // pairs a thread loads before its SetATs
constexpr unsigned long long DEFAULT_SPIN_LIMIT = 1ull << 23;   // x ~128 ns of sleep: about a second

struct GroupState {                       // device-resident
    unsigned long long step;              // the slice last processed (valid once started)
    unsigned int started;                 // set by the first step
    unsigned int status;                  // VATE_GROUP_* bits (sticky)
    unsigned int q_items;                 // work items handed out in the running launch
    unsigned int blocks_done;             // blocks of the running launch that have finished
    unsigned int poisoned;                // a wait of the running launch gave up
    unsigned int pad;
};

struct StepArgs {
    const Geom *descs;
    GroupState *st;
    unsigned int *done;                   // [M]: items of the monitor finished in the running launch
    const uint32_t *pairs;
    const uint64_t *poff;
    uint64_t pcap;
    const uint32_t *hosts;
    const uint64_t *hoff;
    uint64_t hcap;
    const uint32_t *kprimes;
    uint64_t *hist;                       // [M][maxbins]
    float *out;
    uint8_t *flags;
    unsigned long long spin_limit;
    uint32_t M, maxbins;
    uint32_t census_tile, ingest_tile, gather_grab, preserve_tile;
    unsigned long long *qhost;            // [M]: hosts of the monitor handed out in the running launch
    uint64_t wave_bytes;                  // pools per wave of monitors (0: one wave of all monitors)
    unsigned long long *trace;            // NULL, or 4 words per item and per block (vate_group_set_trace)
    uint32_t trace_cap;                   // items the trace buffer holds
    uint32_t advance;                     // 1: the next slice; 0: repeat the last slice (autotuner)
    uint32_t missing;                     // added to every wait's target (tests of the timeout path)
    uint32_t u1, u2, u3;                  // run-time ones (the vector gather's multiply-adds)
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

// the last index m < M with pre[m] <= i (pre non-decreasing, pre[0] <= i < pre[M]): with runs of equal
// entries (empty segments) that is the segment holding i
template <typename T>
__device__ __forceinline__ uint32_t find_monitor(const T *pre, uint32_t M, uint64_t i) {
    uint32_t lo = 0, hi = M;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((uint64_t)pre[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// The 16-byte chunks PreserveAT visits for the slide to `step`: the chunks
// covering [s0, e0) (the block whose ACT became 0) then those covering
// [s1, e1) (ACT k), as in the single-pool preserve_kernel.
struct PreserveSpan {
    uint64_t s0, e0, s1, e1, c0s, c0e, c1s, n0, n;
    uint32_t b0;
};
__device__ __forceinline__ PreserveSpan preserve_span(const Geom &G, unsigned long long step) {
    PreserveSpan p;
    p.b0 = bact0_of(step, G.twok);
    const uint32_t i0 = (G.twok - p.b0) % G.twok, i1 = (G.k + G.twok - p.b0) % G.twok;
    block_range_of(G, i0, &p.s0, &p.e0);
    block_range_of(G, i1, &p.s1, &p.e1);
    p.c0s = p.s0 >> 4;
    p.c0e = (p.e0 + 15) >> 4;
    p.c1s = p.s1 >> 4;
    const uint64_t c1e = (p.e1 + 15) >> 4;
    p.n0 = p.e0 > p.s0 ? p.c0e - p.c0s : 0;
    p.n = p.n0 + (p.e1 > p.s1 ? c1e - p.c1s : 0);
    return p;
}

// Thread 0 of a block: wait until *done >= target, with at most `limit`
// sleeps of ~128 ns.  A wait that gives up marks the launch (poisoned) and
// the group (VATE_GROUP_TIMEOUT); a wait in a marked launch gives up at once.
// Hosts a warp takes at a time from a monitor with g VATs per host: the
// tuning's figure is for g = 4096, scaled by 4096 / g so that a batch is
// about the same work whatever g, in [1, 32] (a lane keeps one host's count).
__device__ __forceinline__ uint32_t gather_grab_of(uint32_t grab, uint32_t g) {
    const uint64_t t = (uint64_t)grab * 4096u / (g ? g : 1u);
    return (uint32_t)(t < 1u ? 1u : (t > 32u ? 32u : t));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t sm_id() {
    uint32_t id;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(id));
    return id;
}

__device__ bool wait_done(const unsigned int *done, unsigned int target, GroupState *st, unsigned long long limit) {
    for (unsigned long long spins = 0;; spins++) {
        if (*reinterpret_cast<const volatile unsigned int *>(done) >= target) {
            __threadfence();                      // the finished items' writes before ours
            return true;
        }
        if (*reinterpret_cast<volatile unsigned int *>(&st->poisoned)) return false;
        if (spins >= limit) {
            atomicOr(&st->status, VATE_GROUP_TIMEOUT);
            atomicExch(&st->poisoned, 1u);
            return false;
        }
        __nanosleep(128);
    }
}

// GK: the gather of the group's segment length: 0, 1, 2 = 16, 32, 64-byte
// segments (gather_host_vec); 3, 4, 5 = 2, 4, 8-byte segments
// (gather_host_seg); 6 = one byte per VAT (gather_host_scalar).
template <int GK>
__device__ __forceinline__ uint32_t gather_one(const Geom &G, const RangeConsts &rc, uint32_t c2k, uint32_t bact0,
                                               uint32_t kp, uint32_t aip, uint32_t lane, const StepArgs &a) {
    // the read-only path: no L1 copy of the pool predates this launch's writes (see the top of the file)
    if constexpr (GK <= 2) {
        const uint32_t nseg = G.g >> G.log2L;
        constexpr bool CG = VATE_GROUP_GATHER_CG != 0;
        if (nseg % (32u * 2u) == 0)
            return gather_host_vec<GK, 2, true, 1, false, CG>(G, rc, c2k, aip, a.u1, a.u2, a.u3, lane);
        return gather_host_vec<GK, 2, false, 1, false, CG>(G, rc, c2k, aip, a.u1, a.u2, a.u3, lane);
    } else if constexpr (GK <= 5) {
        constexpr int SB = GK == 3 ? 2 : (GK == 4 ? 4 : 8);
        return gather_host_seg<SB, 1, false>(G, rc, c2k, G.twok * ONES, aip, lane);
    } else {
        return gather_host_scalar(G, bact0, kp, aip, lane);
    }
}

template <int GK>
__global__ void __launch_bounds__(G_THREADS, G_MIN_BLOCKS) group_step_kernel(StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t M = a.M;
    uint64_t *po = reinterpret_cast<uint64_t *>(smem);              // M + 1 pair offsets (clamped)
    uint64_t *ho = po + (M + 1);                                      // M + 1 host offsets (clamped)
    uint32_t *cum = reinterpret_cast<uint32_t *>(ho + (M + 1));       // [M][NPHASE + 1]: items before each phase
    uint32_t *kp = cum + M * (NPHASE + 1);                            // M: k' (clamped)
    uint32_t *seg_start = kp + M;                                     // NPHASE * M + 1: first item of each segment
    uint32_t *seg_mp = seg_start + (NPHASE * M + 1);                  // NPHASE * M: (monitor << 3) | phase
    uint32_t *wave_lo = seg_mp + NPHASE * M;                          // M + 1: first monitor of each wave
    uint32_t *cols = wave_lo + (M + 1);                               // census lane columns [C_WARPS][pairs][32]
    const uint32_t maxpairs = (a.maxbins + 1u) / 2u;

    __shared__ unsigned long long s_step, s_t0, s_t1;
    __shared__ uint32_t s_j, s_m, s_p, s_t, s_ok, s_gm;
    __shared__ Geom sG, sGw[G_WARPS];
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    GroupState *st = a.st;

    if (tid == 0) {
        // a group whose earlier step timed out (poisoned stays set) does no more work
        s_ok = *reinterpret_cast<volatile unsigned int *>(&st->poisoned) ? 0u : 1u;
        s_step = a.advance ? (st->started ? st->step + 1ull : 0ull) : st->step;
    }
    __syncthreads();
    const unsigned long long step = s_step;
    if (s_ok) {

    // ---- per-block set-up: offsets, k', the item counts of every monitor ----
    for (uint32_t t = tid; t <= M; t += blockDim.x) {
        po[t] = a.poff[t];
        ho[t] = a.hoff[t];
    }
    __syncthreads();
    if (tid == 0) {                           // clamp to the capacities, make non-decreasing
        bool bad = false;
        uint64_t pp = 0, hp = 0;
        for (uint32_t t = 0; t <= M; t++) {
            uint64_t v = po[t], w = ho[t];
            if (v > a.pcap) { v = a.pcap; bad = true; }
            if (t && v < pp) { v = pp; bad = true; }
            if (w > a.hcap) { w = a.hcap; bad = true; }
            if (t && w < hp) { w = hp; bad = true; }
            po[t] = pp = v;
            ho[t] = hp = w;
        }
        if (bad && blockIdx.x == 0) atomicOr(&st->status, VATE_GROUP_BAD_OFFSETS);
    }
    __syncthreads();
    for (uint32_t m = tid; m < M; m += blockDim.x) {
        const Geom &G = a.descs[m];
        uint32_t x = a.kprimes[m];
        if (x < 1u || x > G.k) {
            if (blockIdx.x == 0) atomicOr(&st->status, VATE_GROUP_BAD_KPRIME);
            x = G.k;
        }
        kp[m] = x;
        uint32_t n[NPHASE];
        n[0] = 1u;
        n[1] = step == 0ull ? 0u
                            : (uint32_t)((preserve_span(G, step).n + a.preserve_tile - 1) / a.preserve_tile);
        n[2] = (uint32_t)((po[m + 1] - po[m] + a.ingest_tile - 1) / a.ingest_tile);
        n[3] = (uint32_t)(((G.P >> 4) + a.census_tile - 1) / a.census_tile);
        n[4] = 0u;                            // G runs after the list, warp by warp
        uint32_t c = 0;
        for (int p = 0; p < NPHASE; p++) {
            cum[m * (NPHASE + 1) + p] = c;
            c += n[p];
        }
        cum[m * (NPHASE + 1) + NPHASE] = c;
    }
    __syncthreads();
    if (tid == 0) {
        // waves of consecutive monitors whose pools add up to at most wave_bytes (one monitor at least)
        uint32_t nw = 0;
        for (uint32_t m0 = 0; m0 < M; nw++) {
            wave_lo[nw] = m0;
            uint32_t m1 = m0 + 1;
            uint64_t bytes = a.descs[m0].P;
            if (!a.wave_bytes) m1 = M;
            while (m1 < M && bytes + a.descs[m1].P <= a.wave_bytes) bytes += a.descs[m1++].P;
            m0 = m1;
        }
        wave_lo[nw] = M;
        // segments = (monitor, phase) runs of items: step s lists B, P, I of wave s, C of wave s - 1,
        // each phase monitor after monitor
        uint32_t ns = 0, run = 0;
        auto emit = [&](uint32_t w, int p0, int p1) {
            for (int p = p0; p <= p1; p++)
                for (uint32_t m = wave_lo[w]; m < wave_lo[w + 1]; m++) {
                    seg_start[ns] = run;
                    seg_mp[ns] = (m << 3) | (uint32_t)p;
                    run += cum[m * (NPHASE + 1) + p + 1] - cum[m * (NPHASE + 1) + p];
                    ns++;
                }
        };
        for (uint32_t st2 = 0; st2 < nw + 1; st2++) {
            if (st2 < nw) emit(st2, 0, 2);
            if (st2 >= 1) emit(st2 - 1, 3, 3);
        }
        seg_start[ns] = run;                  // ns = 4 M: the total
    }
    __syncthreads();
    const uint32_t nsegs = 4u * M;
    const uint32_t total = seg_start[nsegs];

    // ---- the items ----
    for (;;) {
        if (tid == 0) {
            const uint32_t j = atomicAdd(&st->q_items, 1u);
            s_j = j;
            if (a.trace) s_t0 = global_ns();
            if (j < total) {
                const uint32_t sg = find_monitor(seg_start, nsegs, j);   // the segment holding item j
                const uint32_t m = seg_mp[sg] >> 3, p = seg_mp[sg] & 7u;
                const uint32_t *cm = cum + m * (NPHASE + 1);
                s_m = m;
                s_p = p;
                s_t = j - seg_start[sg];
                s_ok = wait_done(a.done + m, cm[p] + a.missing, st, a.spin_limit) ? 1u : 0u;
                if (a.trace) s_t1 = global_ns();
            }
        }
        __syncthreads();
        if (s_j >= total) break;
        if (warp == 0 && s_ok) {                                 // the item's descriptor, copied by one warp
            const uint32_t *src = reinterpret_cast<const uint32_t *>(a.descs + s_m);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sG);
            for (uint32_t w = lane; w < sizeof(Geom) / 4; w += 32u) dst[w] = src[w];
        }
        __syncthreads();
        if (s_ok) {
            const uint32_t m = s_m, p = s_p, t = s_t;
            const Geom G = sG;
            const uint32_t bact0 = bact0_of(step, G.twok);
            if (p == 0) {                                        // B: clear the monitor's census
                for (uint32_t b = tid; b <= G.twok; b += blockDim.x) a.hist[(size_t)m * a.maxbins + b] = 0ull;
            } else if (p == 1) {                                 // P: PreserveAT, chunks [t*T, (t+1)*T)
                const PreserveSpan ps = preserve_span(G, step);
                const RangeConsts pc = preserve_consts_frame0(ps.b0, G.k);
                const uint64_t u1 = min((uint64_t)(t + 1) * a.preserve_tile, ps.n);
                for (uint64_t u = (uint64_t)t * a.preserve_tile + tid; u < u1; u += blockDim.x) {
                    const uint64_t chunk = u < ps.n0 ? ps.c0s + u : ps.c1s + (u - ps.n0);
                    if (u >= ps.n0 && ps.n0 && chunk >= ps.c0s && chunk < ps.c0e) continue;   // range 0's chunk
                    preserve_chunk<true>(G.pool, chunk << 4, pc, G.twok, ps.s0, ps.e0, ps.s1, ps.e1);
                }
            } else if (p == 2) {                                 // I: SetAT (frame 0: the value BACT^0)
                const uint2 *p2 = reinterpret_cast<const uint2 *>(a.pairs);   // 8-byte aligned (host check)
                const uint64_t i0 = po[m] + (uint64_t)t * a.ingest_tile;
                const uint64_t i1 = min(i0 + a.ingest_tile, po[m + 1]);
                const uint8_t v = (uint8_t)bact0;
                // I_BATCH pairs loaded before any store: a byte store may alias the pairs, so the
                // compiler would not move a later load above it
                for (uint64_t i = i0 + tid; i < i1; i += (uint64_t)I_BATCH * G_THREADS) {
                    uint2 q[I_BATCH];
#pragma unroll
                    for (int u = 0; u < I_BATCH; u++) {
                        const uint64_t j = i + (uint64_t)u * G_THREADS;
                        q[u] = j < i1 ? __ldcs(p2 + j) : make_uint2(0u, 0u);
                    }
#pragma unroll
                    for (int u = 0; u < I_BATCH; u++) {
                        if (i + (uint64_t)u * G_THREADS >= i1) break;
                        const uint32_t pid = vat_pid(G, q[u].x, bh(G, q[u].y));
                        if (VATE_CHECK_POSITION(G, pid)) G.pool[pid] = v;
                    }
                }
            } else {                                             // C: census tile into lane columns
                const uint32_t nbins = G.twok + 1u, npairs = (nbins + 1u) / 2u;
                const bool counts = warp < (uint32_t)C_WARPS;      // the counting warps (the others wait)
                uint32_t *col = cols + (size_t)(counts ? warp : 0u) * maxpairs * 32u + lane;
                if (counts)
                    for (uint32_t b = 0; b < npairs; b++) col[b * 32u] = 0u;
                const uint32_t pat = G.twok * ONES;
                uint32_t runs = 0;
                const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
                // a tile holds at most 65,536 chunks, over C_WARPS * 32 lanes: at most 2^20 / (32 C_WARPS)
                // ATs a lane (8,192 for four warps), so every 16-bit counter stays exact
                static_assert(C_WARPS >= 1 && (1u << 20) / (32u * C_WARPS) < 65536u, "16-bit census counters");
                constexpr int U = 8;
                constexpr uint32_t CT = C_WARPS * 32u;           // counting threads
                const uint64_t q0 = (uint64_t)t * a.census_tile;
                const uint64_t qend = min(q0 + a.census_tile, G.P >> 4);
                if (counts) {
                    for (uint64_t q = q0 + tid; q < qend; q += (uint64_t)U * CT) {
                        uint4 w[U];
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const uint64_t qu = q + (uint64_t)u * CT;
                            w[u] = qu < qend ? __ldcg(pool16 + qu) : make_uint4(pat, pat, pat, pat);
                        }
#pragma unroll
                        for (int u = 0; u < U; u++) {
                            const uint64_t qu = q + (uint64_t)u * CT;
                            if (qu < qend) census_chunk_raw_pairs(w[u], pat, G.twok, col, runs);
                        }
                    }
                    col[(G.twok >> 1) * 32u] += 16u * runs;      // 2k is even: the low half of pair k
                }
                __syncthreads();
                unsigned long long *h = reinterpret_cast<unsigned long long *>(a.hist) + (size_t)m * a.maxbins;
                for (uint32_t r = warp; r < npairs; r += G_WARPS) {
                    uint32_t lo = 0, hi = 0;
                    for (uint32_t wv = 0; wv < (uint32_t)C_WARPS; wv++) {
                        const uint32_t x = cols[((size_t)wv * maxpairs + r) * 32u + lane];
                        lo += x & 0xFFFFu;
                        hi += x >> 16;
                    }
                    lo = __reduce_add_sync(0xFFFFFFFFu, lo);
                    hi = __reduce_add_sync(0xFFFFFFFFu, hi);
                    if (lane == 0 && lo) atomicAdd(h + census_raw_bin(G, bact0, 2u * r), (unsigned long long)lo);
                    if (lane == 0 && hi && 2u * r + 1u < nbins)
                        atomicAdd(h + census_raw_bin(G, bact0, 2u * r + 1u), (unsigned long long)hi);
                }
            }
        }
        // the item's writes, then its completion (release to the waits of later items)
        __threadfence();
        __syncthreads();
        if (tid == 0 && s_ok) atomicAdd(a.done + s_m, 1u);
        if (tid == 0 && a.trace && s_j < a.trace_cap) {        // handed out, started, finished, what and where
            unsigned long long *tr = a.trace + 4ull * s_j;
            tr[0] = s_t0;
            tr[1] = s_t1;
            tr[2] = global_ns();
            tr[3] = ((unsigned long long)sm_id() << 32) | ((unsigned long long)s_m << 8) | s_p;
        }
    }

    // ---- G: CheckAT gather + Eq. 11, warp by warp over the hosts ----
    if (tid == 0) {
        s_gm = 0u;                            // monitors below s_gm: this block has seen their hosts run out
        if (a.trace) s_t0 = global_ns();
    }
    __syncthreads();
    {
        Geom &G = sGw[warp];                  // the descriptor of the warp's monitor
        uint32_t m = 0, have = 0xFFFFFFFFu;
        bool ready = false;                   // every item of monitor `have` has finished
        RangeConsts rc = {};
        uint32_t c2k = 0, k1 = 1, bact0 = 0, grab = 1;
        uint64_t N0 = 0;
        for (;;) {
            m = max(m, *reinterpret_cast<volatile uint32_t *>(&s_gm));
            if (m >= M) break;
            if (m != have) {
                __syncwarp();
                const uint32_t *src = reinterpret_cast<const uint32_t *>(a.descs + m);
                uint32_t *dst = reinterpret_cast<uint32_t *>(&G);
                for (uint32_t w = lane; w < sizeof(Geom) / 4; w += 32u) dst[w] = src[w];
                __syncwarp();
                have = m;
                ready = false;
                k1 = kp[m];
                bact0 = bact0_of(step, G.twok);
                rc = range_consts(bact0, k1, G.twok);            // frame 0: ACT = BACT^0
                c2k = (128u - G.twok) * ONES;
                grab = gather_grab_of(a.gather_grab, G.g);
            }
            const uint64_t nh = ho[m + 1] - ho[m];
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(a.qhost + m, (unsigned long long)grab);
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            if (b >= nh) {                                       // the monitor's hosts are all handed out
                if (lane == 0) atomicMax(&s_gm, m + 1u);
                m++;
                continue;
            }
            if (!ready) {
                uint32_t ok = 0;
                if (lane == 0)
                    ok = wait_done(a.done + m, cum[m * (NPHASE + 1) + NPHASE] + a.missing, st, a.spin_limit) ? 1u : 0u;
                if (!__shfl_sync(0xFFFFFFFFu, ok, 0)) break;
                // N0 of Eq. 11 from the census (written in this launch: read from L2)
                unsigned long long act = 0;
                for (uint32_t d = lane; d < k1; d += 32u) act += __ldcg(a.hist + (size_t)m * a.maxbins + d);
                for (int o = 16; o; o >>= 1) act += __shfl_xor_sync(0xFFFFFFFFu, act, o);
                N0 = (1ull << G.c) - act;
                ready = true;
            }
            // lane j keeps host b0 + j's count; the Eq. 11 epilogues run side by side
            const uint64_t b0 = ho[m] + b, b1 = ho[m] + min((uint64_t)b + grab, nh);
            const uint32_t my_aip = b0 + lane < b1 ? a.hosts[b0 + lane] : 0u;
            uint32_t myA = 0;
            for (uint32_t j = 0; j < (uint32_t)(b1 - b0); j++) {
                const uint32_t aip = __shfl_sync(0xFFFFFFFFu, my_aip, j);
                const uint32_t A = __reduce_add_sync(0xFFFFFFFFu, gather_one<GK>(G, rc, c2k, bact0, k1, aip, lane, a));
                if (lane == j) myA = A;
            }
            if (b0 + lane < b1) {
                uint8_t f;
                a.out[b0 + lane] = estimate_eq11(G.g, G.P, N0, myA, f);
                if (a.flags) a.flags[b0 + lane] = f;
            }
        }
    }
    __syncthreads();
    if (tid == 0 && a.trace && total + blockIdx.x < a.trace_cap) {   // the block's gather: entry n_items + block
        unsigned long long *tr = a.trace + 4ull * (total + blockIdx.x);
        tr[0] = s_t0;
        tr[1] = s_t0;
        tr[2] = global_ns();
        tr[3] = ((unsigned long long)sm_id() << 32) | (0xFFFFFFull << 8) | 4u;
    }
    }   // s_ok

    // ---- the last block to finish closes the launch ----
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const unsigned int t = atomicAdd(&st->blocks_done, 1u);
        if (t == gridDim.x - 1u) {
            __threadfence();
            for (uint32_t m = 0; m < M; m++) {
                a.done[m] = 0u;
                a.qhost[m] = 0ull;
            }
            st->q_items = 0u;
            st->blocks_done = 0u;
            if (!*reinterpret_cast<volatile unsigned int *>(&st->poisoned)) {   // a timed-out step is not one
                st->step = step;
                st->started = 1u;
            }
            __threadfence();
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
    unsigned int *d_done = nullptr;  // M
    unsigned long long *d_qhost = nullptr;   // M: host counters of the gather
    uint64_t *d_hist = nullptr;      // M x maxbins
    uint32_t maxbins = 0;
    uint32_t L = 1;
    int gk = 1;                      // gather form (group_step_kernel<GK>)
    int sms = 148;
    int max_blocks_per_sm = 1;       // occupancy of group_step_kernel
    uint32_t steps = 0;              // steps queued so far (host count)
    vate_group_tuning tuning;
    unsigned long long spin_limit = DEFAULT_SPIN_LIMIT;
    uint32_t missing = 0;
    unsigned long long *trace = nullptr;   // vate_group_set_trace
    uint32_t trace_cap = 0;
    bool persist_l2 = false;         // holds the persisting limit (VATE_OPT_PERSIST_L2 in some monitor's options)
    int device = 0;
    // CUDA graph of one step
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint32_t graph_nodes = 0;
    uint64_t graph_key[16] = {};
};

namespace {

// dynamic shared memory of group_step_kernel: two uint64 offset arrays, then
// cum, kp, seg_start, seg_mp and wave_lo (uint32), then the census lane columns
size_t step_smem(uint32_t M, uint32_t maxbins) {
    const size_t words = 4 * (size_t)(M + 1) + (size_t)M * (NPHASE + 1) + M + 2 * (size_t)NPHASE * M + 1 + (M + 1);
    return words * 4 + (size_t)C_WARPS * ((maxbins + 1) / 2) * 32 * sizeof(uint32_t);
}

void *kernel_of(int gk) {
    switch (gk) {
    case 0: return (void *)group_step_kernel<0>;
    case 1: return (void *)group_step_kernel<1>;
    case 2: return (void *)group_step_kernel<2>;
    case 3: return (void *)group_step_kernel<3>;
    case 4: return (void *)group_step_kernel<4>;
    case 5: return (void *)group_step_kernel<5>;
    default: return (void *)group_step_kernel<6>;
    }
}

int gather_form(uint32_t L) {
    switch (L) {
    case 16: return 0;
    case 32: return 1;
    case 64: return 2;
    case 2: return 3;
    case 4: return 4;
    case 8: return 5;
    default: return 6;
    }
}

int check_tuning(const vate_group_tuning *t, int max_bps) {
    if (!t) return vate::set_error(VATE_EINVAL, "tuning is NULL");
    const uint32_t c = t->census_tile_chunks;
    if (c < 256 || c > 65536 || (c & (c - 1)))
        return vate::set_error(VATE_EINVAL, "census_tile_chunks: a power of two in [256, 65536]");
    if (t->blocks_per_sm < 1 || (int)t->blocks_per_sm > max_bps) {
        static thread_local char msg[96];
        snprintf(msg, sizeof msg, "blocks_per_sm must be in [1, %d] (the step kernel's occupancy)", max_bps);
        return vate::set_error(VATE_EINVAL, msg);
    }
    for (uint32_t v : {t->ingest_tile_pairs, t->preserve_tile_chunks})
        if (v < 256 || v > 65536 || v % 256)
            return vate::set_error(VATE_EINVAL, "ingest and preserve tiles: multiples of 256 in [256, 65536]");
    if (t->gather_grab_hosts < 1 || t->gather_grab_hosts > 32)
        return vate::set_error(VATE_EINVAL, "gather_grab_hosts must be in [1, 32]");
    if (t->wave_pool_mib > 65536) return vate::set_error(VATE_EINVAL, "wave_pool_mib must be in [0, 65536]");
    return VATE_OK;
}

cudaError_t enqueue_step(vate_group *g, const vate_pair *pairs, const uint64_t *poff, uint64_t pcap,
                         const uint32_t *hosts, const uint64_t *hoff, uint64_t hcap, const uint32_t *kprime,
                         float *out, uint8_t *flags, uint32_t advance, cudaStream_t st) {
    StepArgs a;
    a.descs = g->d_descs;
    a.st = g->d_state;
    a.done = g->d_done;
    a.pairs = reinterpret_cast<const uint32_t *>(pairs);
    a.poff = poff;
    a.pcap = pcap;
    a.hosts = hosts;
    a.hoff = hoff;
    a.hcap = hcap;
    a.kprimes = kprime;
    a.hist = g->d_hist;
    a.out = out;
    a.flags = flags;
    a.spin_limit = g->spin_limit;
    a.M = g->M;
    a.maxbins = g->maxbins;
    a.census_tile = g->tuning.census_tile_chunks;
    a.ingest_tile = g->tuning.ingest_tile_pairs;
    a.gather_grab = g->tuning.gather_grab_hosts;
    a.qhost = g->d_qhost;
    a.preserve_tile = g->tuning.preserve_tile_chunks;
    a.wave_bytes = (uint64_t)g->tuning.wave_pool_mib << 20;
    a.advance = advance;
    a.missing = g->missing;
    a.trace = g->trace;
    a.trace_cap = g->trace_cap;
    a.u1 = a.u2 = a.u3 = 1u;
    const size_t smem = step_smem(g->M, g->maxbins);
    const int grid = g->sms * (int)g->tuning.blocks_per_sm;
    switch (g->gk) {
    case 0: return vate::launch_pool(g->arena_geom, group_step_kernel<0>, grid, G_THREADS, smem, st, a);
    case 1: return vate::launch_pool(g->arena_geom, group_step_kernel<1>, grid, G_THREADS, smem, st, a);
    case 2: return vate::launch_pool(g->arena_geom, group_step_kernel<2>, grid, G_THREADS, smem, st, a);
    case 3: return vate::launch_pool(g->arena_geom, group_step_kernel<3>, grid, G_THREADS, smem, st, a);
    case 4: return vate::launch_pool(g->arena_geom, group_step_kernel<4>, grid, G_THREADS, smem, st, a);
    case 5: return vate::launch_pool(g->arena_geom, group_step_kernel<5>, grid, G_THREADS, smem, st, a);
    default: return vate::launch_pool(g->arena_geom, group_step_kernel<6>, grid, G_THREADS, smem, st, a);
    }
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
    bool want_persist = false;
    for (uint32_t m = 0; m < n_monitors; m++)
        if (params[m].options & VATE_OPT_PERSIST_L2) want_persist = true;
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
    g->gk = gather_form(g->L);
    g->arena_bytes = (off + 255) & ~255ull;
    g->sms = sm_count_current();
    const size_t smem = step_smem(g->M, g->maxbins);
    cudaError_t ea = cudaFuncSetAttribute(kernel_of(g->gk), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    if (ea == cudaSuccess) ea = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel_of(g->gk), G_THREADS, smem);
    if (ea != cudaSuccess || occ < 1) {
        cudaGetLastError();
        delete g;
        return vate::set_error(VATE_ECUDA, "group step kernel: shared-memory attribute or occupancy query failed");
    }
    g->max_blocks_per_sm = occ;
    g->tuning.census_tile_chunks = 16384;
    g->tuning.blocks_per_sm = (uint32_t)std::min(occ, 3);
    g->tuning.gather_grab_hosts = 8;
    g->tuning.ingest_tile_pairs = 16384;
    g->tuning.preserve_tile_chunks = 4096;
    g->tuning.wave_pool_mib = 0;
    bool ok = cudaMalloc(&g->arena, g->arena_bytes) == cudaSuccess &&
              cudaMalloc(&g->d_descs, n_monitors * sizeof(Geom)) == cudaSuccess &&
              cudaMalloc(&g->d_state, sizeof(GroupState)) == cudaSuccess &&
              cudaMalloc(&g->d_done, n_monitors * sizeof(unsigned int)) == cudaSuccess &&
              cudaMalloc(&g->d_qhost, n_monitors * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&g->d_hist, (size_t)n_monitors * g->maxbins * sizeof(uint64_t)) == cudaSuccess &&
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
    if (want_persist) {
        // the arena's window and the device's persisting limit only on request (VATE_OPT_PERSIST_L2 in any
        // monitor's options); the limit is held until the group is destroyed
        int persist_max = 0, window_max = 0;
        cudaGetDevice(&g->device);
        cudaDeviceGetAttribute(&persist_max, cudaDevAttrMaxPersistingL2CacheSize, g->device);
        cudaDeviceGetAttribute(&window_max, cudaDevAttrMaxAccessPolicyWindowSize, g->device);
        cudaGetLastError();
        g->persist_l2 = persist_max > 0 && window_max > 0 && vate::persist_acquire(g->device, (size_t)persist_max);
        if (g->persist_l2) {
            g->arena_geom.l2_window_bytes = std::min<uint64_t>(g->arena_bytes, (uint64_t)window_max);
            double ratio = (double)persist_max / (double)g->arena_geom.l2_window_bytes;
            g->arena_geom.l2_hit_ratio = ratio >= 1.0 ? 1.0f : (float)ratio;
        }
    }
    GroupState s0;
    memset(&s0, 0, sizeof s0);
    cudaError_t e = cudaMemcpyAsync(g->d_descs, g->geoms.data(), n_monitors * sizeof(Geom), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->d_state, &s0, sizeof s0, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_done, 0, n_monitors * sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_qhost, 0, n_monitors * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_hist, 0, (size_t)n_monitors * g->maxbins * sizeof(uint64_t), st);
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
    *out = g;
    return VATE_OK;
}

int vate_group_destroy(vate_group *g) {
    if (!g) return VATE_OK;
    cudaDeviceSynchronize();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->persist_l2) vate::persist_release(g->device);
    cudaFree(g->arena);
    cudaFree(g->d_descs);
    cudaFree(g->d_state);
    cudaFree(g->d_done);
    cudaFree(g->d_qhost);
    cudaFree(g->d_hist);
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
                                 d_kprime, d_out, d_flags, 1u, (cudaStream_t)stream);
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
    uint64_t key[16] = {(uint64_t)d_pairs, (uint64_t)d_pair_offsets, pair_capacity, (uint64_t)d_hosts,
                        (uint64_t)d_host_offsets, host_capacity, (uint64_t)d_kprime, (uint64_t)d_out,
                        (uint64_t)d_flags, ((uint64_t)t.census_tile_chunks << 32) | t.blocks_per_sm,
                        ((uint64_t)t.gather_grab_hosts << 32) | t.ingest_tile_pairs,
                        ((uint64_t)t.wave_pool_mib << 32) | t.preserve_tile_chunks,
                        g->spin_limit, g->missing, (uint64_t)g->trace, g->trace_cap};
    if (!g->exec || memcmp(key, g->graph_key, sizeof key) != 0) {
        if (g->exec) {
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t le = enqueue_step(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets,
                                          host_capacity, d_kprime, d_out, d_flags, 1u, g->cap_stream);
            e = cudaStreamEndCapture(g->cap_stream, &graph);
            if (e == cudaSuccess) e = le;
        }
        size_t nodes = 0;
        if (e == cudaSuccess) e = cudaGraphGetNodes(graph, nullptr, &nodes);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            g->exec = nullptr;
            return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
        }
        g->graph_nodes = (uint32_t)nodes;
        memcpy(g->graph_key, key, sizeof key);
    }
    cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    g->steps++;
    return VATE_OK;
}

int vate_group_graph_nodes(const vate_group *g, uint32_t *nodes) {
    if (!g || !nodes) return vate::set_error(VATE_EINVAL, "NULL argument");
    *nodes = g->exec ? g->graph_nodes : 0u;
    return VATE_OK;
}

int vate_group_set_trace(vate_group *g, uint64_t *d_trace, uint32_t capacity) {
    if (!g || (capacity && !d_trace)) return vate::set_error(VATE_EINVAL, "bad group or trace buffer");
    g->trace = capacity ? reinterpret_cast<unsigned long long *>(d_trace) : nullptr;
    g->trace_cap = capacity;
    return VATE_OK;
}

int vate_group_set_wait(vate_group *g, uint64_t spin_limit, uint32_t missing) {
    if (!g) return vate::set_error(VATE_EINVAL, "group is NULL");
    g->spin_limit = spin_limit;
    g->missing = missing;
    return VATE_OK;
}

int vate_group_set_tuning(vate_group *g, const vate_group_tuning *t) {
    if (!g) return vate::set_error(VATE_EINVAL, "group is NULL");
    if (int rc = check_tuning(t, g->max_blocks_per_sm)) return rc;
    g->tuning = *t;
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
    auto done = [&](int rc) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) g->tuning = entry;               // an error restores the tiling in force on entry
        return rc;
    };
    // the last step repeated: PreserveAT of the same slide changes nothing more,
    // SetAT of the same pairs writes the same values, the census and the gather
    // recompute the same outputs
    auto replay = [&]() {
        return enqueue_step(g, d_pairs, d_pair_offsets, pair_capacity, d_hosts, d_host_offsets, host_capacity,
                            d_kprime, d_out, d_flags, 0u, st);
    };
    vate_group_tuning best = g->tuning;
    float bt = 1e30f;
    // the candidates, each timed as the best of three replays
    std::vector<vate_group_tuning> cand;
    for (uint32_t bps = 2; bps <= (uint32_t)std::min(g->max_blocks_per_sm, 4); bps++)
        for (uint32_t wv : {0u, 32u})
            for (uint32_t ct : {4096u, 16384u})
                for (uint32_t gr : {2u, 4u, 8u})
                    for (uint32_t it : {4096u, 16384u, 65536u}) {
                        vate_group_tuning t = entry;
                        t.blocks_per_sm = bps;
                        t.wave_pool_mib = wv;
                        t.census_tile_chunks = ct;
                        t.gather_grab_hosts = gr;
                        t.ingest_tile_pairs = it;
                        cand.push_back(t);
                    }
    for (const vate_group_tuning &t : cand) {
        g->tuning = t;
        float ms_best = 1e30f;
        for (int r = 0; r < 3; r++) {
            cudaEventRecord(e0, st);
            cudaError_t e = replay();
            cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) return done(vate::set_error(VATE_ECUDA, cudaGetErrorString(e)));
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_best = std::min(ms_best, ms);
        }
        if (ms_best < bt) {
            bt = ms_best;
            best = t;
        }
    }
    g->tuning = best;
    cudaError_t e = replay();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return done(vate::set_error(VATE_ECUDA, cudaGetErrorString(e)));
    if (chosen) *chosen = best;
    return done(VATE_OK);
}

int vate_group_status(vate_group *g, uint32_t *status, int clear, void *stream) {
    if (!g || !status) return vate::set_error(VATE_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    GroupState s;
    cudaError_t e = cudaMemcpyAsync(&s, g->d_state, sizeof s, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && clear) {
        unsigned int z = s.status & VATE_GROUP_TIMEOUT;    // a timeout stays: the group is unusable
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
