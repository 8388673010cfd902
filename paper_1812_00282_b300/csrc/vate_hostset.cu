// vate_hostset.cu -- the close of a fixed host list through an index of its
// VAT positions (include/vate_hostset.h).
//
// Index.  The pool is cut into regions of REGION_ATS positions (a multiple of
// every segment length, so no segment straddles two).  For region r and host
// h of the list, the entries of cell (r, h) locate, in the region's bitmap,
// the first AT of each of h's segments that lie in r (one entry per segment,
// so a segment met twice by one host counts twice, as in the gather): the
// byte offset of its 32-bit word shifted left by 5, plus its bit (the form
// the lookup uses as it is).  A cell opens with a header HDR | h and is
// padded with PAD to a multiple of four entries, so that every cell starts on
// a 16-byte boundary.  Cells are stored region-major, host-minor;
// off[r][h] is the first entry of cell (r, h) relative to the region's first
// entry rbase[r], and off[r][n] the region's total.  Built in two passes over
// the hosts' segments (count per cell, then place), with an exclusive scan of
// the counts between them.
//
// Close (per call).  hs_bitmap_kernel writes the pool's CheckAT bitmap for k'
// (bit p set when AT p is active: the SWAR range test of CheckAT in the frame
// of block 0, as in the gather).  hs_active_kernel runs one block per SM;
// block b takes an equal share of the cells, in order, so it meets one or two
// regions; for each it loads the region's bitmap into shared memory and its
// warps run through the cells, four at a time (eight lanes each), streaming
// each cell's entries as 16-byte loads and summing the popcounts of the
// segments' bits; a cell's sum is added to its host's count.  Eq. 11 then
// comes from the counts and the census (the kernel of vate_estimate_from_counts).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vate.h"
#include "vate_hostset.h"
#include "vate_internal.h"
#include "vate_device_ops.cuh"
#include "vate_launch.cuh"

using namespace vate;

namespace {

constexpr uint32_t REGION_ATS = 1536u * 1024u;         // one region's bitmap: 192 KiB of shared memory
constexpr uint32_t REGION_WORDS = REGION_ATS / 32u;
constexpr uint32_t PAD = REGION_WORDS << 7;             // the entry of a zero word kept past the region's bitmap
constexpr uint32_t HDR = 0x80000000u;                   // a cell's first entry: HDR | host index
// slabs of 32 quads a warp loads before it counts them; measured at 2^20 hosts, 2^26 ATs: 2 slabs 5.04 /
// 2.70 ms (L = 1 / 2), 4 slabs 4.40 / 2.42 ms, 8 slabs 4.22 / 2.32 ms
#ifndef VATE_HS_SLABS
#define VATE_HS_SLABS 8
#endif
constexpr int HB = VATE_HS_SLABS;                       // slabs of 32 quads a warp has in flight
constexpr int HS_THREADS = 1024;                        // hs_active_kernel: one block of 32 warps per SM
constexpr int BUILD_THREADS = 256;
constexpr uint32_t MAX_REGIONS = 1024;

// Thread per 32 ATs: bit (p mod 32) of word p / 32 is set when AT p is active.
__global__ void __launch_bounds__(256) hs_bitmap_kernel(Geom G, RangeConsts rc, uint32_t c2k, uint64_t words,
                                                        uint32_t *__restrict__ bitmap) {
    const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        const uint4 a = __ldcg(pool16 + 2 * w), b = __ldcg(pool16 + 2 * w + 1);
        VATE_CHECK_WORD(G, a.x, 2 * w);
        VATE_CHECK_WORD(G, b.w, 2 * w + 1);
        const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        uint32_t out = 0;
#pragma unroll
        for (int i = 0; i < 8; i++) {
            // bit 7 of byte j of the word -> bit j of a nibble: the four flags sit at bits 0, 8, 16, 24, and
            // the multiply by 2^28 + 2^21 + 2^14 + 2^7 moves flag j to bit 28 + j; the other products land
            // on distinct bits below 28 or past bit 31, so nothing carries into the nibble
            const uint32_t f = (swar_active(v[i], rc, c2k) >> 7) & 0x01010101u;
            out |= ((f * 0x10204080u) >> 28) << (4 * i);
        }
        bitmap[w] = out;
    }
}

// Warp per host: the size of its cell in each region -- a header and one
// entry per segment, rounded up to a multiple of four; 0 where the host has no
// segment.
__global__ void __launch_bounds__(BUILD_THREADS) hs_count_kernel(Geom G, const uint32_t *__restrict__ aips, uint64_t n,
                                                                 uint32_t nr, uint32_t *__restrict__ off) {
    extern __shared__ uint32_t wh_all[];                 // [warps][nr]
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *wh = wh_all + (size_t)warp * nr;
    const uint32_t nseg = G.g >> G.log2L;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n; h += nwarps) {
        for (uint32_t r = lane; r < nr; r += 32u) wh[r] = 0u;
        __syncwarp();
        const uint64_t hk = host_key(G, aips[h]);
        for (uint32_t j = lane; j < nseg; j += 32u) atomicAdd(&wh[seg_base_k(G, hk, j) / REGION_ATS], 1u);
        __syncwarp();
        for (uint32_t r = lane; r < nr; r += 32u)
            off[(uint64_t)r * (n + 1) + h] = wh[r] ? (wh[r] + 1u + 3u) & ~3u : 0u;
        __syncwarp();
    }
}

// Block per region: off[r][0..n) from cell sizes to exclusive offsets,
// off[r][n] and total[r] the region's entries (in 64 bits, to catch overflow).
__global__ void __launch_bounds__(1024) hs_scan_kernel(uint32_t *__restrict__ off, uint64_t n,
                                                       unsigned long long *__restrict__ total) {
    __shared__ unsigned long long part[1024];
    uint32_t *row = off + (uint64_t)blockIdx.x * (n + 1);
    const uint32_t t = threadIdx.x;
    const uint64_t per = (n + blockDim.x - 1) / blockDim.x;
    const uint64_t i0 = min(n, (uint64_t)t * per), i1 = min(n, i0 + per);
    unsigned long long s = 0;
    for (uint64_t i = i0; i < i1; i++) s += row[i];
    part[t] = s;
    __syncthreads();
    for (uint32_t d = 1; d < blockDim.x; d <<= 1) {
        const unsigned long long v = t >= d ? part[t - d] : 0ull;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    unsigned long long run = part[t] - s;
    for (uint64_t i = i0; i < i1; i++) {
        const uint32_t c = row[i];
        row[i] = (uint32_t)run;
        run += c;
    }
    if (t == blockDim.x - 1) {
        row[n] = (uint32_t)part[t];
        total[blockIdx.x] = part[t];
    }
}

// Warp per host: in each region where it has segments, its cell -- the
// header HDR | h, then each segment's entry (its word's byte offset << 5 | its bit), then PAD up
// to the cell's size.
__global__ void __launch_bounds__(BUILD_THREADS) hs_fill_kernel(Geom G, const uint32_t *__restrict__ aips, uint64_t n,
                                                                uint32_t nr, const uint32_t *__restrict__ off,
                                                                const unsigned long long *__restrict__ rbase,
                                                                uint32_t *__restrict__ entries) {
    extern __shared__ uint32_t wh_all[];                 // [warps][nr]: entries placed so far per region
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *wh = wh_all + (size_t)warp * nr;
    const uint32_t nseg = G.g >> G.log2L;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n; h += nwarps) {
        for (uint32_t r = lane; r < nr; r += 32u) wh[r] = 0u;
        __syncwarp();
        const uint64_t hk = host_key(G, aips[h]);
        for (uint32_t j = lane; j < nseg; j += 32u) {
            const uint32_t pos = seg_base_k(G, hk, j);
            const uint32_t r = pos / REGION_ATS;
            const uint32_t k = atomicAdd(&wh[r], 1u);
            const uint32_t o = pos - r * REGION_ATS;                 // the AT's bit in the region's bitmap
            entries[rbase[r] + off[(uint64_t)r * (n + 1) + h] + 1u + k] = ((o & ~31u) << 2) | (o & 31u);
        }
        __syncwarp();
        for (uint32_t r = lane; r < nr; r += 32u) {
            if (!wh[r]) continue;
            const uint64_t cell = rbase[r] + off[(uint64_t)r * (n + 1) + h];
            entries[cell] = HDR | (uint32_t)h;
            for (uint32_t k = 1u + wh[r]; k & 3u; k++) entries[cell + k] = PAD;
        }
        __syncwarp();
    }
}

// The active ATs of the segment of entry e: e >> 5 is the byte offset of its
// word in the region's bitmap, e mod 32 the bit of its first AT.
template <int L>
__device__ __forceinline__ uint32_t seg_count(const unsigned char *bmb, uint32_t e) {
    const uint32_t w = __funnelshift_r(*reinterpret_cast<const uint32_t *>(bmb + (e >> 5)), 0u, e);
    if (L == 1) return w & 1u;
    return __popc(w & ((1u << L) - 1u));
}

// The first quad at or after x (below limit) that starts a cell, else limit.
__device__ __forceinline__ uint64_t next_cell(const uint32_t *__restrict__ ent, uint64_t x, uint64_t limit,
                                              uint32_t lane) {
    for (uint64_t q = x; q < limit; q += 32u) {
        const uint64_t qq = q + lane;
        const bool head = qq < limit && (__ldcg(ent + 4 * qq) & HDR) != 0u;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, head);
        if (m) return q + (uint64_t)(__ffs(m) - 1);
    }
    return limit;
}

// The block's share of the index (whole cells), region by region: the
// region's bitmap into shared memory, then each warp a run of whole cells,
// read as slabs of 32 quads (one per lane, HB slabs in flight).  A cell
// starts a quad, so a quad holds at most one header, in its first entry; a
// lane's quad adds to the cell of the nearest header at or before it, found
// with a prefix sum over the slab and the ballot of its headers; a cell that
// runs past the slab carries into the next.
template <int L>
__global__ void __launch_bounds__(HS_THREADS, 1) hs_active_kernel(const uint32_t *__restrict__ bitmap, uint64_t bm_words,
                                                                  uint32_t nr,
                                                                  const unsigned long long *__restrict__ rbase,
                                                                  const uint4 *__restrict__ ent4, uint64_t quads,
                                                                  uint32_t *__restrict__ active) {
    extern __shared__ uint4 bm4[];                       // REGION_WORDS words of bitmap, then one zero word (PAD)
    uint32_t *bm = reinterpret_cast<uint32_t *>(bm4);
    const unsigned char *bmb = reinterpret_cast<const unsigned char *>(bm4);
    const uint32_t *ent = reinterpret_cast<const uint32_t *>(ent4);
    __shared__ unsigned long long s_b[2];
    __shared__ uint32_t s_r;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nw = blockDim.x >> 5;
    if (tid == 0) bm[REGION_WORDS] = 0u;
    if (warp < 2) {
        const uint64_t a = quads * (blockIdx.x + warp) / gridDim.x;
        const uint64_t b = next_cell(ent, a, quads, lane);
        if (lane == 0) s_b[warp] = b;
    }
    __syncthreads();
    const uint64_t b0 = s_b[0], b1 = s_b[1];
    for (uint64_t p = b0; p < b1;) {
        if (tid == 0) {                                  // the region holding quad p
            uint32_t lo = 0, hi = nr;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((rbase[mid] >> 2) <= p) lo = mid;
                else hi = mid;
            }
            s_r = lo;
        }
        __syncthreads();                                 // also: the previous region's lookups are done
        const uint32_t r = s_r;
        const uint64_t pe = min(b1, (uint64_t)(rbase[r + 1] >> 2));
        const uint64_t w0 = (uint64_t)r * REGION_WORDS, left = bm_words - w0;
        const uint32_t nwords = left < (uint64_t)REGION_WORDS ? (uint32_t)left : REGION_WORDS;
        const uint4 *src = reinterpret_cast<const uint4 *>(bitmap + w0);   // w0 is a multiple of 4 words
        for (uint32_t i = tid; i < nwords / 4u; i += blockDim.x) bm4[i] = __ldcg(src + i);
        for (uint32_t i = (nwords & ~3u) + tid; i < nwords; i += blockDim.x) bm[i] = __ldcg(bitmap + w0 + i);
        __syncthreads();
        const uint64_t len = pe - p;
        const uint64_t ws = next_cell(ent, p + len * warp / nw, pe, lane);
        const uint64_t we = next_cell(ent, p + len * (warp + 1) / nw, pe, lane);
        uint32_t carry_h = 0u, carry_s = 0u;             // the cell open at the end of the last slab
        const uint32_t nq = (uint32_t)(we - ws);          // quads of the warp's run (a region holds < 2^30)
        const uint4 *wp = ent4 + ws;
        for (uint32_t b0 = 0; b0 < nq; b0 += 32u * HB) {
            uint4 v[HB];
#pragma unroll
            for (int u = 0; u < HB; u++) {
                const uint32_t i = b0 + 32u * u + lane;
                v[u] = i < nq ? __ldcs(wp + i) : make_uint4(PAD, PAD, PAD, PAD);
            }
#pragma unroll
            for (int u = 0; u < HB; u++) {
                const bool head = (v[u].x & HDR) != 0u;
                // a header is looked up as PAD (the zero word past the bitmap), never as an address
                const uint32_t x = head ? PAD : v[u].x;
                const uint32_t val = seg_count<L>(bmb, x) + seg_count<L>(bmb, v[u].y) + seg_count<L>(bmb, v[u].z) +
                                     seg_count<L>(bmb, v[u].w);
                const uint32_t heads = __ballot_sync(0xFFFFFFFFu, head);
                if (heads == 0u) {                       // the open cell runs through the slab
                    carry_s += __reduce_add_sync(0xFFFFFFFFu, val);
                    continue;
                }
                // the open cell ends before the first header: its part in this slab is the sum below it
                const uint32_t first = __ffs(heads) - 1u;
                const uint32_t head_sum = __reduce_add_sync(0xFFFFFFFFu, lane < first ? val : 0u);
                if (lane == 0 && carry_s + head_sum) atomicAdd(active + carry_h, carry_s + head_sum);
                if ((heads & (heads - 1u)) == 0u) {      // one header: the cell it starts stays open
                    carry_h = __shfl_sync(0xFFFFFFFFu, v[u].x & ~HDR, first);
                    carry_s = __reduce_add_sync(0xFFFFFFFFu, lane >= first ? val : 0u);
                    continue;
                }
                // several headers: the cells between them close here, the last one stays open
                uint32_t P = val;                        // inclusive prefix sum over the slab
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, P, d);
                    if (lane >= (uint32_t)d) P += y;
                }
                const uint32_t upto = heads & (0xFFFFFFFFu >> (31u - lane));   // headers at or below this lane
                const uint32_t hl = upto ? 31u - __clz(upto) : 0u;             // the lane of the nearest one
                const uint32_t before = __shfl_sync(0xFFFFFFFFu, P, (hl + 31u) & 31u);
                const uint32_t host = __shfl_sync(0xFFFFFFFFu, v[u].x & ~HDR, hl);
                const uint32_t sum = hl ? P - before : P;
                // lanes from the first header on: a cell that ends here (the next lane starts one) adds its sum
                if (upto && lane < 31u && ((heads >> (lane + 1u)) & 1u) && sum) atomicAdd(active + host, sum);
                carry_h = __shfl_sync(0xFFFFFFFFu, host, 31);
                carry_s = __shfl_sync(0xFFFFFFFFu, sum, 31);
            }
        }
        if (lane == 0 && ws < we && carry_s) atomicAdd(active + carry_h, carry_s);
        p = pe;
    }
}

int sm_count_now() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

}  // namespace

struct vate_hostset {
    const vate_handle *owner = nullptr;
    int device = 0;
    int sms = 148;
    uint64_t n = 0;
    uint32_t nr = 0;
    uint32_t L = 1;
    uint64_t entries = 0;                  // index entries (with padding)
    uint64_t bm_words = 0;
    uint32_t *d_entries = nullptr;
    unsigned long long *d_rbase = nullptr; // [nr + 1]
    uint32_t *d_bitmap = nullptr;
    uint32_t *d_active = nullptr;          // [n]
    float *d_out = nullptr;                // [n], vate_estimate_hostset_host (on first use)
    uint8_t *d_flags = nullptr;            // [n]
    uint64_t bytes = 0;
};

namespace {

void free_hostset(vate_hostset *s) {
    if (!s) return;
    cudaFree(s->d_entries);
    cudaFree(s->d_rbase);
    cudaFree(s->d_bitmap);
    cudaFree(s->d_active);
    cudaFree(s->d_out);
    cudaFree(s->d_flags);
    cudaGetLastError();
    delete s;
}

void *kernel_for(uint32_t L) {
    switch (L) {
    case 1: return (void *)hs_active_kernel<1>;
    case 2: return (void *)hs_active_kernel<2>;
    case 4: return (void *)hs_active_kernel<4>;
    default: return (void *)hs_active_kernel<8>;
    }
}

constexpr size_t ACTIVE_SMEM = (size_t)REGION_WORDS * 4 + 16;

}  // namespace

extern "C" {

int vate_hostset_create(vate_handle *h, const uint32_t *d_aips, uint64_t n, void *stream, vate_hostset **out) {
    if (!out) return set_error(VATE_EINVAL, "out must not be NULL");
    *out = nullptr;
    HandleView v;
    if (int rc = handle_view(h, &v)) return rc;
    const Geom &G = v.G;
    if (n == 0 || !d_aips) return set_error(VATE_EINVAL, "a hostset needs at least one host (d_aips not NULL)");
    if (n >= HDR) return set_error(VATE_EINVAL, "at most 2^31 - 1 hosts");
    if (G.atw != 1u || G.packed || (G.counter == VATE_COUNTER_AT && !G.frame0))
        return set_error(VATE_EINVAL, "a hostset needs a pool of byte ATs (k <= 63)");
    if (G.lo != 0 || G.hi != G.P) return set_error(VATE_EINVAL, "a hostset needs the whole pool, not a shard");
    if (G.L != 1 && G.L != 2 && G.L != 4 && G.L != 8) return set_error(VATE_EINVAL, "a hostset needs seg_len 1, 2, 4 or 8");
    const uint32_t nr = (uint32_t)((G.P + REGION_ATS - 1) / REGION_ATS);
    if (nr > MAX_REGIONS) return set_error(VATE_EINVAL, "pool too large for a hostset (more than 1024 regions)");
    cudaStream_t st = (cudaStream_t)stream;
    vate_hostset *s = new (std::nothrow) vate_hostset();
    if (!s) return set_error(VATE_ENOMEM, "host allocation failed");
    s->owner = h;
    cudaGetDevice(&s->device);
    s->sms = sm_count_now();
    s->n = n;
    s->nr = nr;
    s->L = G.L;
    s->bm_words = G.P / 32u;
    const size_t off_words = (size_t)nr * (n + 1);
    unsigned long long *d_total = nullptr;
    uint32_t *d_off = nullptr;             // [nr][n + 1]: cell offsets within each region (build only)
    bool ok = cudaMalloc(&d_off, off_words * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&s->d_rbase, (nr + 1) * sizeof(unsigned long long)) == cudaSuccess &&
              cudaMalloc(&s->d_bitmap, s->bm_words * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&s->d_active, n * sizeof(uint32_t)) == cudaSuccess &&
              cudaMalloc(&d_total, nr * sizeof(unsigned long long)) == cudaSuccess;
    if (!ok) {
        cudaFree(d_total);
        cudaFree(d_off);
        free_hostset(s);
        return set_error(VATE_ENOMEM, "out of device memory for the hostset's offsets");
    }
    auto fail_cuda = [&](cudaError_t e) {
        cudaFree(d_total);
        cudaFree(d_off);
        free_hostset(s);
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    };
    const size_t build_smem = (size_t)(BUILD_THREADS / 32) * nr * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(hs_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hs_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem);
    if (e != cudaSuccess) return fail_cuda(e);
    const int grid = (int)std::min<uint64_t>((n + BUILD_THREADS / 32 - 1) / (BUILD_THREADS / 32), (uint64_t)s->sms * 16);
    hs_count_kernel<<<grid, BUILD_THREADS, build_smem, st>>>(G, d_aips, n, nr, d_off);
    count_launch();
    hs_scan_kernel<<<nr, 1024, 0, st>>>(d_off, n, d_total);
    count_launch();
    std::vector<unsigned long long> total(nr), rbase(nr + 1);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(total.data(), d_total, nr * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_cuda(e);
    rbase[0] = 0;
    for (uint32_t r = 0; r < nr; r++) {
        if (total[r] >= 0xFFFFFFFFull) {
            cudaFree(d_total);
            cudaFree(d_off);
            free_hostset(s);
            return set_error(VATE_EINVAL, "too many hosts for a hostset: a region would hold 2^32 or more entries");
        }
        rbase[r + 1] = rbase[r] + total[r];
    }
    s->entries = rbase[nr];
    if (cudaMalloc(&s->d_entries, std::max<uint64_t>(s->entries, 4) * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(d_total);
        cudaFree(d_off);
        free_hostset(s);
        return set_error(VATE_ENOMEM, "out of device memory for the hostset's index");
    }
    if ((e = cudaMemcpyAsync(s->d_rbase, rbase.data(), (nr + 1) * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                             st)) != cudaSuccess)
        return fail_cuda(e);
    hs_fill_kernel<<<grid, BUILD_THREADS, build_smem, st>>>(G, d_aips, n, nr, d_off, s->d_rbase, s->d_entries);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return fail_cuda(e);
    cudaFree(d_total);
    cudaFree(d_off);
    if ((e = cudaFuncSetAttribute(kernel_for(s->L), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ACTIVE_SMEM)) !=
        cudaSuccess) {
        free_hostset(s);
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    }
    s->bytes = std::max<uint64_t>(s->entries, 4) * 4 + (nr + 1) * 8 + s->bm_words * 4 + n * 4;
    *out = s;
    return VATE_OK;
}

int vate_hostset_destroy(vate_hostset *s) {
    if (!s) return VATE_OK;
    cudaDeviceSynchronize();
    free_hostset(s);
    return VATE_OK;
}

int vate_hostset_info(const vate_hostset *s, uint64_t *bytes, uint64_t *n_hosts, uint32_t *regions) {
    if (!s) return set_error(VATE_EINVAL, "hostset is NULL");
    if (bytes) *bytes = s->bytes;
    if (n_hosts) *n_hosts = s->n;
    if (regions) *regions = s->nr;
    return VATE_OK;
}

int vate_estimate_hostset(vate_handle *h, vate_hostset *s, uint32_t kprime, float *d_out, uint8_t *d_flags,
                          uint32_t *d_active, void *stream) {
    HandleView v;
    if (int rc = handle_view(h, &v)) return rc;
    if (!s || s->owner != h) return set_error(VATE_EINVAL, "the hostset was not built for this handle");
    if (!d_out) return set_error(VATE_EINVAL, "d_out must not be NULL");
    if (!v.closed) return set_error(VATE_ESLICE, "the current slice has not been closed");
    const Geom &G = v.G;
    if (kprime < 1 || kprime > G.k) return set_error(VATE_EINVAL, "kprime must be in [1, k]");
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *acc = d_active ? d_active : s->d_active;
    cudaError_t e = cudaMemsetAsync(acc, 0, s->n * sizeof(uint32_t), st);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    const RangeConsts rc = G.counter == 1u ? dr_range_consts(kprime) : range_consts(v.bact0, kprime, G.twok);
    const uint32_t c2k = (128u - G.twok) * ONES;
    const int bgrid = (int)std::min<uint64_t>((s->bm_words + 255) / 256, (uint64_t)v.sms * 16);
    e = launch_pool(G, hs_bitmap_kernel, bgrid, 256, 0, st, G, rc, c2k, s->bm_words, s->d_bitmap);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    const uint4 *ent4 = reinterpret_cast<const uint4 *>(s->d_entries);
    const uint64_t quads = s->entries / 4;
    switch (s->L) {
    case 1: hs_active_kernel<1><<<v.sms, HS_THREADS, ACTIVE_SMEM, st>>>(s->d_bitmap, s->bm_words, s->nr, s->d_rbase, ent4, quads, acc); break;
    case 2: hs_active_kernel<2><<<v.sms, HS_THREADS, ACTIVE_SMEM, st>>>(s->d_bitmap, s->bm_words, s->nr, s->d_rbase, ent4, quads, acc); break;
    case 4: hs_active_kernel<4><<<v.sms, HS_THREADS, ACTIVE_SMEM, st>>>(s->d_bitmap, s->bm_words, s->nr, s->d_rbase, ent4, quads, acc); break;
    default: hs_active_kernel<8><<<v.sms, HS_THREADS, ACTIVE_SMEM, st>>>(s->d_bitmap, s->bm_words, s->nr, s->d_rbase, ent4, quads, acc); break;
    }
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    e = launch_estimate_from_counts(G, kprime, v.hist, acc, s->n, d_out, d_flags, st, v.sms);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

int vate_estimate_hostset_host(vate_handle *h, vate_hostset *s, uint32_t kprime, float *h_out, uint8_t *h_flags,
                               void *stream) {
    if (!s || !h_out) return set_error(VATE_EINVAL, "hostset and h_out must not be NULL");
    if (!s->d_out) {
        if (cudaMalloc(&s->d_out, s->n * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&s->d_flags, s->n) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(s->d_out);
            s->d_out = nullptr;
            return set_error(VATE_ENOMEM, "out of device memory for the hostset's result buffers");
        }
        s->bytes += s->n * 5;
    }
    if (int rc = vate_estimate_hostset(h, s, kprime, s->d_out, s->d_flags, nullptr, stream)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h_out, s->d_out, s->n * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && h_flags) e = cudaMemcpyAsync(h_flags, s->d_flags, s->n, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

}  // extern "C"
