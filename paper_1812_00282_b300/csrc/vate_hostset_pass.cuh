// vate_hostset_pass.cuh -- the close of a host list through its index: the
// index's constants, the pool's CheckAT bitmap and the pass over the index's
// tiles (vate_hostset.cu builds the index and launches these; the layout is
// described there).
#pragma once
#include "vate_device_ops.cuh"

namespace {

using namespace vate;

// A region's bitmap sits in shared memory (REGION_ATS / 8 bytes); the rest of the SM's 256 KB of L1 and shared
// memory stays L1, which holds the index loads in flight.  Measured at 2^20 hosts, 2^26 ATs, L = 1: see the
// benchmark notes beside the kernel.
#ifndef VATE_HS_REGION_KATS
#define VATE_HS_REGION_KATS 1536
#endif
constexpr uint32_t REGION_ATS = VATE_HS_REGION_KATS * 1024u;
constexpr uint32_t REGION_WORDS = REGION_ATS / 32u;
static_assert(REGION_WORDS % 4u == 0u && REGION_ATS % 8u == 0u, "a region holds whole quads of words and segments");
static_assert(REGION_ATS + 128u <= (1u << 21), "an entry holds a region's offset + 128 in 21 bits");
constexpr uint32_t BM_SKIP = 16u;                       // bytes of zeros before the bitmap in shared memory
constexpr uint32_t PER_UNIT = 6u;                       // 21-bit entries in a 16-byte unit
constexpr uint32_t NONE = 0xFFFFFFFFu;                  // the host of an empty lane
// rows of 32 units a warp has in flight
#ifndef VATE_HS_ROWS
#define VATE_HS_ROWS 8
#endif
constexpr int HB = VATE_HS_ROWS;
constexpr int HS_THREADS = 1024;                        // hs_tile_kernel: one block of 32 warps per SM
constexpr int BUILD_THREADS = 256;
constexpr uint32_t MAX_REGIONS = 1024;

// An index locates ATs in a shared-memory map of bpa bits per AT (1: the CheckAT bitmap; 4: the age map).
// The entry of pool offset o within its region is the first bit of its field in the map, past the map's 16
// leading bytes: bits 5-20 give the map word, bits 0-4 the field's first bit in it.
__host__ __device__ constexpr uint32_t entry_of(uint32_t o, uint32_t bpa) { return o * bpa + BM_SKIP * 8u; }
constexpr uint32_t AGE_REGION_ATS = REGION_WORDS * 8u;  // the age map of a region (4 bits per AT) fills the same words

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

// The active ATs of the segment whose entry is the low 21 bits of x (the
// bits above are the next entry's): bits 5-20 give its word of the
// shared-memory bitmap, bits 0-4 the bit of its first AT.
template <int L>
__device__ __forceinline__ uint32_t seg_count(const unsigned char *bmb, uint32_t x) {
    const uint32_t w = __funnelshift_r(*reinterpret_cast<const uint32_t *>(bmb + ((x >> 3) & 0x3FFFCu)), 0u, x);
    if (L == 1) return w & 1u;
    return __popc(w & ((1u << L) - 1u));
}

// The six entries of a unit: entry s starts at bit 21 s of its 128 bits.
template <int L>
__device__ __forceinline__ uint32_t unit_count(const unsigned char *bmb, uint4 v) {
    return seg_count<L>(bmb, v.x) + seg_count<L>(bmb, __funnelshift_r(v.x, v.y, 21)) + seg_count<L>(bmb, v.y >> 10) +
           seg_count<L>(bmb, __funnelshift_r(v.y, v.z, 31)) + seg_count<L>(bmb, __funnelshift_r(v.z, v.w, 20)) +
           seg_count<L>(bmb, v.w >> 9);
}

// The first tile t in [lo, hi] whose first row is at or past x (row0
// ascending; hi when none below it is): a 32-way search, each lane probing
// one point per round.  Called by all 32 lanes.
__device__ __forceinline__ uint32_t tile_at_row(const uint32_t *__restrict__ row0, uint32_t lo, uint32_t hi, uint32_t x,
                                                uint32_t lane) {
    while (hi - lo > 31u) {                              // the answer lies in [lo, hi]
        const uint32_t step = (hi - lo + 31u) >> 5;
        const uint32_t p = lo + lane * step;
        const bool past = p >= hi || __ldcg(row0 + p) >= x;
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, past);
        if (m & 1u) return lo;
        if (m == 0u) {
            lo += 31u * step;
        } else {
            const uint32_t f = __ffs(m) - 1u;
            hi = min(hi, lo + f * step);
            lo += (f - 1u) * step;
        }
    }
    const uint32_t p = lo + lane;
    const bool past = p >= hi || __ldcg(row0 + p) >= x;
    return lo + (uint32_t)__ffs(__ballot_sync(0xFFFFFFFFu, past)) - 1u;
}

// The block's share of the rows (whole tiles), region by region: the region's
// bitmap into shared memory, then each warp an equal share of the region's
// rows (whole tiles), HB rows of 32 units in flight, lane j summing column j.
// A tile's rows end at the same row for every lane, where each lane adds its
// sum to its cell's host; the next tile's first row and hosts are loaded one
// tile ahead.
template <int L>
__global__ void __launch_bounds__(HS_THREADS, 1) hs_tile_kernel(const uint32_t *__restrict__ bitmap, uint64_t bm_words,
                                                                uint32_t nr, const uint32_t *__restrict__ rt,
                                                                const uint32_t *__restrict__ row0,
                                                                const uint32_t *__restrict__ hosts,
                                                                const uint4 *__restrict__ ent4, uint32_t T, uint32_t R,
                                                                uint32_t *__restrict__ active) {
    extern __shared__ uint4 bm4[];                       // a zero quad, then REGION_WORDS words of bitmap
    uint32_t *bm = reinterpret_cast<uint32_t *>(bm4 + 1);
    const unsigned char *bmb = reinterpret_cast<const unsigned char *>(bm4);
    __shared__ uint32_t s_t[2];
    __shared__ uint32_t s_r;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nw = blockDim.x >> 5;
    if (tid == 0) bm4[0] = make_uint4(0u, 0u, 0u, 0u);
    if (warp < 2) {
        const uint32_t x = (uint32_t)((uint64_t)R * (blockIdx.x + warp) / gridDim.x);
        const uint32_t t = tile_at_row(row0, 0u, T, x, lane);
        if (lane == 0) s_t[warp] = t;
    }
    __syncthreads();
    const uint32_t ta = s_t[0], tb = s_t[1];
    for (uint32_t t0 = ta; t0 < tb;) {
        if (tid == 0) {                                  // the region holding tile t0
            uint32_t lo = 0, hi = nr;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (rt[mid] <= t0) lo = mid;
                else hi = mid;
            }
            s_r = lo;
        }
        __syncthreads();                                 // also: the previous region's lookups are done
        const uint32_t r = s_r;
        const uint32_t t1 = min(tb, rt[r + 1]);
        const uint64_t w0 = (uint64_t)r * REGION_WORDS, left = bm_words - w0;
        const uint32_t nwords = left < (uint64_t)REGION_WORDS ? (uint32_t)left : REGION_WORDS;
        const uint4 *src = reinterpret_cast<const uint4 *>(bitmap + w0);   // w0 is a multiple of 4 words
        for (uint32_t i = tid; i < nwords / 4u; i += blockDim.x) bm4[1 + i] = __ldcg(src + i);
        for (uint32_t i = (nwords & ~3u) + tid; i < nwords; i += blockDim.x) bm[i] = __ldcg(bitmap + w0 + i);
        __syncthreads();
        const uint32_t xa = __ldcg(row0 + t0), xb = __ldcg(row0 + t1);
        const uint32_t wa = tile_at_row(row0, t0, t1, xa + (uint32_t)((uint64_t)(xb - xa) * warp / nw), lane);
        const uint32_t wb = tile_at_row(row0, t0, t1, xa + (uint32_t)((uint64_t)(xb - xa) * (warp + 1u) / nw), lane);
        if (wa < wb) {
            const uint32_t rowA = __ldcg(row0 + wa), rowB = __ldcg(row0 + wb);
            uint32_t t = wa;
            uint32_t end = __ldcg(row0 + t + 1u);         // first row past tile t
            uint32_t host = __ldcg(hosts + (uint64_t)t * 32u + lane);
            const bool more = t + 1u < wb;
            uint32_t end2 = more ? __ldcg(row0 + t + 2u) : rowB;
            uint32_t host2 = more ? __ldcg(hosts + (uint64_t)(t + 1u) * 32u + lane) : NONE;
            uint32_t sum = 0;
            for (uint32_t row = rowA; row < rowB; row += HB) {
                const uint4 *rp = ent4 + (uint64_t)row * 32u + lane;
                uint4 v[HB];
#pragma unroll
                for (int u = 0; u < HB; u++)
                    v[u] = row + u < rowB ? __ldcs(rp + 32u * u) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int u = 0; u < HB; u++) {
                    if (row + u >= rowB) break;
                    if (row + u == end) {                // tile t ends here, for every lane
                        if (host != NONE && sum) atomicAdd(active + host, sum);
                        sum = 0;
                        t++;
                        end = end2;
                        host = host2;
                        if (t + 1u < wb) {
                            end2 = __ldcg(row0 + t + 2u);
                            host2 = __ldcg(hosts + (uint64_t)(t + 1u) * 32u + lane);
                        } else {
                            end2 = rowB;
                            host2 = NONE;
                        }
                    }
                    sum += unit_count<L>(bmb, v[u]);
                }
            }
            if (host != NONE && sum) atomicAdd(active + host, sum);
        }
        t0 = t1;
    }
}

}  // namespace
