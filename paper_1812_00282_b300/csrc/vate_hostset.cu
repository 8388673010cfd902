// vate_hostset.cu -- the close of a fixed host list through an index of its
// VAT positions (include/vate_hostset.h).
//
// Index.  The pool is cut into regions of REGION_ATS positions (a multiple of
// every segment length, so no segment straddles two).  Cell (r, h) holds one
// 21-bit entry per segment of host h that lies in region r (a segment met
// twice by one host counts twice, as in the gather): the first bit of its
// first AT's field in the block's shared-memory copy of the region's map
// (the offset in the region plus 128 for the bitmap; 4 times the offset plus
// 128 for an age map), which starts with a quad that reads as nothing (zero
// bits; ages 15) -- so the entry 0 pads.  Six entries fill a 16-byte
// unit (bits 21 s .. 21 s + 20 of its 128 bits for entry s; the top two bits
// are 0).  The cells of a region are sorted by their number of units,
// largest first, and dealt in that order to tiles of 32 cells.  Tile t holds
// M_t rows of 32 units; row i holds unit i of each of the tile's cells, lane j
// reading cell j's column; M_t is the units of its first, largest, cell and
// the rest of every column is 0.  Tiles are stored region-major: rt[r] is the
// first tile of region r, row0[t] the first row of tile t (row0[T] the number
// of rows), host[32 t + j] the host of cell j of tile t, NONE for an empty
// lane of a region's last tile.  Built in passes over the hosts' segments:
// count per cell, a histogram of cell sizes per region and its scan, the
// placement of every cell in its region's order, a scan of the tiles' rows,
// then the entries.
//
// Close (per call).  hs_bitmap_kernel writes the pool's CheckAT bitmap for k'
// (bit p set when AT p is active: the SWAR range test of CheckAT in the frame
// of block 0, as in the gather).  hs_tile_kernel runs one block per SM; block
// b takes an equal share of the rows (whole tiles, in order), so it meets one
// or two regions; for each it loads the region's bitmap into shared memory,
// and each warp streams an equal share of the region's rows: lane j sums the
// bits its column's entries point at, and at the end of a tile -- the same row
// for every lane -- adds the sum to its cell's host.  Eq. 11 then comes from
// the counts and the census (the kernel of vate_estimate_from_counts).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "vate.h"
#include "vate_hostset.h"
#include "vate_internal.h"
#include "vate_device_ops.cuh"
#include "vate_launch.cuh"
#include "vate_hostset_pass.cuh"

using namespace vate;

namespace {

// Warp per host: cnt[r][h] = the host's segments in region r.
__global__ void __launch_bounds__(BUILD_THREADS) hs_count_kernel(Geom G, const uint32_t *__restrict__ aips, uint64_t n,
                                                                 uint32_t nr, uint32_t ra, uint32_t *__restrict__ cnt) {
    extern __shared__ uint32_t wh_all[];                 // [warps][nr]
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *wh = wh_all + (size_t)warp * nr;
    const uint32_t nseg = G.g >> G.log2L;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n; h += nwarps) {
        for (uint32_t r = lane; r < nr; r += 32u) wh[r] = 0u;
        __syncwarp();
        const uint64_t hk = host_key(G, aips[h]);
        for (uint32_t j = lane; j < nseg; j += 32u) atomicAdd(&wh[seg_base_k(G, hk, j) / ra], 1u);
        __syncwarp();
        for (uint32_t r = lane; r < nr; r += 32u) cnt[(uint64_t)r * n + h] = wh[r];
        __syncwarp();
    }
}

// Cells by size, per region: qh[r][qm - q] += 1 for a cell of q units (row r of qh has qm + 1 counters).
__global__ void __launch_bounds__(BUILD_THREADS) hs_qhist_kernel(const uint32_t *__restrict__ cnt, uint64_t n,
                                                                 uint32_t qm, uint32_t *__restrict__ qh) {
    const uint32_t r = blockIdx.y;
    for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n; h += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t q = (cnt[(uint64_t)r * n + h] + PER_UNIT - 1u) / PER_UNIT;
        if (q) atomicAdd(&qh[(uint64_t)r * (qm + 1) + (qm - q)], 1u);
    }
}

// Block per row of `off` (rows of n counters at a stride of n + 1): the row
// from counts to exclusive offsets, off[n] and total[row] its sum (in 64
// bits, to catch overflow).
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

// Every cell its place: the next slot of its size class in its region's order
// (qh holds the classes' first slots and advances), so that the cells of a
// region run from the most units to the fewest.  Slot s of region r is lane
// s mod 32 of tile rt[r] + s / 32; the first cell of a tile is its largest and
// gives the tile's rows.  cnt[r][h] becomes the cell's tile lane 32 t + j.
__global__ void __launch_bounds__(BUILD_THREADS) hs_place_kernel(uint32_t *__restrict__ cnt, uint64_t n, uint32_t qm,
                                                                 uint32_t *__restrict__ qh,
                                                                 const uint32_t *__restrict__ rt,
                                                                 uint32_t *__restrict__ host,
                                                                 uint32_t *__restrict__ rows) {
    const uint32_t r = blockIdx.y;
    for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n; h += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = (uint64_t)r * n + h;
        const uint32_t q = (cnt[i] + PER_UNIT - 1u) / PER_UNIT;
        if (!q) continue;
        const uint32_t s = atomicAdd(&qh[(uint64_t)r * (qm + 1) + (qm - q)], 1u);
        const uint32_t tl = rt[r] * 32u + s;
        host[tl] = (uint32_t)h;
        if ((s & 31u) == 0u) rows[tl >> 5] = q;
        cnt[i] = tl;
    }
}

// Warp per host: each segment's entry at its slot of the host's cell in its
// region -- entry k of the cell in lane j = tl mod 32 of tile t = tl / 32 is
// field k mod 6 of that lane's unit in row row0[t] + k / 6, OR-ed into the
// (zeroed) words it spans.  A cell's entries go in the order of their
// shared-memory bank less the lane, mod 32 (a counting sort: a histogram per
// region and key, its scan, then each entry to the next slot of its key), so
// that at any step the 32 lanes of a tile -- cells of about the same size --
// look up words in different banks rather than in 32 random ones.
__global__ void hs_fill_kernel(Geom G, const uint32_t *__restrict__ aips, uint64_t n, uint32_t nr, uint32_t ra,
                               uint32_t bpa, const uint32_t *__restrict__ tlpos, const uint32_t *__restrict__ row0,
                               uint32_t *__restrict__ entries) {
    extern __shared__ uint32_t wk_all[];                 // [warps][nr][33]: per region and key, counts, then slots
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *wk = wk_all + (size_t)warp * nr * 33u;
    const uint32_t nseg = G.g >> G.log2L;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n; h += nwarps) {
        for (uint32_t i = lane; i < nr * 33u; i += 32u) wk[i] = 0u;
        __syncwarp();
        const uint64_t hk = host_key(G, aips[h]);
        for (int pass = 0; pass < 2; pass++) {
            for (uint32_t j = lane; j < nseg; j += 32u) {
                const uint32_t pos = seg_base_k(G, hk, j);
                const uint32_t r = pos / ra;
                const uint32_t e = entry_of(pos - r * ra, bpa);
                const uint32_t tl = tlpos[(uint64_t)r * n + h];
                uint32_t *slot = wk + r * 33u + (((e >> 5) - tl) & 31u);
                if (pass == 0) {
                    atomicAdd(slot, 1u);
                    continue;
                }
                const uint32_t k = atomicAdd(slot, 1u);
                const uint64_t row = (uint64_t)row0[tl >> 5] + k / PER_UNIT;
                const uint32_t b = 21u * (k % PER_UNIT);
                uint32_t *u = entries + row * 128u + (tl & 31u) * 4u + (b >> 5);
                atomicOr(u, e << (b & 31u));
                if ((b & 31u) > 11u) atomicOr(u + 1, e >> (32u - (b & 31u)));
            }
            __syncwarp();
            if (pass == 0) {
                for (uint32_t r = lane; r < nr; r += 32u) {   // counts -> first slots, key by key
                    uint32_t run = 0;
                    for (uint32_t q = 0; q < 32u; q++) {
                        const uint32_t c = wk[r * 33u + q];
                        wk[r * 33u + q] = run;
                        run += c;
                    }
                }
                __syncwarp();
            }
        }
    }
}

constexpr uint32_t ORDER_ROWS = 24;                    // tiles of up to this many rows are dealt again
constexpr uint32_t ORDER_CAP = ORDER_ROWS * PER_UNIT;  // entries of a column, at most
constexpr int ORDER_WARPS = 4;                          // hs_order_kernel: warps per block, a tile each
constexpr size_t ORDER_WARP_BYTES = (32u * ORDER_CAP + 2u * 32u * 33u) * 4u;

// The six 21-bit entries of a unit (0 = pad).
__device__ __forceinline__ void unit_entries(uint4 v, uint32_t (&x)[PER_UNIT]) {
    x[0] = v.x & 0x1FFFFFu;
    x[1] = __funnelshift_r(v.x, v.y, 21) & 0x1FFFFFu;
    x[2] = (v.y >> 10) & 0x1FFFFFu;
    x[3] = __funnelshift_r(v.y, v.z, 31) & 0x1FFFFFu;
    x[4] = __funnelshift_r(v.z, v.w, 20) & 0x1FFFFFu;
    x[5] = v.w >> 9;
}

// Warp per tile: the entries of each column dealt again, step by step (step
// 6 i + s is field s of row i), so that at a step the 32 lanes look up words
// in different shared-memory banks where they can.  At each step the lanes
// choose in turn, the lane with the fewest banks left first (then the one
// with the most entries left); a lane takes the bank, not yet taken at this
// step, of which it holds the most entries (ties: the bank most entries of
// the tile still wait for), or, when all of its banks are taken, the one of
// which it holds the most.  A column keeps its entries, reordered, so every
// count is unchanged.  Tiles of more than ORDER_ROWS rows keep the fill's
// order.
__global__ void __launch_bounds__(32 * ORDER_WARPS) hs_order_kernel(const uint32_t *__restrict__ row0, uint32_t T,
                                                                    uint4 *__restrict__ ent4) {
    extern __shared__ uint32_t order_smem[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t *srt = order_smem + (size_t)warp * (ORDER_WARP_BYTES / 4u);   // [32][ORDER_CAP]: a column by bank
    uint32_t *cnt = srt + 32u * ORDER_CAP;                                   // [32][33]: entries left per bank
    uint32_t *mysrt = srt + lane * ORDER_CAP, *mycnt = cnt + lane * 33u;
    uint32_t *mybeg = cnt + 32u * 33u + lane * 33u;                          // first entry of each bank
    const uint32_t nwarps = gridDim.x * ORDER_WARPS;
    for (uint32_t t = blockIdx.x * ORDER_WARPS + warp; t < T; t += nwarps) {
        const uint32_t r0 = row0[t], M = row0[t + 1] - r0;
        if (M > ORDER_ROWS) continue;
        uint4 *col = ent4 + (uint64_t)r0 * 32u + lane;
        for (uint32_t b = 0; b < 32u; b++) mycnt[b] = 0u;
        for (uint32_t i = 0; i < M; i++) {
            uint32_t x[PER_UNIT];
            unit_entries(col[32u * i], x);
#pragma unroll
            for (int f = 0; f < (int)PER_UNIT; f++)
                if (x[f]) mycnt[(x[f] >> 5) & 31u]++;
        }
        uint32_t rem = 0, nav = 0;
        for (uint32_t b = 0; b < 32u; b++) {
            mybeg[b] = rem;
            rem += mycnt[b];
            nav += mycnt[b] != 0u;
        }
        for (uint32_t i = 0; i < M; i++) {
            uint32_t x[PER_UNIT];
            unit_entries(col[32u * i], x);
#pragma unroll
            for (int f = 0; f < (int)PER_UNIT; f++)
                if (x[f]) mysrt[mybeg[(x[f] >> 5) & 31u]++] = x[f];
        }
        for (uint32_t b = 0; b < 32u; b++) mybeg[b] -= mycnt[b];
        __syncwarp();
        uint32_t glob = 0;                               // lane b: entries of bank b the tile has left
        for (uint32_t j = 0; j < 32u; j++) glob += cnt[j * 33u + lane];
        for (uint32_t i = 0; i < M; i++) {
            uint32_t y[PER_UNIT];
#pragma unroll
            for (int f = 0; f < (int)PER_UNIT; f++) {
                uint32_t taken = 0u, done = 0u, mine = 0u;
                for (int turn = 0; turn < 32; turn++) {
                    const bool waiting = rem != 0u && !((done >> lane) & 1u);
                    const uint32_t m = __reduce_min_sync(0xFFFFFFFFu, waiting ? ((nav << 8 | (255u - rem)) << 5 | lane) : 0xFFFFFFFFu);
                    if (m == 0xFFFFFFFFu) break;
                    const uint32_t j = m & 31u;
                    const uint32_t c = cnt[j * 33u + lane];          // lane b looks at bank b of lane j
                    const uint32_t sc = c ? ((c << 16 | glob) << 5 | lane) : 0u;
                    uint32_t best = __reduce_max_sync(0xFFFFFFFFu, ((taken >> lane) & 1u) ? 0u : sc);
                    if (!best) best = __reduce_max_sync(0xFFFFFFFFu, sc);
                    const uint32_t b = best & 31u;
                    taken |= 1u << b;
                    done |= 1u << j;
                    if (lane == b) glob--;
                    if (lane == j) {
                        const uint32_t left = --mycnt[b];
                        mine = mysrt[mybeg[b] + left];
                        rem--;
                        nav -= left == 0u;
                    }
                    __syncwarp();
                }
                y[f] = mine;
            }
            col[32u * i] = make_uint4(y[0] | y[1] << 21, y[1] >> 11 | y[2] << 10 | y[3] << 31, y[3] >> 1 | y[4] << 20,
                                      y[4] >> 12 | y[5] << 9);
        }
        __syncwarp();
    }
}

// Thread per 8 ATs: nibble j of word w is the age of AT 8 w + j -- its
// distance d (Eq. 5 in frame 0; a recorder's value) when d < k, else 15.
__global__ void __launch_bounds__(256) hs_agemap_kernel(Geom G, uint32_t bact0, uint64_t words, uint32_t *__restrict__ map) {
    const uint2 *pool8 = reinterpret_cast<const uint2 *>(G.pool);
    for (uint64_t w = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; w < words; w += (uint64_t)gridDim.x * blockDim.x) {
        const uint2 v = __ldcg(pool8 + w);
        VATE_CHECK_WORD(G, v.x, w >> 1);
        uint32_t half[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            const uint32_t raw = i ? v.y : v.x;
            const uint32_t d = G.counter == 1u ? raw : swar_bins(raw, bact0, G.twok);    // a distance per byte
            const uint32_t old = ((d + (128u - G.k) * ONES) & HIGH) >> 7;               // d >= k
            const uint32_t nb = (d | (old * 0xFFu)) & 0x0F0F0F0Fu;                      // d, or 15
            const uint32_t t = (nb | (nb >> 4)) & 0x00FF00FFu;                           // nibble pairs
            half[i] = (t | (t >> 8)) & 0xFFFFu;
        }
        map[w] = half[0] | half[1] << 16;
    }
}

// One AT age (a < 16) into accumulators of 6-bit fields: one is added to
// field a mod 5 of accumulator a / 5 (bits 6 (a mod 5) ..); ages 15 and, past
// the accumulators in use, ages at or above 5 NACC add nothing (a shift of 32
// or more), and an age that lands on the top two bits of an accumulator is one
// no window counts.
template <int NACC>
__device__ __forceinline__ void add_age(uint32_t (&acc)[3], uint32_t a) {
    acc[0] += __funnelshift_lc(0u, 1u, a * 6u);
    if (NACC > 1) acc[1] += __funnelshift_lc(0u, 1u, a * 6u - 30u);
    if (NACC > 2) acc[2] += __funnelshift_lc(0u, 1u, a * 6u - 60u);
}

// The 6-bit fields into 16-bit ones (ages 2 j, 2 j + 1 in wide[j]); then zero.
template <int NACC>
__device__ __forceinline__ void spill_ages(uint32_t (&acc)[3], uint32_t (&wide)[8]) {
#pragma unroll
    for (int j = 0; j < NACC; j++) {
#pragma unroll
        for (int f = 0; f < 5; f++) {
            const int a = 5 * j + f;
            wide[a >> 1] += ((acc[j] >> (6 * f)) & 63u) << (16 * (a & 1));
        }
        acc[j] = 0u;
    }
}

// The lane's counts added to its host's 16-bit fields (ages 4 i .. 4 i + 3 in
// counts[i n + h]: a host's fields in separate arrays, so that its atomics
// meet different sectors); then zero.
template <int NACC>
__device__ __forceinline__ void flush_ages(uint32_t (&acc)[3], uint32_t (&wide)[8], uint32_t host, uint64_t n,
                                           unsigned long long *__restrict__ counts) {
    spill_ages<NACC>(acc, wide);
    constexpr int NW = (5 * NACC + 3) / 4;              // 64-bit words of four ages
#pragma unroll
    for (int i = 0; i < NW; i++) {
        const unsigned long long v = (unsigned long long)wide[2 * i + 1] << 32 | wide[2 * i];
        if (v && host != NONE) atomicAdd(counts + (uint64_t)i * n + host, v);
        wide[2 * i] = wide[2 * i + 1] = 0u;
    }
}

// hs_tile_kernel over the age map (4 bits per AT, 384 K ATs per region in the
// same shared memory): lane j adds the age of every AT of its column's
// segments to 6-bit fields, moves them into 16-bit fields in registers before
// any could reach 64, and adds those to its cell's host at the end of the
// tile.  NACC = accumulators of five ages in use (k <= 5 NACC).
template <int L, int NACC>
__global__ void __launch_bounds__(HS_THREADS, 1) hs_age_kernel(const uint32_t *__restrict__ agemap, uint64_t map_words,
                                                               uint32_t nr, const uint32_t *__restrict__ rt,
                                                               const uint32_t *__restrict__ row0,
                                                               const uint32_t *__restrict__ hosts,
                                                               const uint4 *__restrict__ ent4, uint32_t T, uint32_t R,
                                                               uint64_t n, unsigned long long *__restrict__ counts) {
    constexpr uint32_t SPILL_ROWS = 63u / (PER_UNIT * L);    // rows a 6-bit field can take before it could overflow
    extern __shared__ uint4 bm4[];                       // a zero quad, then REGION_WORDS words of age map
    uint32_t *bm = reinterpret_cast<uint32_t *>(bm4 + 1);
    const unsigned char *bmb = reinterpret_cast<const unsigned char *>(bm4);
    __shared__ uint32_t s_t[2];
    __shared__ uint32_t s_r;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t nw = blockDim.x >> 5;
    if (tid == 0) bm4[0] = make_uint4(0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu);   // pads: age 15
    if (warp < 2) {
        const uint32_t x = (uint32_t)((uint64_t)R * (blockIdx.x + warp) / gridDim.x);
        const uint32_t t = tile_at_row(row0, 0u, T, x, lane);
        if (lane == 0) s_t[warp] = t;
    }
    __syncthreads();
    const uint32_t ta = s_t[0], tb = s_t[1];
    for (uint32_t t0 = ta; t0 < tb;) {
        if (tid == 0) {
            uint32_t lo = 0, hi = nr;
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (rt[mid] <= t0) lo = mid;
                else hi = mid;
            }
            s_r = lo;
        }
        __syncthreads();
        const uint32_t r = s_r;
        const uint32_t t1 = min(tb, rt[r + 1]);
        const uint64_t w0 = (uint64_t)r * REGION_WORDS, left = map_words - w0;
        const uint32_t nwords = left < (uint64_t)REGION_WORDS ? (uint32_t)left : REGION_WORDS;
        const uint4 *src = reinterpret_cast<const uint4 *>(agemap + w0);
        for (uint32_t i = tid; i < nwords / 4u; i += blockDim.x) bm4[1 + i] = __ldcg(src + i);
        for (uint32_t i = (nwords & ~3u) + tid; i < nwords; i += blockDim.x) bm[i] = __ldcg(agemap + w0 + i);
        __syncthreads();
        const uint32_t xa = __ldcg(row0 + t0), xb = __ldcg(row0 + t1);
        const uint32_t wa = tile_at_row(row0, t0, t1, xa + (uint32_t)((uint64_t)(xb - xa) * warp / nw), lane);
        const uint32_t wb = tile_at_row(row0, t0, t1, xa + (uint32_t)((uint64_t)(xb - xa) * (warp + 1u) / nw), lane);
        if (wa < wb) {
            const uint32_t rowA = __ldcg(row0 + wa), rowB = __ldcg(row0 + wb);
            uint32_t t = wa;
            uint32_t end = __ldcg(row0 + t + 1u);
            uint32_t host = __ldcg(hosts + (uint64_t)t * 32u + lane);
            const bool more = t + 1u < wb;
            uint32_t end2 = more ? __ldcg(row0 + t + 2u) : rowB;
            uint32_t host2 = more ? __ldcg(hosts + (uint64_t)(t + 1u) * 32u + lane) : NONE;
            uint32_t acc[3] = {0u, 0u, 0u};
            uint32_t wide[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
            uint32_t since = 0;                          // rows added since the last flush (the same in every lane)
            for (uint32_t row = rowA; row < rowB; row += HB) {
                const uint4 *rp = ent4 + (uint64_t)row * 32u + lane;
                uint4 v[HB];
#pragma unroll
                for (int u = 0; u < HB; u++)
                    v[u] = row + u < rowB ? __ldcs(rp + 32u * u) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
                for (int u = 0; u < HB; u++) {
                    if (row + u >= rowB) break;
                    if (row + u == end) {
                        flush_ages<NACC>(acc, wide, host, n, counts);
                        since = 0;
                    } else if (since == SPILL_ROWS) {
                        spill_ages<NACC>(acc, wide);
                        since = 0;
                    }
                    if (row + u == end) {
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
                    const uint32_t x[PER_UNIT] = {v[u].x, __funnelshift_r(v[u].x, v[u].y, 21), v[u].y >> 10,
                                                  __funnelshift_r(v[u].y, v[u].z, 31),
                                                  __funnelshift_r(v[u].z, v[u].w, 20), v[u].w >> 9};
#pragma unroll
                    for (int f = 0; f < (int)PER_UNIT; f++) {
                        // bits 5-20 of the entry: its word of the map; bits 0-4: the first bit of the segment's nibbles
                        const uint32_t w = __funnelshift_r(
                            *reinterpret_cast<const uint32_t *>(bmb + ((x[f] >> 3) & 0x3FFFCu)), 0u, x[f]);
#pragma unroll
                        for (int a = 0; a < L; a++) add_age<NACC>(acc, (w >> (4 * a)) & 15u);
                    }
                    since++;
                }
            }
            flush_ages<NACC>(acc, wide, host, n, counts);
        }
        t0 = t1;
    }
}

// Per-host sums of the 16-bit age fields (counts[i n + h]): active[h] = the ages below kprime.
__global__ void hs_counts_active_kernel(const unsigned long long *__restrict__ counts, uint64_t n, uint32_t kprime,
                                        uint32_t *__restrict__ active) {
    for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n; h += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t a = 0;
        for (uint32_t d = 0; d < kprime; d++) a += (uint32_t)(counts[(d >> 2) * n + h] >> (16u * (d & 3u))) & 0xFFFFu;
        active[h] = a;
    }
}

// The 16-bit age fields as vate_age_counts writes them: out[h k + d], d < k.
__global__ void hs_counts_u16_kernel(const unsigned long long *__restrict__ counts, uint64_t n, uint32_t k,
                                     uint16_t *__restrict__ out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n * k; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t h = i / k;
        const uint32_t d = (uint32_t)(i - h * k);
        out[i] = (uint16_t)(counts[(d >> 2) * n + h] >> (16u * (d & 3u)));
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
    uint32_t T = 0;                        // tiles
    uint32_t R = 0;                        // rows of 32 units
    bool ages = false;                     // an age index (4-bit age map) rather than a CheckAT bitmap index
    uint32_t ra = 0;                       // ATs per region
    uint32_t bpa = 1;                      // bits per AT of the region's map (1: bitmap, 4: age map)
    uint64_t bm_words = 0;                 // words of the pool's map (bitmap or age map)
    uint32_t *d_entries = nullptr;         // [R][32][4]
    uint32_t *d_rt = nullptr;              // [nr + 1]: first tile of each region
    uint32_t *d_row0 = nullptr;            // [T + 1]: first row of each tile
    uint32_t *d_host = nullptr;            // [T][32]: host of each cell, NONE for an empty lane
    uint32_t *d_bitmap = nullptr;
    uint32_t *d_active = nullptr;          // [n]
    unsigned long long *d_ages = nullptr;  // [4][n]: an age index's per-age counts, 16-bit fields
    float *d_out = nullptr;                // [n], vate_estimate_hostset_host (on first use)
    uint8_t *d_flags = nullptr;            // [n]
    // vate_estimate_hostset_host_async (on first use): results of two calls in turn, copied on a stream of
    // the hostset; done[b]: the copy out of buffer b; ready: the kernels of the last call
    float *d_out2[2] = {nullptr, nullptr};
    uint8_t *d_flags2[2] = {nullptr, nullptr};
    cudaStream_t d2h = nullptr;
    cudaEvent_t done[2] = {nullptr, nullptr};
    cudaEvent_t ready = nullptr;
    bool used[2] = {false, false};
    uint32_t flip = 0;
    // vate_hostset_time_passes: event pairs around the index pass of the next calls
    std::vector<cudaEvent_t> pass_ev;      // [2 * n]
    uint32_t pass_want = 0, pass_done = 0;
    uint64_t bytes = 0;
};

namespace {

void free_hostset(vate_hostset *s) {
    if (!s) return;
    cudaFree(s->d_entries);
    cudaFree(s->d_rt);
    cudaFree(s->d_row0);
    cudaFree(s->d_host);
    cudaFree(s->d_bitmap);
    cudaFree(s->d_active);
    cudaFree(s->d_ages);
    cudaFree(s->d_out);
    cudaFree(s->d_flags);
    for (int b = 0; b < 2; b++) {
        cudaFree(s->d_out2[b]);
        cudaFree(s->d_flags2[b]);
        if (s->done[b]) cudaEventDestroy(s->done[b]);
    }
    if (s->ready) cudaEventDestroy(s->ready);
    for (cudaEvent_t e : s->pass_ev) cudaEventDestroy(e);
    if (s->d2h) cudaStreamDestroy(s->d2h);
    cudaGetLastError();
    delete s;
}

// accumulators of five ages an age pass needs for window k
uint32_t nacc_for(uint32_t k) { return std::max(1u, (k + 4u) / 5u); }

template <int NACC>
void *age_kernel_for(uint32_t L) {
    switch (L) {
    case 1: return (void *)hs_age_kernel<1, NACC>;
    case 2: return (void *)hs_age_kernel<2, NACC>;
    case 4: return (void *)hs_age_kernel<4, NACC>;
    default: return (void *)hs_age_kernel<8, NACC>;
    }
}

// The index pass for segment length L: the bitmap's (nacc 0) or the age map's with nacc accumulators.
void *kernel_for(uint32_t L, uint32_t nacc) {
    if (nacc == 1u) return age_kernel_for<1>(L);
    if (nacc == 2u) return age_kernel_for<2>(L);
    if (nacc >= 3u) return age_kernel_for<3>(L);
    switch (L) {
    case 1: return (void *)hs_tile_kernel<1>;
    case 2: return (void *)hs_tile_kernel<2>;
    case 4: return (void *)hs_tile_kernel<4>;
    default: return (void *)hs_tile_kernel<8>;
    }
}

constexpr size_t TILE_SMEM = (size_t)REGION_WORDS * 4 + BM_SKIP;

// Shared memory for the region's bitmap and no more: the carveout (in percent
// of the SM's shared memory) that holds one block, so that the rest stays L1.
int tile_carveout() {
#ifdef VATE_HS_CARVEOUT
    return VATE_HS_CARVEOUT;
#endif
    int dev = 0, smem_sm = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess || smem_sm <= 0)
        return 100;
    const size_t need = TILE_SMEM + 64 + 1024;          // dynamic, static and the block's reserved kilobyte
    return (int)std::min<size_t>(100, (need * 100 + smem_sm - 1) / smem_sm);
}

}  // namespace

namespace {

int create_hostset(vate_handle *h, const uint32_t *d_aips, uint64_t n, void *stream, vate_hostset **out, bool ages) {
    if (!out) return set_error(VATE_EINVAL, "out must not be NULL");
    *out = nullptr;
    HandleView v;
    if (int rc = handle_view(h, &v)) return rc;
    const Geom &G = v.G;
    if (n == 0 || !d_aips) return set_error(VATE_EINVAL, "a hostset needs at least one host (d_aips not NULL)");
    if (n >= 0x80000000ull) return set_error(VATE_EINVAL, "at most 2^31 - 1 hosts");
    if (G.atw != 1u || G.packed || (G.counter == VATE_COUNTER_AT && !G.frame0))
        return set_error(VATE_EINVAL, "a hostset needs a pool of byte ATs (k <= 63)");
    if (G.lo != 0 || G.hi != G.P) return set_error(VATE_EINVAL, "a hostset needs the whole pool, not a shard");
    if (G.L != 1 && G.L != 2 && G.L != 4 && G.L != 8) return set_error(VATE_EINVAL, "a hostset needs seg_len 1, 2, 4 or 8");
    if (ages && (G.k > 15u || G.g > 65535u))
        return set_error(VATE_EINVAL, "an age index needs k <= 15 and g <= 65535");
    const uint32_t ra = ages ? AGE_REGION_ATS : REGION_ATS, bpa = ages ? 4u : 1u;
    const uint32_t nr = (uint32_t)((G.P + ra - 1) / ra);
    if (nr > MAX_REGIONS) return set_error(VATE_EINVAL, "pool too large for a hostset (more than 1024 regions)");
    const uint32_t qm = ((G.g >> G.log2L) + PER_UNIT - 1u) / PER_UNIT;   // the most units a cell can have
    cudaStream_t st = (cudaStream_t)stream;
    vate_hostset *s = new (std::nothrow) vate_hostset();
    if (!s) return set_error(VATE_ENOMEM, "host allocation failed");
    s->owner = h;
    cudaGetDevice(&s->device);
    s->sms = sm_count_now();
    s->n = n;
    s->nr = nr;
    s->L = G.L;
    s->ages = ages;
    s->ra = ra;
    s->bpa = bpa;
    s->bm_words = G.P * bpa / 32u;
    // build-only buffers: cnt[r][h] (segments per cell, then the cell's tile lane), qh[r][qm + 1] (cells by size,
    // then each size's next slot), total[] (sums of the scans)
    uint32_t *d_cnt = nullptr, *d_qh = nullptr;
    unsigned long long *d_total = nullptr;
    auto release = [&]() {
        cudaFree(d_cnt);
        cudaFree(d_qh);
        cudaFree(d_total);
        free_hostset(s);
    };
    auto fail_cuda = [&](cudaError_t e) {
        release();
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    };
    auto fail_mem = [&](const char *what) {
        cudaGetLastError();
        release();
        return set_error(VATE_ENOMEM, what);
    };
    if (cudaMalloc(&d_cnt, (size_t)nr * n * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&d_qh, (size_t)nr * (qm + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&d_total, nr * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&s->d_rt, (nr + 1) * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&s->d_bitmap, s->bm_words * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&s->d_active, n * sizeof(uint32_t)) != cudaSuccess ||
        (ages && cudaMalloc(&s->d_ages, n * 4 * sizeof(unsigned long long)) != cudaSuccess))
        return fail_mem("out of device memory for the hostset's build");
    const size_t build_smem = (size_t)(BUILD_THREADS / 32) * nr * sizeof(uint32_t);
    // the fill's warps each hold nr x 33 counters: as many warps per block (1-8) as fit in 200 KB
    const uint32_t fill_warps = (uint32_t)std::max<size_t>(1, std::min<size_t>(8, (200u << 10) / ((size_t)nr * 132u)));
    const size_t fill_smem = (size_t)fill_warps * nr * 132u;
    cudaError_t e = cudaFuncSetAttribute(hs_count_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)build_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(hs_fill_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fill_smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_qh, 0, (size_t)nr * (qm + 1) * sizeof(uint32_t), st);
    if (e != cudaSuccess) return fail_cuda(e);
    const int grid = (int)std::min<uint64_t>((n + BUILD_THREADS / 32 - 1) / (BUILD_THREADS / 32), (uint64_t)s->sms * 16);
    const dim3 rgrid((unsigned)std::min<uint64_t>((n + BUILD_THREADS - 1) / BUILD_THREADS, 256), nr);
    hs_count_kernel<<<grid, BUILD_THREADS, build_smem, st>>>(G, d_aips, n, nr, ra, d_cnt);
    count_launch();
    hs_qhist_kernel<<<rgrid, BUILD_THREADS, 0, st>>>(d_cnt, n, qm, d_qh);
    count_launch();
    hs_scan_kernel<<<nr, 1024, 0, st>>>(d_qh, qm, d_total);
    count_launch();
    std::vector<unsigned long long> cells(nr);
    std::vector<uint32_t> rt(nr + 1);
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(cells.data(), d_total, nr * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_cuda(e);
    uint64_t tiles = 0;
    for (uint32_t r = 0; r < nr; r++) {
        rt[r] = (uint32_t)tiles;
        tiles += (cells[r] + 31u) / 32u;
        if (tiles > (0xFFFFFFFFull >> 5) - 1u) {
            release();
            return set_error(VATE_EINVAL, "too many hosts for a hostset: 2^27 or more tiles of 32 cells");
        }
    }
    rt[nr] = (uint32_t)tiles;
    s->T = (uint32_t)tiles;
    if (cudaMalloc(&s->d_host, (size_t)s->T * 32u * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc(&s->d_row0, ((size_t)s->T + 1) * sizeof(uint32_t)) != cudaSuccess)
        return fail_mem("out of device memory for the hostset's tiles");
    if ((e = cudaMemcpyAsync(s->d_rt, rt.data(), (nr + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess ||
        (e = cudaMemsetAsync(s->d_host, 0xFF, (size_t)s->T * 32u * sizeof(uint32_t), st)) != cudaSuccess)
        return fail_cuda(e);
    hs_place_kernel<<<rgrid, BUILD_THREADS, 0, st>>>(d_cnt, n, qm, d_qh, s->d_rt, s->d_host, s->d_row0);
    count_launch();
    hs_scan_kernel<<<1, 1024, 0, st>>>(s->d_row0, s->T, d_total);
    count_launch();
    unsigned long long rows = 0;
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(&rows, d_total, sizeof(rows), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail_cuda(e);
    if (rows > 0xFFFFFFFFull - 64u) {
        release();
        return set_error(VATE_EINVAL, "too many hosts for a hostset: 2^32 or more rows of index");
    }
    s->R = (uint32_t)rows;
    const size_t ebytes = (size_t)s->R * 512u;
    if (cudaMalloc(&s->d_entries, ebytes) != cudaSuccess) return fail_mem("out of device memory for the hostset's index");
    if ((e = cudaMemsetAsync(s->d_entries, 0, ebytes, st)) != cudaSuccess) return fail_cuda(e);
    const int fgrid = (int)std::min<uint64_t>((n + fill_warps - 1) / fill_warps, (uint64_t)s->sms * 16 * (8 / fill_warps));
    hs_fill_kernel<<<fgrid, 32 * fill_warps, fill_smem, st>>>(G, d_aips, n, nr, ra, bpa, d_cnt, s->d_row0,
                                                              s->d_entries);
    count_launch();
    const size_t order_smem = ORDER_WARPS * ORDER_WARP_BYTES;
    if ((e = cudaFuncSetAttribute(hs_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)order_smem)) !=
        cudaSuccess)
        return fail_cuda(e);
    const int ogrid = (int)std::min<uint64_t>((s->T + ORDER_WARPS - 1) / ORDER_WARPS, (uint64_t)s->sms * 2);
    hs_order_kernel<<<ogrid, 32 * ORDER_WARPS, order_smem, st>>>(s->d_row0, s->T,
                                                                  reinterpret_cast<uint4 *>(s->d_entries));
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return fail_cuda(e);
    cudaFree(d_cnt);
    cudaFree(d_qh);
    cudaFree(d_total);
    d_cnt = d_qh = nullptr;
    d_total = nullptr;
    void *kern = kernel_for(s->L, ages ? nacc_for(G.k) : 0u);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TILE_SMEM)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, tile_carveout())) != cudaSuccess)
        return fail_cuda(e);
    s->bytes = ebytes + (uint64_t)s->T * 32u * 4u + ((uint64_t)s->T + 1) * 4u + (nr + 1) * 4u + s->bm_words * 4 + n * 4 +
               (ages ? n * 32 : 0);
    *out = s;
    return VATE_OK;
}

}  // namespace

extern "C" {

int vate_hostset_create(vate_handle *h, const uint32_t *d_aips, uint64_t n, void *stream, vate_hostset **out) {
    return create_hostset(h, d_aips, n, stream, out, false);
}

int vate_hostset_create_ages(vate_handle *h, const uint32_t *d_aips, uint64_t n, void *stream, vate_hostset **out) {
    return create_hostset(h, d_aips, n, stream, out, true);
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

}  // extern "C"

namespace {

// The per-age counts of an age index's hosts into s->d_ages: the pool's age map, then the tile pass.
cudaError_t age_pass(const HandleView &v, vate_hostset *s, cudaStream_t st) {
    const Geom &G = v.G;
    cudaError_t e = cudaMemsetAsync(s->d_ages, 0, s->n * 4 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    const int mgrid = (int)std::min<uint64_t>((s->bm_words + 255) / 256, (uint64_t)v.sms * 16);
    if ((e = launch_pool(G, hs_agemap_kernel, mgrid, 256, 0, st, G, v.bact0, s->bm_words, s->d_bitmap)) != cudaSuccess)
        return e;
    // the arguments of hs_age_kernel<L, NACC>, in its parameters' types
    const uint32_t *map = s->d_bitmap, *rt = s->d_rt, *row0 = s->d_row0, *hosts = s->d_host;
    const uint4 *ent4 = reinterpret_cast<const uint4 *>(s->d_entries);
    uint64_t words = s->bm_words, n = s->n;
    uint32_t nr = s->nr, T = s->T, R = s->R;
    unsigned long long *counts = s->d_ages;
    void *args[] = {&map, &words, &nr, &rt, &row0, &hosts, &ent4, &T, &R, &n, &counts};
    const bool timed = s->pass_done < s->pass_want;
    if (timed) cudaEventRecord(s->pass_ev[2 * s->pass_done], st);
    e = cudaLaunchKernel(kernel_for(s->L, nacc_for(G.k)), dim3(v.sms), dim3(HS_THREADS), args, TILE_SMEM, st);
    count_launch();
    if (timed && e == cudaSuccess) cudaEventRecord(s->pass_ev[2 * s->pass_done++ + 1], st);
    return e;
}

int check_call(vate_handle *h, vate_hostset *s, HandleView &v) {
    if (int rc = handle_view(h, &v)) return rc;
    if (!s || s->owner != h) return set_error(VATE_EINVAL, "the hostset was not built for this handle");
    if (!v.closed) return set_error(VATE_ESLICE, "the current slice has not been closed");
    return VATE_OK;
}

}  // namespace

extern "C" {

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
    cudaError_t e;
    if (s->ages) {
        // the active count for k' is the sum of the ages below k'
        if ((e = age_pass(v, s, st)) != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
        const int cgrid = (int)std::min<uint64_t>((s->n + 255) / 256, (uint64_t)v.sms * 8);
        hs_counts_active_kernel<<<cgrid, 256, 0, st>>>(s->d_ages, s->n, kprime, acc);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    } else {
        if ((e = cudaMemsetAsync(acc, 0, s->n * sizeof(uint32_t), st)) != cudaSuccess)
            return set_error(VATE_ECUDA, cudaGetErrorString(e));
        const RangeConsts rc = G.counter == 1u ? dr_range_consts(kprime) : range_consts(v.bact0, kprime, G.twok);
        const uint32_t c2k = (128u - G.twok) * ONES;
        const int bgrid = (int)std::min<uint64_t>((s->bm_words + 255) / 256, (uint64_t)v.sms * 16);
        e = launch_pool(G, hs_bitmap_kernel, bgrid, 256, 0, st, G, rc, c2k, s->bm_words, s->d_bitmap);
        if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
        const uint4 *ent4 = reinterpret_cast<const uint4 *>(s->d_entries);
        const bool timed = s->pass_done < s->pass_want;
        if (timed) cudaEventRecord(s->pass_ev[2 * s->pass_done], st);
#define VATE_HS_LAUNCH(LL)                                                                                          \
    hs_tile_kernel<LL><<<v.sms, HS_THREADS, TILE_SMEM, st>>>(s->d_bitmap, s->bm_words, s->nr, s->d_rt, s->d_row0,   \
                                                             s->d_host, ent4, s->T, s->R, acc)
        switch (s->L) {
        case 1: VATE_HS_LAUNCH(1); break;
        case 2: VATE_HS_LAUNCH(2); break;
        case 4: VATE_HS_LAUNCH(4); break;
        default: VATE_HS_LAUNCH(8); break;
        }
#undef VATE_HS_LAUNCH
        count_launch();
        if (timed) cudaEventRecord(s->pass_ev[2 * s->pass_done++ + 1], st);
        if ((e = cudaGetLastError()) != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    }
    e = launch_estimate_from_counts(G, kprime, v.hist, acc, s->n, d_out, d_flags, st, v.sms);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

int vate_age_counts_hostset(vate_handle *h, vate_hostset *s, uint16_t *d_counts, void *stream) {
    HandleView v;
    if (int rc = check_call(h, s, v)) return rc;
    if (!s->ages) return set_error(VATE_EINVAL, "per-age counts need an age index (vate_hostset_create_ages)");
    if (!d_counts) return set_error(VATE_EINVAL, "d_counts must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = age_pass(v, s, st);
    if (e == cudaSuccess) {
        const int cgrid = (int)std::min<uint64_t>((s->n * v.G.k + 255) / 256, (uint64_t)v.sms * 8);
        hs_counts_u16_kernel<<<cgrid, 256, 0, st>>>(s->d_ages, s->n, v.G.k, d_counts);
        count_launch();
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_estimate_learned_hostset(vate_handle *h, vate_hostset *s, const float *d_params, float *d_out,
                                  uint8_t *d_flags, void *stream) {
    HandleView v;
    if (int rc = check_call(h, s, v)) return rc;
    if (!s->ages) return set_error(VATE_EINVAL, "the learned close needs an age index (vate_hostset_create_ages)");
    if (!d_params || !d_out) return set_error(VATE_EINVAL, "d_params and d_out must not be NULL");
    if (int rc = learned_handle_ok(h)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = age_pass(v, s, st);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    return learned_from_age_counts(h, v, s->d_ages, s->n, d_params, d_out, d_flags, st);   // fields counts[i n + h]
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

int vate_estimate_hostset_host_async(vate_handle *h, vate_hostset *s, uint32_t kprime, float *h_out, uint8_t *h_flags,
                                     void *stream) {
    if (!s || !h_out) return set_error(VATE_EINVAL, "hostset and h_out must not be NULL");
    if (!s->d2h) {
        bool ok = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaEventCreateWithFlags(&s->ready, cudaEventDisableTiming) == cudaSuccess;
        for (int b = 0; b < 2 && ok; b++)
            ok = cudaEventCreateWithFlags(&s->done[b], cudaEventDisableTiming) == cudaSuccess &&
                 cudaMalloc(&s->d_out2[b], s->n * sizeof(float)) == cudaSuccess &&
                 cudaMalloc(&s->d_flags2[b], s->n) == cudaSuccess;
        if (!ok) {                                       // undo it all, so that a later call starts over
            cudaGetLastError();
            for (int b = 0; b < 2; b++) {
                cudaFree(s->d_out2[b]);
                cudaFree(s->d_flags2[b]);
                if (s->done[b]) cudaEventDestroy(s->done[b]);
                s->d_out2[b] = nullptr;
                s->d_flags2[b] = nullptr;
                s->done[b] = nullptr;
            }
            if (s->ready) cudaEventDestroy(s->ready);
            if (s->d2h) cudaStreamDestroy(s->d2h);
            s->ready = nullptr;
            s->d2h = nullptr;
            cudaGetLastError();
            return set_error(VATE_ENOMEM, "out of device memory (or streams) for the hostset's copies");
        }
        s->bytes += 2 * s->n * 5;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t b = s->flip;
    // the kernels of this call rewrite buffer b: after the copy that read it two calls ago
    cudaError_t e = s->used[b] ? cudaStreamWaitEvent(st, s->done[b], 0) : cudaSuccess;
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    if (int rc = vate_estimate_hostset(h, s, kprime, s->d_out2[b], s->d_flags2[b], nullptr, stream)) return rc;
    if ((e = cudaEventRecord(s->ready, st)) == cudaSuccess && (e = cudaStreamWaitEvent(s->d2h, s->ready, 0)) == cudaSuccess &&
        (e = cudaMemcpyAsync(h_out, s->d_out2[b], s->n * sizeof(float), cudaMemcpyDeviceToHost, s->d2h)) == cudaSuccess &&
        (!h_flags || (e = cudaMemcpyAsync(h_flags, s->d_flags2[b], s->n, cudaMemcpyDeviceToHost, s->d2h)) == cudaSuccess))
        e = cudaEventRecord(s->done[b], s->d2h);
    if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    s->used[b] = true;
    s->flip = b ^ 1u;
    return VATE_OK;
}

int vate_hostset_wait(vate_hostset *s) {
    if (!s) return set_error(VATE_EINVAL, "hostset is NULL");
    if (!s->d2h) return VATE_OK;
    cudaError_t e = cudaStreamSynchronize(s->d2h);
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_hostset_time_passes(vate_hostset *s, uint32_t n) {
    if (!s) return set_error(VATE_EINVAL, "hostset is NULL");
    if (n > 4096u) return set_error(VATE_EINVAL, "at most 4096 passes are timed at once");
    while (s->pass_ev.size() < 2u * n) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return set_error(VATE_ENOMEM, "CUDA events for the pass timings");
        }
        s->pass_ev.push_back(e);
    }
    s->pass_want = n;
    s->pass_done = 0;
    return VATE_OK;
}

int vate_hostset_pass_times(vate_hostset *s, float *ms, uint32_t max, uint32_t *count) {
    if (!s || (!ms && max) || !count) return set_error(VATE_EINVAL, "hostset, ms and count must not be NULL");
    const uint32_t n = std::min(max, s->pass_done);
    for (uint32_t i = 0; i < n; i++) {
        cudaError_t e = cudaEventSynchronize(s->pass_ev[2 * i + 1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms + i, s->pass_ev[2 * i], s->pass_ev[2 * i + 1]);
        if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    }
    *count = n;
    return VATE_OK;
}

}  // extern "C"
