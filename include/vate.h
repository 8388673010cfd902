/*
 * vate.h -- C ABI of the B300 (sm_103a) VATE library.
 *
 * VATE (virtual asynchronous timestamp estimator, arXiv 1812.00282) estimates,
 * at the end of every time slice t, the number of distinct opposite hosts bip
 * that each host aip has exchanged packets with during the last k' <= k
 * slices, |OP(aip, t-k'+1, k')| (Sec. 1, Def. 1).  Each host owns g virtual
 * asynchronous timestamps (ATs) drawn from one shared pool of 2^c ATs
 * (Sec. 4.1); an AT stores the asynchronous current timestamp (ACT) of the
 * slice in which it was last set, and value 2k means "inactive" (Sec. 3).
 *
 * Conventions for every entry point below
 *   - Pointers named d_* are DEVICE pointers (cudaMalloc / torch CUDA
 *     tensors) on the device that was current at vate_create; h_* are HOST
 *     pointers (page-locked memory gives copy/compute overlap; pageable
 *     memory works but the copies become synchronous).
 *   - Caller-owned buffers stay owned by the caller and must stay valid until
 *     the work queued on `stream` has finished.  The library owns the AT pool,
 *     BACT^0, the census and its staging buffers.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  All device work is queued asynchronously on it, in
 *     call order.  Calls on one handle must be made from one host thread at a
 *     time, in slice order (the slice state machine lives on the host).
 *   - Every function returns VATE_OK (0) or one of the VATE_E* codes;
 *     argument and state checks are made on the host before anything is
 *     queued, so an error return leaves the handle unchanged.
 *     vate_last_error() gives a message for the calling thread.
 *   - Numbers follow the paper's notation: c (log2 of the pool size P),
 *     k (longest window), k' (window of one estimate), g (VATs per host).
 *
 * AT width: for k <= 63 the pool is uint8_t[P], one AT value (0..2k) per
 * byte (2k+1 values below 128; the device compares 4 ATs per 32-bit word);
 * for 64 <= k <= 1023 (e.g. the paper's k' = 300, Sec. 5) it is uint16_t[P]
 * (two ATs per word).  The paper packs ceil(log2(2k+1)) bits per AT
 * (Sec. 4.2); the state is the same AT value per index.
 */
#ifndef VATE_H
#define VATE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes --------------------------------------------------- */
#define VATE_OK        0
#define VATE_EINVAL    1   /* bad argument (range, alignment, NULL)            */
#define VATE_ENOMEM    2   /* device or host allocation failed                 */
#define VATE_ESLICE    3   /* slice out of order, slice already closed, or an
                              estimate before any close                        */
#define VATE_ECUDA     4   /* a CUDA runtime call failed (no device, bad stream,
                              launch failure); see vate_last_error()           */
#define VATE_ETIMEOUT  5   /* a bounded device-side wait gave up               */
#define VATE_EDROPPED  6   /* a serving request dropped by an injected fault
                              (vate_server_inject, include/vate_server.h)      */

/* ---- per-host flags written by vate_estimate ------------------------- */
#define VATE_FLAG_SAT       1u  /* every VAT of the host active: V0 read as 1  */
#define VATE_FLAG_POOLFULL  2u  /* no inactive AT in the pool: N0 read as 1    */

/* One IPv4 address pair <aip, bip> extracted from a packet: 8 bytes, aip
 * first (Sec. 4.2: the host-to-GPU buffers hold r such pairs). */
typedef struct {
    uint32_t aip;
    uint32_t bip;
} vate_pair;

/* Construction parameters.
 *   log2_pool  c: the pool holds P = 2^c ATs, 12 <= c <= 32 (Sec. 4.1).
 *   k          longest window in slices, 1 <= k <= 1023; ATs hold 0..2k (Sec. 3),
 *              one byte each for k <= 63, two bytes beyond.
 *   g          virtual ATs per host, 1 <= g <= 65536, a multiple of seg_len.
 *   seg_len    L: VAT i of a host lives at offset (i mod L) of the pool segment
 *              chosen for (aip, floor(i/L)).  L = 1 is fully random placement
 *              (the paper's H); L = 32 puts 32 VATs in one 32-byte L2 sector.
 *              Power of two, 1 <= L <= 64, and c - log2(L) >= 1.
 *   partition  0: blocks of Eq. 9-10 (2k-1 blocks of a = floor(P/(2k-1)) ATs
 *              and a last block of b = P mod (2k-1)); 1: the low-deviation
 *              partition of Sec. 4.1 (block sizes P/(2k) or P/(2k)+1).
 *              Either way every block must hold at least 32 ATs.
 *   counter    0 (VATE_COUNTER_AT): asynchronous timestamps, values 0..2k,
 *              maintained once every k slices per block (Sec. 3, Algorithm 3);
 *              1 (VATE_COUNTER_DR): distance recorders, values 0..k (k =
 *              inactive), reset to 0 by SetAT and aged by one in every slide,
 *              the whole pool each slice (Sec. 1; the VDRE of Sec. 5).  Both
 *              give the same active sets, censuses and estimates; they differ
 *              in the maintenance work per slide.
 *   at_bits    0: one byte per AT for k <= 63, two beyond (the fast layout).
 *              b with ceil(log2(2k+1)) <= b <= 16: the paper's packed layout
 *              (Sec. 4.2) -- floor(32/b) b-bit fields per 32-bit word, no field
 *              across words (5.33 bits per AT for k = 10, 10.67 for k = 300);
 *              b = 8 and b = 16 are the byte and 16-bit layouts themselves.
 *              A packed pool takes SetAT as two atomic bit operations per
 *              pair and reads one field per VAT: less memory, more time.
 *              Packed pools serve the handle API; shards, groups, per-age
 *              counts and the learned estimator need b = 8 or 16.
 *   options    bit set, 0 by default:
 *              VATE_OPT_PERSIST_L2  keep the pool resident in L2 across
 *                slices: the pool's kernels carry a persisting access-policy
 *                window over it, and the handle holds the device's
 *                PROCESS-WIDE persisting-L2 limit (cudaLimitPersistingL2-
 *                CacheSize) at the device maximum: the first such handle (or
 *                monitor group) raises it, the last one destroyed resets the
 *                persisting lines (cudaCtxResetPersistingL2Cache) and puts
 *                back the limit it found.  While held, the set-aside changes
 *                L2 behaviour for every kernel of the calling process, so
 *                the library does it only when asked.  Without the bit no
 *                process-wide setting is touched and the pool's kernels carry
 *                no window.
 *              Other bits must be 0.
 *   seed       keys the hash functions H and BH.
 * The hash functions (Sec. 4.1 leaves them open):
 *   mix(x)    = SplitMix64 output function (Steele, Lea & Flood 2014)
 *   fmix32(x) = MurmurHash3's 32-bit finalizer (Appleby)
 *   BH(bip)   = ((mix(mix(seed+2) ^ bip) >> 32) * g) >> 32
 *   K         = mix(mix(seed+1) ^ (aip << 32))            (one key per host)
 *   seg       = (fmix32(lo32(K) ^ j * 0x9E3779B9) ^ hi32(K)) >> (32 - (c - log2 L)),
 *               j = floor(i/L), arithmetic on 32-bit words
 *   H(aip,i)  = seg * L + (i mod L)                                          */
typedef struct {
    uint32_t log2_pool;
    uint32_t k;
    uint32_t g;
    uint32_t seg_len;
    uint32_t partition;
    uint32_t counter;    /* VATE_COUNTER_AT (0) or VATE_COUNTER_DR (1) */
    uint32_t at_bits;    /* 0: byte / 16-bit ATs by k; else packed b-bit fields */
    uint32_t options;    /* VATE_OPT_* bits, 0 by default */
    uint64_t seed;
} vate_params;

#define VATE_COUNTER_AT 0u
#define VATE_COUNTER_DR 1u

#define VATE_OPT_PERSIST_L2 1u  /* vate_params.options: see above */

/* Read-only view of a handle's geometry and slice state. */
typedef struct {
    uint64_t pool_size;      /* P = 2^c                                       */
    uint64_t block_a;        /* a (Eq. 9) or a' (low-deviation)               */
    uint64_t block_b;        /* b (Eq. 10) or b'                              */
    int64_t  slice;          /* current slice, -1 before the first call       */
    uint32_t bact0;          /* BACT^0 of the current slice (Eq. 7)           */
    uint32_t closed;         /* 1 when the current slice has been closed      */
    uint64_t pid_lo, pid_hi; /* positions held: [0, P), or a shard's range    */
} vate_info;

typedef struct vate_handle vate_handle;

/* Allocate the AT pool (P bytes of device memory, 256-byte aligned) and run
 * InitAT on every AT: all values become 2k, BACT^0 = 0 (Algorithm 4, start).
 * The first slice number passed to vate_ingest/vate_close_slice becomes
 * slice 0 of Algorithm 4.  Errors: VATE_EINVAL (parameters), VATE_ENOMEM,
 * VATE_ECUDA.  *out is set only on success. */
int vate_create(const vate_params *params, void *stream, vate_handle **out);
/* The handle belongs to the device current at creation: every later call that
 * queues work on it must be made with that device current (the library never
 * switches the calling thread's device); otherwise VATE_EINVAL. */

/* Free the pool and every buffer of the handle (synchronises the device work
 * of the handle first).  NULL is accepted. */
int vate_destroy(vate_handle *h);

/* Scan n pairs of slice `slice` (Algorithm 4, scan loop; Sec. 4.2 "scanning
 * IP address pairs"): for each pair, vid = BH(bip), pid = H(aip, vid), and
 * SetAT(ATP[pid]) writes the ACT of pid's block, (BACT^0 + block) mod 2k.
 *   d_pairs  device array of n vate_pair (8-byte aligned); n = 0 is allowed.
 *   slice    >= the current slice.  Moving to a later slice first slides the
 *            window once per slice passed (BACT^0 + 1, then PreserveAT on the
 *            two blocks whose ACT became 0 or k: Algorithm 4, Algorithm 3),
 *            so no maintenance point is skipped (Corollary 1).
 * Several calls per slice are allowed.  Concurrent SetATs on one AT write the
 * same value, so the pool does not depend on pair order (Sec. 4.2).
 * Errors: VATE_ESLICE if slice < current, or == current after it was closed. */
int vate_ingest(vate_handle *h, const vate_pair *d_pairs, uint64_t n, int64_t slice, void *stream);

/* Close slice `slice` (sliding first, as in vate_ingest, if it is later than
 * the current one) and take the pool census used by Z_p (Eq. 11): the number
 * of pool ATs at each distance d = (ACT + 2k - value) mod 2k, 0 <= d < 2k,
 * and the number of inactive ATs.  After a close, vate_estimate may be called
 * any number of times until the next ingest/close moves to a later slice.
 * Errors: VATE_ESLICE if slice < current or already closed. */
int vate_close_slice(vate_handle *h, int64_t slice, void *stream);

/* Estimate |OP(aip, t-k'+1, k')| for n hosts at the end of the closed slice t
 * (Algorithm 4, estimation loop; Eq. 11 read as g ln Z_p - g ln Z_v):
 *   A   = #{ i < g : CheckAT(ATP[H(aip, i)], k') }          (Algorithm 1)
 *   Z_v = (g - A) / g,  Z_p = N0 / P, N0 = inactive pool ATs for k'
 *   out = g * log1p((N0*g - V0*P) / (V0*P)), V0 = g - A, evaluated in FP32
 *         from exact integers (V0 = 0 -> 1 with VATE_FLAG_SAT, N0 = 0 -> 1
 *         with VATE_FLAG_POOLFULL).
 *   d_aips   device uint32[n] host addresses; d_out device float[n];
 *   d_flags  device uint8[n] or NULL.  1 <= kprime <= k.
 * Errors: VATE_ESLICE if the current slice has not been closed. */
int vate_estimate(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint32_t kprime,
                  float *d_out, uint8_t *d_flags, void *stream);

/* Same gather as vate_estimate, returning the active VAT count A of each host
 * (d_active device uint32[n]) instead of the estimate. */
int vate_active_counts(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint32_t kprime,
                       uint32_t *d_active, void *stream);

/* Per-age VAT counts of each host at the end of the closed slice:
 * d_counts[i*k + d] = number of host i's g VATs whose distance is exactly d
 * (last set d slices ago), 0 <= d < k; the active count for window k' is the
 * sum of the first k' entries.  d_counts is device uint16[n*k] (g <= 65535
 * and k <= 63 are required here). */
int vate_age_counts(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint16_t *d_counts, void *stream);

/* Copy the census of the last close into d_hist (device uint64[2k+1]):
 * d_hist[d] for distances 0 <= d < 2k, d_hist[2k] = inactive ATs. */
int vate_census(vate_handle *h, uint64_t *d_hist, void *stream);

/* Copy the AT pool (device uint8[P] for k <= 63, else uint16[P], 2-byte
 * aligned) to d_dst, or overwrite it from d_src, in the paper's form: byte pid holds the AT value of pool
 * position pid (an ACT of its block, Sec. 3, or 2k when inactive; a distance
 * recorder's value for VATE_COUNTER_DR).  Inside the library a timestamp pool
 * is kept in the frame of block 0 -- value minus block index, mod 2k -- so
 * that every AT is read with ACT = BACT^0; these calls convert.  Values above
 * the counter's range in d_src are loaded as inactive. */
int vate_copy_pool(vate_handle *h, uint8_t *d_dst, void *stream);
int vate_load_pool(vate_handle *h, const uint8_t *d_src, void *stream);

/* End-to-end forms with host buffers: the pairs (or hosts) are copied to the
 * device in chunks through device staging buffers on internal copy streams,
 * overlapping the copy of chunk i+1 with the kernel of chunk i (the double
 * buffer of Sec. 4.2, with larger chunks and more buffers).
 * vate_ingest_host: 2^20 pairs per chunk, a ring of six 8 MiB buffers on a
 * stream of their own, so that the pairs of the next slice (up to 6M) are
 * copied while the current slice is still being estimated.
 * vate_estimate_host: 2^18 hosts per chunk through two buffers; the estimates
 * (and flags, if h_flags is not NULL) go back on a third internal stream,
 * overlapping the gather of the next chunk.
 * The staging buffers (52 MiB) are allocated on the first call.  Results are
 * valid once `stream` has been synchronised; host buffers in page-locked
 * memory let the copies run asynchronously.  The host buffer of a call must
 * stay unchanged until `stream` reaches the call. */
int vate_ingest_host(vate_handle *h, const vate_pair *h_pairs, uint64_t n, int64_t slice, void *stream);
int vate_estimate_host(vate_handle *h, const uint32_t *h_aips, uint64_t n, uint32_t kprime,
                       float *h_out, uint8_t *h_flags, void *stream);

/* Geometry and slice state of a handle (host only, never blocks). */
int vate_get_info(const vate_handle *h, vate_info *out);

/* Host-side evaluation of the mapping the device uses, for checks without a
 * GPU: H(aip, i), BH(bip) and the block of a pool position for `params`. */
int vate_host_h(const vate_params *params, uint32_t aip, uint32_t i, uint64_t *pid);
int vate_host_bh(const vate_params *params, uint32_t bip, uint32_t *vid);
int vate_host_block(const vate_params *params, uint64_t pid, uint32_t *block);

/* Pool census into caller-owned buffers, allocating no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let a library call cudaMalloc -- a packet-processing loop with a
 * latency budget (cudaMalloc can synchronise the device and its duration is
 * unbounded), or an application whose device memory is owned entirely by its
 * own allocator (a caching allocator or a fixed arena), so that nothing is
 * left for a library to request.  It needs no handle either.
 *   params   geometry of the pool (log2_pool, k and partition are used; the
 *            whole struct is validated as for vate_create).
 *   d_pool   device uint8[P], 16-byte aligned, in the paper's form: AT values
 *            in [0, 2k] (a distance recorder's in [0, k]); larger bytes are
 *            counted as inactive.
 *   bact0    BACT^0 of the slice the pool belongs to, 0 <= bact0 < 2k.
 *   d_hist   device uint64[2k+1]: receives the same census as vate_census
 *            (d_hist[d] for distances 0 <= d < 2k, d_hist[2k] inactive).
 * Scratch: the counters the census blocks add into (127 x 8 bytes) and a
 * "blocks finished" counter live in one static device array of 1,272 bytes,
 * which every GPU that loads the library holds until the process exits.  A
 * request needing more than 127 bins (k > 63) is rejected with VATE_EINVAL.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current) and caches it; make that
 * first call before any stream capture.  Every call reuses the same array and
 * clears it first, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race: order them on one stream.  No
 * cudaMalloc, cudaFree or allocating library routine is called. */
int vate_census_noalloc(const vate_params *params, const uint8_t *d_pool, uint32_t bact0, uint64_t *d_hist,
                        void *stream);

/* ---- the checked build --------------------------------------------------
 * The paper has no counterpart; these stand in for a memory checker, which
 * this GPU pool does not offer.  Built with VATE_DEBUG defined (the library
 * libvate_debug.so beside libvate.so), the kernels check what their indexing
 * relies on -- every computed pool position below P, every AT value they read
 * within the counter's range (2k for timestamps, k for recorders), every block
 * index below 2k -- and on a violation record it in the handle's status words
 * instead of trapping: a bad position's access is skipped, a bad value is read
 * as it is (no kernel leaves its buffers whatever a value holds).  Without
 * VATE_DEBUG the checks are compiled out and the status stays 0. */
#define VATE_DBG_POSITION 1u   /* a computed pool position outside the pool (access skipped) */
#define VATE_DBG_VALUE    2u   /* an AT value above the counter's range                        */
#define VATE_DBG_BLOCK    4u   /* a block index outside [0, 2k)                                */

/* 1 if this library was built with the checks, else 0. */
int vate_debug_checks(void);

/* The VATE_DBG_* bits recorded on the handle's device work so far (OR-ed) and,
 * in *first (may be NULL), the first report: bit 63 set, the VATE_DBG_* bit in
 * bits 56-62, the pool position (or 16-byte chunk, or segment) in bits 0-55.
 * clear = 1 resets both.  Synchronises `stream`. */
int vate_debug_status(vate_handle *h, uint32_t *bits, uint64_t *first, int clear, void *stream);

/* Checked build only: overwrite the stored value of pool position pid with
 * `value` as it is (no range check, no frame conversion) -- a deliberate
 * corruption for tests of the checks.  Synchronises `stream`.  Elsewhere, and
 * for packed pools, VATE_EINVAL. */
int vate_debug_poke(vate_handle *h, uint64_t pid, uint32_t value, void *stream);

/* Message of the last error on the calling thread ("" if none). */
const char *vate_last_error(void);

/* Number of kernels this library has launched in the process so far. */
uint64_t vate_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* VATE_H */
