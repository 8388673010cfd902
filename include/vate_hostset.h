/*
 * vate_hostset.h -- the close of a fixed list of hosts through a prebuilt
 * index of their VAT positions.
 *
 * A host's virtual vector is fixed: VAT i of host aip always sits at pool
 * position H(aip, i) (Sec. 4.1), whatever the traffic.  A monitor that
 * estimates the same hosts at every close (every host of a link, say) can
 * therefore sort the positions of all their VATs once, by pool region, and
 * at each close compute the same counts A (Algorithm 1 over each host's g
 * VATs) region by region:
 *   1. the pool's CheckAT bitmap for k' -- one bit per AT, set when the AT is
 *      active (Eq. 5 distance below k'), 2^c / 8 bytes -- in one pass over the
 *      pool;
 *   2. for every region of the bitmap that fits in one SM's shared memory
 *      (1.5 M ATs), the region is loaded into shared memory and the index
 *      entries of every host's segments in that region are streamed from HBM,
 *      each looked up in shared memory; a host's count is the sum over the
 *      regions;
 *   3. Eq. 11 from the counts and the census (vate_estimate_from_counts).
 * The counts are the same integers the per-host gather computes, so the
 * estimates and flags equal vate_estimate's bit for bit.  The gather reads
 * g / L random 32-byte sectors per host, and for segments of at most 8 ATs
 * its speed is set by the SMs' random-sector rate; the index is read in
 * order instead, at HBM streaming rate, and the random lookups go to shared
 * memory.  The index holds one 21-bit entry per segment of every host (the
 * segment's offset in its region), six to 16 bytes, with a host's entries of
 * a region (a cell) padded to whole 16-byte units and the cells of a region
 * in tiles of 32 of about the same size, plus 4 bytes per cell: about
 * 2.8 n g / L bytes, 11.9 GB for 2^20 hosts with g = 4096 and L = 1.
 *
 * Conventions are those of vate.h.  A hostset belongs to the handle it was
 * built for and to the device that was current then; destroy it before that
 * handle (it keeps the handle's address to refuse other handles).
 */
#ifndef VATE_HOSTSET_H
#define VATE_HOSTSET_H

#include <stdint.h>
#include "vate.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vate_hostset vate_hostset;

/* Build the index of the n hosts d_aips (device uint32[n], any order,
 * repeats allowed) for the pool of handle h: their positions depend only on
 * the handle's parameters, so the handle's state (slice, pool contents) does
 * not matter and the index stays valid for the handle's whole life.  Needs a
 * handle of byte ATs (k <= 63, at_bits 0 or 8) over the whole pool, seg_len
 * 1, 2, 4 or 8, and at most 2^31 - 1 hosts.  Device memory: the index (about
 * 2.8 n g / seg_len bytes with its tile tables), the bitmap (2^c / 8 bytes)
 * and 4 n bytes of counts, which vate_hostset_info reports; while it builds,
 * also 4 n bytes per region.  Synchronises `stream`; the build takes about a
 * second for 2^20 hosts with g = 4096, seg_len 1.  Errors: VATE_EINVAL
 * (handle, parameters, NULL pointers, more than 2^32 rows of index),
 * VATE_ENOMEM, VATE_ECUDA. */
int vate_hostset_create(vate_handle *h, const uint32_t *d_aips, uint64_t n, void *stream, vate_hostset **out);

/* Free everything of the hostset (after its queued work).  NULL is accepted. */
int vate_hostset_destroy(vate_hostset *s);

/* Device bytes held by the hostset, and its number of hosts and regions. */
int vate_hostset_info(const vate_hostset *s, uint64_t *bytes, uint64_t *n_hosts, uint32_t *regions);

/* The estimates of Eq. 11 for window kprime (1 <= kprime <= k) of the
 * hostset's hosts, in their order, at the end of the closed slice: the same
 * values and flags as vate_estimate(h, d_aips, n, kprime, d_out, d_flags) for
 * the list the hostset was built from.
 *   d_out     device float[n]; d_flags device uint8[n] or NULL;
 *   d_active  device uint32[n] or NULL: the counts A as vate_active_counts.
 * Asynchronous on `stream`; calls on one hostset must not overlap on the GPU
 * (they share its bitmap and counts).  Errors: VATE_EINVAL (another handle's
 * hostset, kprime), VATE_ESLICE (slice not closed), VATE_ECUDA. */
int vate_estimate_hostset(vate_handle *h, vate_hostset *s, uint32_t kprime, float *d_out, uint8_t *d_flags,
                          uint32_t *d_active, void *stream);

/* vate_estimate_hostset with the results in host memory: h_out (float[n])
 * and h_flags (uint8[n], may be NULL) are written by copies queued on
 * `stream` after the kernels (page-locked buffers make them asynchronous;
 * the caller synchronises `stream` before reading).  The device side goes
 * through buffers of the hostset (5 n bytes, allocated on the first call).
 * Errors: as vate_estimate_hostset, and VATE_ENOMEM. */
int vate_estimate_hostset_host(vate_handle *h, vate_hostset *s, uint32_t kprime, float *h_out, uint8_t *h_flags,
                               void *stream);

/* vate_estimate_hostset_host whose copies overlap the caller's next work:
 * the kernels run on `stream` into one of two device buffers of the hostset
 * (in turn), and the copies to h_out / h_flags are queued on a stream of the
 * hostset after them, so that work queued next on `stream` (the next slice's
 * ingest and close) does not wait for them.  The host buffers hold the
 * results once vate_hostset_wait returns (synchronising `stream` is not
 * enough); a call waits on the device for the copies of the call before last,
 * whose buffer it reuses.  The buffers of two calls in flight must differ.
 * Device memory: 10 n bytes, allocated on the first call.  Errors: as
 * vate_estimate_hostset_host. */
int vate_estimate_hostset_host_async(vate_handle *h, vate_hostset *s, uint32_t kprime, float *h_out, uint8_t *h_flags,
                                     void *stream);

/* Block until every copy queued by vate_estimate_hostset_host_async on this
 * hostset is in host memory.  Errors: VATE_EINVAL (NULL), VATE_ECUDA. */
int vate_hostset_wait(vate_hostset *s);

/* Time the index pass (the tile pass over the bitmap, or the age pass) of
 * the next n calls that run it through this hostset (vate_estimate_hostset
 * and its host forms; vate_age_counts_hostset, vate_estimate_learned_hostset)
 * (n <= 4096; 0 stops):
 * CUDA events recorded on the caller's stream before and after it, so that
 * the pass's own duration is known beside the whole call's.  Restarts the
 * count.  Errors: VATE_EINVAL, VATE_ENOMEM (events). */
int vate_hostset_time_passes(vate_hostset *s, uint32_t n);

/* The pass durations recorded since vate_hostset_time_passes, in ms, in the
 * order of the calls: min(max, recorded) of them into ms[], their number in
 * *count.  Waits for the recorded events.  Errors: VATE_EINVAL, VATE_ECUDA. */
int vate_hostset_pass_times(vate_hostset *s, float *ms, uint32_t max, uint32_t *count);

/* An age index: the same index over regions of 384 K ATs, looked up in the
 * pool's age map (4 bits per AT: the AT's distance d when d < k, else 15;
 * 192 KiB per region) instead of the CheckAT bitmap, so that one pass gives
 * every host's per-age counts.  It serves vate_estimate_hostset (A for k' is
 * the sum of the ages below k'), vate_age_counts_hostset and
 * vate_estimate_learned_hostset.  Needs, beyond vate_hostset_create's
 * conditions, k <= 15 and g <= 65535; device memory as vate_hostset_create's
 * (with an age map of 2^c / 2 bytes) and 32 n bytes of counts.  Errors: as
 * vate_hostset_create. */
int vate_hostset_create_ages(vate_handle *h, const uint32_t *d_aips, uint64_t n, void *stream, vate_hostset **out);

/* vate_age_counts for an age index's hosts, in their order: d_counts device
 * uint16[n * k], d_counts[i k + d] the host's VATs at distance d.
 * Asynchronous on `stream`.  Errors: VATE_EINVAL (not an age index, another
 * handle's hostset, NULL d_counts), VATE_ESLICE (slice not closed),
 * VATE_ECUDA. */
int vate_age_counts_hostset(vate_handle *h, vate_hostset *s, uint16_t *d_counts, void *stream);

/* vate_estimate_learned (include/vate_learned.h) for an age index's hosts:
 * the same values and flags bit for bit, from the per-age counts of one pass
 * over the index; each host's feature row is built from its counts in shared
 * memory, beside the model (no scratch).  Errors: as
 * vate_estimate_learned, and VATE_EINVAL for a hostset that is not an age
 * index or was built for another handle. */
int vate_estimate_learned_hostset(vate_handle *h, vate_hostset *s, const float *d_params, float *d_out,
                                  uint8_t *d_flags, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VATE_HOSTSET_H */
