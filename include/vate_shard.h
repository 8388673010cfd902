/*
 * vate_shard.h -- one VATE pool held by several devices, split by position.
 *
 * The paper runs one pool on one GPU (Sec. 4.2).  A pool larger than one
 * device's memory, or a monitor whose gather must run on several devices,
 * can be split by pool position: shard r holds the ATs of positions
 * [lo_r, hi_r), and every shard sees every pair.  All of the method's
 * per-position work is local:
 *   - SetAT (Algorithm 4, scan) writes a position only on the shard that holds
 *     it;
 *   - a slide (BACT^0 + 1, Algorithm 3) maintains each shard's part of the two
 *     blocks whose ACT became 0 or k -- blocks are ranges of positions
 *     (Eq. 9-10), so a block may span shards;
 *   - the census (the Z_p of Eq. 11) and the count A of a host's active VATs
 *     (Algorithm 1 over its g VATs) are sums over positions, so each shard
 *     gives the part over its own positions (vate_census, vate_active_counts
 *     on the shard handle).
 * Summing the shards' censuses and counts (one all-reduce each, integers, so
 * the order of the sums does not matter) gives exactly the census and counts
 * of one undivided pool; vate_estimate_from_counts turns them into the
 * estimates of Eq. 11, equal bit for bit to vate_estimate on one handle.
 *
 * Shard boundaries are multiples of 64 positions, so a segment of L <= 64
 * VATs (and a 16-byte chunk) lies on one shard.  A shard handle accepts
 * vate_ingest(_host), vate_close_slice, vate_active_counts, vate_census,
 * vate_copy_pool / vate_load_pool (its own positions) and vate_get_info;
 * vate_estimate(_host), vate_age_counts, checkpoints and the learned
 * estimator need the whole pool and return VATE_EINVAL on a shard.
 */
#ifndef VATE_SHARD_H
#define VATE_SHARD_H

#include <stdint.h>
#include "vate.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Create the shard of the pool described by `params` that holds positions
 * [pid_lo, pid_hi) on the current device: pid_lo < pid_hi <= P, pid_lo a
 * multiple of 64, pid_hi a multiple of 64 or P.  Device memory: (pid_hi -
 * pid_lo) ATs plus the census buffers.  Every shard of one pool must get the
 * same params (the same hashes and blocks) and the same pairs, slices and
 * calls.  Errors: VATE_EINVAL, VATE_ENOMEM, VATE_ECUDA. */
int vate_create_shard(const vate_params *params, uint64_t pid_lo, uint64_t pid_hi, void *stream, vate_handle **out);

/* Eq. 11 from counts: d_out[i] = g ln(Z_p / Z_v) with Z_v = (g - d_active[i]) / g
 * and Z_p = N0 / P, N0 = P - sum_{d < kprime} d_hist[d]; the same FP32
 * evaluation and SAT / POOLFULL flags as vate_estimate.
 *   params    the pool's parameters (g, k and P are used; validated as for
 *             vate_create).
 *   d_active  device uint32[n], A of each host, d_active[i] <= g.
 *   d_hist    device uint64[2k+1], the census of the whole pool.
 *   d_out     device float[n]; d_flags device uint8[n] or NULL.
 * Needs no handle and allocates nothing.  Errors: VATE_EINVAL, VATE_ECUDA. */
int vate_estimate_from_counts(const vate_params *params, const uint32_t *d_active, const uint64_t *d_hist, uint64_t n,
                              uint32_t kprime, float *d_out, uint8_t *d_flags, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VATE_SHARD_H */
