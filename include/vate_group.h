/*
 * vate_group.h -- many independent VATE monitors advanced together.
 *
 * A group holds M independent monitors (for instance one per router or link),
 * each with its own pool size 2^c, window k, virtual-vector length g and hash
 * seed, and runs the per-slice pipeline of Algorithm 4 -- slide (BACT^0 + 1,
 * PreserveAT on the two blocks whose ACT became 0 or k), SetAT for every pair,
 * pool census, CheckAT gather and Eq. 11 for every host -- for all of them in
 * ONE persistent launch per slice.  Its blocks take (monitor, phase, tile)
 * work items -- begin, PreserveAT, SetAT, census -- in order from a device
 * queue, monitor after monitor; an item starts once the earlier phases of its
 * monitor have finished (a bounded device-side wait on a per-monitor count of
 * finished items, which can only wait on items already handed to running
 * blocks).  A block that finds the queue empty gathers: each of its warps
 * takes a few hosts at a time, monitor after monitor, once every item of the
 * monitor has finished (the same bounded wait).  Every monitor computes
 * exactly what a single vate_handle with the same parameters computes (the
 * same device arithmetic); a monitor's result does not depend on the other
 * monitors in the group.
 *
 * All monitors advance in lock step, one slice per vate_group_step call: the
 * first step is slice 0 (BACT^0 = 0 for every monitor), step s is slice s.
 * Everything a step reads that changes from slice to slice -- the slice
 * number, the per-monitor batch boundaries, k' -- lives in device memory, so a
 * step can be captured once as a CUDA graph and replayed every slice
 * (vate_group_step_graph) while batch sizes vary.
 *
 * Conventions are those of vate.h (device pointers d_*, asynchronous on
 * `stream`, VATE_* return codes, vate_last_error()).  Values that live in
 * device memory cannot be checked on the host: a step clamps them to the
 * capacities it was given and records what it found in a status word
 * (vate_group_status); it never reads or writes outside the caller's buffers.
 */
#ifndef VATE_GROUP_H
#define VATE_GROUP_H

#include <stdint.h>
#include "vate.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vate_group vate_group;

/* Status bits recorded by a step (sticky until read with clear = 1). */
#define VATE_GROUP_BAD_OFFSETS  1u   /* pair or host offsets decreasing or beyond capacity (clamped) */
#define VATE_GROUP_BAD_KPRIME   2u   /* k' outside [1, k] for some monitor (k used instead)          */
#define VATE_GROUP_TIMEOUT      4u   /* a device-side wait of a step gave up (see vate_group_set_wait):
                                        that step is incomplete and the group does no further work --
                                        destroy it (a checkpoint of each monitor is the way back)      */

/* Tiling of the step kernel, chosen by vate_group_autotune or set by hand.
 *   census_tile_chunks    16-byte chunks per census work item (power of two, 256..65536)
 *   blocks_per_sm         persistent grid: blocks of 256 threads per SM (1 .. the kernel's occupancy)
 *   gather_grab_hosts     hosts a warp takes at a time for g = 4096 (1..32); a monitor with g VATs
 *                         per host gives 4096 / g times as many (at least 1, at most 32)
 *   ingest_tile_pairs     pairs per SetAT work item (multiple of 256, 256..65536)
 *   preserve_tile_chunks  16-byte chunks per PreserveAT work item (multiple of 256, 256..65536)
 *   wave_pool_mib         work order: consecutive monitors whose pools add up to at most this many MiB
 *                         form a wave; the SetAT items of wave s are listed before the census
 *                         items of wave s - 1, so that a census reads pools SetAT has just
 *                         written; 0: one wave of all monitors (0..65536) */
typedef struct {
    uint32_t census_tile_chunks;
    uint32_t blocks_per_sm;
    uint32_t gather_grab_hosts;
    uint32_t ingest_tile_pairs;
    uint32_t preserve_tile_chunks;
    uint32_t wave_pool_mib;
} vate_group_tuning;

/* Create a group of n_monitors (1..256) monitors; params[m] as for
 * vate_create, all with the same seg_len.  The pools live in one device
 * allocation (each 256-byte aligned) and are initialised (InitAT) on `stream`.
 * Errors: VATE_EINVAL (any parameter, mixed seg_len), VATE_ENOMEM, VATE_ECUDA. */
int vate_group_create(const vate_params *params, uint32_t n_monitors, void *stream, vate_group **out);

/* Free everything of the group (synchronises its device work first).  NULL is accepted. */
int vate_group_destroy(vate_group *g);

/* One slice for every monitor.
 *   d_pairs         device vate_pair[pair_capacity]: the pairs of monitor m are
 *                   d_pairs[d_pair_offsets[m] .. d_pair_offsets[m+1]).
 *   d_pair_offsets  device uint64[M+1], non-decreasing, last <= pair_capacity.
 *   d_hosts         device uint32[host_capacity]: hosts of monitor m at
 *                   d_hosts[d_host_offsets[m] .. d_host_offsets[m+1]).
 *   d_host_offsets  device uint64[M+1], non-decreasing, last <= host_capacity.
 *   d_kprime        device uint32[M]: window k' of each monitor's estimates.
 *   d_out, d_flags  device float[host_capacity], uint8[host_capacity] (flags may
 *                   be NULL): estimate and VATE_FLAG_* of each host, same index.
 * Capacities are host values (buffer sizes); the offsets are read on the device. */
int vate_group_step(vate_group *g, const vate_pair *d_pairs, const uint64_t *d_pair_offsets, uint64_t pair_capacity,
                    const uint32_t *d_hosts, const uint64_t *d_host_offsets, uint64_t host_capacity,
                    const uint32_t *d_kprime, float *d_out, uint8_t *d_flags, void *stream);

/* The same step as a CUDA graph: the first call (and any call whose buffers,
 * tuning or wait settings differ from the previous one) captures the step's
 * one launch on an internal stream and instantiates the graph; every call
 * launches the graph on `stream`.  Refill the same buffers (pairs, offsets,
 * hosts, k') between slices to keep replaying one graph. */
int vate_group_step_graph(vate_group *g, const vate_pair *d_pairs, const uint64_t *d_pair_offsets,
                          uint64_t pair_capacity, const uint32_t *d_hosts, const uint64_t *d_host_offsets,
                          uint64_t host_capacity, const uint32_t *d_kprime, float *d_out, uint8_t *d_flags,
                          void *stream);

/* Project-written autotuner: after at least one step, repeats that step (same
 * slice: a second PreserveAT of the same slide changes nothing, a repeat of
 * the same SetATs writes the same values, the census and the gather recompute
 * the same outputs) under candidate tilings -- blocks per SM {2 .. 4} within
 * the kernel's occupancy, waves {0, 32 MiB}, census tiles {4,096, 16,384},
 * gather grabs {2, 4, 8}, ingest tiles {4,096, 16,384, 65,536} -- times each
 * as the best of three replays with CUDA events on `stream` (synchronising
 * it), keeps the fastest and writes it to *chosen (may be NULL).  The
 * monitors' state and the outputs end exactly as the last step left them.
 * The inputs MUST be exactly those of the last vate_group_step (same pairs,
 * offsets, hosts, host offsets and k'): other pairs would be stamped into the
 * current slice, which is not checked.  On an error the tiling in force on
 * entry is restored. */
int vate_group_autotune(vate_group *g, const vate_pair *d_pairs, const uint64_t *d_pair_offsets,
                        uint64_t pair_capacity, const uint32_t *d_hosts, const uint64_t *d_host_offsets,
                        uint64_t host_capacity, const uint32_t *d_kprime, float *d_out, uint8_t *d_flags,
                        vate_group_tuning *chosen, void *stream);

int vate_group_set_tuning(vate_group *g, const vate_group_tuning *t);
int vate_group_get_tuning(const vate_group *g, vate_group_tuning *t);

/* Bounded waits of the step kernel.  Each work item's wait for the earlier
 * phases of its monitor sleeps ~128 ns between looks and gives up after
 * spin_limit looks (default 2^23, about a second; 0 gives up at the first
 * unsatisfied look): the step then sets VATE_GROUP_TIMEOUT, every later wait
 * of the launch gives up at once, and the kernel returns instead of hanging.
 * `missing` > 0 raises every wait's target by that many items, a target no
 * step can reach: a test of the timeout path that needs no fault.  Both
 * apply to later steps (a graph is re-captured).  Errors: VATE_EINVAL. */
int vate_group_set_wait(vate_group *g, uint64_t spin_limit, uint32_t missing);

/* Trace of later steps, for tuning: work item j of a step writes four words
 * at d_trace[4j..4j+3] (device uint64): the %globaltimer nanoseconds when it
 * was handed out, when its wait for the earlier phases of its monitor ended
 * and when it finished, then (SM << 32) | (monitor << 8) | phase (0 begin,
 * 1 PreserveAT, 2 SetAT, 3 census).  Then, with n the step's item count,
 * block b writes its gather at d_trace[4(n + b)..]: the start twice, the
 * end, then (SM << 32) | (0xFFFFFF << 8) | 4.  Only entries below capacity
 * are written (clear the buffer first to tell them apart); capacity 0 stops
 * tracing.  Errors: VATE_EINVAL. */
int vate_group_set_trace(vate_group *g, uint64_t *d_trace, uint32_t capacity);

/* Kernel nodes of the captured step graph (0 before the first
 * vate_group_step_graph): one, the step's persistent launch. */
int vate_group_graph_nodes(const vate_group *g, uint32_t *nodes);

/* Status bits of the steps since the last clear (synchronises `stream`);
 * VATE_GROUP_TIMEOUT is never cleared. */
int vate_group_status(vate_group *g, uint32_t *status, int clear, void *stream);

/* Per-monitor views for checking: the pool (P_m bytes), the census of the last
 * step (uint64[2k_m+1]), and geometry + slice (slice from the device; synchronises `stream`). */
int vate_group_copy_pool(vate_group *g, uint32_t m, uint8_t *d_dst, void *stream);
int vate_group_census(vate_group *g, uint32_t m, uint64_t *d_hist, void *stream);
int vate_group_monitor_info(vate_group *g, uint32_t m, vate_info *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VATE_GROUP_H */
