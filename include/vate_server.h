/*
 * vate_server.h -- a serving loop for many VATE monitors on one GPU.
 *
 * The paper runs one monitor whose host thread copies fixed buffers of pairs
 * to the GPU (Sec. 4.2).  A server hosts many monitors (one per link or
 * router), each a vate_handle with its own CUDA stream, and keeps all AT
 * state on the device:
 *   - admission: a monitor is admitted only if its pool and census buffers fit
 *     in the memory budget left (VATE_ENOMEM otherwise; release frees its share);
 *   - requests: ingest (pairs of one slice) and close (census + estimate of a
 *     host list) are submitted from host buffers and return a ticket at once;
 *   - continuous batching: a scheduler thread dispatches requests in arrival
 *     order onto a fixed set of slots (device staging buffers); a request that
 *     arrives while others are on the GPU is dispatched as soon as a slot is
 *     free, consecutive small ingests of the same monitor and slice are merged
 *     into one copy and one launch, and requests of different monitors overlap
 *     on the device (separate streams; copies overlap kernels);
 *   - close runs the learned estimator (include/vate_learned.h) when the
 *     monitor has a model, with the closed form of Eq. 11 as its fallback, and
 *     the closed form otherwise;
 *   - latency: per request, from submission to completion seen by the
 *     scheduler (queueing included); p50/p99 per request kind;
 *   - order: requests go to the device in arrival order per monitor (a
 *     monitor whose next request is held back does not hold up the others).
 * A monitor's results do not depend on the other monitors or on the timing of
 * the requests: every monitor computes what its vate_handle computes alone.
 *
 * Threading: the server's functions may be called from any host thread;
 * the handles are driven only by the scheduler thread.  Host buffers passed to
 * a submit must stay valid until the request completes (vate_server_wait).
 */
#ifndef VATE_SERVER_H
#define VATE_SERVER_H

#include <stdint.h>
#include "vate.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vate_server vate_server;

typedef struct {
    uint64_t memory_budget_bytes;   /* device memory for pools, census buffers and slots   */
    uint32_t slots;                 /* requests in flight at once (2..64)                    */
    uint32_t slot_records;          /* records (pairs or hosts) per slot (>= 1024)           */
} vate_server_config;

typedef struct {
    uint64_t ingests_done, closes_done, pairs_done, hosts_done;
    uint64_t merged_ingests;        /* ingest requests that shared a launch with an earlier one */
    double ingest_p50_ms, ingest_p99_ms, close_p50_ms, close_p99_ms;
    uint64_t memory_in_use;         /* bytes counted against the budget                       */
    uint32_t monitors;              /* monitors admitted now                                  */
    uint32_t max_in_flight;         /* most slots busy at once                                */
} vate_server_stats;

/* Submit flag: the host buffer is page-locked and stays untouched until the
 * request completes, so it is copied to the device directly (no staging copy). */
#define VATE_SUBMIT_PINNED 1u

/* Create the server on the current device; the slots' device buffers are
 * counted against the budget.  Starts the scheduler thread. */
int vate_server_create(const vate_server_config *cfg, vate_server **out);

/* Drain every request, stop the scheduler, free everything.  NULL is accepted. */
int vate_server_destroy(vate_server *s);

/* Admit a monitor with these parameters (vate_create) if it fits in the
 * budget left; *id receives its number.  VATE_ENOMEM if it does not fit. */
int vate_server_admit(vate_server *s, const vate_params *params, int32_t *id);

/* Wait for the monitor's requests, then destroy it and return its memory. */
int vate_server_release(vate_server *s, int32_t id);

/* Use a learned model (device floats, vate_mlp_param_count(2k+2), kept valid
 * by the caller) for the monitor's closes; NULL returns to the closed form. */
int vate_server_set_model(vate_server *s, int32_t id, const float *d_params);

/* Queue the pairs of slice `slice` for monitor id (n <= slot_records). */
int vate_server_submit_ingest(vate_server *s, int32_t id, const vate_pair *h_pairs, uint64_t n, int64_t slice,
                              uint32_t flags, uint64_t *ticket);

/* Queue the close of slice `slice` and the estimates of n hosts (n <= slot_records)
 * for window kprime (a monitor's learned model estimates k' = k; other k' use
 * the closed form).  h_out (float[n]) and h_flags (uint8[n], may be NULL) are
 * written when the request completes. */
int vate_server_submit_close(vate_server *s, int32_t id, int64_t slice, const uint32_t *h_hosts, uint64_t n,
                             uint32_t kprime, float *h_out, uint8_t *h_flags, uint32_t flags, uint64_t *ticket);

/* Wait up to timeout_ms for a request; returns the request's own status
 * (VATE_OK, or e.g. VATE_ESLICE for an out-of-order slice), VATE_ETIMEOUT if
 * it has not completed, VATE_EINVAL for an unknown ticket. */
int vate_server_wait(vate_server *s, uint64_t ticket, uint32_t timeout_ms);

/* Wait up to timeout_ms for every submitted request. */
int vate_server_drain(vate_server *s, uint32_t timeout_ms);

/* Host-side fault injection, for tests of failure handling that need no GPU
 * fault (the paper has no counterpart).  Faults act in the scheduler:
 *   VATE_FAULT_STALL  the scheduler neither retires nor dispatches anything for
 *                     `ms` milliseconds (a stalled host thread); requests queue.
 *   VATE_FAULT_DROP   the next `count` ingest requests of monitor `mon` are
 *                     dropped when their turn comes: they complete with
 *                     VATE_EDROPPED through vate_server_wait and never reach
 *                     the device (lost batches); the monitor's state is that
 *                     of a stream without them.
 *   VATE_FAULT_HOLD   the next `count` requests of monitor `mon` are each held
 *                     back `ms` milliseconds when they reach the front of the
 *                     monitor's line (late batches); the monitor's later
 *                     requests wait behind them, other monitors' pass them.
 * Requests are dispatched in arrival order per monitor, so no fault changes
 * the results of a monitor it does not drop batches of.  Errors: VATE_EINVAL
 * (unknown kind or monitor). */
#define VATE_FAULT_STALL 1u
#define VATE_FAULT_DROP  2u
#define VATE_FAULT_HOLD  3u
typedef struct {
    uint32_t kind;
    int32_t mon;
    uint32_t count;
    uint32_t ms;
} vate_server_fault;
int vate_server_inject(vate_server *s, const vate_server_fault *f);

/* Counters and latency percentiles since creation or the last reset. */
int vate_server_get_stats(vate_server *s, vate_server_stats *out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* VATE_SERVER_H */
