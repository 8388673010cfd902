/*
 * vate_checkpoint.h -- checkpoint and resume of one VATE handle.
 *
 * The paper has no counterpart: its monitor runs until it is stopped
 * (Algorithm 4).  A long-running monitor still has to survive a process
 * restart or a move to another GPU without losing its window, and the state
 * that decides every later answer is small and exact: the AT pool (one byte
 * per AT), BACT^0 of the current slice (Eq. 7), the slice number, whether the
 * slice has been closed, and the census of the last close (the Z_p term of
 * Eq. 11).  A checkpoint is that state as one host byte image; a handle
 * restored from it answers every later ingest, close and estimate exactly as
 * the handle it was taken from would have.
 *
 * Image layout (little-endian, as written by this library on x86-64/aarch64):
 *   vate_checkpoint_header   (fixed size, header_bytes)
 *   uint64_t hist[2k+1]      census of the last close (zeros before any close)
 *   pool[2^c]                AT values in the paper's form, pool position
 *                            order: uint8 for k <= 63, uint16 beyond (also
 *                            for a packed pool, whose image is unpacked)
 * The checksum is FNV-1a (64-bit, Fowler/Noll/Vo) taken over the whole image
 * 8 bytes at a time with the checksum field read as zero.
 */
#ifndef VATE_CHECKPOINT_H
#define VATE_CHECKPOINT_H

#include <stdint.h>
#include "vate.h"

#ifdef __cplusplus
extern "C" {
#endif

#define VATE_CHECKPOINT_MAGIC   0x31544B4345544156ull   /* "VATECKT1" read as a little-endian uint64 */
#define VATE_CHECKPOINT_VERSION 2u

typedef struct {
    uint64_t   magic;          /* VATE_CHECKPOINT_MAGIC                                   */
    uint32_t   version;        /* VATE_CHECKPOINT_VERSION                                 */
    uint32_t   header_bytes;   /* sizeof(vate_checkpoint_header)                          */
    vate_params params;        /* geometry, hash seed and counter kind of the handle      */
    int64_t    slice;          /* current slice, -1 before the first call                 */
    uint32_t   bact0;          /* BACT^0 of the current slice                             */
    uint32_t   closed;         /* 1 when the current slice has been closed                */
    uint64_t   hist_bytes;     /* (2k+1) * 8                                              */
    uint64_t   pool_bytes;     /* 2^c times the AT width (1 or 2 bytes)                   */
    uint64_t   checksum;       /* FNV-1a over the image with this field taken as zero     */
} vate_checkpoint_header;

/* Bytes a checkpoint of h occupies (header + census + pool).  No GPU work. */
int vate_checkpoint_size(const vate_handle *h, uint64_t *bytes);

/* Write the state of h into the host buffer h_buf (`bytes` >= the size above;
 * any alignment).  Work already queued on `stream` for the handle is part of
 * the image: the call waits for the stream, copies the pool and census to the
 * host and returns when the image is complete.  The handle is left unchanged.
 * Errors: VATE_EINVAL (NULL or short buffer), VATE_ECUDA. */
int vate_checkpoint(vate_handle *h, void *h_buf, uint64_t bytes, void *stream);

/* Create a handle on the current device from a checkpoint image.  The image
 * is checked before any device memory is taken: magic, version, sizes that
 * agree with the parameters, parameters that vate_create accepts, slice and
 * BACT^0 in range, and the checksum.  Errors: VATE_EINVAL (any check fails;
 * vate_last_error names which), VATE_ENOMEM, VATE_ECUDA.  *out is set only on
 * success; the handle is ready when work queued on `stream` completes. */
int vate_restore(const void *h_buf, uint64_t bytes, void *stream, vate_handle **out);

#ifdef __cplusplus
}
#endif
#endif /* VATE_CHECKPOINT_H */
