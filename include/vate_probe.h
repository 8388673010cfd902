/*
 * vate_probe.h -- measurement helpers of the VATE library.
 *
 * These entry points have no counterpart in the paper.  They measure, on the
 * GPU at hand, the two memory-system rates that bound the VATE kernels, so
 * that a benchmark can state each kernel's achieved rate as a fraction of
 * what the hardware sustains for the same access pattern:
 *   - random 32-byte sector reads from an L2-resident buffer (the gather of
 *     vate_estimate with 32-AT segments reads one such sector per segment);
 *   - random 1-byte stores into an L2-resident buffer (the SetAT of
 *     vate_ingest writes one byte per pair).
 * Positions come from a fixed integer mixer of the access index; every access
 * stays inside [d_buf, d_buf + buf_bytes).  Same conventions as vate.h:
 * device pointers, asynchronous on `stream`, VATE_* return codes.
 */
#ifndef VATE_PROBE_H
#define VATE_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Read n_sectors pseudo-random 32-byte sectors of d_buf (buf_bytes: a power
 * of two, >= 4096; d_buf 32-byte aligned), two lanes per sector, and write a
 * checksum to d_sink[0] (device uint32) so the reads cannot be elided. */
int vate_probe_sector_read(const uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_sectors, uint32_t *d_sink,
                           void *stream);

/* Store n_writes bytes at pseudo-random positions of d_buf (buf_bytes: a
 * power of two, >= 4096). */
int vate_probe_byte_write(uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_writes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VATE_PROBE_H */
