/*
 * vate_probe.h -- memory-system probes beside the VATE library
 * (libvate_probe.so, a measurement library of its own).
 *
 * These entry points have no counterpart in the paper.  They measure, on the
 * GPU at hand, the memory-system rates that bound the VATE kernels, so that a
 * benchmark can state each kernel's achieved rate as a fraction of what the
 * hardware sustains for the same access pattern:
 *   - random 32-byte sector reads (the gather of vate_estimate with 32-AT
 *     segments reads one such sector per segment, two lanes per sector);
 *   - random 1-byte stores (the SetAT of vate_ingest writes one byte per pair);
 *   - a coalesced read of a whole buffer (the pool census reads the pool once).
 * Each probe issues U independent accesses per thread per loop trip (U in
 * {1, 2, 4, 8}) from blocks_per_sm (1..32) blocks of 256 threads per SM; a
 * benchmark sweeps both and keeps the fastest, so the figure is a ceiling for
 * the pattern rather than one launch shape's rate.  Positions come from a
 * fixed integer mixer of the access index; every access stays inside
 * [d_buf, d_buf + buf_bytes).  Device pointers, asynchronous on `stream`
 * (a cudaStream_t as void*), VATE_OK / VATE_EINVAL / VATE_ECUDA returns
 * (vate.h codes).
 */
#ifndef VATE_PROBE_H
#define VATE_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Read n_sectors (<= 2^32) pseudo-random 32-byte sectors of d_buf
 * (buf_bytes: a power of two, 4096..2^34; d_buf 32-byte aligned), two
 * consecutive threads per sector, and write a checksum-dependent value to
 * d_sink[0] (device uint32) so that the reads cannot be elided. */
int vate_probe_sector_read(const uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_sectors, uint32_t *d_sink,
                           uint32_t loads_in_flight, uint32_t blocks_per_sm, void *stream);

/* Store n_writes (<= 2^32) bytes at pseudo-random positions of d_buf
 * (buf_bytes: a power of two, 4096..2^34). */
int vate_probe_byte_write(uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_writes, uint32_t stores_per_trip,
                          uint32_t blocks_per_sm, void *stream);

/* Read every 16-byte chunk of d_buf once (buf_bytes: a power of two,
 * 4096..2^34; d_buf 16-byte aligned), coalesced, L2-cached loads. */
int vate_probe_stream_read(const uint8_t *d_buf, uint64_t buf_bytes, uint32_t *d_sink, uint32_t loads_in_flight,
                           uint32_t blocks_per_sm, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* VATE_PROBE_H */
