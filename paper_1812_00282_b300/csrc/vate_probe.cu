// vate_probe.cu -- memory-system probes for the roofline denominators of the
// VATE kernels (include/vate_probe.h).  Built into libvate_probe.so, a
// measurement library of its own: not part of the VATE method and not linked
// into libvate.so.
//
// Each probe issues U independent accesses per thread per loop trip (U = 1,
// 2, 4 or 8), so that several are in flight before any result is used, and
// runs blocks_per_sm blocks of 256 threads per SM: the caller sweeps both and
// keeps the best, which is the ceiling a kernel of the same access pattern
// can be held to.
#include <cstdint>
#include <cuda_runtime.h>

#include "vate.h"
#include "vate_probe.h"

namespace {

__device__ __forceinline__ uint32_t probe_mix(uint32_t h) {   // MurmurHash3 32-bit finalizer
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

// 16-byte load number i reads half (i & 1) of the pseudo-random 32-byte sector
// mix(i >> 1): consecutive threads read the two halves of one sector, the
// gather's lane-pair pattern.  Read-only cached loads, as in the gather.
template <int U>
__global__ void __launch_bounds__(256) sector_read_kernel(const uint4 *__restrict__ buf, uint64_t sector_mask,
                                                          uint64_t n_loads, uint32_t *sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < n_loads; i0 += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t i = i0 + (uint64_t)u * stride;
            v[u] = make_uint4(0u, 0u, 0u, 0u);
            if (i < n_loads) {
                const uint64_t s = (uint64_t)probe_mix((uint32_t)(i >> 1) * 0x9E3779B9u + 7u) & sector_mask;
                v[u] = __ldg(buf + 2 * s + (i & 1));
            }
        }
#pragma unroll
        for (int u = 0; u < U; u++) acc += v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;   // practically never; keeps the loads live
}

// Byte store number i writes position mix(i) of the buffer.
template <int U>
__global__ void __launch_bounds__(256) byte_write_kernel(uint8_t *__restrict__ buf, uint64_t mask, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < n; i0 += U * stride) {
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t i = i0 + (uint64_t)u * stride;
            if (i < n) buf[(uint64_t)probe_mix((uint32_t)i * 0x9E3779B9u + 13u) & mask] = (uint8_t)i;
        }
    }
}

// Every 16-byte chunk of the buffer once, coalesced, L2-cached loads (the
// census's pattern).
template <int U>
__global__ void __launch_bounds__(256) stream_read_kernel(const uint4 *__restrict__ buf, uint64_t n16, uint32_t *sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < n16; i0 += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint64_t i = i0 + (uint64_t)u * stride;
            v[u] = i < n16 ? __ldcg(buf + i) : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < U; u++) acc += v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;
}

int grid_of(uint32_t blocks_per_sm) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms * (int)blocks_per_sm;
}

bool pow2_buffer(uint64_t b) { return b >= 4096 && (b & (b - 1)) == 0 && b <= (1ull << 34); }
bool valid_shape(uint32_t u, uint32_t bps) { return (u == 1 || u == 2 || u == 4 || u == 8) && bps >= 1 && bps <= 32; }

int finish() { return cudaGetLastError() == cudaSuccess ? VATE_OK : VATE_ECUDA; }

}  // namespace

extern "C" int vate_probe_sector_read(const uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_sectors, uint32_t *d_sink,
                                      uint32_t loads_in_flight, uint32_t blocks_per_sm, void *stream) {
    if (!d_buf || !d_sink || !pow2_buffer(buf_bytes) || (reinterpret_cast<uintptr_t>(d_buf) & 31u) ||
        !valid_shape(loads_in_flight, blocks_per_sm) || n_sectors > (1ull << 32))
        return VATE_EINVAL;
    if (n_sectors == 0) return VATE_OK;
    const uint64_t mask = (buf_bytes >> 5) - 1;
    const uint4 *b = reinterpret_cast<const uint4 *>(d_buf);
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_of(blocks_per_sm);
    switch (loads_in_flight) {
    case 1: sector_read_kernel<1><<<grid, 256, 0, st>>>(b, mask, 2 * n_sectors, d_sink); break;
    case 2: sector_read_kernel<2><<<grid, 256, 0, st>>>(b, mask, 2 * n_sectors, d_sink); break;
    case 4: sector_read_kernel<4><<<grid, 256, 0, st>>>(b, mask, 2 * n_sectors, d_sink); break;
    default: sector_read_kernel<8><<<grid, 256, 0, st>>>(b, mask, 2 * n_sectors, d_sink); break;
    }
    return finish();
}

extern "C" int vate_probe_byte_write(uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_writes, uint32_t stores_per_trip,
                                     uint32_t blocks_per_sm, void *stream) {
    if (!d_buf || !pow2_buffer(buf_bytes) || !valid_shape(stores_per_trip, blocks_per_sm) || n_writes > (1ull << 32))
        return VATE_EINVAL;
    if (n_writes == 0) return VATE_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_of(blocks_per_sm);
    switch (stores_per_trip) {
    case 1: byte_write_kernel<1><<<grid, 256, 0, st>>>(d_buf, buf_bytes - 1, n_writes); break;
    case 2: byte_write_kernel<2><<<grid, 256, 0, st>>>(d_buf, buf_bytes - 1, n_writes); break;
    case 4: byte_write_kernel<4><<<grid, 256, 0, st>>>(d_buf, buf_bytes - 1, n_writes); break;
    default: byte_write_kernel<8><<<grid, 256, 0, st>>>(d_buf, buf_bytes - 1, n_writes); break;
    }
    return finish();
}

extern "C" int vate_probe_stream_read(const uint8_t *d_buf, uint64_t buf_bytes, uint32_t *d_sink,
                                      uint32_t loads_in_flight, uint32_t blocks_per_sm, void *stream) {
    if (!d_buf || !d_sink || !pow2_buffer(buf_bytes) || (reinterpret_cast<uintptr_t>(d_buf) & 15u) ||
        !valid_shape(loads_in_flight, blocks_per_sm))
        return VATE_EINVAL;
    const uint64_t n16 = buf_bytes >> 4;
    const uint4 *b = reinterpret_cast<const uint4 *>(d_buf);
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = grid_of(blocks_per_sm);
    switch (loads_in_flight) {
    case 1: stream_read_kernel<1><<<grid, 256, 0, st>>>(b, n16, d_sink); break;
    case 2: stream_read_kernel<2><<<grid, 256, 0, st>>>(b, n16, d_sink); break;
    case 4: stream_read_kernel<4><<<grid, 256, 0, st>>>(b, n16, d_sink); break;
    default: stream_read_kernel<8><<<grid, 256, 0, st>>>(b, n16, d_sink); break;
    }
    return finish();
}
