// vate_probe.cu -- memory-system probes for the roofline denominators
// (see include/vate_probe.h).  Not part of the VATE method.
#include <cstdint>
#include <cuda_runtime.h>

#include "vate.h"
#include "vate_probe.h"
#include "vate_internal.h"

namespace {

__device__ __forceinline__ uint32_t probe_mix(uint32_t h) {   // MurmurHash3 32-bit finalizer
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__global__ void __launch_bounds__(256) sector_read_kernel(const uint4 *__restrict__ buf, uint64_t sector_mask,
                                                          uint64_t n_sectors, uint32_t *sink) {
    uint32_t acc = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < 2 * n_sectors; i += stride) {
        uint64_t s = (uint64_t)probe_mix((uint32_t)(i >> 1) * 0x9E3779B9u + 7u) & sector_mask;
        uint4 v = __ldg(buf + 2 * s + (i & 1));
        acc += __popc(v.x ^ v.y ^ v.z ^ v.w);
    }
    if (acc == 0xFFFFFFFFu) sink[0] = acc;   // practically never; keeps the loads live
}

__global__ void __launch_bounds__(256) byte_write_kernel(uint8_t *__restrict__ buf, uint64_t mask, uint64_t n) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t s = (uint64_t)probe_mix((uint32_t)i * 0x9E3779B9u + 13u) & mask;
        buf[s] = (uint8_t)i;
    }
}

int sm_count() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

bool pow2_at_least_4k(uint64_t b) { return b >= 4096 && (b & (b - 1)) == 0 && b <= (1ull << 34); }

}  // namespace

extern "C" int vate_probe_sector_read(const uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_sectors, uint32_t *d_sink,
                                      void *stream) {
    if (!d_buf || !d_sink || !pow2_at_least_4k(buf_bytes) || (reinterpret_cast<uintptr_t>(d_buf) & 31u))
        return VATE_EINVAL;
    if (n_sectors == 0) return VATE_OK;
    uint64_t mask = (buf_bytes >> 5) - 1;
    sector_read_kernel<<<sm_count() * 16, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const uint4 *>(d_buf), mask,
                                                                         n_sectors, d_sink);
    vate::count_launch();
    return cudaGetLastError() == cudaSuccess ? VATE_OK : VATE_ECUDA;
}

extern "C" int vate_probe_byte_write(uint8_t *d_buf, uint64_t buf_bytes, uint64_t n_writes, void *stream) {
    if (!d_buf || !pow2_at_least_4k(buf_bytes)) return VATE_EINVAL;
    if (n_writes == 0) return VATE_OK;
    byte_write_kernel<<<sm_count() * 16, 256, 0, (cudaStream_t)stream>>>(d_buf, buf_bytes - 1, n_writes);
    vate::count_launch();
    return cudaGetLastError() == cudaSuccess ? VATE_OK : VATE_ECUDA;
}
