// vate_noalloc.cu -- a pool census that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: a packet-processing loop
// with a latency budget (cudaMalloc can synchronise the device and takes an
// unbounded time), or a host application whose device memory is owned
// entirely by its own allocator (a framework's caching allocator or a fixed
// arena) and which therefore has nothing left for a library to ask the
// driver for.  vate_census_noalloc serves them: it takes the caller's pool
// and output buffers and keeps its only scratch -- the 2k + 1 counters the
// census blocks add into and the "blocks finished" ticket of the census
// kernel -- in a file-scope device array of fixed size.  That array exists
// once on every device that loads the library and stays allocated until the
// process exits.
//
// In host code the array's name is only a host-side stand-in, not a device
// address.  The first call on each device (with that device current) looks
// the address up with cudaGetSymbolAddress and caches it; every launch is
// given that address.  Device code in this file names the array directly.
#include <cstdio>
#include <mutex>

#include "vate.h"
#include "vate_internal.h"

using vate::Geom;

namespace {

constexpr int NOALLOC_MAX_BINS = 127;                   // 2k + 1 with k <= 63
constexpr size_t NOALLOC_TICKET_BYTES = 256;            // ticket, padded to the alignment
constexpr size_t NOALLOC_SCRATCH_BYTES =
    NOALLOC_TICKET_BYTES + (size_t)NOALLOC_MAX_BINS * sizeof(uint64_t);   // 1,272 bytes

static __device__ __align__(256) unsigned char census_scratch[NOALLOC_SCRATCH_BYTES];

// The ticket and the counters must be 0 when the census kernel starts.  A
// completed call leaves them at 0; they are cleared before every call anyway
// so that nothing a previous call left behind can leak into this one.
__global__ void clear_scratch_kernel() {
    if (threadIdx.x == 0) *reinterpret_cast<unsigned int *>(census_scratch) = 0u;
    if (threadIdx.x < NOALLOC_MAX_BINS)
        reinterpret_cast<uint64_t *>(census_scratch + NOALLOC_TICKET_BYTES)[threadIdx.x] = 0u;
}

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_scratch_addr[MAX_DEVICES] = {};
int g_sms[MAX_DEVICES] = {};
thread_local char g_msg[256];

// Once per device: the device address of the scratch array, the SM count,
// and the census kernel's shared-memory attribute.
int setup_device(void **addr_out, int *sms_out, const char **why) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        *why = "no-alloc census: no current CUDA device (cudaGetDevice failed)";
        return VATE_ECUDA;
    }
    if (dev >= MAX_DEVICES) {
        *why = "no-alloc census: device index beyond the 64 devices this entry point keeps addresses for";
        return VATE_EINVAL;
    }
    *why = "no-alloc census: device set-up (cudaGetSymbolAddress, SM count or kernel attribute) failed";
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&ptr, census_scratch);
        if (e != cudaSuccess || !ptr) return VATE_ECUDA;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || sms <= 0) return VATE_ECUDA;
        if (vate::census_prepare(126) != cudaSuccess) return VATE_ECUDA;
        g_sms[dev] = sms;
        g_scratch_addr[dev] = ptr;
    }
    *addr_out = g_scratch_addr[dev];
    *sms_out = g_sms[dev];
    return VATE_OK;
}

}  // namespace

namespace vate {
int make_geom_checked(const vate_params *p, Geom *G);   // vate_api.cu
int set_error(int code, const char *msg);               // vate_api.cu
}  // namespace vate

extern "C" int vate_census_noalloc(const vate_params *params, const uint8_t *d_pool, uint32_t bact0, uint64_t *d_hist,
                                   void *stream) {
    Geom G;
    int rc = vate::make_geom_checked(params, &G);
    if (rc) return rc;
    if (!d_pool || !d_hist) return vate::set_error(VATE_EINVAL, "d_pool and d_hist must not be NULL");
    if ((reinterpret_cast<uintptr_t>(d_pool) & 15u) != 0)
        return vate::set_error(VATE_EINVAL, "d_pool must be 16-byte aligned");
    if (bact0 >= G.twok) return vate::set_error(VATE_EINVAL, "bact0 must be below 2k");
    if (G.twok + 1 > (uint32_t)NOALLOC_MAX_BINS) {
        snprintf(g_msg, sizeof g_msg, "no-alloc census keeps at most %d bins (k <= 63)", NOALLOC_MAX_BINS);
        return vate::set_error(VATE_EINVAL, g_msg);
    }
    // every argument is checked before the device is touched
    int sms = 0;
    void *scratch = nullptr;
    const char *why = "";
    rc = setup_device(&scratch, &sms, &why);
    if (rc != VATE_OK) return vate::set_error(rc, why);
    G.pool = const_cast<uint8_t *>(d_pool);
    G.packed = 0;                                // the caller's pool: one byte per AT in the paper's form
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char *base = static_cast<unsigned char *>(scratch);
    clear_scratch_kernel<<<1, 128, 0, st>>>();
    vate::count_launch();
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = vate::launch_census(G, bact0, reinterpret_cast<uint64_t *>(base + NOALLOC_TICKET_BYTES), sms, d_hist,
                                reinterpret_cast<unsigned int *>(base), st);
    if (e != cudaSuccess) return vate::set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}
