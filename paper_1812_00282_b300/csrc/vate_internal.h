// vate_internal.h -- declarations shared by the kernel file and the C-ABI file.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "vate_device.cuh"

namespace vate {

constexpr int GATHER_THREADS = 256;
constexpr int CENSUS_THREADS = 256;
constexpr int AGE_THREADS = 256;
constexpr int GATHER_ESTIMATE = 0;
constexpr int GATHER_ACTIVE = 1;

void count_launch();

// Read-only view of a vate_handle (defined in vate_api.cu).
struct HandleView {
    Geom G;
    uint32_t bact0;
    const uint64_t *hist;
    bool closed;
    int sms;
};
}  // namespace vate
struct vate_handle;
namespace vate {
int handle_view(const vate_handle *h, HandleView *v);
int set_error(int code, const char *msg);
// A device scratch of at least `bytes` owned by the handle: allocated on the
// first request (and grown if a later one is larger), freed by vate_destroy.
int handle_scratch(vate_handle *h, uint64_t bytes, void **ptr);
// The device's persisting-L2 limit, held by the handles and groups made with
// VATE_OPT_PERSIST_L2: the first raises it to `want`, the last released puts
// back the limit it found (vate_api.cu).  acquire returns false when the
// device index is out of range (nothing changed).
bool persist_acquire(int dev, size_t want);
void persist_release(int dev);
// VATE_OK when the handle can serve the learned estimator (its checks and
// error messages), else the error (vate_learned.cu).
int learned_handle_ok(const vate_handle *h);
// The learned estimate (vate_estimate_learned) of n hosts from their per-age
// counts, given as 16-bit fields (ages 4 i .. 4 i + 3 in counts[i n + h]):
// feature rows, Eq. 11 and the output rule in one kernel (vate_learned.cu).
int learned_from_age_counts(vate_handle *h, const HandleView &v, const unsigned long long *counts, uint64_t n,
                            const float *d_params, float *d_out, uint8_t *d_flags, cudaStream_t st);

cudaError_t launch_init(const Geom &G, cudaStream_t st, int sms);
cudaError_t launch_ingest(const Geom &G, uint32_t bact0, const uint32_t *pairs, uint64_t n, cudaStream_t st, int sms);
cudaError_t launch_dr_age(const Geom &G, cudaStream_t st, int sms);
cudaError_t launch_preserve(const Geom &G, uint32_t bact0, uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1,
                            cudaStream_t st, int sms);
// frame 0 -> the paper's per-block values (to_paper) or back, for pool positions pid0 .. pid0 + n - 1
cudaError_t launch_frame_convert(const Geom &G, const uint8_t *src, uint8_t *dst, uint64_t pid0, uint64_t n,
                                 bool to_paper, cudaStream_t st, int sms);
size_t census_smem_bytes(uint32_t twok);
cudaError_t census_prepare(uint32_t twok);
// the pool census into hist (2k + 1 counters); acc (2k + 1 counters) and
// ticket are scratch that must be zero before the first call and are left zero
cudaError_t launch_census(const Geom &G, uint32_t bact0, uint64_t *acc, int sms, uint64_t *hist,
                          unsigned int *ticket, cudaStream_t st);
cudaError_t launch_gather(int mode, const Geom &G, uint32_t bact0, uint32_t kprime, const uint64_t *hist,
                          const uint32_t *aips, uint64_t n, float *out, uint8_t *flags, uint32_t *active,
                          cudaStream_t st, int sms);
cudaError_t age_prepare(uint32_t k);
// packed pools (vate_packed.cu)
uint32_t packed_pattern(const Geom &G);
cudaError_t launch_packed_init(const Geom &G, cudaStream_t st, int sms);
cudaError_t launch_packed_preserve(const Geom &G, uint32_t bact0, uint64_t s0, uint64_t e0, uint64_t s1, uint64_t e1,
                                   cudaStream_t st, int sms);
cudaError_t launch_packed_dr_age(const Geom &G, cudaStream_t st, int sms);
cudaError_t packed_census_prepare(uint32_t twok);   // shared-memory attribute of the lane-column packed census
cudaError_t launch_packed_census(const Geom &G, uint32_t bact0, uint64_t *acc, int sms, uint64_t *hist,
                                 unsigned int *ticket, cudaStream_t st);
cudaError_t launch_packed_gather(int mode, const Geom &G, uint32_t bact0, uint32_t kprime, const uint64_t *hist,
                                 const uint32_t *aips, uint64_t n, float *out, uint8_t *flags, uint32_t *active,
                                 cudaStream_t st, int sms);
cudaError_t launch_packed_to_paper(const Geom &G, uint8_t *dst, uint64_t pos0, uint64_t n, cudaStream_t st, int sms);
cudaError_t launch_paper_to_packed(const Geom &G, const uint8_t *src, uint64_t pos0, uint64_t n, cudaStream_t st,
                                   int sms);
// Eq. 11 from active counts and a census (both summed over the shards of one pool)
cudaError_t launch_estimate_from_counts(const Geom &G, uint32_t kprime, const uint64_t *hist, const uint32_t *active,
                                        uint64_t n, float *out, uint8_t *flags, cudaStream_t st, int sms);
cudaError_t launch_age_counts(const Geom &G, uint32_t bact0, const uint32_t *aips, uint64_t n, uint16_t *counts,
                              cudaStream_t st, int sms);

}  // namespace vate
