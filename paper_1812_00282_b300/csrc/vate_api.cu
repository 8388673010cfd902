// vate_api.cu -- C ABI of the VATE library: argument checks, the slice state
// machine of Algorithm 4 on the host, device buffers, kernel launches.
#include <atomic>
#include <mutex>
#include <cstddef>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "vate.h"
#include "vate_checkpoint.h"
#include "vate_shard.h"
#include "vate_internal.h"

using vate::Geom;

namespace {
thread_local std::string g_err;
std::atomic<uint64_t> g_launches{0};
constexpr uint64_t STAGE_RECORDS = 1ull << 20;   // pairs per chunk of vate_ingest_host (staging buffer size)
constexpr int INGEST_RING = 6;                   // pair staging buffers: one 6M-pair slice copied ahead
constexpr uint64_t EST_RECORDS = 1ull << 18;     // hosts per chunk of vate_estimate_host's pipeline

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(VATE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// Parameter checks and derived geometry; no device needed.
int make_geom(const vate_params *p, Geom *G) {
    if (!p) return fail(VATE_EINVAL, "params is NULL");
    if (p->counter > 1) return fail(VATE_EINVAL, "params.counter must be VATE_COUNTER_AT (0) or VATE_COUNTER_DR (1)");
    if (p->log2_pool < 12 || p->log2_pool > 32) return fail(VATE_EINVAL, "log2_pool (c) must be in [12, 32], got %u", p->log2_pool);
    if (p->k < 1 || p->k > 1023) return fail(VATE_EINVAL, "k must be in [1, 1023], got %u", p->k);
    if (p->g < 1 || p->g > 65536) return fail(VATE_EINVAL, "g must be in [1, 65536], got %u", p->g);
    uint32_t L = p->seg_len;
    if (L < 1 || L > 64 || (L & (L - 1)) != 0) return fail(VATE_EINVAL, "seg_len must be a power of two in [1, 64], got %u", L);
    if (p->g % L != 0) return fail(VATE_EINVAL, "g (%u) must be a multiple of seg_len (%u)", p->g, L);
    if (p->partition > 1) return fail(VATE_EINVAL, "partition must be 0 or 1, got %u", p->partition);
    uint32_t log2L = 0;
    while ((1u << log2L) < L) log2L++;
    if (p->log2_pool <= log2L) return fail(VATE_EINVAL, "log2_pool must exceed log2(seg_len)");
    memset(G, 0, sizeof *G);
    G->c = p->log2_pool;
    G->k = p->k;
    G->twok = 2 * p->k;
    G->g = p->g;
    G->L = L;
    G->log2L = log2L;
    G->segbits = p->log2_pool - log2L;
    G->partition = p->partition;
    G->counter = p->counter;
    G->atw = p->k <= 63 ? 1u : 2u;             // byte ATs up to k = 63, 16-bit ones beyond
    if (p->options & ~VATE_OPT_PERSIST_L2)
        return fail(VATE_EINVAL, "params.options has unknown bits (0x%x)", p->options & ~VATE_OPT_PERSIST_L2);
    if (p->at_bits != 0) {
        uint32_t bmin = 1;
        while ((1u << bmin) < 2 * p->k + 1) bmin++;          // ceil(log2(2k + 1))
        if (p->at_bits < bmin || p->at_bits > 16)
            return fail(VATE_EINVAL, "at_bits must be 0 or in [%u, 16] for k = %u, got %u", bmin, p->k, p->at_bits);
        const bool natural = (p->at_bits == 8 && p->k <= 63) || (p->at_bits == 16 && p->k >= 64);
        if (!natural) {                          // the paper's packed layout (vate_packed.cu)
            G->packed = 1;
            G->atb = p->at_bits;
            G->pn = 32 / p->at_bits;
        }
    }
    G->P = 1ull << p->log2_pool;
    G->key_h = vate::mix64(p->seed + 1);
    G->key_bh = vate::mix64(p->seed + 2);
    uint64_t twok = G->twok;
    if (p->partition == 0) {               // Eq. 9, Eq. 10
        G->a = G->P / (twok - 1);
        G->b = G->P % (twok - 1);
        G->first = G->P;
    } else {                               // low-deviation partition
        G->a = G->P / twok;
        G->b = G->P % twok;
        G->first = G->a * (twok - G->b);
    }
    if (G->a < 32) return fail(VATE_EINVAL, "blocks must hold at least 32 ATs (a = %llu)", (unsigned long long)G->a);
    G->lo = 0;
    G->hi = G->P;
    G->ma = vate::magic_for(G->a);
    if (G->packed) G->mpn = vate::magic_for(G->pn);
    G->ma1 = vate::magic_for(G->a + 1);
    return VATE_OK;
}

}  // namespace

void vate::count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace vate {
// parameter checks and error reporting for entry points without a handle
int make_geom_checked(const vate_params *p, Geom *G) { return make_geom(p, G); }
int set_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace vate

struct vate_handle {
    vate_params prm;
    Geom G;
    bool persist_l2 = false;         // VATE_OPT_PERSIST_L2: holds the device's persisting-L2 limit (persist_acquire)
    int device = 0;
    int sms = 148;
    int64_t slice = -1;
    bool closed = false;
    uint32_t bact0 = 0;
    uint64_t *d_hist = nullptr;       // census of the last close, 2k+1 counters
    uint64_t *d_acc = nullptr;        // census scratch: 2k+1 counters the blocks add into, zero between calls
    unsigned int *d_ticket = nullptr; // census scratch: blocks finished
    unsigned long long *d_dbg = nullptr;   // checked build: [VATE_DBG_* bits, first report]
    // host-copy staging (allocated on first use)
    // pairs: a ring of staging buffers filled on their own stream, so that the
    // pairs of the next slice are copied while this slice is estimated
    cudaStream_t pairs_stream = nullptr;                 // host -> device (pairs)
    cudaEvent_t ev_in_ready[INGEST_RING] = {};           // chunk copied
    cudaEvent_t ev_in_free[INGEST_RING] = {};            // chunk ingested: the buffer may be refilled
    vate_pair *d_in[INGEST_RING] = {};
    uint32_t in_next = 0;                                // next ring slot
    // estimates: two host-list buffers in, two result buffers out
    cudaStream_t copy_stream = nullptr;      // host -> device (hosts)
    cudaStream_t d2h_stream = nullptr;       // device -> host (estimates)
    cudaEvent_t ev_ready[2] = {nullptr, nullptr};
    cudaEvent_t ev_free[2] = {nullptr, nullptr};
    cudaEvent_t ev_done[2] = {nullptr, nullptr};
    uint32_t *d_stage[2] = {nullptr, nullptr};   // hosts in
    float *d_stage_out[2] = {nullptr, nullptr};  // estimates out
    uint8_t *d_stage_flags[2] = {nullptr, nullptr};
    // device scratch of other translation units (the learned estimator's feature rows), on first use
    void *d_scratch = nullptr;
    uint64_t scratch_bytes = 0;
};

namespace vate {
// read-only view of a handle for the other translation units of the library
int handle_view(const vate_handle *h, HandleView *v) {
    if (!h) return fail(VATE_EINVAL, "handle is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
        return fail(VATE_EINVAL, "the handle lives on device %d but device %d is current (cudaSetDevice first)",
                    h->device, dev);
    v->G = h->G;
    v->bact0 = h->bact0;
    v->hist = h->d_hist;
    v->closed = h->closed;
    v->sms = h->sms;
    return VATE_OK;
}

int handle_scratch(vate_handle *h, uint64_t bytes, void **ptr) {
    if (h->scratch_bytes < bytes) {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(VATE_ENOMEM, "out of device memory for a scratch of %llu bytes", (unsigned long long)bytes);
        }
        if (h->d_scratch) {
            cudaDeviceSynchronize();           // work queued on the old scratch ends first
            cudaFree(h->d_scratch);
        }
        h->d_scratch = p;
        h->scratch_bytes = bytes;
    }
    *ptr = h->d_scratch;
    return VATE_OK;
}

// Handles and groups made with VATE_OPT_PERSIST_L2, per device: the first one
// raises the device's persisting-L2 limit to `want` (remembering the limit it
// found), the last one released puts that limit back, so that no L2 stays set
// aside once none of them is left.
namespace {
constexpr int PERSIST_DEVICES = 64;
std::mutex g_persist_mu;
int g_persist_users[PERSIST_DEVICES];
size_t g_persist_prev[PERSIST_DEVICES];
}  // namespace

bool persist_acquire(int dev, size_t want) {
    std::lock_guard<std::mutex> lock(g_persist_mu);
    if (dev < 0 || dev >= PERSIST_DEVICES) return false;
    if (g_persist_users[dev]++ == 0) {
        size_t cur = 0;
        if (cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize) != cudaSuccess) cur = 0;
        g_persist_prev[dev] = cur;
        if (cur < want) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want);
        cudaGetLastError();
    }
    return true;
}

void persist_release(int dev) {
    std::lock_guard<std::mutex> lock(g_persist_mu);
    if (dev < 0 || dev >= PERSIST_DEVICES || g_persist_users[dev] == 0) return;
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    if (cur_dev != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    cudaCtxResetPersistingL2Cache();                   // lines of the freed memory must not stay set aside
    if (--g_persist_users[dev] == 0) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_persist_prev[dev]);
    if (cur_dev != dev) cudaSetDevice(cur_dev);
    cudaGetLastError();
}
}  // namespace vate

namespace {

// A handle's memory and streams belong to the device it was created on; the
// library never switches the calling thread's device, so calls that queue
// work on a handle must be made with that device current.
int check_handle(const vate_handle *h) {
    if (!h) return fail(VATE_EINVAL, "handle is NULL");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device)
        return fail(VATE_EINVAL, "the handle lives on device %d but device %d is current (cudaSetDevice first)",
                    h->device, dev);
    return VATE_OK;
}

// [s, e) intersected with the positions the handle holds (empty: s = e)
void clip(const Geom &G, uint64_t *s, uint64_t *e) {
    uint64_t a = *s > G.lo ? *s : G.lo, b = *e < G.hi ? *e : G.hi;
    if (a >= b) a = b = G.lo;
    *s = a;
    *e = b;
}

bool is_shard(const vate_handle *h) { return h->G.lo != 0 || h->G.hi != h->G.P; }

// Slide the window until `slice` is the current slice: each step is
// BACT^0 <- BACT^0 + 1 and PreserveAT on the blocks whose ACT became 0 or k
// (Algorithm 4, last lines).  After 2k steps with no SetAT every AT is
// inactive, which every further step leaves unchanged, so longer gaps only
// advance BACT^0.
int advance_to(vate_handle *h, int64_t slice, cudaStream_t st) {
    if (h->slice < 0) {            // first call fixes the origin (slice 0 of Algorithm 4)
        h->slice = slice;
        h->closed = false;
        return VATE_OK;
    }
    const Geom &G = h->G;
    int64_t steps = slice - h->slice;
    // distance recorders all reach k (inactive) after k slides, timestamps after 2k
    const int64_t settle = G.counter == 1u ? (int64_t)G.k : (int64_t)G.twok;
    int64_t run = steps > settle ? settle : steps;
    for (int64_t s = 0; s < run; s++) {
        h->bact0 = (h->bact0 + 1) % G.twok;
        cudaError_t e;
        if (G.counter == 1u) {
            e = vate::launch_dr_age(G, st, h->sms);                // VDRE: age the whole pool
        } else {
            uint32_t i0 = (G.twok - h->bact0) % G.twok;          // BACT = 0
            uint32_t i1 = (G.k + G.twok - h->bact0) % G.twok;    // BACT = k
            uint64_t s0, e0, s1, e1;
            vate::block_range_of(G, i0, &s0, &e0);
            vate::block_range_of(G, i1, &s1, &e1);
            clip(G, &s0, &e0);                                 // a shard maintains its part of each block
            clip(G, &s1, &e1);
            e = vate::launch_preserve(G, h->bact0, s0, e0, s1, e1, st, h->sms);
        }
        if (e != cudaSuccess) return cuda_fail(e, "maintenance launch");
    }
    if (steps > run) h->bact0 = (uint32_t)((h->bact0 + (uint64_t)(steps - run)) % G.twok);
    h->slice = slice;
    h->closed = false;
    return VATE_OK;
}

int check_slice(const vate_handle *h, int64_t slice) {
    if (slice < 0) return fail(VATE_ESLICE, "slice numbers start at 0 (got %lld)", (long long)slice);
    if (h->slice >= 0 && slice < h->slice)
        return fail(VATE_ESLICE, "slice %lld is before the current slice %lld", (long long)slice, (long long)h->slice);
    if (h->slice >= 0 && slice == h->slice && h->closed)
        return fail(VATE_ESLICE, "slice %lld is already closed", (long long)slice);
    return VATE_OK;
}

// The kernels' shared-memory limits are attributes of the current device:
// set them once per device, under a lock (handles may be created from
// several threads and on several devices).
std::mutex g_prep_mu;
bool g_prepared[256] = {};

cudaError_t prepare_device(int dev) {
    std::lock_guard<std::mutex> lock(g_prep_mu);
    if (dev >= 0 && dev < 256 && g_prepared[dev]) return cudaSuccess;
    cudaError_t e = vate::census_prepare(126);
    if (e == cudaSuccess) e = vate::age_prepare(63);
    if (e == cudaSuccess && dev >= 0 && dev < 256) g_prepared[dev] = true;
    return e;
}

// The staging of the host-buffer entry points (and of checkpoints), created
// on first use.  Each piece is created only if missing, so a call after a
// failed one finishes the set-up; copy_stream, created last, marks it done.
int ensure_staging(vate_handle *h) {
    if (h->copy_stream) return VATE_OK;
    auto stream = [](cudaStream_t *s) { return *s ? cudaSuccess : cudaStreamCreateWithFlags(s, cudaStreamNonBlocking); };
    auto event = [](cudaEvent_t *e) { return *e ? cudaSuccess : cudaEventCreateWithFlags(e, cudaEventDisableTiming); };
    auto alloc = [](auto **p, size_t bytes) {
        return *p ? cudaSuccess : cudaMalloc(reinterpret_cast<void **>(p), bytes);
    };
    CU(stream(&h->pairs_stream), "copy stream");
    CU(stream(&h->d2h_stream), "copy stream");
    for (int i = 0; i < INGEST_RING; i++) {
        CU(event(&h->ev_in_ready[i]), "event");
        CU(event(&h->ev_in_free[i]), "event");
        if (alloc(&h->d_in[i], STAGE_RECORDS * sizeof(vate_pair)) != cudaSuccess) {
            cudaGetLastError();
            return fail(VATE_ENOMEM, "staging buffers: out of device memory");
        }
    }
    for (int i = 0; i < 2; i++) {
        CU(event(&h->ev_ready[i]), "event");
        CU(event(&h->ev_free[i]), "event");
        CU(event(&h->ev_done[i]), "event");
        if (alloc(&h->d_stage[i], EST_RECORDS * sizeof(uint32_t)) != cudaSuccess ||
            alloc(&h->d_stage_out[i], EST_RECORDS * sizeof(float)) != cudaSuccess ||
            alloc(&h->d_stage_flags[i], EST_RECORDS) != cudaSuccess) {
            cudaGetLastError();
            return fail(VATE_ENOMEM, "staging buffers: out of device memory");
        }
    }
    CU(stream(&h->copy_stream), "copy stream");
    return VATE_OK;
}

}  // namespace

extern "C" {

const char *vate_last_error(void) { return g_err.c_str(); }

uint64_t vate_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int vate_host_h(const vate_params *params, uint32_t aip, uint32_t i, uint64_t *pid) {
    Geom G;
    int rc = make_geom(params, &G);
    if (rc) return rc;
    if (!pid || i >= G.g) return fail(VATE_EINVAL, "bad pid pointer or i >= g");
    *pid = vate::vat_pid(G, aip, i);
    return VATE_OK;
}

int vate_host_bh(const vate_params *params, uint32_t bip, uint32_t *vid) {
    Geom G;
    int rc = make_geom(params, &G);
    if (rc) return rc;
    if (!vid) return fail(VATE_EINVAL, "vid is NULL");
    *vid = vate::bh(G, bip);
    return VATE_OK;
}

int vate_host_block(const vate_params *params, uint64_t pid, uint32_t *block) {
    Geom G;
    int rc = make_geom(params, &G);
    if (rc) return rc;
    if (!block || pid >= G.P) return fail(VATE_EINVAL, "bad block pointer or pid >= P");
    *block = vate::block_of(G, (uint32_t)pid);
    return VATE_OK;
}

// The handle of a whole pool (hi = ~0: up to P) or of the shard that holds
// the positions [lo, hi).
static int create_range(const vate_params *params, uint64_t lo, uint64_t hi, void *stream, vate_handle **out) {
    if (!out) return fail(VATE_EINVAL, "out is NULL");
    Geom G;
    int rc = make_geom(params, &G);
    if (rc) return rc;
    G.lo = lo;
    G.hi = hi > G.P ? G.P : hi;
    const uint64_t held_bytes = vate::held_bytes(G);

    cudaStream_t st = (cudaStream_t)stream;
    vate_handle *h = new (std::nothrow) vate_handle();
    if (!h) return fail(VATE_ENOMEM, "host allocation failed");
    h->prm = *params;
    h->G = G;
    h->G.frame0 = G.counter == VATE_COUNTER_AT ? 1u : 0u;    // timestamps kept in the frame of block 0
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "no usable CUDA device");
    }
    e = prepare_device(h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "kernel attributes");
    }
    // With VATE_OPT_PERSIST_L2 the pool's kernels launch with a persisting
    // access-policy window over it (hit ratio = persisting capacity / pool),
    // and the handle holds the device's persisting limit that gives the window
    // its effect (persist_acquire); without it, neither.
    if (params->options & VATE_OPT_PERSIST_L2) {
        int persist_max = 0, window_max = 0;
        cudaDeviceGetAttribute(&persist_max, cudaDevAttrMaxPersistingL2CacheSize, h->device);
        cudaDeviceGetAttribute(&window_max, cudaDevAttrMaxAccessPolicyWindowSize, h->device);
        cudaGetLastError();
        if (persist_max > 0 && window_max > 0 && vate::persist_acquire(h->device, (size_t)persist_max)) {
            h->persist_l2 = true;
            h->G.l2_window_bytes = held_bytes < (uint64_t)window_max ? held_bytes : (uint64_t)window_max;
            double ratio = (double)persist_max / (double)h->G.l2_window_bytes;
            h->G.l2_hit_ratio = ratio >= 1.0 ? 1.0f : (float)ratio;
        }
    }
    size_t nbins = G.twok + 1;
    uint8_t *mem = nullptr;
    if (cudaMalloc(&mem, held_bytes) == cudaSuccess) h->G.pool = mem - G.lo * G.atw;   // position 0's address
    if (!mem || cudaMalloc(&h->d_hist, nbins * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&h->d_acc, nbins * sizeof(uint64_t)) != cudaSuccess ||
        cudaMalloc(&h->d_ticket, sizeof(unsigned int)) != cudaSuccess ||
        cudaMalloc(&h->d_dbg, 2 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        vate_destroy(h);
        return fail(VATE_ENOMEM, "out of device memory for a pool of 2^%u ATs", G.c);
    }
    h->G.dbg = h->d_dbg;
    e = cudaMemsetAsync(h->d_ticket, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_dbg, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_hist, 0, nbins * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_acc, 0, nbins * sizeof(uint64_t), st);
    if (e == cudaSuccess) e = vate::launch_init(h->G, st, h->sms);
    if (e != cudaSuccess) {
        vate_destroy(h);
        return cuda_fail(e, "pool initialisation");
    }
    *out = h;
    return VATE_OK;
}


int vate_create(const vate_params *params, void *stream, vate_handle **out) {
    return create_range(params, 0, ~0ull, stream, out);
}

int vate_create_shard(const vate_params *params, uint64_t pid_lo, uint64_t pid_hi, void *stream, vate_handle **out) {
    Geom G;
    if (int rc = make_geom(params, &G)) return rc;
    if (G.packed) return fail(VATE_EINVAL, "shards hold byte or 16-bit ATs (at_bits 0, 8 or 16)");
    if (pid_lo >= pid_hi || pid_hi > G.P || (pid_lo & 63u) != 0 || ((pid_hi & 63u) != 0 && pid_hi != G.P))
        return fail(VATE_EINVAL, "a shard holds positions [lo, hi) with lo < hi <= P, both multiples of 64 "
                                 "(got [%llu, %llu), P = %llu)", (unsigned long long)pid_lo,
                    (unsigned long long)pid_hi, (unsigned long long)G.P);
    return create_range(params, pid_lo, pid_hi, stream, out);
}

int vate_destroy(vate_handle *h) {
    if (!h) return VATE_OK;
    if (h->pairs_stream) cudaStreamSynchronize(h->pairs_stream);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    if (h->d2h_stream) cudaStreamSynchronize(h->d2h_stream);
    if (h->persist_l2) vate::persist_release(h->device);
    if (h->G.pool) cudaFree(vate::pool_mem(h->G));
    cudaFree(h->d_hist);
    cudaFree(h->d_acc);
    cudaFree(h->d_ticket);
    cudaFree(h->d_dbg);
    cudaFree(h->d_scratch);
    for (int i = 0; i < 2; i++) {
        cudaFree(h->d_stage[i]);
        cudaFree(h->d_stage_out[i]);
        cudaFree(h->d_stage_flags[i]);
        if (h->ev_ready[i]) cudaEventDestroy(h->ev_ready[i]);
        if (h->ev_free[i]) cudaEventDestroy(h->ev_free[i]);
        if (h->ev_done[i]) cudaEventDestroy(h->ev_done[i]);
    }
    for (int i = 0; i < INGEST_RING; i++) {
        cudaFree(h->d_in[i]);
        if (h->ev_in_ready[i]) cudaEventDestroy(h->ev_in_ready[i]);
        if (h->ev_in_free[i]) cudaEventDestroy(h->ev_in_free[i]);
    }
    if (h->pairs_stream) cudaStreamDestroy(h->pairs_stream);
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
    delete h;
    return VATE_OK;
}

int vate_debug_checks(void) {
#ifdef VATE_DEBUG
    return 1;
#else
    return 0;
#endif
}

int vate_debug_status(vate_handle *h, uint32_t *bits, uint64_t *first, int clear, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (!bits) return fail(VATE_EINVAL, "bits is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long w[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(w, h->d_dbg, sizeof w, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && clear) {
        e = cudaMemsetAsync(h->d_dbg, 0, sizeof w, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "debug status");
    *bits = (uint32_t)w[0];
    if (first) *first = w[1];
    return VATE_OK;
}

int vate_debug_poke(vate_handle *h, uint64_t pid, uint32_t value, void *stream) {
#ifndef VATE_DEBUG
    (void)h; (void)pid; (void)value; (void)stream;
    return fail(VATE_EINVAL, "vate_debug_poke exists in the checked build (VATE_DEBUG) only");
#else
    if (int rc = check_handle(h)) return rc;
    if (h->G.packed) return fail(VATE_EINVAL, "a packed pool cannot be poked");
    if (pid < h->G.lo || pid >= h->G.hi) return fail(VATE_EINVAL, "pid outside the positions held");
    if (value > (h->G.atw == 1u ? 0xFFu : 0xFFFFu)) return fail(VATE_EINVAL, "value wider than an AT");
    const uint16_t v16 = (uint16_t)value;
    const uint8_t v8 = (uint8_t)value;
    cudaError_t e = cudaMemcpyAsync(h->G.pool + pid * h->G.atw, h->G.atw == 1u ? (const void *)&v8 : (const void *)&v16,
                                    h->G.atw, cudaMemcpyHostToDevice, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "poke");
    return VATE_OK;
#endif
}

int vate_get_info(const vate_handle *h, vate_info *out) {
    if (!h) return fail(VATE_EINVAL, "handle is NULL");
    if (!out) return fail(VATE_EINVAL, "out is NULL");
    out->pool_size = h->G.P;
    out->block_a = h->G.a;
    out->block_b = h->G.b;
    out->slice = h->slice;
    out->bact0 = h->bact0;
    out->closed = h->closed ? 1u : 0u;
    out->pid_lo = h->G.lo;
    out->pid_hi = h->G.hi;
    return VATE_OK;
}

int vate_ingest(vate_handle *h, const vate_pair *d_pairs, uint64_t n, int64_t slice, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (n && !d_pairs) return fail(VATE_EINVAL, "d_pairs is NULL");
    if ((reinterpret_cast<uintptr_t>(d_pairs) & 7u) != 0) return fail(VATE_EINVAL, "d_pairs must be 8-byte aligned");
    if (int rc = check_slice(h, slice)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = advance_to(h, slice, st)) return rc;
    cudaError_t e = vate::launch_ingest(h->G, h->bact0, reinterpret_cast<const uint32_t *>(d_pairs), n, st, h->sms);
    if (e != cudaSuccess) return cuda_fail(e, "ingest launch");
    return VATE_OK;
}

int vate_close_slice(vate_handle *h, int64_t slice, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (int rc = check_slice(h, slice)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = advance_to(h, slice, st)) return rc;
    cudaError_t e = vate::launch_census(h->G, h->bact0, h->d_acc, h->sms, h->d_hist, h->d_ticket, st);
    if (e != cudaSuccess) return cuda_fail(e, "census launch");
    h->closed = true;
    return VATE_OK;
}

static int gather_common(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint32_t kprime) {
    if (int rc = check_handle(h)) return rc;
    if (!h->closed) return fail(VATE_ESLICE, "the current slice has not been closed");
    if (kprime < 1 || kprime > h->G.k) return fail(VATE_EINVAL, "kprime must be in [1, k=%u], got %u", h->G.k, kprime);
    if (n && !d_aips) return fail(VATE_EINVAL, "d_aips is NULL");
    return VATE_OK;
}

static int whole_pool_only(const vate_handle *h, const char *what) {
    if (is_shard(h))
        return fail(VATE_EINVAL, "%s needs the whole pool; a shard gives vate_active_counts and vate_census, "
                                 "summed over the shards and passed to vate_estimate_from_counts", what);
    return VATE_OK;
}

int vate_estimate(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint32_t kprime, float *d_out,
                  uint8_t *d_flags, void *stream) {
    if (int rc = gather_common(h, d_aips, n, kprime)) return rc;
    if (int rc = whole_pool_only(h, "vate_estimate")) return rc;
    if (n && !d_out) return fail(VATE_EINVAL, "d_out is NULL");
    cudaError_t e = vate::launch_gather(vate::GATHER_ESTIMATE, h->G, h->bact0, kprime, h->d_hist, d_aips, n, d_out,
                                        d_flags, nullptr, (cudaStream_t)stream, h->sms);
    if (e != cudaSuccess) return cuda_fail(e, "estimate launch");
    return VATE_OK;
}

int vate_active_counts(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint32_t kprime, uint32_t *d_active,
                       void *stream) {
    if (int rc = gather_common(h, d_aips, n, kprime)) return rc;
    if (n && !d_active) return fail(VATE_EINVAL, "d_active is NULL");
    cudaError_t e = vate::launch_gather(vate::GATHER_ACTIVE, h->G, h->bact0, kprime, h->d_hist, d_aips, n, nullptr,
                                        nullptr, d_active, (cudaStream_t)stream, h->sms);
    if (e != cudaSuccess) return cuda_fail(e, "active-count launch");
    return VATE_OK;
}

int vate_age_counts(vate_handle *h, const uint32_t *d_aips, uint64_t n, uint16_t *d_counts, void *stream) {
    if (int rc = gather_common(h, d_aips, n, 1)) return rc;
    if (h->G.g > 65535) return fail(VATE_EINVAL, "vate_age_counts needs g <= 65535");
    if (h->G.atw != 1u || h->G.packed) return fail(VATE_EINVAL, "vate_age_counts needs byte ATs (k <= 63, at_bits 0 or 8)");
    if (int rc = whole_pool_only(h, "vate_age_counts")) return rc;
    if (n && !d_counts) return fail(VATE_EINVAL, "d_counts is NULL");
    cudaError_t e = vate::launch_age_counts(h->G, h->bact0, d_aips, n, d_counts, (cudaStream_t)stream, h->sms);
    if (e != cudaSuccess) return cuda_fail(e, "age-count launch");
    return VATE_OK;
}

int vate_estimate_from_counts(const vate_params *params, const uint32_t *d_active, const uint64_t *d_hist, uint64_t n,
                              uint32_t kprime, float *d_out, uint8_t *d_flags, void *stream) {
    Geom G;
    if (int rc = make_geom(params, &G)) return rc;
    if (kprime < 1 || kprime > G.k) return fail(VATE_EINVAL, "kprime must be in [1, k=%u], got %u", G.k, kprime);
    if (!d_hist) return fail(VATE_EINVAL, "d_hist is NULL");
    if (n && (!d_active || !d_out)) return fail(VATE_EINVAL, "d_active and d_out must not be NULL");
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    CU(vate::launch_estimate_from_counts(G, kprime, d_hist, d_active, n, d_out, d_flags, (cudaStream_t)stream, sms),
       "estimate launch");
    return VATE_OK;
}

int vate_census(vate_handle *h, uint64_t *d_hist, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (!h->closed) return fail(VATE_ESLICE, "the current slice has not been closed");
    if (!d_hist) return fail(VATE_EINVAL, "d_hist is NULL");
    CU(cudaMemcpyAsync(d_hist, h->d_hist, (h->G.twok + 1) * sizeof(uint64_t), cudaMemcpyDeviceToDevice,
                       (cudaStream_t)stream), "census copy");
    return VATE_OK;
}

int vate_copy_pool(vate_handle *h, uint8_t *d_dst, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (!d_dst) return fail(VATE_EINVAL, "d_dst is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((reinterpret_cast<uintptr_t>(d_dst) & (h->G.atw - 1u)) != 0) return fail(VATE_EINVAL, "d_dst must be 2-byte aligned");
    const uint64_t n = h->G.hi - h->G.lo;
    if (h->G.packed) {
        CU(vate::launch_packed_to_paper(h->G, d_dst, 0, n, st, h->sms), "pool copy");
        return VATE_OK;
    }
    CU(cudaMemcpyAsync(d_dst, vate::pool_mem(h->G), n * h->G.atw, cudaMemcpyDeviceToDevice, st), "pool copy");
    if (h->G.frame0) CU(vate::launch_frame_convert(h->G, d_dst, d_dst, h->G.lo, n, true, st, h->sms), "pool convert");
    return VATE_OK;
}

int vate_load_pool(vate_handle *h, const uint8_t *d_src, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (!d_src) return fail(VATE_EINVAL, "d_src is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((reinterpret_cast<uintptr_t>(d_src) & (h->G.atw - 1u)) != 0) return fail(VATE_EINVAL, "d_src must be 2-byte aligned");
    if (h->G.packed) {
        CU(vate::launch_paper_to_packed(h->G, d_src, 0, h->G.P, st, h->sms), "pool load");
        return VATE_OK;
    }
    CU(vate::launch_frame_convert(h->G, d_src, vate::pool_mem(h->G), h->G.lo, h->G.hi - h->G.lo, false, st, h->sms),
       "pool load");
    return VATE_OK;
}

int vate_ingest_host(vate_handle *h, const vate_pair *h_pairs, uint64_t n, int64_t slice, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (n && !h_pairs) return fail(VATE_EINVAL, "h_pairs is NULL");
    if (int rc = check_slice(h, slice)) return rc;
    if (int rc = ensure_staging(h)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = advance_to(h, slice, st)) return rc;
    // chunk copies on the pairs stream into the next free ring buffer; each
    // chunk's SetAT on `stream` waits for its copy, and a buffer is refilled
    // only after the kernel that read it
    for (uint64_t off = 0; off < n; off += STAGE_RECORDS) {
        const uint32_t b = h->in_next;
        h->in_next = (b + 1u) % INGEST_RING;
        uint64_t m = (n - off) < STAGE_RECORDS ? (n - off) : STAGE_RECORDS;
        CU(cudaStreamWaitEvent(h->pairs_stream, h->ev_in_free[b], 0), "wait");
        CU(cudaMemcpyAsync(h->d_in[b], h_pairs + off, m * sizeof(vate_pair), cudaMemcpyHostToDevice, h->pairs_stream),
           "pairs H2D");
        CU(cudaEventRecord(h->ev_in_ready[b], h->pairs_stream), "record");
        CU(cudaStreamWaitEvent(st, h->ev_in_ready[b], 0), "wait");
        cudaError_t e = vate::launch_ingest(h->G, h->bact0, reinterpret_cast<const uint32_t *>(h->d_in[b]), m, st,
                                            h->sms);
        if (e != cudaSuccess) return cuda_fail(e, "ingest launch");
        CU(cudaEventRecord(h->ev_in_free[b], st), "record");
    }
    return VATE_OK;
}

int vate_estimate_host(vate_handle *h, const uint32_t *h_aips, uint64_t n, uint32_t kprime, float *h_out,
                       uint8_t *h_flags, void *stream) {
    if (int rc = gather_common(h, h_aips, n, kprime)) return rc;
    if (int rc = whole_pool_only(h, "vate_estimate_host")) return rc;
    if (n && !h_out) return fail(VATE_EINVAL, "h_out is NULL");
    if (int rc = ensure_staging(h)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    // Three-stage pipeline over chunks of EST_RECORDS hosts and two staging
    // buffers: hosts in on the copy stream, gather + Eq. 11 on `stream`,
    // estimates out on the D2H stream, so that the copies of chunks i+1 and
    // i-1 overlap the gather of chunk i.
    int used = 0;
    for (uint64_t off = 0, i = 0; off < n; off += EST_RECORDS, i++) {
        int b = (int)(i & 1);
        uint64_t m = (n - off) < EST_RECORDS ? (n - off) : EST_RECORDS;
        uint32_t *din = h->d_stage[b];
        CU(cudaStreamWaitEvent(h->copy_stream, h->ev_free[b], 0), "wait");
        CU(cudaMemcpyAsync(din, h_aips + off, m * sizeof(uint32_t), cudaMemcpyHostToDevice, h->copy_stream), "hosts H2D");
        CU(cudaEventRecord(h->ev_ready[b], h->copy_stream), "record");
        CU(cudaStreamWaitEvent(st, h->ev_ready[b], 0), "wait");
        cudaError_t e = vate::launch_gather(vate::GATHER_ESTIMATE, h->G, h->bact0, kprime, h->d_hist, din, m,
                                            h->d_stage_out[b], h_flags ? h->d_stage_flags[b] : nullptr, nullptr, st,
                                            h->sms);
        if (e != cudaSuccess) return cuda_fail(e, "estimate launch");
        CU(cudaEventRecord(h->ev_done[b], st), "record");
        CU(cudaStreamWaitEvent(h->d2h_stream, h->ev_done[b], 0), "wait");
        CU(cudaMemcpyAsync(h_out + off, h->d_stage_out[b], m * sizeof(float), cudaMemcpyDeviceToHost, h->d2h_stream),
           "D2H");
        if (h_flags)
            CU(cudaMemcpyAsync(h_flags + off, h->d_stage_flags[b], m, cudaMemcpyDeviceToHost, h->d2h_stream), "D2H");
        CU(cudaEventRecord(h->ev_free[b], h->d2h_stream), "record");
        used |= 1 << b;
    }
    for (int b = 0; b < 2; b++)            // the caller's stream completes after the last copy out
        if (used & (1 << b)) CU(cudaStreamWaitEvent(st, h->ev_free[b], 0), "wait");
    return VATE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint and resume (include/vate_checkpoint.h)
// ---------------------------------------------------------------------------
namespace {

static_assert(sizeof(vate_checkpoint_header) % 8 == 0, "the image is hashed 8 bytes at a time");

// FNV-1a (Fowler/Noll/Vo), 64-bit offset basis and prime, one 8-byte word per
// round.  `skip` is the byte offset of a word read as zero (the checksum).
struct Fnv {
    uint64_t h = 0xcbf29ce484222325ull;
    void words(const uint8_t *p, uint64_t n_bytes, uint64_t base, uint64_t skip) {
        for (uint64_t o = 0; o < n_bytes; o += 8) {
            uint64_t w;
            std::memcpy(&w, p + o, 8);
            if (base + o == skip) w = 0;
            h = (h ^ w) * 0x100000001b3ull;
        }
    }
};

uint64_t image_bytes(uint32_t twok, uint64_t P) {
    return sizeof(vate_checkpoint_header) + (uint64_t)(twok + 1) * sizeof(uint64_t) + P;
}

constexpr uint64_t CHECKSUM_AT = offsetof(vate_checkpoint_header, checksum);

}  // namespace

extern "C" {

int vate_checkpoint_size(const vate_handle *h, uint64_t *bytes) {
    if (!h) return fail(VATE_EINVAL, "handle is NULL");
    if (int rc = whole_pool_only(h, "a checkpoint")) return rc;
    if (!bytes) return fail(VATE_EINVAL, "bytes is NULL");
    *bytes = image_bytes(h->G.twok, h->G.P * h->G.atw);
    return VATE_OK;
}

int vate_checkpoint(vate_handle *h, void *h_buf, uint64_t bytes, void *stream) {
    if (int rc = check_handle(h)) return rc;
    if (int rc = whole_pool_only(h, "a checkpoint")) return rc;
    if (!h_buf) return fail(VATE_EINVAL, "h_buf is NULL");
    const uint64_t need = image_bytes(h->G.twok, h->G.P * h->G.atw);
    if (bytes < need) return fail(VATE_EINVAL, "checkpoint buffer holds %llu bytes, %llu needed",
                                  (unsigned long long)bytes, (unsigned long long)need);
    uint8_t *img = static_cast<uint8_t *>(h_buf);
    vate_checkpoint_header hd;
    std::memset(&hd, 0, sizeof hd);
    hd.magic = VATE_CHECKPOINT_MAGIC;
    hd.version = VATE_CHECKPOINT_VERSION;
    hd.header_bytes = (uint32_t)sizeof hd;
    hd.params = h->prm;
    hd.slice = h->slice;
    hd.bact0 = h->bact0;
    hd.closed = h->closed ? 1u : 0u;
    hd.hist_bytes = (uint64_t)(h->G.twok + 1) * sizeof(uint64_t);
    hd.pool_bytes = h->G.P * h->G.atw;
    uint8_t *hist = img + sizeof hd, *pool = hist + hd.hist_bytes;
    cudaStream_t st = (cudaStream_t)stream;
    CU(cudaMemcpyAsync(hist, h->d_hist, hd.hist_bytes, cudaMemcpyDeviceToHost, st), "census D2H");
    if (!h->G.frame0 && !h->G.packed) {
        CU(cudaMemcpyAsync(pool, vate::pool_mem(h->G), hd.pool_bytes, cudaMemcpyDeviceToHost, st), "pool D2H");
    } else {                   // the image holds the paper's form: convert piece by piece through a staging buffer
        if (int rc = ensure_staging(h)) return rc;
        const uint32_t w = h->G.atw;
        const uint64_t piece = STAGE_RECORDS * sizeof(vate_pair) / w;    // positions per piece
        uint8_t *stage = reinterpret_cast<uint8_t *>(h->d_in[0]);          // a pair buffer, once its last reader is done
        CU(cudaStreamWaitEvent(st, h->ev_in_free[0], 0), "wait");
        for (uint64_t pos = 0; pos < h->G.P; pos += piece) {
            const uint64_t n = h->G.P - pos < piece ? h->G.P - pos : piece;
            if (h->G.packed)
                CU(vate::launch_packed_to_paper(h->G, stage, pos, n, st, h->sms), "pool convert");
            else
                CU(vate::launch_frame_convert(h->G, h->G.pool + pos * w, stage, pos, n, true, st, h->sms),
                   "pool convert");
            CU(cudaMemcpyAsync(pool + pos * w, stage, n * w, cudaMemcpyDeviceToHost, st), "pool D2H");
            CU(cudaStreamSynchronize(st), "checkpoint");
        }
    }
    CU(cudaStreamSynchronize(st), "checkpoint");
    std::memcpy(img, &hd, sizeof hd);
    Fnv f;
    f.words(img, need, 0, CHECKSUM_AT);
    hd.checksum = f.h;
    std::memcpy(img, &hd, sizeof hd);
    return VATE_OK;
}

int vate_restore(const void *h_buf, uint64_t bytes, void *stream, vate_handle **out) {
    if (!out) return fail(VATE_EINVAL, "out is NULL");
    if (!h_buf) return fail(VATE_EINVAL, "h_buf is NULL");
    if (bytes < sizeof(vate_checkpoint_header))
        return fail(VATE_EINVAL, "checkpoint image of %llu bytes is shorter than its header", (unsigned long long)bytes);
    const uint8_t *img = static_cast<const uint8_t *>(h_buf);
    vate_checkpoint_header hd;
    std::memcpy(&hd, img, sizeof hd);
    if (hd.magic != VATE_CHECKPOINT_MAGIC) return fail(VATE_EINVAL, "not a VATE checkpoint (bad magic)");
    if (hd.version != VATE_CHECKPOINT_VERSION || hd.header_bytes != sizeof hd)
        return fail(VATE_EINVAL, "checkpoint version %u / header of %u bytes is not supported", hd.version,
                    hd.header_bytes);
    Geom G;
    if (int rc = make_geom(&hd.params, &G)) return rc;
    if (hd.pool_bytes != G.P * G.atw || hd.hist_bytes != (uint64_t)(G.twok + 1) * sizeof(uint64_t))
        return fail(VATE_EINVAL, "checkpoint sizes do not match its parameters");
    const uint64_t need = image_bytes(G.twok, G.P * G.atw);
    if (bytes < need)
        return fail(VATE_EINVAL, "checkpoint image truncated: %llu of %llu bytes", (unsigned long long)bytes,
                    (unsigned long long)need);
    if (hd.slice < -1 || hd.bact0 >= G.twok || hd.closed > 1u || (hd.slice < 0 && (hd.bact0 != 0 || hd.closed)))
        return fail(VATE_EINVAL, "checkpoint slice state is inconsistent");
    Fnv f;
    f.words(img, need, 0, CHECKSUM_AT);
    if (f.h != hd.checksum) return fail(VATE_EINVAL, "checkpoint checksum mismatch");
    // AT values beyond the counter's range would index past the census bins
    const uint8_t *hist = img + sizeof hd, *pool = hist + hd.hist_bytes;
    const uint32_t vmax = G.counter == VATE_COUNTER_DR ? G.k : G.twok;
    uint32_t worst = 0;
    if (G.atw == 1u) {
        for (uint64_t i = 0; i < G.P; i++) worst = pool[i] > worst ? pool[i] : worst;
    } else {
        for (uint64_t i = 0; i < G.P; i++) {
            uint16_t v;
            std::memcpy(&v, pool + 2 * i, 2);
            worst = v > worst ? v : worst;
        }
    }
    if (worst > vmax) return fail(VATE_EINVAL, "checkpoint pool holds the value %u, above %u", worst, vmax);
    vate_handle *h = nullptr;
    if (int rc = vate_create(&hd.params, stream, &h)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!h->G.packed) {
        e = cudaMemcpyAsync(h->G.pool, pool, G.P * G.atw, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && h->G.frame0)      // the image holds the paper's form
            e = vate::launch_frame_convert(h->G, h->G.pool, h->G.pool, 0, G.P, false, st, h->sms);
    } else {                                      // pack piece by piece through a staging buffer
        if (int rc = ensure_staging(h)) {
            vate_destroy(h);
            return rc;
        }
        const uint64_t piece = STAGE_RECORDS * sizeof(vate_pair) / G.atw / G.pn * G.pn;   // whole words
        uint8_t *stage = reinterpret_cast<uint8_t *>(h->d_in[0]);
        for (uint64_t pos = 0; e == cudaSuccess && pos < G.P; pos += piece) {
            const uint64_t n = G.P - pos < piece ? G.P - pos : piece;
            e = cudaMemcpyAsync(stage, pool + pos * G.atw, n * G.atw, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = vate::launch_paper_to_packed(h->G, stage, pos, n, st, h->sms);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->d_hist, hist, hd.hist_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        vate_destroy(h);
        return cuda_fail(e, "checkpoint H2D");
    }
    h->slice = hd.slice;
    h->bact0 = hd.bact0;
    h->closed = hd.closed != 0;
    *out = h;
    return VATE_OK;
}

}  // extern "C"
