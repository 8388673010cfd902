// vate_server.cu -- serving loop for many monitors on one GPU (include/vate_server.h).
//
// One scheduler thread owns every vate_handle of the server.  Submitters only
// append requests to a FIFO queue; the scheduler, in a loop:
//   1. retires slots whose completion event has fired (copying estimates back
//      to the caller's buffers for closes) and wakes waiters;
//   2. dispatches queued requests in arrival order while a slot is free: an
//      ingest is copied (through the slot's page-locked buffer unless the
//      caller's buffer is page-locked) to the slot's device buffer and scanned
//      on the monitor's stream; queued ingests that follow it for the same
//      monitor and slice are merged into the same copy and launch; a close
//      copies the host list, takes the census and runs the learned estimate
//      (or Eq. 11) and copies the results back, all on the monitor's stream.
// Requests of different monitors therefore overlap on the device, and new
// requests enter as soon as slots free up.
//
// Host-side fault injection (vate_server_inject) exercises failure handling
// without touching a GPU: the scheduler can be stalled, a monitor's next
// ingest batches dropped (they complete with VATE_EDROPPED and never reach the
// device), or a monitor's next requests held back for a while (late batches).
// Requests are dispatched in arrival order per monitor: a held request holds
// up the later requests of its own monitor only.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vate.h"
#include "vate_learned.h"
#include "vate_server.h"
#include "vate_internal.h"

namespace vate {
int make_geom_checked(const vate_params *p, Geom *G);   // vate_api.cu
}  // namespace vate

using vate::Geom;

namespace {

using Clock = std::chrono::steady_clock;
enum { REQ_INGEST = 0, REQ_CLOSE = 1 };
constexpr int PENDING = -1;

struct Req {
    uint64_t ticket = 0;
    Clock::time_point hold_until{};   // a held (late) request is not dispatched before this
    int kind = REQ_INGEST;
    int32_t mon = -1;
    int64_t slice = 0;
    const void *in = nullptr;
    uint64_t n = 0;
    uint32_t kprime = 0;
    float *out = nullptr;
    uint8_t *flags = nullptr;
    uint32_t sflags = 0;
    Clock::time_point t_submit;
    int err = VATE_OK;             // set when dispatch fails; reported at retirement
    int status = PENDING;          // set once, at retirement (waiters look only at this)
    std::string msg;
};

struct Slot {
    void *d_in = nullptr;
    float *d_out = nullptr;
    uint8_t *d_flags = nullptr;
    void *h_in = nullptr;          // page-locked staging
    float *h_out = nullptr;
    uint8_t *h_flags = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    int kind = REQ_INGEST;
    std::vector<Req *> reqs;
};

struct Mon {
    vate_handle *h = nullptr;
    cudaStream_t st = nullptr;
    const float *model = nullptr;
    uint64_t bytes = 0;
    uint32_t k = 0;
    bool alive = false;
    uint64_t pending = 0;          // queued + in flight
    uint32_t drop_next = 0;        // injected: ingest batches still to drop
    uint32_t hold_next = 0;        // injected: requests still to hold back ...
    uint32_t hold_ms = 0;          // ... for this long each
};

double pct(std::vector<double> v, double p) {
    if (v.empty()) return 0.0;
    size_t i = (size_t)std::min<double>(v.size() - 1, std::max(0.0, p * (v.size() - 1) + 0.5));
    std::nth_element(v.begin(), v.begin() + i, v.end());
    return v[i];
}

}  // namespace

struct vate_server {
    vate_server_config cfg{};
    int device = 0;
    int sms = 148;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> queue;
    std::unordered_map<uint64_t, Req *> reqs;
    std::vector<Slot> slots;
    std::vector<Mon> mons;
    uint64_t next_ticket = 1;
    uint64_t mem_in_use = 0;
    bool stop = false;
    Clock::time_point stall_until{};   // injected: the scheduler does nothing before this
    std::thread th;
    // statistics
    std::vector<double> lat_ingest, lat_close;
    uint64_t ingests = 0, closes = 0, pairs = 0, hosts = 0, merged = 0;
    uint32_t max_in_flight = 0;
};

namespace {

void complete(vate_server *s, Req *r, int status, const char *msg) {
    r->status = status;
    if (msg) r->msg = msg;
    const double ms = std::chrono::duration<double, std::milli>(Clock::now() - r->t_submit).count();
    if (status == VATE_OK) {
        if (r->kind == REQ_INGEST) {
            s->lat_ingest.push_back(ms);
            s->ingests++;
            s->pairs += r->n;
        } else {
            s->lat_close.push_back(ms);
            s->closes++;
            s->hosts += r->n;
        }
    }
    if (r->mon >= 0 && r->mon < (int32_t)s->mons.size()) s->mons[r->mon].pending--;
}

// Retire finished slots (lock held).
bool retire(vate_server *s) {
    bool any = false;
    for (Slot &sl : s->slots) {
        if (!sl.busy) continue;
        cudaError_t e = cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        for (Req *r : sl.reqs) {
            int st = r->err != VATE_OK ? r->err : (e == cudaSuccess ? VATE_OK : VATE_ECUDA);
            if (st == VATE_OK && r->kind == REQ_CLOSE) {
                memcpy(r->out, sl.h_out, r->n * sizeof(float));
                if (r->flags) memcpy(r->flags, sl.h_flags, r->n);
            }
            complete(s, r, st, e == cudaSuccess ? nullptr : cudaGetErrorString(e));
        }
        sl.reqs.clear();
        sl.busy = false;
        any = true;
    }
    if (any) s->cv_done.notify_all();
    return any;
}

// Dispatch queued request number i (plus mergeable followers) into slot `sl`
// (lock held).
void dispatch(vate_server *s, Slot &sl, size_t i) {
    Req *r = s->queue[i];
    s->queue.erase(s->queue.begin() + (long)i);
    Mon &m = s->mons[r->mon];
    sl.reqs.clear();
    sl.reqs.push_back(r);
    sl.kind = r->kind;
    const uint64_t cap = s->cfg.slot_records;
    int rc = VATE_OK;
    cudaError_t e = cudaSuccess;
    if (r->kind == REQ_INGEST) {
        uint64_t total = r->n;
        while (i < s->queue.size()) {      // merge consecutive ingests of the same monitor and slice
            Req *q = s->queue[i];
            if (q->kind != REQ_INGEST || q->mon != r->mon || q->slice != r->slice || total + q->n > cap ||
                m.drop_next || m.hold_next || q->hold_until > Clock::now())
                break;
            s->queue.erase(s->queue.begin() + (long)i);
            sl.reqs.push_back(q);
            total += q->n;
            s->merged++;
        }
        const void *src = r->in;
        if (sl.reqs.size() > 1 || !(r->sflags & VATE_SUBMIT_PINNED)) {
            uint64_t off = 0;
            for (Req *q : sl.reqs) {
                memcpy(static_cast<char *>(sl.h_in) + off * sizeof(vate_pair), q->in, q->n * sizeof(vate_pair));
                off += q->n;
            }
            src = sl.h_in;
        }
        if (total) e = cudaMemcpyAsync(sl.d_in, src, total * sizeof(vate_pair), cudaMemcpyHostToDevice, m.st);
        if (e == cudaSuccess)
            rc = vate_ingest(m.h, static_cast<const vate_pair *>(sl.d_in), total, r->slice, m.st);
    } else {
        const void *src = r->in;
        if (!(r->sflags & VATE_SUBMIT_PINNED) && r->n) {
            memcpy(sl.h_in, r->in, r->n * sizeof(uint32_t));
            src = sl.h_in;
        }
        if (r->n) e = cudaMemcpyAsync(sl.d_in, src, r->n * sizeof(uint32_t), cudaMemcpyHostToDevice, m.st);
        if (e == cudaSuccess) rc = vate_close_slice(m.h, r->slice, m.st);
        if (e == cudaSuccess && rc == VATE_OK && r->n) {
            const uint32_t *d_hosts = static_cast<const uint32_t *>(sl.d_in);
            if (m.model && r->kprime == m.k)
                rc = vate_estimate_learned(m.h, d_hosts, r->n, m.model, sl.d_out, sl.d_flags, m.st);
            else
                rc = vate_estimate(m.h, d_hosts, r->n, r->kprime, sl.d_out, sl.d_flags, m.st);
            if (rc == VATE_OK) e = cudaMemcpyAsync(sl.h_out, sl.d_out, r->n * sizeof(float), cudaMemcpyDeviceToHost, m.st);
            if (rc == VATE_OK && e == cudaSuccess)
                e = cudaMemcpyAsync(sl.h_flags, sl.d_flags, r->n, cudaMemcpyDeviceToHost, m.st);
        }
    }
    if (e != cudaSuccess) {
        rc = VATE_ECUDA;
        cudaGetLastError();
    }
    if (rc != VATE_OK) {
        std::string msg = e != cudaSuccess ? cudaGetErrorString(e) : vate_last_error();
        for (Req *q : sl.reqs) {
            q->err = rc;
            q->msg = msg;
        }
    }
    // retire through the event even on error, after whatever was queued has run
    cudaEventRecord(sl.done, m.st);
    sl.busy = true;
}

// The first queued request that may go now (lock held): requests of one
// monitor go in arrival order, so a monitor whose earliest queued request is
// held back waits, while other monitors' requests pass it.  An injected hold
// is stamped on a monitor's request when it first reaches the front of that
// monitor's line.  Returns the queue size when nothing may go.
size_t next_dispatchable(vate_server *s, Clock::time_point now) {
    std::vector<char> blocked(s->mons.size(), 0);
    for (size_t i = 0; i < s->queue.size(); i++) {
        Req *r = s->queue[i];
        if (blocked[r->mon]) continue;
        Mon &m = s->mons[r->mon];
        if (r->hold_until == Clock::time_point{} && m.hold_next) {
            m.hold_next--;
            r->hold_until = now + std::chrono::milliseconds(m.hold_ms);
        }
        if (r->hold_until > now) {
            blocked[r->mon] = 1;
            continue;
        }
        return i;
    }
    return s->queue.size();
}

// An injected drop: the monitor's next ingest completes with VATE_EDROPPED
// without reaching the device (lock held).  Returns true if it dropped r.
bool drop_injected(vate_server *s, Req *r) {
    Mon &m = s->mons[r->mon];
    if (r->kind != REQ_INGEST || !m.drop_next) return false;
    m.drop_next--;
    complete(s, r, VATE_EDROPPED, "ingest batch dropped (injected fault)");
    return true;
}

void scheduler(vate_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        const Clock::time_point now = Clock::now();
        if (now < s->stall_until) {             // injected stall: neither retire nor dispatch
            lk.unlock();
            std::this_thread::sleep_until(std::min(s->stall_until, now + std::chrono::milliseconds(5)));
            lk.lock();
            continue;
        }
        retire(s);
        uint32_t busy = 0;
        for (Slot &sl : s->slots) busy += sl.busy ? 1u : 0u;
        bool dropped = false;
        while (!s->queue.empty()) {
            const size_t i = next_dispatchable(s, Clock::now());
            if (i == s->queue.size()) break;
            if (drop_injected(s, s->queue[i])) {
                s->queue.erase(s->queue.begin() + (long)i);
                dropped = true;
                continue;
            }
            Slot *free_slot = nullptr;
            for (Slot &sl : s->slots)
                if (!sl.busy) { free_slot = &sl; break; }
            if (!free_slot) break;
            dispatch(s, *free_slot, i);
            busy++;
        }
        if (dropped) s->cv_done.notify_all();
        s->max_in_flight = std::max(s->max_in_flight, busy);
        if (s->stop && s->queue.empty() && busy == 0) break;
        if (busy == 0 && s->queue.empty())
            s->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        else {                               // work on the GPU or held requests: poll briskly
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        }
    }
}

uint64_t monitor_bytes(const vate_params *p, int sms) {
    const uint64_t bins = 2ull * p->k + 1;
    vate::Geom G;
    const uint64_t pool = vate::make_geom_checked(p, &G) == VATE_OK ? vate::held_bytes(G) : (2ull << p->log2_pool);
    return pool + bins * 8 * (1 + 4ull * sms) + 256;
}

int enqueue(vate_server *s, Req *r, uint64_t *ticket) {
    std::lock_guard<std::mutex> g(s->mu);
    if (r->mon < 0 || r->mon >= (int32_t)s->mons.size() || !s->mons[r->mon].alive) {
        delete r;
        return vate::set_error(VATE_EINVAL, "unknown monitor");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->mons[r->mon].pending++;
    s->reqs[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
    s->cv_work.notify_one();
    return VATE_OK;
}

}  // namespace

extern "C" {

int vate_server_create(const vate_server_config *cfg, vate_server **out) {
    if (!cfg || !out) return vate::set_error(VATE_EINVAL, "cfg and out must not be NULL");
    if (cfg->slots < 2 || cfg->slots > 64 || cfg->slot_records < 1024)
        return vate::set_error(VATE_EINVAL, "slots must be in [2, 64] and slot_records >= 1024");
    vate_server *s = new (std::nothrow) vate_server();
    if (!s) return vate::set_error(VATE_ENOMEM, "host allocation failed");
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
        delete s;
        return vate::set_error(VATE_ECUDA, "no usable CUDA device");
    }
    const uint64_t rec = cfg->slot_records;
    const uint64_t slot_bytes = rec * sizeof(vate_pair) + rec * sizeof(float) + rec;
    if (slot_bytes * cfg->slots > cfg->memory_budget_bytes) {
        delete s;
        return vate::set_error(VATE_ENOMEM, "the slots alone exceed the memory budget");
    }
    s->slots.resize(cfg->slots);
    for (Slot &sl : s->slots) {
        bool ok = cudaMalloc(&sl.d_in, rec * sizeof(vate_pair)) == cudaSuccess &&
                  cudaMalloc(&sl.d_out, rec * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&sl.d_flags, rec) == cudaSuccess &&
                  cudaMallocHost(&sl.h_in, rec * sizeof(vate_pair)) == cudaSuccess &&
                  cudaMallocHost(&sl.h_out, rec * sizeof(float)) == cudaSuccess &&
                  cudaMallocHost(&sl.h_flags, rec) == cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            vate_server_destroy(s);
            return vate::set_error(VATE_ENOMEM, "out of memory for the server's slots");
        }
    }
    s->mem_in_use = slot_bytes * cfg->slots;
    s->th = std::thread(scheduler, s);
    *out = s;
    return VATE_OK;
}

int vate_server_destroy(vate_server *s) {
    if (!s) return VATE_OK;
    if (s->th.joinable()) {
        {
            std::lock_guard<std::mutex> g(s->mu);
            s->stop = true;
            s->cv_work.notify_one();
        }
        s->th.join();
    }
    for (Mon &m : s->mons) {
        if (m.h) vate_destroy(m.h);
        if (m.st) cudaStreamDestroy(m.st);
    }
    for (Slot &sl : s->slots) {
        cudaFree(sl.d_in);
        cudaFree(sl.d_out);
        cudaFree(sl.d_flags);
        cudaFreeHost(sl.h_in);
        cudaFreeHost(sl.h_out);
        cudaFreeHost(sl.h_flags);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return VATE_OK;
}

int vate_server_admit(vate_server *s, const vate_params *params, int32_t *id) {
    if (!s || !params || !id) return vate::set_error(VATE_EINVAL, "NULL argument");
    Geom G;
    if (int rc = vate::make_geom_checked(params, &G)) return rc;
    const uint64_t need = monitor_bytes(params, s->sms);
    std::lock_guard<std::mutex> g(s->mu);
    if (s->mem_in_use + need > s->cfg.memory_budget_bytes)
        return vate::set_error(VATE_ENOMEM, "the monitor does not fit in the memory budget left");
    Mon m;
    m.bytes = need;
    m.k = params->k;
    if (cudaStreamCreateWithFlags(&m.st, cudaStreamNonBlocking) != cudaSuccess)
        return vate::set_error(VATE_ECUDA, "stream creation failed");
    int rc = vate_create(params, m.st, &m.h);
    if (rc) {
        cudaStreamDestroy(m.st);
        return rc;
    }
    m.alive = true;
    s->mem_in_use += need;
    s->mons.push_back(m);
    *id = (int32_t)s->mons.size() - 1;
    return VATE_OK;
}

int vate_server_release(vate_server *s, int32_t id) {
    if (!s) return vate::set_error(VATE_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int32_t)s->mons.size() || !s->mons[id].alive) return vate::set_error(VATE_EINVAL, "unknown monitor");
    s->cv_done.wait(lk, [&] { return s->mons[id].pending == 0; });
    Mon &m = s->mons[id];
    cudaStreamSynchronize(m.st);
    vate_destroy(m.h);
    cudaStreamDestroy(m.st);
    m.h = nullptr;
    m.st = nullptr;
    m.alive = false;
    s->mem_in_use -= m.bytes;
    return VATE_OK;
}

int vate_server_set_model(vate_server *s, int32_t id, const float *d_params) {
    if (!s) return vate::set_error(VATE_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> g(s->mu);
    if (id < 0 || id >= (int32_t)s->mons.size() || !s->mons[id].alive) return vate::set_error(VATE_EINVAL, "unknown monitor");
    if (d_params && s->mons[id].k > 15) return vate::set_error(VATE_EINVAL, "the learned estimator needs k <= 15");
    s->mons[id].model = d_params;
    return VATE_OK;
}

int vate_server_submit_ingest(vate_server *s, int32_t id, const vate_pair *h_pairs, uint64_t n, int64_t slice,
                              uint32_t flags, uint64_t *ticket) {
    if (!s || !ticket || (n && !h_pairs)) return vate::set_error(VATE_EINVAL, "NULL argument");
    if (n > s->cfg.slot_records) return vate::set_error(VATE_EINVAL, "batch larger than a slot");
    Req *r = new (std::nothrow) Req();
    if (!r) return vate::set_error(VATE_ENOMEM, "host allocation failed");
    r->kind = REQ_INGEST;
    r->mon = id;
    r->slice = slice;
    r->in = h_pairs;
    r->n = n;
    r->sflags = flags;
    return enqueue(s, r, ticket);
}

int vate_server_submit_close(vate_server *s, int32_t id, int64_t slice, const uint32_t *h_hosts, uint64_t n,
                             uint32_t kprime, float *h_out, uint8_t *h_flags, uint32_t flags, uint64_t *ticket) {
    if (!s || !ticket || (n && (!h_hosts || !h_out))) return vate::set_error(VATE_EINVAL, "NULL argument");
    if (n > s->cfg.slot_records) return vate::set_error(VATE_EINVAL, "host list larger than a slot");
    Req *r = new (std::nothrow) Req();
    if (!r) return vate::set_error(VATE_ENOMEM, "host allocation failed");
    r->kind = REQ_CLOSE;
    r->mon = id;
    r->slice = slice;
    r->in = h_hosts;
    r->n = n;
    r->kprime = kprime;
    r->out = h_out;
    r->flags = h_flags;
    r->sflags = flags;
    return enqueue(s, r, ticket);
}

int vate_server_wait(vate_server *s, uint64_t ticket, uint32_t timeout_ms) {
    if (!s) return vate::set_error(VATE_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return vate::set_error(VATE_EINVAL, "unknown ticket");
    Req *r = it->second;
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->status != PENDING; }))
        return vate::set_error(VATE_ETIMEOUT, "the request has not completed yet");
    int st = r->status;
    std::string msg = r->msg;
    s->reqs.erase(it);
    delete r;
    if (st != VATE_OK) return vate::set_error(st, msg.c_str());
    return VATE_OK;
}

int vate_server_drain(vate_server *s, uint32_t timeout_ms) {
    if (!s) return vate::set_error(VATE_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto idle = [&] {
        if (!s->queue.empty()) return false;
        for (Slot &sl : s->slots)
            if (sl.busy) return false;
        return true;
    };
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
        return vate::set_error(VATE_ETIMEOUT, "requests still in flight");
    return VATE_OK;
}

int vate_server_inject(vate_server *s, const vate_server_fault *f) {
    if (!s || !f) return vate::set_error(VATE_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    if (f->kind == VATE_FAULT_STALL) {
        s->stall_until = Clock::now() + std::chrono::milliseconds(f->ms);
        return VATE_OK;
    }
    if (f->kind != VATE_FAULT_DROP && f->kind != VATE_FAULT_HOLD) return vate::set_error(VATE_EINVAL, "unknown fault kind");
    if (f->mon < 0 || f->mon >= (int32_t)s->mons.size() || !s->mons[f->mon].alive)
        return vate::set_error(VATE_EINVAL, "unknown monitor");
    Mon &m = s->mons[f->mon];
    if (f->kind == VATE_FAULT_DROP) {
        m.drop_next += f->count;
    } else {
        m.hold_next += f->count;
        m.hold_ms = f->ms;
    }
    s->cv_work.notify_one();
    return VATE_OK;
}

int vate_server_get_stats(vate_server *s, vate_server_stats *out, int reset) {
    if (!s || !out) return vate::set_error(VATE_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> g(s->mu);
    out->ingests_done = s->ingests;
    out->closes_done = s->closes;
    out->pairs_done = s->pairs;
    out->hosts_done = s->hosts;
    out->merged_ingests = s->merged;
    out->ingest_p50_ms = pct(s->lat_ingest, 0.50);
    out->ingest_p99_ms = pct(s->lat_ingest, 0.99);
    out->close_p50_ms = pct(s->lat_close, 0.50);
    out->close_p99_ms = pct(s->lat_close, 0.99);
    out->memory_in_use = s->mem_in_use;
    uint32_t live = 0;
    for (Mon &m : s->mons) live += m.alive ? 1u : 0u;
    out->monitors = live;
    out->max_in_flight = s->max_in_flight;
    if (reset) {
        s->lat_ingest.clear();
        s->lat_close.clear();
        s->ingests = s->closes = s->pairs = s->hosts = s->merged = 0;
        s->max_in_flight = 0;
    }
    return VATE_OK;
}

}  // extern "C"
