// Served recognition: resident programs, a device text arena with a pinned host mirror, and a
// scheduler thread that batches whatever is pending onto free launch slots (continuous batching).
//
// Each request is recognised by the batched reach and join (the same kernels as ridfa_batch, one
// item per request), so its accept bit is exactly what ridfa_recognize gives for the same text,
// whatever else shares its batch.  The paper has no serving layer; this is the runtime around its
// recogniser (Sec. 3.2).
//
// Flow of one request: submit() reserves [off, off + len) of the arena ring (E_BUSY when full),
// copies a host text into the pinned mirror and queues the request.  The scheduler, whenever a
// launch slot is free, takes every pending request (up to the batch limits), issues one
// host-to-device copy per contiguous arena run, plans the batch into the slot's device block,
// copies the plan's image, launches the reach groups and the join, copies the accept bytes and
// status word back and records an event.  When the event has completed the results are posted and
// the arena ranges released.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <random>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ridfa.h"
#include "ridfa_batch_plan.h"
#include "ridfa_internal.h"

namespace ridfa {
namespace {

using Clock = std::chrono::steady_clock;
constexpr uint64_t kNoArena = ~0ull;
constexpr uint32_t kStatusBadBit = 2u;       // the kernels' status bits
constexpr uint32_t kStatusTimeoutBit = 4u;

inline uint64_t round16(uint64_t x) { return (x + 15) & ~15ull; }

struct Request {
    uint64_t id = 0;
    uint32_t prog = 0;
    const uint8_t *dtext = nullptr;   // device address of the text (arena or the caller's)
    uint64_t len = 0;
    uint64_t arena_seq = kNoArena;    // ring entry holding the text
    uint64_t arena_off = 0;
    uint64_t charge = 0;              // bytes charged to the device budget until posted
    Clock::time_point t0;
};

// Device bytes of a program's tables as uploaded (the same count as ridfa_info.table_bytes).
uint64_t table_bytes_of(const ridfa_program *prog) {
    const HostAutomaton &A = prog->rid;
    return static_cast<uint64_t>(A.trans.size() * 2 + 256 + A.final_bits.size() * 4 + A.ifmask.size() * 4 +
                                 A.slot_state.size() * 2);
}

// Ring allocator over [0, cap): ranges are handed out in order and released in any order; space
// is reclaimed from the oldest live range forward.
class Ring {
  public:
    void reset(uint64_t cap) {
        cap_ = cap;
        head_ = tail_ = 0;
        wrapped_ = false;
        live_.clear();
    }
    bool alloc(uint64_t bytes, uint64_t *off, uint64_t *seq) {
        const uint64_t size = round16(bytes);
        if (size == 0 || size > cap_) return false;
        uint64_t o;
        if (live_.empty()) {
            head_ = tail_ = 0;
            wrapped_ = false;
            o = 0;
        } else if (!wrapped_) {                 // live: [tail, head)
            if (head_ + size <= cap_) {
                o = head_;
            } else if (size <= tail_) {
                o = 0;
                wrapped_ = true;
            } else {
                return false;
            }
        } else {                                // live: [tail, cap) and [0, head)
            if (head_ + size <= tail_) o = head_;
            else return false;
        }
        live_.push_back(Entry{o, size, false});
        head_ = o + size;
        *off = o;
        *seq = seq0_ + live_.size() - 1;
        return true;
    }
    void release(uint64_t seq) {
        if (seq < seq0_ || seq - seq0_ >= live_.size()) return;
        live_[seq - seq0_].freed = true;
        while (!live_.empty() && live_.front().freed) {
            live_.pop_front();
            ++seq0_;
        }
        if (live_.empty()) {
            head_ = tail_ = 0;
            wrapped_ = false;
            return;
        }
        const uint64_t t = live_.front().off;
        if (wrapped_ && t < tail_) wrapped_ = false;    // the oldest range is past the wrap
        tail_ = t;
    }

  private:
    struct Entry {
        uint64_t off, size;
        bool freed;
    };
    uint64_t cap_ = 0, head_ = 0, tail_ = 0, seq0_ = 0;
    bool wrapped_ = false;
    std::deque<Entry> live_;
};

struct Slot {                          // one launch slot: a batch in flight at most
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    BatchPlan *plan = nullptr;
    uint8_t *dblock = nullptr;         // plan's device block
    size_t dcap = 0;
    uint8_t *himg = nullptr;           // pinned image of the block's descriptors
    size_t hcap = 0;
    uint8_t *dacc = nullptr;           // device accept bytes [max_batch_requests]
    uint8_t *hacc = nullptr;           // pinned: accept bytes, then the status word
    LaunchFork fork;                   // the batch's reach groups run concurrently
    std::vector<Request> reqs;
    bool busy = false;
};

}  // namespace
}  // namespace ridfa

struct ridfa_server {
    int device = 0;
    int sms = 1;
    ridfa_server_opts o{};
    std::vector<const ridfa_program *> progs;     // guarded by mu; only appended
    uint8_t *darena = nullptr, *harena = nullptr;
    ridfa::Ring ring;                              // guarded by mu
    std::vector<ridfa::Slot> slots;                // scheduler thread only (after create)
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ridfa::Request> pending;
    std::deque<ridfa_result> done;
    uint64_t next_id = 1, outstanding = 0, in_flight = 0;
    uint64_t tables = 0, charged = 0;              // device budget: resident tables, requests
    ridfa_server_stats stats{};
    size_t slot_bytes = 0;
    bool stop = false;
    std::thread th;
};

namespace ridfa {
namespace {

struct DeviceGuard {                   // switch the calling thread to a device for a scope
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Post results for the requests of one batch (status rs, or per-request accept bytes from acc).
void post(ridfa_server *S, const std::vector<Request> &reqs, int rs, const uint8_t *acc) {
    const Clock::time_point now = Clock::now();
    std::lock_guard<std::mutex> lock(S->mu);
    for (size_t i = 0; i < reqs.size(); ++i) {
        const Request &r = reqs[i];
        ridfa_result res{};
        res.req_id = r.id;
        res.status = rs;
        res.accept = (rs == RIDFA_OK && acc) ? acc[i] : 0u;
        res.latency_us = std::chrono::duration<double, std::micro>(now - r.t0).count();
        S->done.push_back(res);
        if (r.arena_seq != kNoArena) S->ring.release(r.arena_seq);
        S->charged -= r.charge;
        --S->in_flight;
        ++S->stats.completed;
    }
    S->cv_done.notify_all();
}

int grow_slot(ridfa_server *S, Slot &sl, size_t dneed, size_t hneed) {
    if (dneed > sl.dcap) {
        if (sl.dblock) cudaFree(sl.dblock);
        sl.dblock = nullptr;
        const size_t old = sl.dcap;
        sl.dcap = 0;
        const size_t cap = dneed + dneed / 4;
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&sl.dblock), cap);
        if (e != cudaSuccess) sl.dblock = nullptr;
        else sl.dcap = cap;
        {
            std::lock_guard<std::mutex> lock(S->mu);
            S->slot_bytes = S->slot_bytes - old + sl.dcap;
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    if (hneed > sl.hcap) {
        if (sl.himg) cudaFreeHost(sl.himg);
        sl.himg = nullptr;
        sl.hcap = 0;
        const size_t cap = hneed + hneed / 4;
        cudaError_t e = cudaHostAlloc(reinterpret_cast<void **>(&sl.himg), cap, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            sl.himg = nullptr;
            return cuda_fail(e);
        }
        sl.hcap = cap;
    }
    return RIDFA_OK;
}

// Enqueue one batch on a free slot.  On failure the requests are posted with the error.
void launch(ridfa_server *S, Slot &sl, std::vector<Request> &batch) {
    NvtxRange range("ridfa server batch");
    std::vector<const ridfa_program *> progs;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        progs = S->progs;
    }
    const uint32_t n = static_cast<uint32_t>(batch.size());
    int err = RIDFA_OK;
    // the batch's host texts to the device, one copy per contiguous arena run
    uint64_t run_off = 0, run_len = 0;
    auto flush = [&]() {
        if (run_len && err == RIDFA_OK) {
            cudaError_t e = cudaMemcpyAsync(S->darena + run_off, S->harena + run_off, run_len,
                                            cudaMemcpyHostToDevice, sl.st);
            if (e != cudaSuccess) err = cuda_fail(e);
        }
        run_len = 0;
    };
    for (const Request &r : batch) {
        if (r.arena_seq == kNoArena) continue;
        const uint64_t sz = round16(r.len);
        if (run_len && r.arena_off == run_off + run_len) {
            run_len += sz;
        } else {
            flush();
            run_off = r.arena_off;
            run_len = sz;
        }
    }
    flush();
    std::vector<ridfa_batch_item> items(n);
    uint64_t bytes = 0;
    for (uint32_t i = 0; i < n; ++i) {
        items[i] = ridfa_batch_item{batch[i].dtext, batch[i].len, batch[i].prog, 0};
        bytes += batch[i].len;
    }
    // chunk length: the configured one, else adapted to the batch -- about two chunks per resident
    // lane of the GPU (short chunks keep a small batch's latency low, long ones cut the
    // speculation overhead of a large batch), a power of two in [1 KiB, 8 KiB]
    uint32_t L = S->o.chunk_len;
    if (L == 0) {
        const uint64_t per = bytes / (2ull * static_cast<uint64_t>(S->sms) * 1024);
        L = 1024;
        while (L < 8192 && L < per) L <<= 1;
    }
    if (err == RIDFA_OK)
        err = plan_build(sl.plan, progs.data(), static_cast<uint32_t>(progs.size()), items.data(), n, L, S->device);
    if (err == RIDFA_OK) err = grow_slot(S, sl, plan_device_bytes(sl.plan), plan_image_bytes(sl.plan));
    if (err == RIDFA_OK) {
        const size_t img = plan_image_bytes(sl.plan);
        plan_image(sl.plan, sl.dblock, sl.himg);
        cudaError_t e = cudaMemcpyAsync(sl.dblock, sl.himg, img, cudaMemcpyHostToDevice, sl.st);
        if (e != cudaSuccess) err = cuda_fail(e);
    }
    if (err == RIDFA_OK) err = plan_enqueue(sl.plan, sl.dblock, sl.dacc, sl.st, false, &sl.fork);
    if (err == RIDFA_OK) {
        const size_t so = (static_cast<size_t>(S->o.max_batch_requests) + 15) & ~static_cast<size_t>(15);
        cudaError_t e = cudaMemcpyAsync(sl.hacc, sl.dacc, n, cudaMemcpyDeviceToHost, sl.st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.hacc + so, sl.dblock + plan_status_offset(sl.plan), 4, cudaMemcpyDeviceToHost, sl.st);
        if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.st);
        if (e != cudaSuccess) err = cuda_fail(e);
    }
    if (err != RIDFA_OK) {
        cudaStreamSynchronize(sl.st);          // nothing of this batch may still read its buffers
        (void)cudaGetLastError();
        post(S, batch, err, nullptr);
        return;
    }
    {
        std::lock_guard<std::mutex> lock(S->mu);
        ++S->stats.batches;
        if (n > S->stats.max_batch) S->stats.max_batch = n;
        uint32_t b = 0;
        while (b < 15 && (2u << b) <= n) ++b;
        ++S->stats.batch_hist[b];
    }
    sl.reqs.swap(batch);
    sl.busy = true;
}

void finish(ridfa_server *S, Slot &sl, cudaError_t q) {
    int rs = RIDFA_OK;
    if (q != cudaSuccess) {
        (void)cudaGetLastError();
        rs = RIDFA_E_CUDA;
    } else {
        const size_t so = (static_cast<size_t>(S->o.max_batch_requests) + 15) & ~static_cast<size_t>(15);
        uint32_t status = 0;
        std::memcpy(&status, sl.hacc + so, 4);
        if (status & kStatusBadBit) rs = RIDFA_E_STATE;
        else if (status & kStatusTimeoutBit) rs = RIDFA_E_TIMEOUT;
    }
    post(S, sl.reqs, rs, sl.hacc);
    sl.reqs.clear();
    sl.busy = false;
}

void scheduler(ridfa_server *S) {
    cudaSetDevice(S->device);
    std::vector<Request> batch;
    for (;;) {
        bool progressed = false, any_busy = false;
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            finish(S, sl, q);
            progressed = true;
        }
        for (Slot &sl : S->slots) {
            if (sl.busy) continue;
            batch.clear();
            {
                std::lock_guard<std::mutex> lock(S->mu);
                if (S->stop) break;
                uint64_t bytes = 0;
                while (!S->pending.empty() && batch.size() < S->o.max_batch_requests) {
                    const Request &r = S->pending.front();
                    if (!batch.empty() && bytes + r.len > S->o.max_batch_bytes) break;
                    bytes += r.len;
                    batch.push_back(r);
                    S->pending.pop_front();
                }
                S->in_flight += batch.size();
                S->stats.bytes += bytes;
            }
            if (batch.empty()) break;
            launch(S, sl, batch);
            any_busy = any_busy || sl.busy;
            progressed = true;
        }
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop && !any_busy) break;
        if (progressed) continue;
        if (any_busy) {
            // batches in flight: poll their events again soon
            lk.unlock();
            std::this_thread::yield();
        } else {
            S->cv_work.wait(lk, [&] { return S->stop || !S->pending.empty(); });
        }
    }
}

void release_server(ridfa_server *S) {
    DeviceGuard g(S->device);
    for (Slot &sl : S->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.dblock) cudaFree(sl.dblock);
        if (sl.himg) cudaFreeHost(sl.himg);
        if (sl.dacc) cudaFree(sl.dacc);
        if (sl.hacc) cudaFreeHost(sl.hacc);
        free_fork(&sl.fork);
        plan_delete(sl.plan);
    }
    S->slots.clear();
    if (S->darena) cudaFree(S->darena);
    if (S->harena) cudaFreeHost(S->harena);
    S->darena = S->harena = nullptr;
    (void)cudaGetLastError();
}

}  // namespace
}  // namespace ridfa

extern "C" int ridfa_server_create(const ridfa_server_opts *opts, ridfa_server **out) {
    if (!out) return RIDFA_E_ARG;
    ridfa_server *S = new (std::nothrow) ridfa_server();
    if (!S) return RIDFA_E_NOMEM;
    ridfa_server_opts o = opts ? *opts : ridfa_server_opts{-1, 0, 0, 0, 0, 0, 0, 0, 0};
    if (o.device < 0) {
        int d = 0;
        if (cudaGetDevice(&d) != cudaSuccess) {
            delete S;
            return ridfa::cuda_fail(cudaGetLastError());
        }
        o.device = d;
    }
    if (!o.n_streams) o.n_streams = 3;
    if (!o.arena_bytes) o.arena_bytes = 1ull << 30;
    if (!o.max_requests) o.max_requests = 1u << 20;
    if (!o.max_batch_requests) o.max_batch_requests = 8192;
    if (!o.max_batch_bytes) o.max_batch_bytes = 512ull << 20;
    o.arena_bytes = ridfa::round16(o.arena_bytes);
    S->o = o;
    S->device = o.device;
    ridfa::DeviceGuard g(S->device);
    cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
    if (S->sms < 1) S->sms = 1;
    int err = RIDFA_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&S->darena), o.arena_bytes);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&S->harena), o.arena_bytes, cudaHostAllocDefault);
    if (e != cudaSuccess) err = ridfa::cuda_fail(e);
    S->ring.reset(o.arena_bytes);
    S->slots.resize(o.n_streams);
    const size_t so = (static_cast<size_t>(o.max_batch_requests) + 15) & ~static_cast<size_t>(15);
    for (ridfa::Slot &sl : S->slots) {
        if (err != RIDFA_OK) break;
        sl.plan = ridfa::plan_new();
        if (!sl.plan) {
            err = RIDFA_E_NOMEM;
            break;
        }
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&sl.dacc), o.max_batch_requests);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&sl.hacc), so + 16, cudaHostAllocDefault);
        if (e != cudaSuccess) err = ridfa::cuda_fail(e);
        if (err == RIDFA_OK) err = ridfa::make_fork(&sl.fork);
    }
    if (err != RIDFA_OK) {
        ridfa::release_server(S);
        delete S;
        return err;
    }
    S->stats.device_bytes = o.arena_bytes;
    try {
        S->th = std::thread(ridfa::scheduler, S);
    } catch (...) {
        ridfa::release_server(S);
        delete S;
        return RIDFA_E_NOMEM;
    }
    *out = S;
    return RIDFA_OK;
}

extern "C" int ridfa_server_add_program(ridfa_server *S, const ridfa_program *prog, uint32_t *prog_slot) {
    if (!S || !prog || !prog_slot) return RIDFA_E_ARG;
    if (prog->rid.k > RIDFA_MAX_SLOTS) return RIDFA_E_UNSUPPORTED;
    {
        ridfa::DeviceGuard g(S->device);
        std::lock_guard<std::mutex> lock(prog->mu);
        int err = RIDFA_OK;
        if (!ridfa::device_copy(prog, false, S->device, &err)) return err;
    }
    std::lock_guard<std::mutex> lock(S->mu);
    const uint64_t tb = ridfa::table_bytes_of(prog);
    if (S->o.device_budget && S->tables + S->charged + tb > S->o.device_budget) {
        ++S->stats.rejected;
        return RIDFA_E_BUSY;
    }
    S->tables += tb;
    S->stats.table_bytes = S->tables;
    S->stats.budget_peak = std::max(S->stats.budget_peak, S->tables + S->charged);
    *prog_slot = static_cast<uint32_t>(S->progs.size());
    S->progs.push_back(prog);
    S->stats.n_programs = static_cast<uint32_t>(S->progs.size());
    return RIDFA_OK;
}

extern "C" int ridfa_server_submit(ridfa_server *S, uint32_t prog_slot, const uint8_t *text, uint64_t len,
                                   uint32_t flags, uint64_t *req_id) {
    if (!S || !req_id || (len && !text)) return RIDFA_E_ARG;
    const bool on_device = (flags & RIDFA_SUBMIT_DEVICE_TEXT) != 0;
    ridfa::Request r;
    r.len = len;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        if (S->stop || prog_slot >= S->progs.size()) return RIDFA_E_ARG;
        if (len > S->o.max_batch_bytes || (!on_device && ridfa::round16(len) > S->o.arena_bytes))
            return RIDFA_E_TOO_LARGE;
        if (S->outstanding >= S->o.max_requests) {
            ++S->stats.rejected;
            return RIDFA_E_BUSY;
        }
        if (S->o.device_budget) {
            // the arena text (a device text is the caller's) and the kernels' per-chunk scratch:
            // chunk maps (k entries of 2 bytes) and summaries (4 bytes), chunks of at least
            // chunk_len bytes (1 KiB when adaptive), plus descriptors
            const uint64_t L = S->o.chunk_len ? S->o.chunk_len : 1024;
            const uint64_t chunks = len ? (len + L - 1) / L : 0;
            r.charge = (on_device ? 0 : ridfa::round16(len)) + chunks * (2ull * S->progs[prog_slot]->rid.k + 4) + 64;
            if (S->tables + r.charge > S->o.device_budget) return RIDFA_E_TOO_LARGE;
            if (S->tables + S->charged + r.charge > S->o.device_budget) {
                ++S->stats.rejected;
                return RIDFA_E_BUSY;
            }
        }
        if (!on_device && len) {
            uint64_t off = 0, seq = 0;
            if (!S->ring.alloc(len, &off, &seq)) {
                ++S->stats.rejected;
                return RIDFA_E_BUSY;
            }
            r.arena_off = off;
            r.arena_seq = seq;
            r.dtext = S->darena + off;
        } else {
            r.dtext = text;
        }
        r.id = S->next_id++;
        r.prog = prog_slot;
        S->charged += r.charge;
        S->stats.budget_peak = std::max(S->stats.budget_peak, S->tables + S->charged);
        ++S->outstanding;
        ++S->stats.submitted;
    }
    // the copy into the reserved range needs no lock: the request is not queued yet
    if (r.arena_seq != ridfa::kNoArena) std::memcpy(S->harena + r.arena_off, text, len);
    r.t0 = ridfa::Clock::now();
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->pending.push_back(r);
    }
    S->cv_work.notify_one();
    *req_id = r.id;
    return RIDFA_OK;
}

extern "C" int ridfa_server_poll(ridfa_server *S, ridfa_result *out, uint32_t max, uint32_t *n_out,
                                 uint32_t wait_us) {
    if (!S || !n_out || (max && !out)) return RIDFA_E_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_us)
        S->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !S->done.empty(); });
    uint32_t n = 0;
    while (n < max && !S->done.empty()) {
        out[n++] = S->done.front();
        S->done.pop_front();
    }
    S->outstanding -= n;
    *n_out = n;
    return RIDFA_OK;
}

extern "C" int ridfa_server_drain(ridfa_server *S, uint32_t timeout_ms) {
    if (!S) return RIDFA_E_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    const bool ok = S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return S->pending.empty() && S->in_flight == 0; });
    return ok ? RIDFA_OK : RIDFA_E_TIMEOUT;
}

extern "C" int ridfa_server_get_stats(const ridfa_server *S, ridfa_server_stats *out) {
    if (!S || !out) return RIDFA_E_ARG;
    ridfa_server *M = const_cast<ridfa_server *>(S);
    std::lock_guard<std::mutex> lock(M->mu);
    *out = M->stats;
    out->device_bytes = M->o.arena_bytes + M->slot_bytes;
    out->table_bytes = M->tables;
    out->budget_used = M->tables + M->charged;
    return RIDFA_OK;
}

extern "C" void ridfa_server_destroy(ridfa_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    ridfa::release_server(S);
    delete S;
}

extern "C" int ridfa_bench_served_poisson(ridfa_server *S, const uint32_t *prog_slots,
                                          const uint8_t *const *texts, const uint64_t *lens, uint32_t n_texts,
                                          double rate_rps, double seconds, uint64_t seed,
                                          ridfa_loadgen_record *out, uint32_t cap, uint32_t *n_out,
                                          double *wall_s, uint32_t submit_flags) {
    using ridfa::Clock;
    if (!S || !prog_slots || !texts || !lens || !n_texts || !(rate_rps > 0) || !(seconds > 0) || !out ||
        !n_out)
        return RIDFA_E_ARG;
    // the arrival schedule and the text picks, drawn before the clock starts
    std::mt19937_64 rng(seed);
    std::exponential_distribution<double> gap(rate_rps);
    std::uniform_int_distribution<uint32_t> pick(0, n_texts - 1);
    std::vector<double> sched;
    std::vector<uint32_t> which;
    for (double t = gap(rng); t < seconds; t += gap(rng)) {
        if (sched.size() == cap) return RIDFA_E_ARG;
        sched.push_back(t);
        which.push_back(pick(rng));
    }
    const size_t n = sched.size();
    for (size_t i = 0; i < n; ++i) out[i] = ridfa_loadgen_record{which[i], 0, 0, 0, 0.0, 0.0};
    std::unordered_map<uint64_t, size_t> of_req;
    of_req.reserve(n * 2 + 16);
    std::vector<double> submit_s(n, 0.0);
    std::vector<ridfa_result> res(4096);
    size_t next = 0, got = 0;
    int err = RIDFA_OK;
    const Clock::time_point t0 = Clock::now();
    auto now_s = [&] { return std::chrono::duration<double>(Clock::now() - t0).count(); };
    auto drain_results = [&](uint32_t wait_us) {
        uint32_t m = 0;
        const int e = ridfa_server_poll(S, res.data(), static_cast<uint32_t>(res.size()), &m, wait_us);
        if (e != RIDFA_OK) return e;
        for (uint32_t q = 0; q < m; ++q) {
            auto it = of_req.find(res[q].req_id);
            if (it == of_req.end()) continue;        // not one of this run's requests
            const size_t i = it->second;
            of_req.erase(it);
            ridfa_loadgen_record &rec = out[i];
            rec.status = res[q].status;
            rec.accept = res[q].accept;
            rec.server_us = res[q].latency_us;
            rec.latency_us = (submit_s[i] - sched[i]) * 1e6 + res[q].latency_us;
            ++got;
        }
        return RIDFA_OK;
    };
    while (err == RIDFA_OK && (next < n || got < n)) {
        if (next < n && now_s() >= sched[next]) {
            const uint32_t j = which[next];
            uint64_t id = 0;
            const int e = ridfa_server_submit(S, prog_slots[j], texts[j], lens[j], submit_flags, &id);
            if (e == RIDFA_OK) {
                submit_s[next] = now_s();
                of_req.emplace(id, next);
                ++next;
                continue;
            }
            if (e != RIDFA_E_BUSY) {
                err = e;
                break;
            }
            ++out[next].busy_retries;                // full: collect results, then retry
            err = drain_results(50);
            continue;
        }
        err = drain_results(next < n ? 0 : 1000);
    }
    if (wall_s) *wall_s = now_s();
    *n_out = static_cast<uint32_t>(next);
    return err;
}
