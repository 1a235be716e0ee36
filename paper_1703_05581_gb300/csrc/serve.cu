// Serving runtime: a request loop over the FFA search with continuous
// batching.  Requests (a host series plus its own search configuration)
// queue on submit; n_slots worker threads, each owning a non-blocking CUDA
// stream, admit them as soon as a slot and enough of the caller's device
// arena (the HBM admission budget) are free, so searches of uneven lengths
// and period ranges run concurrently on the device.  Each admitted request
// gets one contiguous arena block holding its series, its workspace (octave
// series and fold planes stay on the device for the whole search) and its
// periodogram; the block returns to the arena when the request completes.
//
// Admission: first fit in arrival order, except that once the oldest waiting
// request has been passed over MAX_BYPASS times, nothing is admitted ahead of
// it (bounded waiting for large requests).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace ffa {
namespace {

constexpr int MAX_SLOTS = 32;
constexpr int MAX_BYPASS = 8;
constexpr size_t ALIGN = 256;

size_t al(size_t x) { return (x + ALIGN - 1) & ~(ALIGN - 1); }

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// First-fit allocator of 256-byte-aligned blocks over [0, cap), free blocks
// coalesced on release.
class Arena {
  public:
    explicit Arena(size_t cap) : cap_(cap) {
        if (cap > 0) free_[0] = cap;
    }
    static constexpr size_t none = ~(size_t)0;
    size_t alloc(size_t bytes) {
        bytes = al(std::max<size_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[off + bytes] = rest;
                used_ += bytes;
                return off;
            }
        }
        return none;
    }
    void release(size_t off, size_t bytes) {
        bytes = al(std::max<size_t>(bytes, 1));
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }

  private:
    size_t cap_, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Request {
    int64_t ticket = 0;
    ffa_search_config cfg{};
    const void* host_series = nullptr;
    int64_t n = 0;
    double snr_min = 0.0;
    int32_t top_k = 0;
    ffa_record* host_records = nullptr;
    ffa_plan* plan = nullptr;
    size_t need = 0, off = 0, in_bytes = 0, rec_bytes = 0;
    int bypassed = 0;
    // result
    bool done = false;
    ffa_status status = FFA_OK;
    std::string err;
    std::vector<ffa_candidate> cands;
    int64_t best = -1;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

size_t in_bytes_of(const ffa_search_config& c, int64_t n) {
    return (size_t)n * (c.in_type == FFA_IN_U8 ? 1 : 4);
}

}  // namespace
}  // namespace ffa

struct ffa_server {
    ffa_server_config cfg{};
    int device = 0;
    std::unique_ptr<ffa::Arena> arena;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ffa::Request*> queue;
    std::map<int64_t, std::unique_ptr<ffa::Request>> reqs;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;
    char* base = nullptr;     // arena after the per-slot status words
    int32_t* status = nullptr;
    bool stop = false;
    int64_t next_ticket = 1;
    int64_t in_flight = 0;
};

namespace ffa {
namespace {

// Pick the next admissible request (caller holds the lock).
Request* admit(ffa_server* s) {
    if (s->queue.empty()) return nullptr;
    Request* head = s->queue.front();
    const bool head_only = head->bypassed >= MAX_BYPASS;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        Request* r = *it;
        const size_t off = s->arena->alloc(r->need);
        if (off != Arena::none) {
            r->off = off;
            if (r != head) ++head->bypassed;
            s->queue.erase(it);
            return r;
        }
        if (head_only) break;
    }
    return nullptr;
}

void run_request(ffa_server* s, int slot, Request* r) {
    cudaStream_t st = s->streams[(size_t)slot];
    int32_t* d_status = s->status + (size_t)slot * (ALIGN / sizeof(int32_t));
    char* blk = s->base + r->off;
    void* d_series = blk;
    ffa_record* d_rec = (ffa_record*)(blk + al(r->in_bytes));
    void* d_ws = blk + al(r->in_bytes) + al(r->rec_bytes);
    size_t ws_bytes = 0;
    int64_t n_trials = 0;
    ffa_plan_info(r->plan, nullptr, &n_trials, nullptr, nullptr, &ws_bytes);
    ffa_status st_ = FFA_OK;
    auto check = [&](ffa_status x) {
        if (st_ == FFA_OK && x != FFA_OK) {
            st_ = x;
            r->err = ffa_last_error();
        }
    };
    auto cuda = [&](cudaError_t e, const char* what) {
        if (st_ == FFA_OK && e != cudaSuccess) {
            st_ = FFA_ERR_CUDA;
            r->err = std::string(what) + ": " + cudaGetErrorString(e);
        }
    };
    cuda(cudaMemsetAsync(d_status, 0, sizeof(int32_t), st), "serve: status reset");
    cuda(cudaMemcpyAsync(d_series, r->host_series, r->in_bytes, cudaMemcpyHostToDevice, st), "serve: series copy");
    if (st_ == FFA_OK) check(ffa_search(r->plan, d_series, d_ws, ws_bytes, d_rec, d_status, st));
    if (st_ == FFA_OK) {
        r->cands.resize((size_t)std::max(r->top_k, 1));
        int32_t n_out = 0;
        check(ffa_candidates(r->plan, d_rec, r->snr_min, r->top_k, d_ws, ws_bytes, r->cands.data(), &n_out,
                             &r->best, d_status, st, s->cfg.timeout_ms));
        r->cands.resize(st_ == FFA_OK ? (size_t)n_out : 0);
    }
    if (st_ == FFA_OK && r->host_records && n_trials > 0) {
        cuda(cudaMemcpyAsync(r->host_records, d_rec, sizeof(ffa_record) * (size_t)n_trials,
                             cudaMemcpyDeviceToHost, st), "serve: records copy");
        if (st_ == FFA_OK) check(ffa_wait(st, nullptr, s->cfg.timeout_ms));
    }
    if (st_ != FFA_OK) ffa_wait(st, nullptr, s->cfg.timeout_ms);  // nothing of it still in flight
    r->status = st_;
}

void worker(ffa_server* s, int slot) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        Request* r = nullptr;
        s->cv_work.wait(lk, [&] { return s->stop || (r = admit(s)) != nullptr; });
        if (!r) return;  // stopping with nothing admissible
        r->t_admit = now_ms();
        ++s->in_flight;
        if (!s->queue.empty()) s->cv_work.notify_one();  // another idle slot may admit the next
        lk.unlock();
        run_request(s, slot, r);
        lk.lock();
        s->arena->release(r->off, r->need);
        ffa_plan_destroy(r->plan);
        r->plan = nullptr;
        r->t_done = now_ms();
        r->done = true;
        --s->in_flight;
        s->cv_done.notify_all();
        s->cv_work.notify_all();  // memory came back: others may fit now
    }
}

}  // namespace
}  // namespace ffa

using namespace ffa;

extern "C" {

ffa_status ffa_server_request_bytes(const ffa_search_config* cfg, int64_t n, size_t* bytes) {
    if (!cfg || !bytes) return fail(FFA_ERR_ARG, "server_request_bytes: null argument");
    ffa_plan* p = nullptr;
    ffa_status s = ffa_plan_create(cfg, n, &p);
    if (s != FFA_OK) return s;
    int64_t nt = 0;
    size_t ws = 0;
    ffa_plan_info(p, nullptr, &nt, nullptr, nullptr, &ws);
    ffa_plan_destroy(p);
    *bytes = al(in_bytes_of(*cfg, n)) + al(sizeof(ffa_record) * (size_t)std::max<int64_t>(nt, 1)) + al(ws);
    return FFA_OK;
}

ffa_status ffa_server_create(const ffa_server_config* cfg, ffa_server** out) {
    if (!cfg || !out) return fail(FFA_ERR_ARG, "server_create: null argument");
    *out = nullptr;
    if (cfg->n_slots < 1 || cfg->n_slots > MAX_SLOTS) return fail(FFA_ERR_ARG, "server_create: n_slots in [1, 32]");
    if (!cfg->d_arena || (uintptr_t)cfg->d_arena % ALIGN != 0)
        return fail(FFA_ERR_ARG, "server_create: arena must be 256-byte aligned device memory");
    const size_t status_bytes = ALIGN * (size_t)cfg->n_slots;
    if (cfg->arena_bytes <= status_bytes) return fail(FFA_ERR_OOM, "server_create: arena too small");
    std::unique_ptr<ffa_server> s(new (std::nothrow) ffa_server());
    if (!s) return fail(FFA_ERR_OOM, "server_create: host allocation failed");
    s->cfg = *cfg;
    if (s->cfg.timeout_ms <= 0) s->cfg.timeout_ms = 600000;
    FFA_CUDA_TRY(cudaGetDevice(&s->device));
    s->status = (int32_t*)cfg->d_arena;
    s->base = (char*)cfg->d_arena + status_bytes;
    s->arena.reset(new Arena(cfg->arena_bytes - status_bytes));
    for (int i = 0; i < cfg->n_slots; ++i) {
        cudaStream_t st = nullptr;
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            return cuda_fail(e, "server_create: stream");
        }
        s->streams.push_back(st);
    }
    ffa_server* raw = s.get();
    for (int i = 0; i < cfg->n_slots; ++i) raw->workers.emplace_back(worker, raw, i);
    *out = s.release();
    return FFA_OK;
}

ffa_status ffa_server_submit(ffa_server* s, const ffa_search_config* cfg, const void* host_series, int64_t n,
                             double snr_min, int32_t top_k, ffa_record* host_records, int64_t* ticket) {
    if (!s || !cfg || !ticket || (n > 0 && !host_series)) return fail(FFA_ERR_ARG, "server_submit: null argument");
    if (top_k < 0 || top_k > 4096) return fail(FFA_ERR_ARG, "server_submit: top_k in [0, 4096]");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return fail(FFA_ERR_OOM, "server_submit: host allocation failed");
    ffa_status st = ffa_plan_create(cfg, n, &r->plan);
    if (st != FFA_OK) return st;
    r->cfg = *cfg;
    r->host_series = host_series;
    r->n = n;
    r->snr_min = snr_min;
    r->top_k = top_k;
    r->host_records = host_records;
    int64_t nt = 0;
    size_t ws = 0;
    ffa_plan_info(r->plan, nullptr, &nt, nullptr, nullptr, &ws);
    r->in_bytes = in_bytes_of(*cfg, n);
    r->rec_bytes = sizeof(ffa_record) * (size_t)std::max<int64_t>(nt, 1);
    r->need = al(r->in_bytes) + al(r->rec_bytes) + al(ws);
    std::lock_guard<std::mutex> lk(s->mu);
    if (r->need > s->arena->capacity()) {
        ffa_plan_destroy(r->plan);
        return fail(FFA_ERR_OOM, "server_submit: request larger than the whole arena");
    }
    r->ticket = s->next_ticket++;
    r->t_submit = now_ms();
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
    s->cv_work.notify_one();
    return FFA_OK;
}

ffa_status ffa_server_wait(ffa_server* s, int64_t ticket, int32_t timeout_ms, ffa_candidate* out, int32_t cap,
                           int32_t* n_out, int64_t* best, double* times_ms) {
    if (!s) return fail(FFA_ERR_ARG, "server_wait: null server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(FFA_ERR_ARG, "server_wait: unknown ticket");
    Request* r = it->second.get();
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(FFA_ERR_TIMEOUT, "server_wait: request not finished in time");
    const ffa_status st = r->status;
    const std::string err = r->err;
    if (st == FFA_OK) {
        const int32_t m = std::min<int32_t>((int32_t)r->cands.size(), std::max(cap, 0));
        if (m > 0 && !out) return fail(FFA_ERR_ARG, "server_wait: null output");
        for (int32_t i = 0; i < m; ++i) out[i] = r->cands[(size_t)i];
        if (n_out) *n_out = m;
        if (best) *best = r->best;
    }
    if (times_ms) {
        times_ms[0] = r->t_admit - r->t_submit;  // queued
        times_ms[1] = r->t_done - r->t_admit;    // on the device
        times_ms[2] = r->t_done - r->t_submit;   // latency
    }
    s->reqs.erase(it);
    if (st != FFA_OK) return fail(st, "server request failed: " + err);
    return FFA_OK;
}

ffa_status ffa_server_stats(ffa_server* s, int64_t* queued, int64_t* in_flight, size_t* arena_used) {
    if (!s) return fail(FFA_ERR_ARG, "server_stats: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (in_flight) *in_flight = s->in_flight;
    if (arena_used) *arena_used = s->arena->used();
    return FFA_OK;
}

void ffa_server_destroy(ffa_server* s) {
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // finish what is admitted or queued, then stop
        s->cv_done.wait(lk, [&] { return s->queue.empty() && s->in_flight == 0; });
        s->stop = true;
        s->cv_work.notify_all();
    }
    for (auto& t : s->workers) t.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    for (auto& kv : s->reqs)
        if (kv.second->plan) ffa_plan_destroy(kv.second->plan);
    delete s;
}

}  // extern "C"
