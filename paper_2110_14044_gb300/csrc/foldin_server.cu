// Fold-in server (ials_foldin_*): continuous batching of new-user solves
// against frozen, device-resident item factors.
//
// submit() copies a request into a host queue and returns a ticket.  A
// scheduler thread owns the device side.  It admits queued requests in arrival
// order into a batch as long as the batch's device memory fits the free part of
// a fixed workspace arena (memory admission), uploads the batch's inputs with
// one copy and launches two fold-in kernels on one of several stream pairs:
// short requests on one CTA each, long ones (more than kFoldLong interactions)
// on a cluster of kFoldCluster CTAs each, so a long history no longer sets the
// latency of everything batched with it.  Up to kSlots batches are in flight at
// once, so requests that arrive while others run are admitted as soon as a
// stream slot and memory free up and their work overlaps on the device.  Every
// request writes its embedding and a completion flag to mapped host memory as
// it finishes; the scheduler publishes it at once (waking poll() callers) and
// returns the batch's memory when the whole batch is done.  Which kernel a
// request takes depends on its length alone, so its result does not depend on
// the batch it lands in.
#include "ials_internal.cuh"
#include "../../include/ials.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

using namespace ials;

namespace ials {
void set_last_error(const std::string &msg);
}

namespace {

constexpr int kSlots = 4;               // batches in flight
constexpr int kMaxBatch = 2048;         // requests per batch
constexpr size_t kAlign = 256;
constexpr size_t kMaxPending = 1 << 20;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

ials_status sfail(ials_status st, const std::string &msg) {
    ials::set_last_error(msg);
    return st;
}

struct Request {
    uint64_t ticket = 0;
    std::chrono::steady_clock::time_point t_submit, t_done;
    std::vector<int32_t> items;
    std::vector<float> y;
    bool has_y = false;
    bool done = false;
    int status = 0;
    std::vector<float> w;
    uint64_t batch = 0;   // batch it ran in
    int batch_size = 0;   // requests in that batch
    bool cluster = false;  // ran on a CTA cluster
};

// First-fit allocator over [0, size) with coalescing frees.
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> length
    void reset(size_t size) {
        free_.clear();
        free_[0] = size;
    }
    bool alloc(size_t bytes, size_t &off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                const size_t noff = it->first + bytes;
                free_.erase(it);
                if (rest) free_[noff] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
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
};

struct Slot {
    cudaStream_t stream = nullptr, stream2 = nullptr;  // short requests; long requests
    cudaEvent_t ev = nullptr, ev_in = nullptr, ev2 = nullptr;
    bool busy = false;
    std::vector<std::shared_ptr<Request>> reqs;
    size_t off = 0, bytes = 0, out_off = 0;
    // pinned host staging (grown on demand) and device request table
    void *h_in = nullptr;
    size_t h_in_cap = 0;
    FoldReq *h_req = nullptr, *d_req = nullptr;
    int32_t *h_list = nullptr, *d_list = nullptr;
    int32_t *d_st = nullptr;
    // mapped host memory the kernels write: embeddings (kMaxBatch x d), flags
    float *h_out = nullptr, *m_out = nullptr;
    int32_t *h_done = nullptr, *m_done = nullptr;
};

}  // namespace

struct ials_srv {
    int device = 0;
    int32_t d = 0, b = 0, n_items = 0, sweeps = 0;
    float alpha0 = 0, lambda = 0, nu = 0;
    float *H = nullptr, *G = nullptr;
    uint8_t *arena = nullptr;
    size_t arena_bytes = 0;
    Arena alloc;
    Slot slots[kSlots];
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<uint64_t, std::shared_ptr<Request>> table;
    uint64_t next_ticket = 1, next_batch = 1;
    bool stop = false;
    std::string error;
    std::thread worker;

    size_t req_bytes(int n) const {
        return align_up(8 * (size_t)n) + align_up(4 * (size_t)n) +
               align_up(4 * (size_t)foldin_factor_floats(d, b)) + align_up(4 * (size_t)d);
    }

    // Publish the requests of slot s whose completion flag the kernels have set.
    bool publish(Slot &s) {
        bool any = false;
        const auto now = std::chrono::steady_clock::now();
        for (size_t i = 0; i < s.reqs.size(); ++i) {
            Request &r = *s.reqs[i];
            if (r.done) continue;
            const int32_t f = reinterpret_cast<volatile int32_t *>(s.h_done)[i];
            if (f == 0) continue;
            std::atomic_thread_fence(std::memory_order_acquire);
            r.w.assign(s.h_out + i * d, s.h_out + (i + 1) * d);
            r.status = f - 1;
            r.t_done = now;
            r.done = true;
            any = true;
        }
        return any;
    }

    // The whole batch is done: every request is published; the memory returns.
    void retire(Slot &s) {
        publish(s);
        const auto now = std::chrono::steady_clock::now();
        for (auto &r : s.reqs)
            if (!r->done) {  // a finished batch without the request's flag: report it as failed
                r->t_done = now;
                r->status = IALS_ECUDA;
                r->done = true;
                error = "fold-in request finished without its completion flag";
            }
        alloc.release(s.off, s.bytes);
        s.reqs.clear();
        s.busy = false;
    }

    // A batch whose stream reported an error: its requests finish with IALS_ECUDA
    // (instead of staying pending), and its memory returns to the arena.
    void fail_slot(Slot &s, cudaError_t err) {
        error = std::string("fold-in batch: ") + cudaGetErrorString(err);
        const auto now = std::chrono::steady_clock::now();
        for (auto &r : s.reqs) {
            if (r->done) continue;
            r->t_done = now;
            r->status = IALS_ECUDA;
            r->done = true;
        }
        alloc.release(s.off, s.bytes);
        s.reqs.clear();
        s.busy = false;
    }

    // Build and launch one batch on slot s from the head of the queue.  Caller holds mu.
    bool launch(Slot &s) {
        size_t total = 0, in_bytes = 0;
        int k = 0;
        std::vector<size_t> sizes;
        while (k < (int)pending.size() && k < kMaxBatch) {
            const int n = (int)pending[k]->items.size();
            const size_t add = req_bytes(n);
            size_t off;
            if (!alloc.alloc(total + add, off)) break;  // probe that the grown batch still fits
            alloc.release(off, total + add);
            total += add;
            sizes.push_back(add);
            ++k;
        }
        if (k == 0) return false;
        size_t off;
        if (!alloc.alloc(total, off)) return false;
        // layout: [inputs of all requests | outputs (k x d, unused: results go to mapped
        // host memory) | e and factors]
        std::vector<size_t> in_off(k), sc_off(k);
        size_t cur = 0;
        for (int i = 0; i < k; ++i) {
            in_off[i] = cur;
            cur += align_up(8 * pending[i]->items.size());
        }
        in_bytes = cur;
        const size_t out_off = cur;
        cur += align_up(4 * (size_t)d * k);
        for (int i = 0; i < k; ++i) {
            sc_off[i] = cur;
            cur += align_up(4 * pending[i]->items.size()) + align_up(4 * (size_t)foldin_factor_floats(d, b));
        }
        if (cur > total) {  // the packed layout never exceeds the per-request sum; keep it safe anyway
            alloc.release(off, total);
            return false;
        }
        if (in_bytes > s.h_in_cap) {
            if (s.h_in) cudaFreeHost(s.h_in);
            s.h_in_cap = std::max(in_bytes, 2 * s.h_in_cap);
            if (cudaHostAlloc(&s.h_in, s.h_in_cap, cudaHostAllocDefault) != cudaSuccess) {
                cudaGetLastError();
                s.h_in = nullptr;
                s.h_in_cap = 0;
                alloc.release(off, total);
                error = "pinned staging allocation failed";
                return false;
            }
        }
        s.reqs.assign(pending.begin(), pending.begin() + k);
        pending.erase(pending.begin(), pending.begin() + k);
        const uint64_t batch = next_batch++;
        int n_short = 0;
        for (int i = 0; i < k; ++i) {
            s.reqs[i]->batch = batch;
            s.reqs[i]->batch_size = k;
            s.reqs[i]->cluster = (int)s.reqs[i]->items.size() > kFoldLong;
            if (!s.reqs[i]->cluster) s.h_list[n_short++] = i;
        }
        for (int i = 0, j = n_short; i < k; ++i)  // short requests first, then long ones
            if (s.reqs[i]->cluster) s.h_list[j++] = i;
        std::memset(s.h_done, 0, sizeof(int32_t) * k);
        uint8_t *hin = static_cast<uint8_t *>(s.h_in);
        for (int i = 0; i < k; ++i) {
            const Request &r = *s.reqs[i];
            const size_t n = r.items.size();
            std::memcpy(hin + in_off[i], r.items.data(), 4 * n);
            if (r.has_y) std::memcpy(hin + in_off[i] + 4 * n, r.y.data(), 4 * n);
            FoldReq q;
            q.off = (int64_t)(off + in_off[i]);
            q.y_off = (int64_t)(4 * n);
            q.e_off = (int64_t)(off + sc_off[i]) - q.off;
            q.l_off = q.e_off + (int64_t)align_up(4 * n);
            q.w_off = (int64_t)(off + out_off + 4 * (size_t)d * i) - q.off;
            q.n = (int32_t)n;
            q.has_y = r.has_y ? 1 : 0;
            s.h_req[i] = q;
        }
        FoldArgs a;
        a.req = s.d_req;
        a.n_req = k;
        a.list = s.d_list;
        a.n_list = n_short;
        a.w_host = s.m_out;
        a.done_host = s.m_done;
        a.arena = arena;
        a.H = H;
        a.G = G;
        a.d = d;
        a.b = b;
        a.sweeps = sweeps;
        a.alpha0 = alpha0;
        a.lambda = lambda;
        a.nu = nu;
        a.status = s.d_st;
        cudaError_t e = cudaMemcpyAsync(arena + off, hin, in_bytes, cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.d_req, s.h_req, sizeof(FoldReq) * k, cudaMemcpyHostToDevice, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.d_list, s.h_list, sizeof(int32_t) * k, cudaMemcpyHostToDevice, s.stream);
        const bool any_long = n_short < k;
        if (e == cudaSuccess && any_long) e = cudaEventRecord(s.ev_in, s.stream);
        if (e == cudaSuccess && any_long) e = cudaStreamWaitEvent(s.stream2, s.ev_in, 0);
        if (e == cudaSuccess && any_long) {  // long requests: one CTA cluster each, on the second stream
            FoldArgs al = a;
            al.list = s.d_list + n_short;
            al.n_list = k - n_short;
            e = launch_foldin(al, true, s.stream2);
        }
        if (e == cudaSuccess) e = launch_foldin(a, false, s.stream);
        if (e == cudaSuccess && any_long) e = cudaEventRecord(s.ev2, s.stream2);
        if (e == cudaSuccess && any_long) e = cudaStreamWaitEvent(s.stream, s.ev2, 0);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
        if (e != cudaSuccess) {
            error = std::string("fold-in launch: ") + cudaGetErrorString(e);
            cudaGetLastError();
            cudaStreamSynchronize(s.stream);
            cudaStreamSynchronize(s.stream2);
            const auto now = std::chrono::steady_clock::now();
            for (auto &r : s.reqs) {
                r->t_done = now;
                r->status = IALS_ECUDA;
                r->done = true;
            }
            s.reqs.clear();
            alloc.release(off, total);
            return true;
        }
        s.off = off;
        s.bytes = total;
        s.out_off = out_off;
        s.busy = true;
        return true;
    }

    void run() {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        while (!stop) {
            bool progressed = false;
            for (Slot &s : slots) {
                if (!s.busy) continue;
                const cudaError_t q = cudaEventQuery(s.ev);
                if (q == cudaSuccess) {
                    retire(s);
                    progressed = true;
                } else if (q != cudaErrorNotReady) {
                    fail_slot(s, q);
                    progressed = true;
                } else if (publish(s)) {
                    cv_done.notify_all();  // requests finished ahead of their batch
                }
            }
            cudaGetLastError();  // a not-ready query is not an error
            if (progressed) cv_done.notify_all();
            for (Slot &s : slots) {
                if (!s.busy && !pending.empty()) {
                    if (launch(s)) progressed = true;
                    else break;  // the head of the queue does not fit yet
                }
            }
            if (progressed) cv_done.notify_all();
            bool any_busy = false;
            for (Slot &s : slots) any_busy = any_busy || s.busy;
            if (!progressed) {
                if (any_busy) cv_sched.wait_for(lk, std::chrono::microseconds(20));
                else cv_sched.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
        lk.unlock();
        for (Slot &s : slots) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            if (s.stream2) cudaStreamSynchronize(s.stream2);
        }
    }

    ~ials_srv() {
        {
            std::lock_guard<std::mutex> g(mu);
            stop = true;
        }
        cv_sched.notify_all();
        if (worker.joinable()) worker.join();
        for (Slot &s : slots) {
            if (s.ev) cudaEventDestroy(s.ev);
            if (s.ev_in) cudaEventDestroy(s.ev_in);
            if (s.ev2) cudaEventDestroy(s.ev2);
            if (s.stream) cudaStreamDestroy(s.stream);
            if (s.stream2) cudaStreamDestroy(s.stream2);
            if (s.h_in) cudaFreeHost(s.h_in);
            if (s.h_out) cudaFreeHost(s.h_out);
            if (s.h_done) cudaFreeHost(s.h_done);
            if (s.h_req) cudaFreeHost(s.h_req);
            if (s.h_list) cudaFreeHost(s.h_list);
            if (s.d_req) cudaFree(s.d_req);
            if (s.d_list) cudaFree(s.d_list);
            if (s.d_st) cudaFree(s.d_st);
        }
        if (H) cudaFree(H);
        if (G) cudaFree(G);
        if (arena) cudaFree(arena);
        cv_done.notify_all();
    }
};

extern "C" {

ials_status ials_foldin_open(const float *H, int32_t n_items, const ials_params *params,
                             size_t workspace_bytes, int32_t sweeps, void *cuda_stream, ials_srv **out) {
    if (!H || !params || !out || n_items <= 0 || sweeps < 0) return sfail(IALS_EINVAL, "bad fold-in arguments");
    *out = nullptr;
    const ials_params p = *params;
    if (p.d < 8 || p.d > 4096 || p.d % 4 != 0 || (p.b != 16 && p.b != 32 && p.b != 64 && p.b != 128) ||
        p.d % p.b != 0)
        return sfail(IALS_EINVAL, "fold-in needs b in {16, 32, 64, 128} dividing d (d % 4 == 0, d <= 4096)");
    if (!(p.alpha0 >= 0) || !(p.lambda >= 0) || !(p.nu >= 0)) return sfail(IALS_EINVAL, "negative weights");
    std::unique_ptr<ials_srv> s(new (std::nothrow) ials_srv);
    if (!s) return sfail(IALS_ENOMEM, "server");
    cudaGetDevice(&s->device);
    s->d = p.d;
    s->b = p.b;
    s->n_items = n_items;
    s->sweeps = sweeps;
    s->alpha0 = (float)p.alpha0;
    s->lambda = (float)p.lambda;
    s->nu = (float)p.nu;
    const size_t hb = sizeof(float) * (size_t)n_items * p.d;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    float *ws = nullptr;
    const int64_t wsn = gram_ws_floats(n_items, p.d, p.d);
    if (cudaMalloc(&s->H, hb) != cudaSuccess || cudaMalloc(&s->G, sizeof(float) * (size_t)p.d * p.d) != cudaSuccess ||
        cudaMalloc(&ws, sizeof(float) * (size_t)std::max<int64_t>(wsn, 1)) != cudaSuccess ||
        cudaMalloc(&s->arena, workspace_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (ws) cudaFree(ws);
        return sfail(IALS_ENOMEM, "fold-in device memory (H, G^I or the workspace)");
    }
    s->arena_bytes = workspace_bytes;
    s->alloc.reset(workspace_bytes);
    cudaError_t e = cudaMemcpyAsync(s->H, H, hb, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = launch_gram(s->H, n_items, p.d, 0, p.d, s->G, ws, st);  // G^I (Eq. 4)
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(ws);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(IALS_ECUDA, std::string("fold-in set-up: ") + cudaGetErrorString(e));
    }
    for (Slot &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&sl.stream2, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev2, cudaEventDisableTiming) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_req, sizeof(FoldReq) * kMaxBatch, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_list, sizeof(int32_t) * kMaxBatch, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_out, sizeof(float) * (size_t)kMaxBatch * p.d, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostAlloc((void **)&sl.h_done, sizeof(int32_t) * kMaxBatch, cudaHostAllocMapped) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&sl.m_out, sl.h_out, 0) != cudaSuccess ||
            cudaHostGetDevicePointer((void **)&sl.m_done, sl.h_done, 0) != cudaSuccess ||
            cudaMalloc(&sl.d_req, sizeof(FoldReq) * kMaxBatch) != cudaSuccess ||
            cudaMalloc(&sl.d_list, sizeof(int32_t) * kMaxBatch) != cudaSuccess ||
            cudaMalloc(&sl.d_st, sizeof(int32_t) * kMaxBatch) != cudaSuccess) {
            cudaGetLastError();
            return sfail(IALS_ENOMEM, "fold-in streams or staging");
        }
    }
    ials_srv *raw = s.get();
    try {
        s->worker = std::thread([raw] { raw->run(); });
    } catch (...) {
        return sfail(IALS_ENOMEM, "fold-in scheduler thread");
    }
    *out = s.release();
    return IALS_OK;
}

ials_status ials_foldin_submit(ials_srv *s, const int32_t *items, const float *y, int32_t n,
                               uint64_t *ticket) {
    if (!s || !ticket || n < 0 || (n > 0 && !items)) return sfail(IALS_EINVAL, "bad fold-in request");
    auto r = std::make_shared<Request>();
    try {
        r->items.assign(items, items + n);
        if (y) r->y.assign(y, y + n);
    } catch (...) {
        return sfail(IALS_ENOMEM, "request copy");
    }
    for (int32_t v : r->items)
        if (v < 0 || v >= s->n_items) return sfail(IALS_EINVAL, "item id out of range");
    r->has_y = y != nullptr;
    if (s->req_bytes(n) > s->arena_bytes) return sfail(IALS_EINVAL, "request larger than the fold-in workspace");
    {
        std::lock_guard<std::mutex> g(s->mu);
        if (s->pending.size() >= kMaxPending) return sfail(IALS_EAGAIN, "fold-in queue full");
        r->ticket = s->next_ticket++;
        r->t_submit = std::chrono::steady_clock::now();
        s->table[r->ticket] = r;
        s->pending.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_sched.notify_one();
    return IALS_OK;
}

ials_status ials_foldin_poll_info(ials_srv *s, uint64_t ticket, float *w_out, int32_t timeout_us,
                                  ials_foldin_info *info);

ials_status ials_foldin_poll_timed(ials_srv *s, uint64_t ticket, float *w_out, int32_t timeout_us,
                                   double *latency_us) {
    ials_foldin_info info;
    const ials_status st = ials_foldin_poll_info(s, ticket, w_out, timeout_us, &info);
    if (latency_us && (st == IALS_OK || st == IALS_ENOTPD)) *latency_us = info.latency_us;
    return st;
}

ials_status ials_foldin_poll_info(ials_srv *s, uint64_t ticket, float *w_out, int32_t timeout_us,
                                  ials_foldin_info *info) {
    if (!s || !w_out) return sfail(IALS_EINVAL, "bad poll arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->table.find(ticket);
    if (it == s->table.end()) return sfail(IALS_ENOTFOUND, "unknown ticket");
    std::shared_ptr<Request> r = it->second;
    if (!r->done && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; });
    if (!r->done) return timeout_us > 0 ? sfail(IALS_ETIMEDOUT, "result not ready") : IALS_EAGAIN;
    std::memcpy(w_out, r->w.data(), sizeof(float) * (size_t)s->d);
    if (info) {
        info->latency_us = std::chrono::duration<double, std::micro>(r->t_done - r->t_submit).count();
        info->batch = r->batch;
        info->batch_size = r->batch_size;
        info->cluster = r->cluster ? 1 : 0;
    }
    const int st = r->status;
    s->table.erase(it);
    if (st == 4) return sfail(IALS_ENOTPD, "a block Hessian was not positive definite");
    if (st == IALS_ECUDA) return sfail(IALS_ECUDA, s->error.empty() ? "fold-in batch failed" : s->error);
    if (st != 0) return sfail((ials_status)st, "fold-in failed");
    return IALS_OK;
}

ials_status ials_foldin_poll(ials_srv *s, uint64_t ticket, float *w_out, int32_t timeout_us) {
    return ials_foldin_poll_timed(s, ticket, w_out, timeout_us, nullptr);
}

ials_status ials_foldin_close(ials_srv *s) {
    delete s;
    return IALS_OK;
}

}  // extern "C"
