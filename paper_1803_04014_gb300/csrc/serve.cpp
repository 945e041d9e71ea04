// Serving loop: continuous batching of GEMM requests (beyond the paper).
//
// A request names FP32 operands already resident on the device and a mode
// (FP16, BF16, E4M3 with per-tensor scales, or the 3-product FP16 split of
// Eq. 2).  serve_submit() queues it; one scheduler thread
//   1. retires finished requests (their completion event has fired) and
//      returns their workspace to the arena,
//   2. admits queued requests in arrival order while an in-flight slot is
//      free and their workspace fits in the HBM budget (a first-fit arena
//      carved out of one allocation made at serve_open),
//   3. launches each admitted request on the least-recently used of S streams
//      (round robin), so requests that arrive while others run overlap them
//      on the GPU.  Launches happen outside the lock that submit and poll
//      take.
// A request's kernels and tile shapes depend only on (mode, m, n, k), so its
// result is bitwise the same alone and in any mix.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tcgemm.h"

namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int64_t pad_k(int64_t k, int64_t to) { return (k + to - 1) / to * to; }

// Workspace a request needs in the arena (quantised copies or split pieces).
size_t request_bytes(const tc_request& r) {
    switch (r.mode) {
        case TC_MODE_F16:
        case TC_MODE_BF16: {
            const int64_t kp = pad_k(r.k, 8);
            return round_up(static_cast<size_t>(r.m * kp * 2), kAlign) + round_up(static_cast<size_t>(r.n * kp * 2), kAlign);
        }
        case TC_MODE_E4M3: {
            const int64_t kp = pad_k(r.k, 16);
            return round_up(static_cast<size_t>(r.m * kp), kAlign) + round_up(static_cast<size_t>(r.n * kp), kAlign) + kAlign;
        }
        case TC_MODE_SPLIT3:
            return round_up(gemm_split_workspace_bytes(TC_F16, 3, r.m, r.n, r.k), kAlign);
        default:
            return 0;
    }
}

struct Arena {
    uint8_t* base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_;  // offset -> length

    void init(uint8_t* b, size_t s) {
        base = b;
        size = s;
        free_.clear();
        if (s) free_[0] = s;
    }
    void* alloc(size_t bytes) {
        bytes = round_up(bytes ? bytes : kAlign, kAlign);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used += bytes;
                if (used > peak) peak = used;
                return base + off;
            }
        }
        return nullptr;
    }
    void release(void* p, size_t bytes) {
        bytes = round_up(bytes ? bytes : kAlign, kAlign);
        size_t off = static_cast<uint8_t*>(p) - base;
        used -= bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
};

enum class State { Queued, Running, Done };

struct Req {
    uint64_t ticket = 0;
    tc_request r{};
    size_t ws_bytes = 0;
    void* ws = nullptr;
    State state = State::Queued;
    int status = TC_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    cudaEvent_t ev = nullptr;
};

// Enqueue one request's kernels on `st` using workspace `ws`.
tc_status launch_request(const tc_request& r, void* ws, cudaStream_t st) {
    uint8_t* w = static_cast<uint8_t*>(ws);
    tc_status s;
    switch (r.mode) {
        case TC_MODE_F16:
        case TC_MODE_BF16: {
            const int32_t dt = r.mode == TC_MODE_F16 ? TC_F16 : TC_BF16;
            const int64_t kp = pad_k(r.k, 8);
            void* aq = w;
            void* bq = w + round_up(static_cast<size_t>(r.m * kp * 2), kAlign);
            if ((s = tc_quantize(dt, r.m, r.k, r.A, r.lda, aq, kp, 0, nullptr, st)) != TC_OK) return s;
            if ((s = tc_quantize(dt, r.k, r.n, r.B, r.ldb, bq, kp, 1, nullptr, st)) != TC_OK) return s;
            return gemm_mixed(dt, r.m, r.n, r.k, r.alpha, aq, kp, TC_ROW_MAJOR, bq, kp, TC_COL_MAJOR, r.beta, r.C,
                              r.ldc, nullptr, nullptr, st);
        }
        case TC_MODE_E4M3: {
            const int64_t kp = pad_k(r.k, 16);
            void* aq = w;
            void* bq = w + round_up(static_cast<size_t>(r.m * kp), kAlign);
            float* scales = reinterpret_cast<float*>(static_cast<uint8_t*>(bq) + round_up(static_cast<size_t>(r.n * kp), kAlign));
            if ((s = tc_quantize(TC_E4M3, r.m, r.k, r.A, r.lda, aq, kp, 0, scales, st)) != TC_OK) return s;
            if ((s = tc_quantize(TC_E4M3, r.k, r.n, r.B, r.ldb, bq, kp, 1, scales + 1, st)) != TC_OK) return s;
            return gemm_mixed(TC_E4M3, r.m, r.n, r.k, r.alpha, aq, kp, TC_ROW_MAJOR, bq, kp, TC_COL_MAJOR, r.beta,
                              r.C, r.ldc, scales, scales + 1, st);
        }
        case TC_MODE_SPLIT3:
            return gemm_split(TC_F16, 3, r.m, r.n, r.k, r.alpha, r.A, r.lda, TC_ROW_MAJOR, r.B, r.ldb, TC_ROW_MAJOR,
                              r.beta, r.C, r.ldc, ws, gemm_split_workspace_bytes(TC_F16, 3, r.m, r.n, r.k), st);
        default:
            return TC_ERR_INVALID;
    }
}

}  // namespace

struct tc_server {
    tc_serve_cfg cfg{};
    int dev = 0;
    std::vector<cudaStream_t> streams;
    size_t next_stream = 0;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work;  // scheduler wakes on submit / stop
    std::condition_variable cv_done;  // drain waits on completions
    std::deque<Req*> queue;
    std::vector<Req*> running;
    std::unordered_map<uint64_t, Req*> by_ticket;
    std::vector<cudaEvent_t> event_pool;
    uint64_t next_ticket = 1;
    bool stop = false;
    int64_t submitted = 0, completed = 0, peak_inflight = 0, budget_waits = 0;
    size_t launching = 0;  // admitted requests being launched outside the lock
    std::thread sched;

    struct Admitted {
        Req* q;
        cudaStream_t st;
    };

    void loop() {
        cudaSetDevice(dev);
        std::unique_lock<std::mutex> lk(mu);
        bool blocked_on_budget = false;
        std::vector<Admitted> admitted;
        for (;;) {
            // 1. retire
            bool retired = false;
            for (size_t i = 0; i < running.size();) {
                Req* q = running[i];
                const cudaError_t e = cudaEventQuery(q->ev);
                if (e == cudaErrorNotReady) {
                    ++i;
                    continue;
                }
                q->t_done = now_us();
                if (e != cudaSuccess && q->status == TC_OK) q->status = TC_ERR_CUDA;
                q->state = State::Done;
                arena.release(q->ws, q->ws_bytes);
                q->ws = nullptr;
                event_pool.push_back(q->ev);
                q->ev = nullptr;
                running[i] = running.back();
                running.pop_back();
                ++completed;
                retired = true;
            }
            if (retired) {
                blocked_on_budget = false;
                cv_done.notify_all();
            }
            // 2. admit in arrival order: take the workspace, an event and a stream under the lock ...
            admitted.clear();
            while (!queue.empty() && static_cast<int>(running.size() + admitted.size()) < cfg.max_inflight) {
                Req* q = queue.front();
                void* ws = arena.alloc(q->ws_bytes);
                if (!ws) {
                    if (!blocked_on_budget) ++budget_waits;
                    blocked_on_budget = true;
                    break;
                }
                queue.pop_front();
                q->ws = ws;
                if (event_pool.empty()) {
                    cudaEvent_t ev;
                    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                    event_pool.push_back(ev);
                }
                q->ev = event_pool.back();
                event_pool.pop_back();
                admitted.push_back({q, streams[next_stream]});
                next_stream = (next_stream + 1) % streams.size();
            }
            // ... and launch outside it, so submitters and pollers are not held up by the launches;
            // a request joins `running` (where its event is queried) only once its event is recorded
            if (!admitted.empty()) {
                launching = admitted.size();
                lk.unlock();
                for (auto& a : admitted) {
                    a.q->t_start = now_us();
                    a.q->status = launch_request(a.q->r, a.q->ws, a.st);
                    cudaEventRecord(a.q->ev, a.st);
                }
                lk.lock();
                launching = 0;
                for (auto& a : admitted) {
                    a.q->state = State::Running;
                    running.push_back(a.q);
                }
                if (static_cast<int64_t>(running.size()) > peak_inflight) peak_inflight = running.size();
            }
            if (stop && queue.empty() && running.empty()) break;
            if (running.empty()) {
                cv_work.wait(lk, [&] { return stop || !queue.empty(); });
            } else {
                // poll completions; let submitters in between polls
                lk.unlock();
                std::this_thread::yield();
                lk.lock();
            }
        }
    }
};

extern "C" {

tc_status serve_open(const tc_serve_cfg* cfg, tc_server** out) {
    if (!cfg || !out) return TC_ERR_INVALID;
    *out = nullptr;
    if (cfg->hbm_budget_bytes <= 0 || cfg->max_inflight <= 0 || cfg->num_streams <= 0 || cfg->queue_capacity <= 0)
        return TC_ERR_INVALID;
    auto* s = new tc_server();
    s->cfg = *cfg;
    cudaGetDevice(&s->dev);
    void* base = nullptr;
    if (cudaMalloc(&base, static_cast<size_t>(cfg->hbm_budget_bytes)) != cudaSuccess) {
        delete s;
        return TC_ERR_OOM;
    }
    s->arena.init(static_cast<uint8_t*>(base), static_cast<size_t>(cfg->hbm_budget_bytes));
    for (int i = 0; i < cfg->num_streams; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            cudaFree(base);
            delete s;
            return TC_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    s->sched = std::thread([s] { s->loop(); });
    *out = s;
    return TC_OK;
}

tc_status serve_submit(tc_server* s, const tc_request* req, uint64_t* ticket) {
    if (!s || !req || !ticket) return TC_ERR_INVALID;
    const tc_request& r = *req;
    if (r.mode < TC_MODE_F16 || r.mode > TC_MODE_SPLIT3) return TC_ERR_INVALID;
    if (r.m < 1 || r.n < 1 || r.k < 1 || r.m > 0x7FFFFFFF || r.n > 0x7FFFFFFF || r.k > 0x7FFFFFFF) return TC_ERR_INVALID;
    if (!r.A || !r.B || !r.C || r.lda < r.k || r.ldb < r.n || r.ldc < r.n) return TC_ERR_INVALID;
    const size_t need = request_bytes(r);
    if (need > s->arena.size) return TC_ERR_INVALID;
    auto* q = new Req();
    q->r = r;
    q->ws_bytes = need;
    q->t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete q;
            return TC_ERR_INVALID;
        }
        if (static_cast<int>(s->queue.size()) >= s->cfg.queue_capacity) {
            delete q;
            return TC_ERR_BUSY;
        }
        q->ticket = s->next_ticket++;
        s->by_ticket[q->ticket] = q;
        s->queue.push_back(q);
        ++s->submitted;
    }
    s->cv_work.notify_one();
    *ticket = q->ticket;
    return TC_OK;
}

tc_status serve_poll(tc_server* s, uint64_t ticket, tc_result* out) {
    if (!s) return TC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->by_ticket.find(ticket);
    if (it == s->by_ticket.end()) return TC_ERR_INVALID;
    Req* q = it->second;
    if (q->state != State::Done) return TC_PENDING;
    if (out) {
        out->status = q->status;
        out->reserved = 0;
        out->t_submit_us = q->t_submit;
        out->t_start_us = q->t_start;
        out->t_done_us = q->t_done;
    }
    s->by_ticket.erase(it);
    delete q;
    return TC_OK;
}

tc_status serve_drain(tc_server* s, int64_t timeout_ms) {
    if (!s) return TC_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                                        [&] { return s->queue.empty() && s->running.empty() && s->launching == 0; });
    return ok ? TC_OK : TC_ERR_TIMEOUT;
}

tc_status serve_stats(tc_server* s, int64_t* out5) {
    if (!s || !out5) return TC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out5[0] = s->submitted;
    out5[1] = s->completed;
    out5[2] = static_cast<int64_t>(s->arena.peak);
    out5[3] = s->peak_inflight;
    out5[4] = s->budget_waits;
    return TC_OK;
}

tc_status serve_close(tc_server* s) {
    if (!s) return TC_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->sched.joinable()) s->sched.join();
    cudaSetDevice(s->dev);
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto ev : s->event_pool) cudaEventDestroy(ev);
    for (auto& kv : s->by_ticket) delete kv.second;
    cudaFree(s->arena.base);
    delete s;
    return TC_OK;
}

}  // extern "C"
