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
//   3. launches the admitted requests on S streams in turn, so requests that
//      arrive while others run overlap them on the GPU.  Small requests
//      (m n k <= 2^28, each of m, n, k <= 4096) admitted together are batched
//      by mode, alpha and beta: FP16/BF16 roundings run as one
//      tc_quantize_batch launch and their GEMMs as one grouped launch
//      (gemm_grouped_ws); E4M3 roundings as one tc_quantize_batch_e4m3 (a
//      max-|x| launch and a rounding launch), then a gemm_mixed each.  Small
//      split-3 requests (m n k <= 2^29) run as the one-launch refined GEMM,
//      larger ones in two passes; every other request gets its own launches.
//      Launches happen outside the lock that submit and poll take.
// Whether a request is batched, and its kernels and tile shapes, depend only
// on (mode, m, n, k) and its C alignment, so its result is bitwise the same
// alone and in any mix.
// Requests complete in order on each stream.  After each launch group the
// stream itself writes the group's sequence number into pinned host memory
// (cuStreamWriteValue32), so retiring is a memory read instead of a driver
// call per request (a cudaEventQuery costs about 1.7 us on the Grace host);
// where stream memory operations are unavailable, completion events are
// queried instead, each stream's oldest request only.  A stream whose number
// has not advanced for a second is asked for a sticky error.  The scheduler
// keeps cumulative times of its three phases (serve_timing).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdint>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "serve_batch.h"
#include "tcgemm.h"

namespace {

double now_us() {
    using namespace std::chrono;
    return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int64_t pad_k(int64_t k, int64_t to) { return (k + to - 1) / to * to; }

constexpr int64_t kBatchWork = int64_t(1) << 28;  // m n k of a request run in a batch
constexpr int64_t kBatchDim = 4096;
constexpr size_t kDescBytes = size_t(4) << 20;    // per stream: job tables and tile lists of batches
constexpr size_t kMaxBatch = 64;

bool small_request(const tc_request& r) {
    return r.m <= kBatchDim && r.n <= kBatchDim && r.k <= kBatchDim && r.m * r.n * r.k <= kBatchWork &&
           r.ldc <= 0x7FFFFFFF &&
           ((reinterpret_cast<uintptr_t>(r.A) | reinterpret_cast<uintptr_t>(r.B) |
             reinterpret_cast<uintptr_t>(r.C)) & 3u) == 0;
}

// Requests whose roundings run in a batch: small FP16/BF16 requests (their GEMMs also run as one
// grouped launch) and small E4M3 requests (one max-|x| pass and one rounding launch for all of
// them, then a GEMM each).
bool batched(const tc_request& r) {
    return (r.mode == TC_MODE_F16 || r.mode == TC_MODE_BF16 || r.mode == TC_MODE_E4M3) && small_request(r);
}

// Split-3 requests small enough that launches, not the GPU, bound them run as one launch that forms
// the pieces on chip (gemm_split without a workspace); larger ones in two passes through a
// workspace, which take less GPU time.  Both give the same bits.
constexpr int64_t kFusedSplitWork = int64_t(1) << 29;
bool split_one_launch(const tc_request& r) {
    return r.mode == TC_MODE_SPLIT3 && r.m * r.n * r.k <= kFusedSplitWork && r.lda % 4 == 0 && r.ldb % 4 == 0 &&
           ((reinterpret_cast<uintptr_t>(r.A) | reinterpret_cast<uintptr_t>(r.B)) & 15u) == 0;
}

// Tensor-core work of a request, in FP16 multiply-adds: E4M3 runs at twice the rate, split-3 issues
// three products.
double request_work(const tc_request& r) {
    const double mnk = static_cast<double>(r.m) * static_cast<double>(r.n) * static_cast<double>(r.k);
    return r.mode == TC_MODE_E4M3 ? 0.5 * mnk : r.mode == TC_MODE_SPLIT3 ? 3.0 * mnk : mnk;
}

// Workspace a request needs in the arena (quantised copies or split pieces).
size_t request_bytes(const tc_request& r) {
    if (batched(r) && r.mode == TC_MODE_E4M3) {
        // A (m x kp) and K-major B (n x kp), kp a multiple of 16, then the two scales
        const int64_t kp = pad_k(r.k, 16);
        return round_up(static_cast<size_t>(r.m * kp), kAlign) + round_up(static_cast<size_t>(r.n * kp), kAlign) +
               kAlign;
    }
    if (batched(r)) {
        // row-major A (m x kp) and B (k x np), both 16-byte aligned rows
        return round_up(static_cast<size_t>(r.m * pad_k(r.k, 8) * 2), kAlign) +
               round_up(static_cast<size_t>(r.k * pad_k(r.n, 8) * 2), kAlign);
    }
    if (split_one_launch(r)) return 0;
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
    uint32_t seq = 0;  // the launch group's number on its stream
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
            if (split_one_launch(r))
                return gemm_split(TC_F16, 3, r.m, r.n, r.k, r.alpha, r.A, r.lda, TC_ROW_MAJOR, r.B, r.ldb,
                                  TC_ROW_MAJOR, r.beta, r.C, r.ldc, nullptr, 0, st);
            return gemm_split(TC_F16, 3, r.m, r.n, r.k, r.alpha, r.A, r.lda, TC_ROW_MAJOR, r.B, r.ldb, TC_ROW_MAJOR,
                              r.beta, r.C, r.ldc, ws, gemm_split_workspace_bytes(TC_F16, 3, r.m, r.n, r.k), st);
        default:
            return TC_ERR_INVALID;
    }
}

// One launch pair for `members` (same mode, alpha, beta; all batched): their A and B
// rounded into their workspaces as tc_quantize_batch does, their GEMMs as one
// gemm_grouped_ws with the arena as the A and B base, both schedules in one upload to
// `desc` (kDescBytes of device memory of this stream: stream order keeps an earlier
// batch's kernels ahead of the next upload).  E4M3 members: tc_quantize_batch_e4m3, then
// a gemm_mixed each.
tc_status launch_batch_e4m3(const std::vector<Req*>& members, uint8_t* desc, cudaStream_t st) {
    std::vector<tc_quantize_job> jobs;
    std::vector<float*> scales;
    for (Req* q : members) {
        const tc_request& r = q->r;
        const int64_t kp = pad_k(r.k, 16);
        uint8_t* aq = static_cast<uint8_t*>(q->ws);
        uint8_t* bq = aq + round_up(static_cast<size_t>(r.m * kp), kAlign);
        float* sc = reinterpret_cast<float*>(bq + round_up(static_cast<size_t>(r.n * kp), kAlign));
        jobs.push_back({r.m, r.k, static_cast<const float*>(r.A), r.lda, aq, kp, 0, 0});
        jobs.push_back({r.k, r.n, static_cast<const float*>(r.B), r.ldb, bq, kp, 1, 0});
        scales.push_back(sc);
        scales.push_back(sc + 1);
    }
    const size_t qbytes = tc_quantize_batch_workspace_bytes(static_cast<int32_t>(jobs.size()), jobs.data());
    if (qbytes > kDescBytes) return TC_ERR_INVALID;
    tc_status s = tc_quantize_batch_e4m3(static_cast<int32_t>(jobs.size()), jobs.data(), scales.data(), desc, qbytes,
                                         st);
    for (size_t i = 0; s == TC_OK && i < members.size(); ++i) {
        const tc_request& r = members[i]->r;
        const int64_t kp = pad_k(r.k, 16);
        s = gemm_mixed(TC_E4M3, r.m, r.n, r.k, r.alpha, jobs[2 * i].dst, kp, TC_ROW_MAJOR, jobs[2 * i + 1].dst, kp,
                       TC_COL_MAJOR, r.beta, r.C, r.ldc, scales[2 * i], scales[2 * i + 1], st);
    }
    return s;
}

tc_status launch_batch(const std::vector<Req*>& members, uint8_t* arena_base, uint8_t* desc, cudaStream_t st) {
    const tc_request& r0 = members.front()->r;
    if (r0.mode == TC_MODE_E4M3) return launch_batch_e4m3(members, desc, st);
    const int32_t dt = r0.mode == TC_MODE_F16 ? TC_F16 : TC_BF16;
    std::vector<tc_quantize_job> jobs;
    std::vector<tc_problem> probs;
    uintptr_t c_lo = UINTPTR_MAX;
    for (Req* q : members) c_lo = std::min(c_lo, reinterpret_cast<uintptr_t>(q->r.C));
    c_lo &= ~uintptr_t(7);
    for (Req* q : members) {
        const tc_request& r = q->r;
        const int64_t kp = pad_k(r.k, 8), np = pad_k(r.n, 8);
        uint8_t* aq = static_cast<uint8_t*>(q->ws);
        uint8_t* bq = aq + round_up(static_cast<size_t>(r.m * kp * 2), kAlign);
        jobs.push_back({r.m, r.k, static_cast<const float*>(r.A), r.lda, aq, kp, 0, 0});
        jobs.push_back({r.k, r.n, static_cast<const float*>(r.B), r.ldb, bq, np, 0, 0});
        tc_problem p{};
        p.m = static_cast<int32_t>(r.m);
        p.n = static_cast<int32_t>(r.n);
        p.k = static_cast<int32_t>(r.k);
        p.off_a = (aq - arena_base) / 2;
        p.off_b = (bq - arena_base) / 2;
        p.off_c = static_cast<int64_t>((reinterpret_cast<uintptr_t>(r.C) - c_lo) / 4);
        p.lda = static_cast<int32_t>(kp);
        p.ldb = static_cast<int32_t>(np);
        p.ldc = static_cast<int32_t>(r.ldc);
        probs.push_back(p);
    }
    return tcgserve::round_and_grouped_ws(dt, static_cast<int32_t>(jobs.size()), jobs.data(),
                                          static_cast<int32_t>(probs.size()), probs.data(), arena_base,
                                          reinterpret_cast<float*>(c_lo), r0.alpha, r0.beta, desc, kDescBytes, st);
}

// Descriptor bytes a batch member adds (two rounding jobs of at most 80 bytes and their 64 x 32 tiles
// of at most 32, then for FP16/BF16 the larger of the two grouped layouts: tensor maps and 128 x 256
// tiles, or problem entry and 64 x 64 tiles; an upper bound).
size_t batch_desc_bytes(const tc_request& r) {
    auto tiles = [](int64_t rows, int64_t cols, int64_t tr, int64_t tc) { return ((rows + tr - 1) / tr) * ((cols + tc - 1) / tc); };
    if (r.mode == TC_MODE_E4M3) return 2 * 80 + size_t(tiles(r.m, r.k, 64, 32) + tiles(r.k, r.n, 64, 32)) * 32;
    const size_t mma = 64 + size_t(tiles(r.m, r.n, 64, 64)) * 16;
    const size_t tc = 2 * 128 + size_t(tiles(r.m, r.n, 128, 256)) * 48;
    return 2 * 80 + size_t(tiles(r.m, r.k, 64, 32) + tiles(r.k, r.n, 64, 32)) * 32 + std::max(mma, tc);
}

// The driver's stream-write entry point, if it has one.
PFN_cuStreamWriteValue32_v11070 stream_write_fn() {
    static PFN_cuStreamWriteValue32_v11070 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &p, 11070, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuStreamWriteValue32_v11070>(p);
    });
    return fn;
}

}  // namespace

struct tc_server {
    tc_serve_cfg cfg{};
    int dev = 0;
    std::vector<cudaStream_t> streams;
    std::vector<uint8_t*> desc;  // per stream: kDescBytes for batch descriptors
    size_t next_stream = 0;
    Arena arena;
    std::mutex mu;
    std::condition_variable cv_work;  // scheduler wakes on submit / stop
    std::condition_variable cv_done;  // drain waits on completions
    std::deque<Req*> queue;
    std::vector<std::deque<Req*>> running;  // per stream, in launch order
    size_t n_running = 0;
    // completion numbers: the host's next number per stream, and the last number each stream
    // wrote into pinned host memory (nullptr: completion events instead)
    std::vector<uint32_t> issued_seq;
    volatile uint32_t* done_seq = nullptr;
    std::vector<double> last_progress_us;
    // per stream: the tensor-core work of its admitted, unretired requests, to give each new launch
    // group the least-loaded stream (a request queued behind a long one on its stream waits for it)
    std::vector<double> stream_work;
    std::unordered_map<uint64_t, Req*> by_ticket;
    std::vector<cudaEvent_t> event_pool;
    uint64_t next_ticket = 1;
    bool stop = false;
    int64_t submitted = 0, completed = 0, peak_inflight = 0, budget_waits = 0;
    // scheduler time in retire / admit / launch (ns), launch groups, event queries
    int64_t t_retire_ns = 0, t_admit_ns = 0, t_launch_ns = 0, n_groups = 0, n_queries = 0;
    size_t launching = 0;  // admitted requests being launched outside the lock
    std::thread sched;

    struct Admitted {
        std::vector<Req*> qs;  // one request, or a batch of batched() requests
        size_t si;             // stream index
    };

    void loop() {
        cudaSetDevice(dev);
        std::unique_lock<std::mutex> lk(mu);
        bool blocked_on_budget = false;
        std::vector<Admitted> admitted;
        std::vector<size_t> open_batches;             // indices into `admitted` of batches
        std::map<size_t, size_t> batch_bytes;         // their descriptor bytes so far
        for (;;) {
            // 1. retire: the oldest running requests of each stream, in order
            const double tr0 = now_us();
            bool retired = false;
            for (size_t si = 0; si < running.size(); ++si) {
                auto& fifo = running[si];
                while (!fifo.empty()) {
                    Req* q = fifo.front();
                    cudaError_t e;
                    if (done_seq) {
                        if (static_cast<int32_t>(done_seq[si] - q->seq) >= 0) {
                            e = cudaSuccess;
                        } else if (tr0 - last_progress_us[si] > 1e6) {
                            // no progress for a second: a failed launch never writes its number
                            ++n_queries;
                            e = cudaStreamQuery(streams[si]);
                            if (e == cudaSuccess || e == cudaErrorNotReady) {
                                last_progress_us[si] = tr0;
                                break;
                            }
                        } else {
                            break;
                        }
                    } else {
                        ++n_queries;
                        e = cudaEventQuery(q->ev);
                        if (e == cudaErrorNotReady) break;
                    }
                    last_progress_us[si] = tr0;
                    q->t_done = now_us();
                    if (e != cudaSuccess && q->status == TC_OK) q->status = TC_ERR_CUDA;
                    q->state = State::Done;
                    stream_work[si] -= request_work(q->r);
                    if (fifo.size() == 1) stream_work[si] = 0.0;  // no rounding residue on an idle stream
                    arena.release(q->ws, q->ws_bytes);
                    q->ws = nullptr;
                    if (q->ev) event_pool.push_back(q->ev);
                    q->ev = nullptr;
                    fifo.pop_front();
                    --n_running;
                    ++completed;
                    retired = true;
                }
            }
            const double ta0 = now_us();
            t_retire_ns += static_cast<int64_t>((ta0 - tr0) * 1e3);
            if (retired) {
                blocked_on_budget = false;
                cv_done.notify_all();
            }
            // 2. admit in arrival order: take the workspace, an event and a stream under the lock ...
            admitted.clear();
            open_batches.clear();
            batch_bytes.clear();
            size_t n_admitted = 0;
            while (!queue.empty() && static_cast<int>(n_running + n_admitted) < cfg.max_inflight) {
                Req* q = queue.front();
                void* ws = arena.alloc(q->ws_bytes);
                if (!ws) {
                    if (!blocked_on_budget) ++budget_waits;
                    blocked_on_budget = true;
                    break;
                }
                queue.pop_front();
                q->ws = ws;
                if (!done_seq) {
                    if (event_pool.empty()) {
                        cudaEvent_t ev;
                        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                        event_pool.push_back(ev);
                    }
                    q->ev = event_pool.back();
                    event_pool.pop_back();
                }
                ++n_admitted;
                if (batched(q->r)) {
                    // join an open batch of the same mode, alpha and beta with room left, else open one
                    Admitted* into = nullptr;
                    for (size_t bi : open_batches) {
                        Admitted& a = admitted[bi];
                        const tc_request& r = a.qs.front()->r;
                        if (r.mode == q->r.mode && r.alpha == q->r.alpha && r.beta == q->r.beta &&
                            a.qs.size() < kMaxBatch && batch_bytes[bi] + batch_desc_bytes(q->r) + 1024 <= kDescBytes) {
                            into = &a;
                            batch_bytes[bi] += batch_desc_bytes(q->r);
                            break;
                        }
                    }
                    if (into) {
                        into->qs.push_back(q);
                        stream_work[into->si] += request_work(q->r);
                        continue;
                    }
                    open_batches.push_back(admitted.size());
                    batch_bytes[admitted.size()] = batch_desc_bytes(q->r);
                }
                // the stream with the least work in flight; ties go round-robin
                size_t si = next_stream;
                for (size_t j = 1; j < streams.size(); ++j) {
                    const size_t c = (next_stream + j) % streams.size();
                    if (stream_work[c] < stream_work[si]) si = c;
                }
                next_stream = (si + 1) % streams.size();
                stream_work[si] += request_work(q->r);
                admitted.push_back({{q}, si});
            }
            const double tl0 = now_us();
            t_admit_ns += static_cast<int64_t>((tl0 - ta0) * 1e3);
            // ... and launch outside it, so submitters and pollers are not held up by the launches;
            // a request joins `running` (where its event is queried) only once its event is recorded
            if (!admitted.empty()) {
                launching = n_admitted;
                uint8_t* abase = arena.base;
                lk.unlock();
                for (auto& a : admitted) {
                    const double t0 = now_us();
                    const cudaStream_t st_ = streams[a.si];
                    tc_status st = TC_OK;
                    if (batched(a.qs.front()->r))
                        st = launch_batch(a.qs, abase, desc[a.si], st_);
                    else
                        st = launch_request(a.qs.front()->r, a.qs.front()->ws, st_);
                    if (done_seq) {
                        // the stream writes the group's number once its kernels are done
                        const uint32_t seq = ++issued_seq[a.si];
                        const CUresult wr = stream_write_fn()(
                            reinterpret_cast<CUstream>(st_),
                            static_cast<CUdeviceptr>(reinterpret_cast<uintptr_t>(done_seq + a.si)), seq,
                            CU_STREAM_WRITE_VALUE_DEFAULT);
                        if (wr != CUDA_SUCCESS && st == TC_OK) st = TC_ERR_CUDA;
                        for (Req* q : a.qs) {
                            q->t_start = t0;
                            q->status = st;
                            q->seq = seq;
                        }
                    } else {
                        for (Req* q : a.qs) {
                            q->t_start = t0;
                            q->status = st;
                            cudaEventRecord(q->ev, st_);
                        }
                    }
                }
                const double tl1 = now_us();
                lk.lock();
                t_launch_ns += static_cast<int64_t>((tl1 - tl0) * 1e3);
                n_groups += static_cast<int64_t>(admitted.size());
                launching = 0;
                for (auto& a : admitted)
                    for (Req* q : a.qs) {
                        q->state = State::Running;
                        running[a.si].push_back(q);
                        ++n_running;
                    }
                if (static_cast<int64_t>(n_running) > peak_inflight) peak_inflight = static_cast<int64_t>(n_running);
            }
            if (stop && queue.empty() && n_running == 0) break;
            if (n_running == 0) {
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
        void* d = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            for (auto x : s->desc) cudaFree(x);
            cudaFree(base);
            delete s;
            return TC_ERR_CUDA;
        }
        s->streams.push_back(st);
        if (cudaMalloc(&d, kDescBytes) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            for (auto x : s->desc) cudaFree(x);
            cudaFree(base);
            delete s;
            return TC_ERR_OOM;
        }
        s->desc.push_back(static_cast<uint8_t*>(d));
    }
    s->running.resize(s->streams.size());
    s->issued_seq.assign(s->streams.size(), 0);
    s->last_progress_us.assign(s->streams.size(), now_us());
    s->stream_work.assign(s->streams.size(), 0.0);
    // completion numbers written by the streams into pinned, mapped host memory, where the driver
    // supports stream writes (else completion events)
    void* seq_mem = nullptr;
    if (stream_write_fn() &&
        cudaHostAlloc(&seq_mem, s->streams.size() * sizeof(uint32_t), cudaHostAllocMapped | cudaHostAllocPortable) ==
            cudaSuccess) {
        std::memset(seq_mem, 0, s->streams.size() * sizeof(uint32_t));
        // one write of 0 on the first stream tells whether the driver takes them here
        const CUresult wr = stream_write_fn()(reinterpret_cast<CUstream>(s->streams[0]),
                                              static_cast<CUdeviceptr>(reinterpret_cast<uintptr_t>(seq_mem)), 0u,
                                              CU_STREAM_WRITE_VALUE_DEFAULT);
        if (wr == CUDA_SUCCESS && cudaStreamSynchronize(s->streams[0]) == cudaSuccess)
            s->done_seq = static_cast<volatile uint32_t*>(seq_mem);
        else
            cudaFreeHost(seq_mem);
    }
    cudaGetLastError();
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
                                        [&] { return s->queue.empty() && s->n_running == 0 && s->launching == 0; });
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

tc_status serve_timing(tc_server* s, int64_t* out6) {
    if (!s || !out6) return TC_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out6[0] = s->t_retire_ns;
    out6[1] = s->t_admit_ns;
    out6[2] = s->t_launch_ns;
    out6[3] = s->n_groups;
    out6[4] = s->n_queries;
    out6[5] = s->completed;
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
    if (s->done_seq) cudaFreeHost(const_cast<uint32_t*>(s->done_seq));
    for (auto d : s->desc) cudaFree(d);
    for (auto& kv : s->by_ticket) delete kv.second;
    cudaFree(s->arena.base);
    delete s;
    return TC_OK;
}

}  // extern "C"
