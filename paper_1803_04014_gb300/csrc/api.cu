// Host side of the C ABI (include/tcgemm.h): argument checks, per-device
// state (SM count, status word), TMA descriptor encoding, workspaces,
// grouped-GEMM plans and dispatch to the kernels.
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "grouped_sched.h"
#include "launch.h"
#include "tcgemm.h"
#include "tcgemm_debug.h"

namespace {

thread_local std::string g_err;

tc_status fail(tc_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

tc_status cuda_fail(cudaError_t e, const char* what) {
    return fail(TC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct Device {
    bool ready = false;
    int sm_count = 0;
    int cc_major = 0, cc_minor = 0;
    int* status = nullptr;  // device status word (first error wins)
    // flags of the pair kernels' parts of K, one block per stream (per host thread for
    // cudaStreamPerThread), and the count that gives every launch its token
    std::mutex kmu;
    std::map<std::pair<cudaStream_t, std::thread::id>, unsigned long long*> kflags;
    std::atomic<unsigned long long> ktoken{0};
};

std::mutex g_mu;
Device g_dev[64];
static __device__ __align__(256) int g_status_word[64];  // one copy per device; word 0 is used


tc_status get_device(Device** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(TC_ERR_INVALID, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    Device& d = g_dev[dev];
    if (!d.ready) {
        if ((e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "cudaDeviceGetAttribute");
        cudaDeviceGetAttribute(&d.cc_major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&d.cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
        // the status word is a static device variable (zero at module load): no allocation
        void* sw = nullptr;
        if ((e = cudaGetSymbolAddress(&sw, g_status_word)) != cudaSuccess)
            return cuda_fail(e, "cudaGetSymbolAddress(status)");
        d.status = static_cast<int*>(sw);
        // keep freed stream-ordered workspace cached in the pool instead of returning it each sync
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t threshold = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
        }
        d.ready = true;
    }
    *out = &d;
    return TC_OK;
}

// Flags and token of one launch of the pair kernels with parts of K on `st`.  The first part of a
// cut tile stores the launch's token in its flags and the second waits for that value; tokens count
// up per device from 1, so flags left by earlier launches never match.
//  - An eager launch uses its stream's own block (allocated and zeroed on the stream's first such
//    launch, kept for the process): launches on one stream never run at the same time.
//  - A launch being captured into a graph uses a block the graph allocates and zeroes at each replay
//    and frees after the launch (*owned): a replay may run on another stream beside eager launches on
//    this one, and its token is the same at every replay.
//  - nullptr when neither can be had; the kernels then cut halves of N instead of parts of K.
unsigned long long* kpart_flags(Device* d, cudaStream_t st, unsigned long long* token, bool* owned) {
    *owned = false;
    *token = d->ktoken.fetch_add(1, std::memory_order_relaxed) + 1;
    const size_t bytes = sizeof(unsigned long long) * tcg::kKpartFlags;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    void* p = nullptr;
    if (cs == cudaStreamCaptureStatusActive) {
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        if (cudaMemsetAsync(p, 0, bytes, st) != cudaSuccess) {
            cudaFreeAsync(p, st);
            cudaGetLastError();
            return nullptr;
        }
        *owned = true;
        return static_cast<unsigned long long*>(p);
    }
    if (cs != cudaStreamCaptureStatusNone) return nullptr;
    const auto key = std::make_pair(st, st == cudaStreamPerThread ? std::this_thread::get_id() : std::thread::id());
    std::lock_guard<std::mutex> lk(d->kmu);
    auto it = d->kflags.find(key);
    if (it != d->kflags.end()) return it->second;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (cudaMemsetAsync(p, 0, bytes, st) != cudaSuccess) {
        cudaFree(p);
        cudaGetLastError();
        return nullptr;
    }
    d->kflags[key] = static_cast<unsigned long long*>(p);
    return static_cast<unsigned long long*>(p);
}

// Frees a graph-owned flags block after the launch that used it was enqueued.
struct KpartFlagsGuard {
    unsigned long long* p = nullptr;
    cudaStream_t st = nullptr;
    bool owned = false;
    ~KpartFlagsGuard() {
        if (owned && p) cudaFreeAsync(p, st);
    }
};

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D K-major operand: `pieces` stacked matrices of `rows` x `k` elements,
// row stride ld_bytes, piece stride piece_bytes; box = box_rows x 128 bytes
// with the 128-byte swizzle; out-of-range elements read as zero.
tc_status encode_kmajor(CUtensorMap* map, CUtensorMapDataType dtype, int esz, const void* ptr, int64_t k,
                        int64_t rows, int64_t pieces, int64_t ld_bytes, int64_t piece_bytes, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return fail(TC_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[3] = {static_cast<cuuint64_t>(k), static_cast<cuuint64_t>(rows),
                          static_cast<cuuint64_t>(pieces)};
    cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld_bytes), static_cast<cuuint64_t>(piece_bytes)};
    cuuint32_t box[3] = {static_cast<cuuint32_t>(128 / esz), static_cast<cuuint32_t>(box_rows), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, dtype, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(TC_ERR_INVALID, "cuTensorMapEncodeTiled failed (%d)", static_cast<int>(r));
    return TC_OK;
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }
inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }
constexpr int64_t kMaxDim = 0x7FFFFFFF;

int elem_size(int32_t dt) { return dt == TC_E4M3 ? 1 : 2; }

tc_status check_dims(int64_t m, int64_t n, int64_t k) {
    if (m < 0 || n < 0 || k < 0) return fail(TC_ERR_INVALID, "negative size (m=%lld n=%lld k=%lld)", (long long)m,
                                             (long long)n, (long long)k);
    if (m > kMaxDim || n > kMaxDim || k > kMaxDim) return fail(TC_ERR_INVALID, "size above 2^31-1");
    // the kernels count output tiles (at least 128 x 128) and their halves in 32-bit integers
    if (((m + 127) / 128) * ((n + 127) / 128) > (int64_t(1) << 29))
        return fail(TC_ERR_INVALID, "m x n above 2^43 elements");
    return TC_OK;
}

tc_status enqueue(cudaError_t e, const char* what) { return e == cudaSuccess ? TC_OK : cuda_fail(e, what); }

// ---- autotune table: shape class -> fastest configuration measured in this process
struct TuneKey {
    int dt, lm, ln, lk;  // log2 of m, n, k rounded up to a power of two
    bool operator<(const TuneKey& o) const {
        return dt != o.dt ? dt < o.dt : lm != o.lm ? lm < o.lm : ln != o.ln ? ln < o.ln : lk < o.lk;
    }
};
// A kernel configuration of gemm_mixed: 256 x 256 tiles on CTA pairs or 128 x bn on single CTAs,
// the raster band height in M-tiles, whether a last partial round of pair tiles is cut into
// 256 x 128 halves, whether odd rounds of tiles walk K downwards, and the CTAs per cluster of the
// pair kernel: 2 (one pair per tile) or 4 (two pairs on adjacent tiles of a row band, A multicast
// between them).
struct GemmCfg {
    int pair, group_m, tail, korder, cluster, bn;
};
struct TuneCfg {
    GemmCfg cfg;
    double ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneCfg> g_tune;

int ceil_log2(int64_t v) {
    int l = 0;
    while ((int64_t(1) << l) < v && l < 62) ++l;
    return l;
}
TuneKey tune_key(int dt, int64_t m, int64_t n, int64_t k) { return {dt, ceil_log2(m), ceil_log2(n), ceil_log2(k)}; }

bool tune_lookup(int dt, int64_t m, int64_t n, int64_t k, TuneCfg* out) {
    if (dt < 0) return false;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(tune_key(dt, m, n, k));
    if (it == g_tune.end()) return false;
    *out = it->second;
    return true;
}

// Untuned configuration of gemm_mixed for an m x n output.
//   Tiles: 256 x 256 on CTA pairs, unless 128 x 64 (else 128 x 128) tiles on single CTAs number no
//   more than the SMs: a problem that small is bound by the latency of each CTA's loads and
//   epilogue, not by tensor throughput, and narrow tiles spread it over the most SMs (graph-replayed
//   FP16 GEMMs with beta = 0.5: N = 256 6.3 us against 8.5 on one CTA pair, N = 1024 9.9 against
//   12.3).  Problems of at most 128 rows always take single CTAs (a pair tile would be half empty).
//   Raster bands of 8 M-tiles: the tiles in flight then span 8 M-tiles and about 10 N-tiles, the
//   smallest A-band plus B-panel working set (DRAM reads of the FP16 GEMM at N = 8192: 1.36-1.41 GB
//   against 1.53 GB with bands of 16 and 2.4 GB with bands of 2 or 32, at the same speed).
//   A last round of pair tiles that would keep at most half of the CTA pairs busy runs as two units
//   per tile over parts of K (tail 2): an MMA takes about as long at N = 128 as at N = 256, so
//   256 x 128 halves (tail 1) take as long as whole tiles.
//   K order: a CTA pair takes every ncl-th tile of the raster, so its i-th tile belongs to round i
//   of tiles in flight together; consecutive rounds of a raster band share the band's A panels.
//   Walking K downwards in odd rounds starts each round on the k-blocks the round before it left in
//   L2 (DRAM reads at N = 8192: 1.30 GB against 1.45 GB in one direction).  Each tile's order
//   depends only on its place in the raster and the number of CTA pairs, so results stay bitwise
//   reproducible.
//   Clusters of two CTAs.
GemmCfg default_gemm_cfg(int64_t m, int64_t n, int sm_count) {
    GemmCfg c{1, 8, 2, 1, 2, 256};
    auto tiles = [&](int64_t bn) { return ((m + 127) / 128) * ((n + bn - 1) / bn); };
    if (tiles(64) <= sm_count) {
        c.pair = 0;
        c.bn = 64;
    } else if (tiles(128) <= sm_count) {
        c.pair = 0;
        c.bn = 128;
    } else if (m <= 128) {
        c.pair = 0;
    }
    return c;
}

// Environment overrides of a configuration: TCGEMM_TILE=single|pair, TCGEMM_BN=64|128|256 (single
// CTAs), TCGEMM_GROUP_M, TCGEMM_PAIR_TAIL=full|halves|split (split: parts of K),
// TCGEMM_K_ORDER=forward|serpentine and
// TCGEMM_CLUSTER=2|4.
int env_choice(const char* name, const char* a, int va, const char* b, int vb, int dflt) {
    const char* env = getenv(name);
    if (env && strcmp(env, a) == 0) return va;
    if (env && strcmp(env, b) == 0) return vb;
    return dflt;
}
GemmCfg apply_env(GemmCfg c) {
    const int pair = env_choice("TCGEMM_TILE", "single", 0, "pair", 1, c.pair);
    if (pair != c.pair) c.bn = 256;
    c.pair = pair;
    if (const char* env = getenv("TCGEMM_BN")) {
        const int v = atoi(env);
        if (v == 64 || v == 128 || v == 256) c.bn = v;
    }
    if (const char* env = getenv("TCGEMM_GROUP_M")) {
        const int v = atoi(env);
        if (v >= 1 && v <= 1024) c.group_m = v;
    }
    c.tail = env_choice("TCGEMM_PAIR_TAIL", "full", 0, "split", 2, c.tail);
    c.tail = env_choice("TCGEMM_PAIR_TAIL", "halves", 1, "kparts", 2, c.tail);
    c.korder = env_choice("TCGEMM_K_ORDER", "forward", 0, "serpentine", 1, c.korder);
    c.cluster = env_choice("TCGEMM_CLUSTER", "2", 2, "4", 4, c.cluster);
    return c;
}

// The configuration a gemm_mixed call runs: the environment's overrides of the autotune table's
// entry for the shape class, else of the untuned configuration.
GemmCfg gemm_cfg_for(int dt, int64_t m, int64_t n, int64_t k, int sm_count) {
    TuneCfg t;
    return apply_env(tune_lookup(dt, m, n, k, &t) ? t.cfg : default_gemm_cfg(m, n, sm_count));
}

// Raster band, tail split and K order of the refined GEMMs (CTA pairs): the untuned values unless
// overridden by the environment.
int gemm_group_m() { return apply_env(GemmCfg{1, 8, 2, 1, 2, 256}).group_m; }
int gemm_split_tail() { return apply_env(GemmCfg{1, 8, 2, 1, 2, 256}).tail; }
int gemm_serpentine() { return apply_env(GemmCfg{1, 8, 2, 1, 2, 256}).korder; }

// Pending failure-injection request of this thread (tc_debug_stall_next_gemm).
thread_local int g_stall_next = 0;  // k-block + 1, 0 = none
int take_stall() {
    const int v = g_stall_next;
    g_stall_next = 0;
    return v;
}

// Epilogue of the pair GEMM: stage 32 x 32 chunks in shared memory (default) or store rows
// directly from the accumulator registers (TCGEMM_EPILOGUE=direct).
int gemm_staged_epilogue() {
    const char* env = getenv("TCGEMM_EPILOGUE");
    return (env && strcmp(env, "direct") == 0) ? 0 : 1;
}

// k-blocks of 64 between promotions of the refined GEMM's partial sums out of
// TMEM into round-to-nearest FP32 registers.  TCGEMM_SPLIT_PROMOTE=0|1|2|4
// overrides the default of the scheme: every 128 of K for Eq. 1 / Eq. 2 and
// the three BF16 pieces (below the FP32 CUDA-core GEMM's error at about 3 % of
// the time), every 256 of K for the scaled split, whose single-buffered hi x hi
// accumulator stalls the tensor pipe once per promotion and whose corrections
// are already kept apart.
int split_promote_kb(int dflt = 2) {
    const char* env = getenv("TCGEMM_SPLIT_PROMOTE");
    if (env) {
        const int v = atoi(env);
        if (v == 0 || v == 1 || v == 2 || v == 4) return v;
    }
    return dflt;
}

}  // namespace

extern "C" {

const char* tc_version(void) { return "tcgemm 0.1 (sm_103a)"; }

tc_status tc_debug_stall_next_gemm(int32_t k_block) {
    g_stall_next = k_block >= 0 ? k_block + 1 : 0;
    return TC_OK;
}

const char* tc_last_error(void) { return g_err.c_str(); }

tc_status tc_device_info(int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor) {
    Device* d;
    tc_status s = get_device(&d);
    if (s != TC_OK) return s;
    if (sm_count) *sm_count = d->sm_count;
    if (cc_major) *cc_major = d->cc_major;
    if (cc_minor) *cc_minor = d->cc_minor;
    return TC_OK;
}

tc_status tc_sync_status(void* stream) {
    Device* d;
    tc_status s = get_device(&d);
    if (s != TC_OK) return s;
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    int word = 0;
    if ((e = cudaMemcpy(&word, d->status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if (word != 0) {
        cudaMemset(d->status, 0, sizeof(int));
        return fail(TC_ERR_TIMEOUT, "a kernel gave up on a bounded wait (device status %d)", word);
    }
    return TC_OK;
}

tc_status tc_quantize(int32_t dt, int64_t rows, int64_t cols, const float* src, int64_t ld_src, void* dst,
                      int64_t ld_dst, int32_t transpose, float* scale_out, void* stream) {
    if (dt != TC_F16 && dt != TC_BF16 && dt != TC_E4M3) return fail(TC_ERR_INVALID, "tc_quantize: bad dtype %d", dt);
    if (rows < 0 || cols < 0) return fail(TC_ERR_INVALID, "tc_quantize: negative size");
    if (dt == TC_E4M3 && scale_out == nullptr) return fail(TC_ERR_INVALID, "tc_quantize: E4M3 needs scale_out");
    if (scale_out && !aligned(scale_out, 4)) return fail(TC_ERR_INVALID, "tc_quantize: scale_out misaligned");
    if (rows > 0 && cols > 0) {
        if (!src || !dst) return fail(TC_ERR_INVALID, "tc_quantize: null pointer");
        if (ld_src < cols) return fail(TC_ERR_INVALID, "tc_quantize: ld_src < cols");
        if (ld_dst < (transpose ? rows : cols)) return fail(TC_ERR_INVALID, "tc_quantize: ld_dst too small");
        if (!aligned(src, 4) || !aligned(dst, elem_size(dt)))
            return fail(TC_ERR_INVALID, "tc_quantize: misaligned pointer");
        if (transpose && (cols + 31) / 32 > 0x7FFFFFFF) return fail(TC_ERR_INVALID, "tc_quantize: too many columns");
        if (transpose && (rows + 31) / 32 > 65535) return fail(TC_ERR_INVALID, "tc_quantize: too many rows to transpose");
    }
    Device* d;
    tc_status s = get_device(&d);
    if (s != TC_OK) return s;
    return enqueue(tcg::launch_quantize(dt, rows, cols, src, ld_src, dst, ld_dst, transpose != 0, scale_out,
                                        as_stream(stream)),
                   "tc_quantize launch");
}

}  // extern "C"

namespace {

// Shared checks and launch of the three piece-forming entry points.
tc_status split_entry(const char* name, int scheme, int32_t piece, int64_t rows, int64_t cols, const float* src,
                      int64_t ld_src, int32_t transpose, void* const* dst, int npieces, int64_t ld_dst,
                      void* stream) {
    if (piece != TC_F16 && piece != TC_BF16) return fail(TC_ERR_INVALID, "%s: piece must be F16 or BF16", name);
    if (rows < 0 || cols < 0) return fail(TC_ERR_INVALID, "%s: negative size", name);
    if (rows > 0 && cols > 0) {
        if (!src) return fail(TC_ERR_INVALID, "%s: null pointer", name);
        for (int q = 0; q < npieces; ++q)
            if (!dst[q] || !aligned(dst[q], 2)) return fail(TC_ERR_INVALID, "%s: null or misaligned piece", name);
        if (ld_src < cols) return fail(TC_ERR_INVALID, "%s: ld_src < cols", name);
        if (ld_dst < (transpose ? rows : cols)) return fail(TC_ERR_INVALID, "%s: ld_dst too small", name);
        if (!aligned(src, 4)) return fail(TC_ERR_INVALID, "%s: misaligned pointer", name);
        if (transpose && (rows + 31) / 32 > 65535) return fail(TC_ERR_INVALID, "%s: too many rows to transpose", name);
    }
    Device* d;
    tc_status s = get_device(&d);
    if (s != TC_OK) return s;
    return enqueue(tcg::launch_split(scheme, piece, rows, cols, src, ld_src, transpose != 0, dst, ld_dst,
                                     as_stream(stream)),
                   name);
}

}  // namespace

extern "C" {

tc_status tc_split(int32_t piece, int64_t rows, int64_t cols, const float* src, int64_t ld_src, int32_t transpose,
                   void* dst_hi, void* dst_lo, int64_t ld_dst, void* stream) {
    void* dst[3] = {dst_hi, dst_lo, nullptr};
    return split_entry("tc_split", 0, piece, rows, cols, src, ld_src, transpose, dst, 2, ld_dst, stream);
}

tc_status tc_split_scaled(int32_t piece, int64_t rows, int64_t cols, const float* src, int64_t ld_src,
                          int32_t transpose, void* dst_hi, void* dst_lo, int64_t ld_dst, void* stream) {
    void* dst[3] = {dst_hi, dst_lo, nullptr};
    return split_entry("tc_split_scaled", 1, piece, rows, cols, src, ld_src, transpose, dst, 2, ld_dst, stream);
}

tc_status tc_split_bf16x3(int64_t rows, int64_t cols, const float* src, int64_t ld_src, int32_t transpose,
                          void* dst0, void* dst1, void* dst2, int64_t ld_dst, void* stream) {
    void* dst[3] = {dst0, dst1, dst2};
    return split_entry("tc_split_bf16x3", 2, TC_BF16, rows, cols, src, ld_src, transpose, dst, 3, ld_dst, stream);
}

}  // extern "C"

namespace {

// gemm_mixed with its kernel configuration either resolved from the environment, the autotune
// table and the defaults (force == NULL), or given explicitly (the autotuner's candidates), so
// the autotuner changes nothing that another thread's calls see.
tc_status gemm_mixed_impl(int32_t dt, int64_t m, int64_t n, int64_t k, float alpha, const void* A, int64_t lda,
                          int32_t la, const void* B, int64_t ldb, int32_t lb, float beta, float* C, int64_t ldc,
                          const float* scale_a, const float* scale_b, void* stream, const GemmCfg* force) {
    if (dt != TC_F16 && dt != TC_BF16 && dt != TC_E4M3) return fail(TC_ERR_INVALID, "gemm_mixed: bad dtype %d", dt);
    tc_status s = check_dims(m, n, k);
    if (s != TC_OK) return s;
    if ((la != TC_ROW_MAJOR && la != TC_COL_MAJOR) || (lb != TC_ROW_MAJOR && lb != TC_COL_MAJOR))
        return fail(TC_ERR_INVALID, "gemm_mixed: bad layout");
    if (m == 0 || n == 0) return TC_OK;
    if (!C || ldc < n || !aligned(C, 4)) return fail(TC_ERR_INVALID, "gemm_mixed: bad C / ldc");
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    cudaStream_t st = as_stream(stream);
    if (k == 0) return enqueue(tcg::launch_scale_c(m, n, beta, C, ldc, st), "gemm_mixed scale");
    if (la != TC_ROW_MAJOR)
        return fail(TC_ERR_UNSUPPORTED, "gemm_mixed: A must be row-major (K-major)");
    // B: column-major (K-major), or row-major (MN-major, read by the MMA transposed) for 16-bit types
    const bool b_mn = lb == TC_ROW_MAJOR;
    if (b_mn && dt == TC_E4M3)
        return fail(TC_ERR_UNSUPPORTED, "gemm_mixed: row-major B is supported for F16 and BF16 only");
    const int esz = elem_size(dt);
    if (!A || !B) return fail(TC_ERR_INVALID, "gemm_mixed: null operand");
    if (lda < k || ldb < (b_mn ? n : k)) return fail(TC_ERR_INVALID, "gemm_mixed: lda/ldb too small");
    if (!aligned(A, 16) || !aligned(B, 16) || (lda * esz) % 16 || (ldb * esz) % 16)
        return fail(TC_ERR_INVALID, "gemm_mixed: operands and their row strides must be 16-byte aligned");
    if (dt == TC_E4M3 && (!scale_a || !scale_b)) return fail(TC_ERR_INVALID, "gemm_mixed: E4M3 needs scale_a/scale_b");
    const CUtensorMapDataType tdt = dt == TC_F16    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                    : dt == TC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    tcg::TcGemmLaunch p{};
    p.kind = dt == TC_E4M3 ? 1 : 0;
    p.ab_format = dt == TC_BF16 ? 1 : 0;
    p.na = p.nb = p.nprod = 1;
    p.bn = 256;
    const GemmCfg cfg = force ? *force : gemm_cfg_for(dt, m, n, k, d->sm_count);
    p.pair = (b_mn || cfg.pair) ? 1 : 0;   // the MN-major path exists on CTA pairs only
    if (!p.pair) p.bn = cfg.bn;
    p.b_mn_major = b_mn ? 1 : 0;
    p.group_m = cfg.group_m;
    p.stall_at = take_stall();
    p.staged_epilogue = gemm_staged_epilogue();
    p.split_tail = cfg.tail;
    KpartFlagsGuard kg;
    const int64_t kbk = dt == TC_E4M3 ? 128 : 64;
    if (p.pair && p.split_tail == 2 && (k + kbk - 1) / kbk >= tcg::kKpartMinKb) {
        p.kpart_flags = kpart_flags(d, st, &p.kpart_token, &kg.owned);
        kg.p = p.kpart_flags;
        kg.st = st;
    }
    p.serpentine = cfg.korder;
    p.quad = (p.pair && !b_mn && cfg.cluster == 4) ? 1 : 0;
    p.m = m; p.n = n; p.k = k;
    p.alpha = alpha; p.beta = beta;
    p.C = C; p.ldc = ldc;
    p.scale_a = scale_a; p.scale_b = scale_b;
    p.status = d->status;
    p.sm_count = d->sm_count;
    CUtensorMap ta, tb;
    // the four-CTA kernel loads A in 64-row quarters (each multicast to two CTAs)
    if ((s = encode_kmajor(&ta, tdt, esz, A, k, m, 1, lda * esz, m * lda * esz, p.quad ? 64 : 128)) != TC_OK)
        return s;
    if (b_mn) {
        // dims {n, k}: boxes of 64 n (128 bytes) x 64 k rows
        if ((s = encode_kmajor(&tb, tdt, esz, B, n, k, 1, ldb * esz, k * ldb * esz, 64)) != TC_OK) return s;
    } else if ((s = encode_kmajor(&tb, tdt, esz, B, k, n, 1, ldb * esz, n * ldb * esz, p.pair ? 128 : p.bn)) != TC_OK) {
        return s;
    }
    return enqueue(tcg::launch_tc_gemm(ta, tb, p, st), "gemm_mixed launch");
}

}  // namespace

extern "C" {

tc_status gemm_mixed(int32_t dt, int64_t m, int64_t n, int64_t k, float alpha, const void* A, int64_t lda, int32_t la,
                     const void* B, int64_t ldb, int32_t lb, float beta, float* C, int64_t ldc, const float* scale_a,
                     const float* scale_b, void* stream) {
    return gemm_mixed_impl(dt, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, scale_a, scale_b, stream, nullptr);
}

static int64_t split_kpad(int64_t k) { return (k + 7) / 8 * 8; }

size_t gemm_split_workspace_bytes(int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k) {
    (void)piece;
    if (m < 0 || n < 0 || k < 0) return 0;
    const int64_t kp = split_kpad(k);
    const int64_t np = nprod == 6 ? 3 : 2;
    // np pieces of A (m x kp) and of B (n x kp), 2 bytes each, 256-byte aligned blocks
    const int64_t a_bytes = (np * m * kp * 2 + 255) / 256 * 256;
    const int64_t b_bytes = (np * n * kp * 2 + 255) / 256 * 256;
    return static_cast<size_t>(a_bytes + b_bytes);
}

}  // extern "C"

namespace {

// Phases of a refined GEMM: forming the pieces, the tensor-core GEMM on them, or both.
constexpr int kSplitPhasePieces = 1, kSplitPhaseGemm = 2, kSplitPhaseBoth = 3;

// Path of a one-call refined GEMM.  The one-launch kernel (pieces formed on chip) needs no
// workspace; the two-pass path (split pass into a workspace, then the tensor-core GEMM on the
// pieces) is faster on this GPU (its shared memory moves 160 KB per k-block and CTA against the
// one-launch kernel's 288 KB).  So a call that brings a workspace takes the two-pass path and a
// call without one takes the one-launch path, which allocates nothing; TCGEMM_SPLIT=fused or
// =twopass forces either.  The one-launch kernel streams its operands in by TMA: both 16-byte
// aligned, leading dimensions multiples of 4 (else two passes, with a pooled workspace).
bool split_use_fused(int scheme, int nprod, const void* workspace, const float* A, int64_t lda, const float* B,
                     int64_t ldb) {
    const char* env = getenv("TCGEMM_SPLIT");
    bool want = workspace == nullptr;
    if (env && strcmp(env, "fused") == 0) want = true;
    if (env && strcmp(env, "twopass") == 0) want = false;
    return want && tcg::split_fused_supported(scheme, nprod) && aligned(A, 16) && aligned(B, 16) && lda % 4 == 0 &&
           ldb % 4 == 0;
}

// Refined GEMM of every scheme: form the pieces of A and B (K-major) in the
// workspace with one HBM-bound pass each, then one tcgen05 launch.
//   scheme 0: Eq. 1 / Eq. 2, nprod 2-4;  1: scaled residuals, nprod 2-3;
//   scheme 2: three BF16 pieces, nprod 6.
// phases selects the pass(es); a single phase needs the caller's workspace, and
// the GEMM phase reads pieces that an earlier pieces phase left there.
tc_status split_gemm(const char* name, int scheme, int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k,
                     float alpha, const float* A, int64_t lda, int32_t la, const float* B, int64_t ldb, int32_t lb,
                     float beta, float* C, int64_t ldc, void* workspace, size_t workspace_bytes, void* stream,
                     int phases = kSplitPhaseBoth) {
    if (piece != TC_F16 && piece != TC_BF16) return fail(TC_ERR_INVALID, "%s: piece must be F16 or BF16", name);
    tc_status s = check_dims(m, n, k);
    if (s != TC_OK) return s;
    const bool do_pieces = (phases & kSplitPhasePieces) != 0, do_gemm = (phases & kSplitPhaseGemm) != 0;
    if (do_pieces && ((la != TC_ROW_MAJOR && la != TC_COL_MAJOR) || (lb != TC_ROW_MAJOR && lb != TC_COL_MAJOR)))
        return fail(TC_ERR_INVALID, "%s: bad layout", name);
    if (phases != kSplitPhaseBoth && !workspace)
        return fail(TC_ERR_INVALID, "%s: the pieces live in the caller's workspace: it may not be NULL", name);
    if (m == 0 || n == 0) return TC_OK;
    if (do_gemm && (!C || ldc < n || !aligned(C, 4))) return fail(TC_ERR_INVALID, "%s: bad C / ldc", name);
    // operands, leading dimensions and the workspace are checked before the k = 0 shortcut, so
    // every call with the same arguments is accepted or refused whatever k is; an empty operand
    // (k = 0) may be NULL
    if (do_pieces) {
        if (k > 0 && (!A || !B)) return fail(TC_ERR_INVALID, "%s: null operand", name);
        if (!aligned(A, 4) || !aligned(B, 4)) return fail(TC_ERR_INVALID, "%s: misaligned operand pointer", name);
        if (lda < (la == TC_ROW_MAJOR ? k : m) || ldb < (lb == TC_ROW_MAJOR ? n : k))
            return fail(TC_ERR_INVALID, "%s: leading dimension too small", name);
    }
    const size_t need = gemm_split_workspace_bytes(piece, nprod, m, n, k);
    if (workspace && workspace_bytes < need)
        return fail(TC_ERR_INVALID, "%s: workspace of %zu bytes, need %zu", name, workspace_bytes, need);
    if (workspace && !aligned(workspace, 256)) return fail(TC_ERR_INVALID, "%s: workspace must be 256-byte aligned", name);
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    cudaStream_t st = as_stream(stream);
    if (k == 0) return do_gemm ? enqueue(tcg::launch_scale_c(m, n, beta, C, ldc, st), name) : TC_OK;
    const int np = scheme == 2 ? 3 : 2;
    if (phases == kSplitPhaseBoth && split_use_fused(scheme, nprod, workspace, A, lda, B, ldb)) {
        // one launch: the kernel streams FP32 A and B in by TMA and forms the pieces on chip
        tcg::SplitFusedLaunch f{};
        f.scheme = scheme;
        f.nprod = nprod;
        f.bf16 = piece == TC_BF16 ? 1 : 0;
        f.m = m; f.n = n; f.k = k;
        f.alpha = alpha; f.beta = beta;
        f.a_mn = la == TC_COL_MAJOR ? 1 : 0;
        f.b_mn = lb == TC_ROW_MAJOR ? 1 : 0;
        f.C = C; f.ldc = ldc;
        f.status = d->status;
        f.sm_count = d->sm_count;
        f.group_m = gemm_group_m();
        f.stall_at = take_stall();
        f.serpentine = gemm_serpentine();
        f.split_tail = gemm_split_tail();
        KpartFlagsGuard kg;
        if (f.split_tail == 2 && (k + 63) / 64 >= tcg::kKpartMinKbPromoted) {
            f.kpart_flags = kpart_flags(d, st, &f.kpart_token, &kg.owned);
            kg.p = f.kpart_flags;
            kg.st = st;
        }
        CUtensorMap ta, tb;
        // K-major: rows of k elements, boxes of 32 k x 128 rows; MN-major: k rows of m (or n)
        // elements, boxes of 32 x 32 k-rows
        if ((s = f.a_mn ? encode_kmajor(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, m, k, 1, lda * 4, k * lda * 4, 32)
                        : encode_kmajor(&ta, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, A, k, m, 1, lda * 4, m * lda * 4,
                                        128)) != TC_OK)
            return s;
        if ((s = f.b_mn ? encode_kmajor(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, B, n, k, 1, ldb * 4, k * ldb * 4, 32)
                        : encode_kmajor(&tb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, B, k, n, 1, ldb * 4, n * ldb * 4,
                                        128)) != TC_OK)
            return s;
        return enqueue(tcg::launch_split_fused(ta, tb, f, st), name);
    }
    void* ws = workspace;
    cudaError_t e;
    if (!ws) {
        if ((e = cudaMallocAsync(&ws, need, st)) != cudaSuccess)
            return fail(TC_ERR_OOM, "%s: workspace: %s", name, cudaGetErrorString(e));
    }
    const int64_t kp = split_kpad(k);
    uint8_t* wa = static_cast<uint8_t*>(ws);
    uint8_t* wb = wa + (np * m * kp * 2 + 255) / 256 * 256;
    void* pa[3];
    void* pb[3];
    for (int q = 0; q < np; ++q) {
        pa[q] = reinterpret_cast<uint16_t*>(wa) + q * m * kp;
        pb[q] = reinterpret_cast<uint16_t*>(wb) + q * n * kp;
    }
    tc_status out = TC_OK;
    do {
        if (do_pieces) {
            // A pieces as m x k (K-major): row-major A directly, column-major A (k x m in memory) transposed
            e = (la == TC_ROW_MAJOR) ? tcg::launch_split(scheme, piece, m, k, A, lda, false, pa, kp, st)
                                     : tcg::launch_split(scheme, piece, k, m, A, lda, true, pa, kp, st);
            if (e != cudaSuccess) { out = cuda_fail(e, "split of A"); break; }
            // B pieces as n x k (K-major): row-major B (k x n) transposed, column-major B directly
            e = (lb == TC_ROW_MAJOR) ? tcg::launch_split(scheme, piece, k, n, B, ldb, true, pb, kp, st)
                                     : tcg::launch_split(scheme, piece, n, k, B, ldb, false, pb, kp, st);
            if (e != cudaSuccess) { out = cuda_fail(e, "split of B"); break; }
        }
        if (!do_gemm) break;
        const CUtensorMapDataType tdt = piece == TC_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
        tcg::TcGemmLaunch p{};
        p.kind = 0;
        p.ab_format = piece == TC_BF16 ? 1 : 0;
        p.na = np;
        p.nb = nprod == 2 ? 1 : np;
        p.nprod = nprod;
        p.bn = nprod == 2 ? 256 : 128;
        if (scheme == 0) {
            // the promoted pair kernel for every m, as the one-launch path, so both give the same C
            p.pair = 1;
            p.promote_kb = split_promote_kb();
        } else {
            // the scaled and three-piece schemes run on the promoted CTA-pair kernel only
            p.pair = 1;
            p.promote_kb = split_promote_kb(scheme == 1 ? 4 : 2) == 4 ? 4 : 2;
            p.corr_exp = scheme == 1 ? (piece == TC_F16 ? 11 : 8) : 0;
        }
        p.group_m = gemm_group_m();
        p.stall_at = take_stall();
        p.split_tail = gemm_split_tail();
        KpartFlagsGuard kg;
        if (p.pair && p.split_tail == 2 && (k + 63) / 64 >= tcg::kKpartMinKbPromoted) {
            p.kpart_flags = kpart_flags(d, st, &p.kpart_token, &kg.owned);
            kg.p = p.kpart_flags;
            kg.st = st;
        }
        p.serpentine = gemm_serpentine();
        p.m = m; p.n = n; p.k = k;
        p.alpha = alpha; p.beta = beta;
        p.C = C; p.ldc = ldc;
        p.status = d->status;
        p.sm_count = d->sm_count;
        CUtensorMap ta, tb;
        if ((out = encode_kmajor(&ta, tdt, 2, pa[0], k, m, np, kp * 2, m * kp * 2, 128)) != TC_OK) break;
        if ((out = encode_kmajor(&tb, tdt, 2, pb[0], k, n, p.nb, kp * 2, n * kp * 2, p.pair ? 128 : p.bn)) != TC_OK)
            break;
        e = tcg::launch_tc_gemm(ta, tb, p, st);
        if (e != cudaSuccess) { out = cuda_fail(e, name); break; }
    } while (false);
    if (!workspace) cudaFreeAsync(ws, st);
    return out;
}

}  // namespace

extern "C" {

tc_status gemm_split(int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k, float alpha, const float* A,
                     int64_t lda, int32_t la, const float* B, int64_t ldb, int32_t lb, float beta, float* C,
                     int64_t ldc, void* workspace, size_t workspace_bytes, void* stream) {
    if (nprod < 2 || nprod > 4) return fail(TC_ERR_INVALID, "gemm_split: nprod must be 2, 3 or 4");
    return split_gemm("gemm_split", 0, piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, workspace,
                      workspace_bytes, stream);
}

tc_status gemm_split_scaled(int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k, float alpha,
                            const float* A, int64_t lda, int32_t la, const float* B, int64_t ldb, int32_t lb,
                            float beta, float* C, int64_t ldc, void* workspace, size_t workspace_bytes,
                            void* stream) {
    if (nprod != 2 && nprod != 3) return fail(TC_ERR_INVALID, "gemm_split_scaled: nprod must be 2 or 3");
    return split_gemm("gemm_split_scaled", 1, piece, nprod, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc,
                      workspace, workspace_bytes, stream);
}

tc_status gemm_split_bf16x3(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int32_t la,
                            const float* B, int64_t ldb, int32_t lb, float beta, float* C, int64_t ldc,
                            void* workspace, size_t workspace_bytes, void* stream) {
    return split_gemm("gemm_split_bf16x3", 2, TC_BF16, 6, m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc,
                      workspace, workspace_bytes, stream);
}

}  // extern "C"

namespace {

// The scheme, piece and product count of a two-phase refined GEMM, checked as the one-call
// entry points check them.
tc_status split_scheme_ok(const char* name, int32_t scheme, int32_t piece, int32_t nprod) {
    if (scheme == 0 && (nprod < 2 || nprod > 4)) return fail(TC_ERR_INVALID, "%s: scheme 0 takes nprod 2, 3 or 4", name);
    if (scheme == 1 && nprod != 2 && nprod != 3) return fail(TC_ERR_INVALID, "%s: scheme 1 takes nprod 2 or 3", name);
    if (scheme == 2 && (piece != TC_BF16 || nprod != 6))
        return fail(TC_ERR_INVALID, "%s: scheme 2 takes BF16 pieces and nprod 6", name);
    if (scheme < 0 || scheme > 2) return fail(TC_ERR_INVALID, "%s: scheme must be 0, 1 or 2", name);
    return TC_OK;
}

}  // namespace

extern "C" {

tc_status gemm_split_prepare(int32_t scheme, int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k,
                             const float* A, int64_t lda, int32_t la, const float* B, int64_t ldb, int32_t lb,
                             void* workspace, size_t workspace_bytes, void* stream) {
    tc_status s = split_scheme_ok("gemm_split_prepare", scheme, piece, nprod);
    if (s != TC_OK) return s;
    return split_gemm("gemm_split_prepare", scheme, piece, nprod, m, n, k, 1.0f, A, lda, la, B, ldb, lb, 0.0f, nullptr,
                      0, workspace, workspace_bytes, stream, kSplitPhasePieces);
}

tc_status gemm_split_run(int32_t scheme, int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k, float alpha,
                         float beta, float* C, int64_t ldc, const void* workspace, size_t workspace_bytes,
                         void* stream) {
    tc_status s = split_scheme_ok("gemm_split_run", scheme, piece, nprod);
    if (s != TC_OK) return s;
    return split_gemm("gemm_split_run", scheme, piece, nprod, m, n, k, alpha, nullptr, 0, TC_ROW_MAJOR, nullptr, 0,
                      TC_ROW_MAJOR, beta, C, ldc, const_cast<void*>(workspace), workspace_bytes, stream,
                      kSplitPhaseGemm);
}

tc_status gemm_sgemm(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int32_t la,
                     const float* B, int64_t ldb, int32_t lb, float beta, float* C, int64_t ldc, void* stream) {
    tc_status s = check_dims(m, n, k);
    if (s != TC_OK) return s;
    if ((la != TC_ROW_MAJOR && la != TC_COL_MAJOR) || (lb != TC_ROW_MAJOR && lb != TC_COL_MAJOR))
        return fail(TC_ERR_INVALID, "gemm_sgemm: bad layout");
    if (m == 0 || n == 0) return TC_OK;
    if (!C || ldc < n) return fail(TC_ERR_INVALID, "gemm_sgemm: bad C / ldc");
    if (m > 65535LL * 128) return fail(TC_ERR_INVALID, "gemm_sgemm: m too large");
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    cudaStream_t st = as_stream(stream);
    if (k == 0) return enqueue(tcg::launch_scale_c(m, n, beta, C, ldc, st), "gemm_sgemm scale");
    if (!A || !B) return fail(TC_ERR_INVALID, "gemm_sgemm: null operand");
    if (lda < (la == TC_ROW_MAJOR ? k : m) || ldb < (lb == TC_ROW_MAJOR ? n : k))
        return fail(TC_ERR_INVALID, "gemm_sgemm: leading dimension too small");
    return enqueue(tcg::launch_sgemm(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, st), "gemm_sgemm launch");
}

tc_status gemm_batched_strided(int32_t dt, int64_t batch, int32_t m, int32_t n, int32_t k, float alpha, const void* A,
                               int64_t stride_a, int32_t la, const void* B, int64_t stride_b, int32_t lb, float beta,
                               float* C, int64_t stride_c, void* stream) {
    if (dt != TC_F16 && dt != TC_BF16) return fail(TC_ERR_UNSUPPORTED, "gemm_batched_strided: F16 or BF16 only");
    if (m != 16 || n != 16 || k != 16) return fail(TC_ERR_UNSUPPORTED, "gemm_batched_strided: 16x16x16 problems only");
    if (la != TC_ROW_MAJOR) return fail(TC_ERR_UNSUPPORTED, "gemm_batched_strided: A must be row-major");
    if (lb != TC_ROW_MAJOR && lb != TC_COL_MAJOR) return fail(TC_ERR_INVALID, "gemm_batched_strided: bad layout");
    if (batch < 0) return fail(TC_ERR_INVALID, "gemm_batched_strided: negative batch");
    if (batch == 0) return TC_OK;
    if (!A || !B || !C) return fail(TC_ERR_INVALID, "gemm_batched_strided: null pointer");
    if (stride_a < 256 || stride_b < 256 || stride_c < 256)
        return fail(TC_ERR_INVALID, "gemm_batched_strided: strides must cover a 16x16 problem");
    if (stride_a % 8 || stride_b % 8 || stride_c % 2 || !aligned(A, 16) || !aligned(B, 16) || !aligned(C, 8))
        return fail(TC_ERR_INVALID, "gemm_batched_strided: strides/pointers not aligned");
    Device* d;
    tc_status s = get_device(&d);
    if (s != TC_OK) return s;
    return enqueue(tcg::launch_batched16(dt, batch, alpha, A, stride_a, B, stride_b, lb, beta, C, stride_c, d->status,
                                         d->sm_count, as_stream(stream)),
                   "gemm_batched_strided launch");
}

}  // extern "C"

// ------------------------------------------------------------ grouped plans

struct tc_grouped_plan {
    int dt = 0, la = 0, lb = 0;
    int32_t count = 0, num_tiles = 0;
    int dev = 0, sm_count = 0;
    tcg::GroupedProblemDev* d_probs = nullptr;
    tcg::GroupedTileDev* d_tiles = nullptr;
    // graph of the last run
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    const void* g_a = nullptr;
    const void* g_b = nullptr;
    float* g_c = nullptr;
    float g_alpha = 0.f, g_beta = 0.f;
    // tensor-core path: 128 x 256 tiles and two TMA maps per problem (A, B)
    bool use_tc = false;
    std::vector<tc_problem> host_probs;
    tcg::GroupedTcTile* d_tc_tiles = nullptr;
    int32_t tc_tiles = 0;
    CUtensorMap* d_maps = nullptr;
    const void* maps_a = nullptr;  // bases the device maps were encoded for
    const void* maps_b = nullptr;
    int* status = nullptr;
    int variant = -1;  // autotuned: 0 tensor cores + staged epilogue, 1 tensor cores + direct, 2 mma.sync
};

namespace {

using tcg::grouped_swap;
using tcg::grouped_tall_tiles;
using tcg::grouped_tc_tile_count;
using tcg::grouped_tc_tiles;

// Every problem's tensor maps for these bases, two per problem: A_g (dims {k, m}) and B_g
// (dims {k, n} K-major, or {n, k} row-major); a transposed problem has B_g's map first.
tc_status encode_grouped_maps(int32_t dt, int32_t lb, int32_t count, const tc_problem* problems, const void* a_base,
                              const void* b_base, CUtensorMap* maps) {
    const CUtensorMapDataType tdt = dt == TC_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const uint8_t* a = static_cast<const uint8_t*>(a_base);
    const uint8_t* b = static_cast<const uint8_t*>(b_base);
    constexpr int kM = tcg::kGroupedTcMapsPerProblem;
    for (int32_t g = 0; g < count; ++g) {
        const tc_problem& p = problems[g];
        if (grouped_swap(p, lb)) {   // B_g as the A operand, A_g (m x k) as the K-major B operand
            tc_status s = lb == TC_ROW_MAJOR   // k x n: dims {n, k}, boxes of 64 n x 64 k (MN-major A)
                              ? encode_kmajor(&maps[kM * g], tdt, 2, b + p.off_b * 2, p.n, p.k, 1, int64_t(p.ldb) * 2,
                                              int64_t(p.k) * p.ldb * 2, 64)
                              : encode_kmajor(&maps[kM * g], tdt, 2, b + p.off_b * 2, p.k, p.n, 1, int64_t(p.ldb) * 2,
                                              int64_t(p.n) * p.ldb * 2, tcg::kGroupedTcTileM);
            if (s == TC_OK)
                s = encode_kmajor(&maps[kM * g + 1], tdt, 2, a + p.off_a * 2, p.k, p.m, 1, int64_t(p.lda) * 2,
                                  int64_t(p.m) * p.lda * 2, tcg::grouped_tc_box_rows(p.m));
            if (s != TC_OK) return s;
            continue;
        }
        tc_status s = encode_kmajor(&maps[kM * g], tdt, 2, a + p.off_a * 2, p.k, p.m, 1, int64_t(p.lda) * 2,
                                    int64_t(p.m) * p.lda * 2, tcg::kGroupedTcTileM);
        if (s != TC_OK) return s;
        if (lb == TC_ROW_MAJOR)   // B_g k x n: dims {n, k}, boxes of 64 n (128 bytes) x 64 k
            s = encode_kmajor(&maps[kM * g + 1], tdt, 2, b + p.off_b * 2, p.n, p.k, 1, int64_t(p.ldb) * 2,
                              int64_t(p.k) * p.ldb * 2, 64);
        else
            s = encode_kmajor(&maps[kM * g + 1], tdt, 2, b + p.off_b * 2, p.k, p.n, 1, int64_t(p.ldb) * 2,
                              int64_t(p.n) * p.ldb * 2, tcg::grouped_tc_box_rows(p.n));
        if (s != TC_OK) return s;
    }
    return TC_OK;
}

// Encode every problem's tensor maps for these bases and upload them (stream-ordered).
tc_status grouped_upload_maps(tc_grouped_plan* plan, const void* a_base, const void* b_base, cudaStream_t st) {
    std::vector<CUtensorMap> maps(tcg::kGroupedTcMapsPerProblem * static_cast<size_t>(plan->count));
    tc_status s = encode_grouped_maps(plan->dt, plan->lb, plan->count, plan->host_probs.data(), a_base, b_base,
                                      maps.data());
    if (s != TC_OK) return s;
    // pageable source: returns once the bytes are staged
    cudaError_t e = cudaMemcpyAsync(plan->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "grouped: upload tensor maps");
    plan->maps_a = a_base;
    plan->maps_b = b_base;
    return TC_OK;
}

cudaError_t grouped_launch(tc_grouped_plan* plan, const void* a_base, const void* b_base, float* c_base, float alpha,
                           float beta, cudaStream_t st) {
    if (plan->use_tc && plan->variant != 2)
        return tcg::launch_grouped_tc(plan->dt, plan->d_tc_tiles, plan->tc_tiles, plan->d_maps, c_base, alpha, beta,
                                      plan->status, plan->sm_count, st,
                                      plan->variant < 0 ? -1 : (plan->variant == 0 ? 1 : 0),
                                      plan->lb == TC_ROW_MAJOR);
    return tcg::launch_grouped(plan->dt, plan->lb, plan->d_probs, plan->d_tiles, plan->num_tiles, a_base, b_base,
                               c_base, alpha, beta, plan->sm_count, st);
}

// Grouped GEMMs run on the tensor cores (B K-major, or row-major read as MN-major) unless
// TCGEMM_GROUPED=mma selects the mma.sync kernel.
bool grouped_use_tensor_cores(int32_t lb) {
    (void)lb;
    const char* env = getenv("TCGEMM_GROUPED");
    return !(env && strcmp(env, "mma") == 0);
}


}  // namespace

extern "C" {

tc_status gemm_grouped_plan_create(int32_t dt, int32_t count, const tc_problem* problems, int32_t la, int32_t lb,
                                   tc_grouped_plan** plan_out) {
    if (!plan_out) return fail(TC_ERR_INVALID, "grouped: null plan_out");
    *plan_out = nullptr;
    if (dt != TC_F16 && dt != TC_BF16) return fail(TC_ERR_UNSUPPORTED, "grouped: F16 or BF16 only");
    if (la != TC_ROW_MAJOR) return fail(TC_ERR_UNSUPPORTED, "grouped: A must be row-major");
    if (lb != TC_ROW_MAJOR && lb != TC_COL_MAJOR) return fail(TC_ERR_INVALID, "grouped: bad layout");
    if (count < 0 || (count > 0 && !problems)) return fail(TC_ERR_INVALID, "grouped: bad problem array");
    std::vector<tcg::GroupedProblemDev> probs(count);
    struct P { int64_t cost; int32_t g; };
    std::vector<P> order;
    order.reserve(count);
    size_t ntiles = 0;
    for (int32_t g = 0; g < count; ++g) {
        const tc_problem& p = problems[g];
        if (p.m < 1 || p.n < 1 || p.k < 1) return fail(TC_ERR_INVALID, "grouped: problem %d has a zero size", g);
        if (p.lda < p.k || p.ldb < (lb == TC_ROW_MAJOR ? p.n : p.k) || p.ldc < p.n)
            return fail(TC_ERR_INVALID, "grouped: problem %d leading dimension too small", g);
        if (p.lda % 8 || p.ldb % 8 || p.off_a % 8 || p.off_b % 8)
            return fail(TC_ERR_INVALID, "grouped: problem %d rows not 16-byte aligned", g);
        if (p.off_a < 0 || p.off_b < 0 || p.off_c < 0) return fail(TC_ERR_INVALID, "grouped: problem %d negative offset", g);
        probs[g] = {p.m, p.n, p.k, 0, p.off_a, p.off_b, p.off_c, p.lda, p.ldb, p.ldc, 0};
        const int64_t tm = (p.m + tcg::kGroupedTileM - 1) / tcg::kGroupedTileM;
        const int64_t tn = (p.n + tcg::kGroupedTileN - 1) / tcg::kGroupedTileN;
        ntiles += static_cast<size_t>(tm * tn);
        // bytes every tile of the problem moves together: A panels, B panels, C
        order.push_back({2 * p.k * (p.m * tn + p.n * tm) + 4 * int64_t(p.m) * p.n, g});
    }
    if (ntiles > 0x7FFFFFFF) return fail(TC_ERR_INVALID, "grouped: too many tiles");
    // problems longest first, each problem's tiles next to each other: CTAs that run at the
    // same time share the problem's A and B panels through L2, and the longest problems
    // start first so the static stride of the persistent grid ends evenly
    std::stable_sort(order.begin(), order.end(), [](const P& a, const P& b) { return a.cost > b.cost; });
    std::vector<tcg::GroupedTileDev> tl;
    tl.reserve(ntiles);
    for (const P& o : order) {
        const tc_problem& p = problems[o.g];
        const int tm = (p.m + tcg::kGroupedTileM - 1) / tcg::kGroupedTileM;
        const int tn = (p.n + tcg::kGroupedTileN - 1) / tcg::kGroupedTileN;
        for (int i = 0; i < tm; ++i)
            for (int j = 0; j < tn; ++j) tl.push_back({o.g, i, j, 0});
    }

    Device* d;
    tc_status s = get_device(&d);
    if (s != TC_OK) return s;
    auto* plan = new tc_grouped_plan();
    plan->dt = dt; plan->la = la; plan->lb = lb;
    plan->count = count;
    plan->num_tiles = static_cast<int32_t>(tl.size());
    plan->sm_count = d->sm_count;
    cudaGetDevice(&plan->dev);
    cudaError_t e = cudaSuccess;
    if (count > 0) {
        if ((e = cudaMalloc(&plan->d_probs, probs.size() * sizeof(probs[0]))) == cudaSuccess)
            e = cudaMemcpy(plan->d_probs, probs.data(), probs.size() * sizeof(probs[0]), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && (e = cudaMalloc(&plan->d_tiles, tl.size() * sizeof(tl[0]))) == cudaSuccess)
            e = cudaMemcpy(plan->d_tiles, tl.data(), tl.size() * sizeof(tl[0]), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && count > 0 && grouped_use_tensor_cores(lb)) {
        // the same problem order, cut into 128 x 256 (and tall 256 x 256) tiles
        std::vector<tcg::GroupedTcTile> tc;
        const bool tall = grouped_tall_tiles();
        for (const P& o : order)
            grouped_tc_tiles(problems[o.g], o.g, tall, lb, [&](const tcg::GroupedTcTile& t) { tc.push_back(t); });
        plan->use_tc = true;
        plan->tc_tiles = static_cast<int32_t>(tc.size());
        plan->host_probs.assign(problems, problems + count);
        plan->status = d->status;
        if ((e = cudaMalloc(&plan->d_tc_tiles, tc.size() * sizeof(tc[0]))) == cudaSuccess)
            e = cudaMemcpy(plan->d_tc_tiles, tc.data(), tc.size() * sizeof(tc[0]), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMalloc(&plan->d_maps, tcg::kGroupedTcMapsPerProblem * size_t(count) * sizeof(CUtensorMap));
    }
    if (e != cudaSuccess) {
        gemm_grouped_plan_destroy(plan);
        return fail(TC_ERR_OOM, "grouped: plan upload: %s", cudaGetErrorString(e));
    }
    *plan_out = plan;
    return TC_OK;
}

tc_status gemm_grouped_plan_run(tc_grouped_plan* plan, const void* a_base, const void* b_base, float* c_base,
                                float alpha, float beta, int32_t use_graph, void* stream) {
    if (!plan) return fail(TC_ERR_INVALID, "grouped: null plan");
    if (plan->num_tiles == 0) return TC_OK;
    if (!a_base || !b_base || !c_base) return fail(TC_ERR_INVALID, "grouped: null base pointer");
    if (!aligned(a_base, 16) || !aligned(b_base, 16) || !aligned(c_base, 8))
        return fail(TC_ERR_INVALID, "grouped: base pointers must be 16-byte aligned (C: 8)");
    cudaStream_t st = as_stream(stream);
    if (plan->use_tc && (plan->maps_a != a_base || plan->maps_b != b_base)) {
        tc_status s = grouped_upload_maps(plan, a_base, b_base, st);
        if (s != TC_OK) return s;
    }
    if (!use_graph)
        return enqueue(grouped_launch(plan, a_base, b_base, c_base, alpha, beta, st), "grouped launch");
    const bool same = plan->exec && plan->g_a == a_base && plan->g_b == b_base && plan->g_c == c_base &&
                      plan->g_alpha == alpha && plan->g_beta == beta;
    cudaError_t e;
    if (!same) {
        if (plan->exec) {
            cudaGraphExecDestroy(plan->exec);
            plan->exec = nullptr;
        }
        if (!plan->cap_stream && (e = cudaStreamCreateWithFlags(&plan->cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "grouped: capture stream");
        // only recorded here; the graph is launched on `st`, after the map upload above
        if ((e = cudaStreamBeginCapture(plan->cap_stream, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return cuda_fail(e, "grouped: begin capture");
        cudaError_t le = grouped_launch(plan, a_base, b_base, c_base, alpha, beta, plan->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(plan->cap_stream, &graph);
        if (le != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(le != cudaSuccess ? le : e, "grouped: capture");
        }
        e = cudaGraphInstantiate(&plan->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "grouped: instantiate");
        plan->g_a = a_base; plan->g_b = b_base; plan->g_c = c_base;
        plan->g_alpha = alpha; plan->g_beta = beta;
    }
    return enqueue(cudaGraphLaunch(plan->exec, st), "grouped: graph launch");
}

tc_status gemm_grouped_plan_destroy(tc_grouped_plan* plan) {
    if (!plan) return TC_OK;
    cudaDeviceSynchronize();
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->cap_stream) cudaStreamDestroy(plan->cap_stream);
    if (plan->d_probs) cudaFree(plan->d_probs);
    if (plan->d_tiles) cudaFree(plan->d_tiles);
    if (plan->d_tc_tiles) cudaFree(plan->d_tc_tiles);
    if (plan->d_maps) cudaFree(plan->d_maps);
    delete plan;
    return TC_OK;
}

tc_status gemm_grouped(int32_t dt, int32_t count, const tc_problem* problems, const void* a_base, int32_t la,
                       const void* b_base, int32_t lb, float* c_base, float alpha, float beta, void* stream) {
    tc_grouped_plan* plan = nullptr;
    tc_status s = gemm_grouped_plan_create(dt, count, problems, la, lb, &plan);
    if (s != TC_OK) return s;
    s = gemm_grouped_plan_run(plan, a_base, b_base, c_base, alpha, beta, 0, stream);
    if (s == TC_OK) {
        cudaError_t e = cudaStreamSynchronize(as_stream(stream));
        if (e != cudaSuccess) s = cuda_fail(e, "grouped: synchronize");
    }
    gemm_grouped_plan_destroy(plan);
    return s;
}

size_t tc_error_norm_workspace_bytes(void) { return static_cast<size_t>(3 * tcg::kErrBlocks * 2) * sizeof(double); }

}  // extern "C"

namespace {

tc_status error_norm_checks(const char* name, int64_t m, int64_t n, const float* C, int64_t ldc, const void* Cref,
                            int64_t ldr, int64_t a_rows, int64_t a_cols, const float* A, int64_t lda, int64_t b_rows,
                            int64_t b_cols, const float* B, int64_t ldb) {
    if (m < 0 || n < 0 || a_rows < 0 || a_cols < 0 || b_rows < 0 || b_cols < 0)
        return fail(TC_ERR_INVALID, "%s: negative size", name);
    if (m * n > 0 && (!C || !Cref || ldc < n || ldr < n)) return fail(TC_ERR_INVALID, "%s: bad C / Cref", name);
    if (A && lda < a_cols) return fail(TC_ERR_INVALID, "%s: lda < a_cols", name);
    if (B && ldb < b_cols) return fail(TC_ERR_INVALID, "%s: ldb < b_cols", name);
    return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_error_norm_dev(int64_t m, int64_t n, const float* C, int64_t ldc, const void* Cref, int64_t ldr,
                            int32_t ref_is_f64, const float* A, int64_t a_rows, int64_t a_cols, int64_t lda,
                            const float* B, int64_t b_rows, int64_t b_cols, int64_t ldb, double* out_dev,
                            void* workspace, size_t workspace_bytes, void* stream) {
    tc_status s = error_norm_checks("tc_error_norm_dev", m, n, C, ldc, Cref, ldr, a_rows, a_cols, A, lda, b_rows,
                                    b_cols, B, ldb);
    if (s != TC_OK) return s;
    if (!out_dev || !aligned(out_dev, 8)) return fail(TC_ERR_INVALID, "tc_error_norm_dev: bad out_dev");
    if (!workspace || !aligned(workspace, 8) || workspace_bytes < tc_error_norm_workspace_bytes())
        return fail(TC_ERR_INVALID, "tc_error_norm_dev: workspace of %zu bytes, need %zu (8-byte aligned)",
                    workspace_bytes, tc_error_norm_workspace_bytes());
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    return enqueue(tcg::launch_error_norm(m, n, C, ldc, Cref, ldr, ref_is_f64 != 0, A, A ? a_rows : 0, a_cols, lda, B,
                                          B ? b_rows : 0, b_cols, ldb, static_cast<double*>(workspace), out_dev,
                                          as_stream(stream)),
                   "tc_error_norm_dev");
}

tc_status tc_error_norm(int64_t m, int64_t n, const float* C, int64_t ldc, const void* Cref, int64_t ldr,
                        int32_t ref_is_f64, const float* A, int64_t a_rows, int64_t a_cols, int64_t lda,
                        const float* B, int64_t b_rows, int64_t b_cols, int64_t ldb, double* out, void* stream) {
    if (!out) return fail(TC_ERR_INVALID, "tc_error_norm: null out");
    tc_status s = error_norm_checks("tc_error_norm", m, n, C, ldc, Cref, ldr, a_rows, a_cols, A, lda, b_rows, b_cols,
                                    B, ldb);
    if (s != TC_OK) return s;
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    cudaStream_t st = as_stream(stream);
    double* scratch = nullptr;
    const size_t bytes = tc_error_norm_workspace_bytes() + 4 * sizeof(double);
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&scratch), bytes, st);
    if (e != cudaSuccess) return fail(TC_ERR_OOM, "tc_error_norm: scratch: %s", cudaGetErrorString(e));
    double* out_dev = scratch + 3 * tcg::kErrBlocks * 2;
    e = tcg::launch_error_norm(m, n, C, ldc, Cref, ldr, ref_is_f64 != 0, A, A ? a_rows : 0, a_cols, lda, B,
                               B ? b_rows : 0, b_cols, ldb, scratch, out_dev, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, out_dev, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(scratch, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "tc_error_norm");
    if (e2 != cudaSuccess) return cuda_fail(e2, "tc_error_norm: synchronize");
    return TC_OK;
}

}  // extern "C"

// ------------------------------------------------------------ grouped GEMM without allocation
//
// For callers that may not allocate device memory: the problem descriptors
// and the tile schedule live in a static device array instead of a plan's
// cudaMalloc'd buffers.  The host-side name of the array is only a stand-in;
// its device address comes from cudaGetSymbolAddress, taken once per device
// with that device current.

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;  // 8 MiB on every device that loads the library
static __device__ __align__(256) unsigned char g_grouped_scratch[kNoAllocScratchBytes];

struct NoAllocDevice {
    bool ready = false;
    void* scratch = nullptr;  // device address of g_grouped_scratch on this device
    int* status = nullptr;    // device address of the status word (a static variable as well)
    int sm_count = 0;
};
NoAllocDevice g_noalloc_dev[64];

tc_status noalloc_setup(NoAllocDevice** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "gemm_grouped_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(TC_ERR_INVALID, "gemm_grouped_noalloc: device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        if ((e = cudaGetSymbolAddress(&p, g_grouped_scratch)) != cudaSuccess)
            return cuda_fail(e, "gemm_grouped_noalloc: cudaGetSymbolAddress");
        void* sw = nullptr;
        if ((e = cudaGetSymbolAddress(&sw, g_status_word)) != cudaSuccess)
            return cuda_fail(e, "gemm_grouped_noalloc: cudaGetSymbolAddress(status)");
        if ((e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "gemm_grouped_noalloc: cudaDeviceGetAttribute");
        d.scratch = p;
        d.status = static_cast<int*>(sw);
        d.ready = true;
    }
    *out = &d;
    return TC_OK;
}

}  // namespace

namespace {

// The plan-free entry points below copy their schedule from host memory that the call owns and
// frees on return.  Inside a stream capture that copy would become a graph node reading freed
// host memory at every replay, so a capturing stream is refused before anything is enqueued.
tc_status refuse_capture(const char* name, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e != cudaSuccess) return cuda_fail(e, name);
    if (cs != cudaStreamCaptureStatusNone)
        return fail(TC_ERR_UNSUPPORTED,
                    "%s: the stream is being captured; this call uploads its schedule from host memory it frees "
                    "on return and cannot be recorded in a CUDA graph (gemm_grouped_plan_run can)",
                    name);
    return TC_OK;
}

// Host half of a plan-free grouped GEMM on the mma.sync kernel (64 x 64 tiles): checks the
// call and builds in `host` the problem table (padded to 256 bytes) followed by the tile list,
// tiles in the longest-first order of a plan.
tc_status grouped_mma_host(const char* name, int32_t dt, int32_t count, const tc_problem* problems,
                           const void* a_base, int32_t la, const void* b_base, int32_t lb, const float* c_base,
                           std::vector<unsigned char>& host, size_t* desc_bytes_out, int64_t* tiles_out,
                           bool pack = true) {
    if (dt != TC_F16 && dt != TC_BF16) return fail(TC_ERR_UNSUPPORTED, "%s: F16 or BF16 only", name);
    if (la != TC_ROW_MAJOR) return fail(TC_ERR_UNSUPPORTED, "%s: A must be row-major", name);
    if (lb != TC_ROW_MAJOR && lb != TC_COL_MAJOR) return fail(TC_ERR_INVALID, "%s: bad layout", name);
    if (count < 0 || (count > 0 && !problems)) return fail(TC_ERR_INVALID, "%s: bad problem array", name);
    *tiles_out = 0;
    *desc_bytes_out = 0;
    host.clear();
    if (count == 0) return TC_OK;
    if (!a_base || !b_base || !c_base) return fail(TC_ERR_INVALID, "%s: null base pointer", name);
    if (!aligned(a_base, 16) || !aligned(b_base, 16) || !aligned(c_base, 8))
        return fail(TC_ERR_INVALID, "%s: base pointers must be 16-byte aligned (C: 8)", name);
    int64_t num_tiles = 0;
    for (int32_t g = 0; g < count; ++g) {
        const tc_problem& p = problems[g];
        if (p.m < 1 || p.n < 1 || p.k < 1) return fail(TC_ERR_INVALID, "%s: problem %d has a zero size", name, g);
        if (p.lda < p.k || p.ldb < (lb == TC_ROW_MAJOR ? p.n : p.k) || p.ldc < p.n)
            return fail(TC_ERR_INVALID, "%s: problem %d leading dimension too small", name, g);
        if (p.lda % 8 || p.ldb % 8 || p.off_a % 8 || p.off_b % 8)
            return fail(TC_ERR_INVALID, "%s: problem %d rows not 16-byte aligned", name, g);
        if (p.off_a < 0 || p.off_b < 0 || p.off_c < 0)
            return fail(TC_ERR_INVALID, "%s: problem %d negative offset", name, g);
        num_tiles += int64_t((p.m + tcg::kGroupedTileM - 1) / tcg::kGroupedTileM) *
                     ((p.n + tcg::kGroupedTileN - 1) / tcg::kGroupedTileN);
    }
    if (num_tiles > 0x7FFFFFFF) return fail(TC_ERR_INVALID, "%s: too many tiles", name);
    *tiles_out = num_tiles;
    if (!pack) return TC_OK;  // checked only
    const size_t desc_bytes = (size_t(count) * sizeof(tcg::GroupedProblemDev) + 255) / 256 * 256;
    host.assign(desc_bytes + size_t(num_tiles) * sizeof(tcg::GroupedTileDev), 0);
    auto* hp = reinterpret_cast<tcg::GroupedProblemDev*>(host.data());
    struct T { int64_t cost; tcg::GroupedTileDev t; };
    std::vector<T> tiles;
    tiles.reserve(static_cast<size_t>(num_tiles));
    for (int32_t g = 0; g < count; ++g) {
        const tc_problem& p = problems[g];
        hp[g] = {p.m, p.n, p.k, 0, p.off_a, p.off_b, p.off_c, p.lda, p.ldb, p.ldc, 0};
        const int tm = (p.m + tcg::kGroupedTileM - 1) / tcg::kGroupedTileM;
        const int tn = (p.n + tcg::kGroupedTileN - 1) / tcg::kGroupedTileN;
        for (int i = 0; i < tm; ++i)
            for (int j = 0; j < tn; ++j) {
                const int64_t rows = std::min(tcg::kGroupedTileM, p.m - i * tcg::kGroupedTileM);
                const int64_t cols = std::min(tcg::kGroupedTileN, p.n - j * tcg::kGroupedTileN);
                tiles.push_back({2 * p.k * (rows + cols) + 4 * rows * cols, {g, i, j, 0}});
            }
    }
    std::stable_sort(tiles.begin(), tiles.end(), [](const T& a, const T& b) { return a.cost > b.cost; });
    auto* ht = reinterpret_cast<tcg::GroupedTileDev*>(host.data() + desc_bytes);
    for (size_t i = 0; i < tiles.size(); ++i) ht[i] = tiles[i].t;
    *desc_bytes_out = desc_bytes;
    *tiles_out = num_tiles;
    return TC_OK;
}

// Upload the host half to `dev_base` and launch.
tc_status grouped_mma_enqueue(const char* name, int32_t dt, int32_t lb, const std::vector<unsigned char>& host,
                              size_t desc_bytes, int64_t num_tiles, unsigned char* dev_base, const void* a_base,
                              const void* b_base, float* c_base, float alpha, float beta, int sm_count,
                              cudaStream_t st) {
    // pageable source: the call returns once the bytes are staged, so `host` may go out of scope
    cudaError_t e = cudaMemcpyAsync(dev_base, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, name);
    return enqueue(tcg::launch_grouped(dt, lb, reinterpret_cast<const tcg::GroupedProblemDev*>(dev_base),
                                       reinterpret_cast<const tcg::GroupedTileDev*>(dev_base + desc_bytes),
                                       static_cast<int32_t>(num_tiles), a_base, b_base, c_base, alpha, beta,
                                       sm_count, st),
                   name);
}

// Host half of a plan-free grouped GEMM on the tensor-core kernel: two TMA maps per problem
// (encoded for these bases; 256-byte aligned table first), then the 128 x 256 tiles in the
// longest-first problem order of a plan.  Nothing is built when the result would exceed
// max_bytes (*fits = false).  The problems were checked by grouped_mma_host.
tc_status grouped_tc_host(int32_t dt, int32_t count, const tc_problem* problems, const void* a_base,
                          const void* b_base, int32_t lb, size_t max_bytes, std::vector<unsigned char>& host,
                          size_t* maps_bytes_out, int32_t* tiles_out, bool* fits) {
    const size_t maps_bytes =
        (tcg::kGroupedTcMapsPerProblem * size_t(count) * sizeof(CUtensorMap) + 255) / 256 * 256;
    struct P { int64_t cost; int32_t g; };
    std::vector<P> order;
    order.reserve(count);
    int64_t ntiles = 0;
    const bool tall = grouped_tall_tiles();
    for (int32_t g = 0; g < count; ++g) {
        const tc_problem& p = problems[g];
        const int64_t tm = (p.m + tcg::kGroupedTcTileM - 1) / tcg::kGroupedTcTileM;
        const int64_t tn = (p.n + tcg::kGroupedTcTileN - 1) / tcg::kGroupedTcTileN;
        ntiles += grouped_tc_tile_count(p, tall, lb);
        order.push_back({2 * p.k * (p.m * tn + p.n * tm) + 4 * int64_t(p.m) * p.n, g});
    }
    if (ntiles > 0x7FFFFFFF) return fail(TC_ERR_INVALID, "grouped: too many tiles");
    const size_t total = maps_bytes + size_t(ntiles) * sizeof(tcg::GroupedTcTile);
    *fits = total <= max_bytes;
    if (!*fits) return TC_OK;
    std::stable_sort(order.begin(), order.end(), [](const P& x, const P& y) { return x.cost > y.cost; });
    host.assign(total, 0);
    tc_status st =
        encode_grouped_maps(dt, lb, count, problems, a_base, b_base, reinterpret_cast<CUtensorMap*>(host.data()));
    if (st != TC_OK) return st;
    auto* tl = reinterpret_cast<tcg::GroupedTcTile*>(host.data() + maps_bytes);
    size_t t = 0;
    for (const P& o : order)
        grouped_tc_tiles(problems[o.g], o.g, tall, lb, [&](const tcg::GroupedTcTile& x) { tl[t++] = x; });
    *maps_bytes_out = maps_bytes;
    *tiles_out = static_cast<int32_t>(ntiles);
    return TC_OK;
}

// Upload the tensor-core host half to `dev_base` and launch.
tc_status grouped_tc_enqueue(const char* name, int32_t dt, int32_t lb, const std::vector<unsigned char>& host,
                             size_t maps_bytes, int32_t ntiles, unsigned char* dev_base, float* c_base, float alpha,
                             float beta, int* status, int sm_count, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(dev_base, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, name);
    return enqueue(tcg::launch_grouped_tc(dt, reinterpret_cast<const tcg::GroupedTcTile*>(dev_base + maps_bytes),
                                          ntiles, reinterpret_cast<const CUtensorMap*>(dev_base), c_base, alpha, beta,
                                          status, sm_count, st, -1, lb == TC_ROW_MAJOR),
                   name);
}

}  // namespace

extern "C" tc_status gemm_grouped_noalloc(int32_t dt, int32_t count, const tc_problem* problems, const void* a_base,
                                          int32_t la, const void* b_base, int32_t lb, float* c_base, float alpha,
                                          float beta, void* stream) {
    std::vector<unsigned char> host;
    size_t desc_bytes = 0;
    int64_t num_tiles = 0;
    const bool tc = grouped_use_tensor_cores(lb);
    tc_status s = grouped_mma_host("gemm_grouped_noalloc", dt, count, problems, a_base, la, b_base, lb, c_base, host,
                                   &desc_bytes, &num_tiles, !tc);
    if (s != TC_OK || count == 0) return s;
    if ((s = refuse_capture("gemm_grouped_noalloc", as_stream(stream))) != TC_OK) return s;
    NoAllocDevice* d;
    if ((s = noalloc_setup(&d)) != TC_OK) return s;
    if (tc) {
        std::vector<unsigned char> tch;
        size_t maps_bytes = 0;
        int32_t tc_tiles = 0;
        bool fits = false;
        if ((s = grouped_tc_host(dt, count, problems, a_base, b_base, lb, kNoAllocScratchBytes, tch, &maps_bytes,
                                 &tc_tiles, &fits)) != TC_OK)
            return s;
        if (fits)
            return grouped_tc_enqueue("gemm_grouped_noalloc", dt, lb, tch, maps_bytes, tc_tiles,
                                      static_cast<unsigned char*>(d->scratch), c_base, alpha, beta, d->status,
                                      d->sm_count, as_stream(stream));
        // more problems than the static table holds maps for: the mma.sync schedule is smaller
        if ((s = grouped_mma_host("gemm_grouped_noalloc", dt, count, problems, a_base, la, b_base, lb, c_base, host,
                                  &desc_bytes, &num_tiles)) != TC_OK)
            return s;
    }
    if (host.size() > kNoAllocScratchBytes)
        return fail(TC_ERR_INVALID,
                    "gemm_grouped_noalloc: %d problems (%lld tiles) need %zu bytes of scratch; the static maximum "
                    "is %zu bytes (use gemm_grouped_plan_create for larger groups)",
                    count, (long long)num_tiles, host.size(), kNoAllocScratchBytes);
    return grouped_mma_enqueue("gemm_grouped_noalloc", dt, lb, host, desc_bytes, num_tiles,
                               static_cast<unsigned char*>(d->scratch), a_base, b_base, c_base, alpha, beta,
                               d->sm_count, as_stream(stream));
}

extern "C" size_t gemm_grouped_workspace_bytes(int32_t count, const tc_problem* problems) {
    if (count <= 0 || !problems) return 0;
    int64_t mma_tiles = 0, tc_tiles = 0;
    for (int32_t g = 0; g < count; ++g) {
        const tc_problem& p = problems[g];
        if (p.m < 1 || p.n < 1) continue;
        mma_tiles += int64_t((p.m + tcg::kGroupedTileM - 1) / tcg::kGroupedTileM) *
                     ((p.n + tcg::kGroupedTileN - 1) / tcg::kGroupedTileN);
        tc_tiles += tcg::grouped_tc_tile_bound(p);
    }
    // enough for either kernel: the mma.sync schedule or the tensor-core maps and tiles
    const size_t mma = (size_t(count) * sizeof(tcg::GroupedProblemDev) + 255) / 256 * 256 +
                       size_t(mma_tiles) * sizeof(tcg::GroupedTileDev);
    const size_t tc = (tcg::kGroupedTcMapsPerProblem * size_t(count) * sizeof(CUtensorMap) + 255) / 256 * 256 +
                      size_t(tc_tiles) * sizeof(tcg::GroupedTcTile);
    return mma > tc ? mma : tc;
}

extern "C" tc_status gemm_grouped_ws(int32_t dt, int32_t count, const tc_problem* problems, const void* a_base,
                                     int32_t la, const void* b_base, int32_t lb, float* c_base, float alpha,
                                     float beta, void* workspace, size_t workspace_bytes, void* stream) {
    std::vector<unsigned char> host;
    size_t desc_bytes = 0;
    int64_t num_tiles = 0;
    const bool tc = grouped_use_tensor_cores(lb);
    tc_status s = grouped_mma_host("gemm_grouped_ws", dt, count, problems, a_base, la, b_base, lb, c_base, host,
                                   &desc_bytes, &num_tiles, !tc);
    if (s != TC_OK || count == 0) return s;
    if (!workspace || !aligned(workspace, 256))
        return fail(TC_ERR_INVALID, "gemm_grouped_ws: workspace must be a 256-byte aligned device pointer");
    if ((s = refuse_capture("gemm_grouped_ws", as_stream(stream))) != TC_OK) return s;
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    if (tc) {
        std::vector<unsigned char> tch;
        size_t maps_bytes = 0;
        int32_t tc_tiles = 0;
        bool fits = false;
        if ((s = grouped_tc_host(dt, count, problems, a_base, b_base, lb, workspace_bytes, tch, &maps_bytes, &tc_tiles,
                                 &fits)) != TC_OK)
            return s;
        if (!fits)
            return fail(TC_ERR_INVALID, "gemm_grouped_ws: workspace of %zu bytes is smaller than "
                        "gemm_grouped_workspace_bytes", workspace_bytes);
        return grouped_tc_enqueue("gemm_grouped_ws", dt, lb, tch, maps_bytes, tc_tiles,
                                  static_cast<unsigned char*>(workspace), c_base, alpha, beta, d->status,
                                  d->sm_count, as_stream(stream));
    }
    if (workspace_bytes < host.size())
        return fail(TC_ERR_INVALID, "gemm_grouped_ws: workspace of %zu bytes, need %zu", workspace_bytes, host.size());
    return grouped_mma_enqueue("gemm_grouped_ws", dt, lb, host, desc_bytes, num_tiles,
                               static_cast<unsigned char*>(workspace), a_base, b_base, c_base, alpha, beta,
                               d->sm_count, as_stream(stream));
}

// ------------------------------------------------------------ batched rounding

namespace {

int64_t quant_job_tiles(const tc_quantize_job& j) {
    return ((j.rows + tcg::kQuantTileRows - 1) / tcg::kQuantTileRows) *
           ((j.cols + tcg::kQuantTileCols - 1) / tcg::kQuantTileCols);
}

}  // namespace

extern "C" size_t tc_quantize_batch_workspace_bytes(int32_t count, const tc_quantize_job* jobs) {
    if (count <= 0 || !jobs) return 0;
    int64_t tiles = 0;
    // an empty job of an E4M3 batch still takes one tile (it stores the job's scale)
    for (int32_t j = 0; j < count; ++j)
        tiles += (jobs[j].rows > 0 && jobs[j].cols > 0) ? quant_job_tiles(jobs[j]) : 1;
    return (size_t(count) * sizeof(tcg::QuantJobDev) + 255) / 256 * 256 + size_t(tiles) * sizeof(tcg::QuantTileDev);
}

namespace {

// Checks of a batch of roundings and its job table and tile list built in `host` (job table padded
// to 256 bytes, then the tiles).
tc_status quantize_batch_build(const char* name, int32_t dt, int32_t count, const tc_quantize_job* jobs,
                               float* const* scale_out, std::vector<unsigned char>& host, size_t* desc_bytes_out,
                               int64_t* ntiles_out) {
    if (count < 0 || (count > 0 && !jobs)) return fail(TC_ERR_INVALID, "%s: bad job array", name);
    if (dt == TC_E4M3 && count > 0 && !scale_out) return fail(TC_ERR_INVALID, "%s: null scale array", name);
    const int esz = elem_size(dt);
    const size_t desc_bytes = (size_t(count) * sizeof(tcg::QuantJobDev) + 255) / 256 * 256;
    int64_t ntiles = 0;
    for (int32_t j = 0; j < count; ++j) {
        const tc_quantize_job& J = jobs[j];
        if (J.rows < 0 || J.cols < 0) return fail(TC_ERR_INVALID, "%s: job %d negative size", name, j);
        if (dt == TC_E4M3 && (!scale_out[j] || !aligned(scale_out[j], 4)))
            return fail(TC_ERR_INVALID, "%s: job %d null or misaligned scale", name, j);
        if (J.rows == 0 || J.cols == 0) {
            if (dt == TC_E4M3) ++ntiles;
            continue;
        }
        if (!J.src || !J.dst) return fail(TC_ERR_INVALID, "%s: job %d null pointer", name, j);
        if (J.ld_src < J.cols || J.ld_dst < (J.transpose ? J.rows : J.cols))
            return fail(TC_ERR_INVALID, "%s: job %d leading dimension too small", name, j);
        if (!aligned(J.src, 4) || !aligned(J.dst, esz))
            return fail(TC_ERR_INVALID, "%s: job %d misaligned pointer", name, j);
        ntiles += quant_job_tiles(J);
    }
    if (ntiles > 0x7FFFFFFF) return fail(TC_ERR_INVALID, "%s: too many tiles", name);
    host.assign(desc_bytes + size_t(ntiles) * sizeof(tcg::QuantTileDev), 0);
    auto* hj = reinterpret_cast<tcg::QuantJobDev*>(host.data());
    auto* ht = reinterpret_cast<tcg::QuantTileDev*>(host.data() + desc_bytes);
    int64_t t = 0;
    for (int32_t j = 0; j < count; ++j) {
        const tc_quantize_job& J = jobs[j];
        // 8-element chunks of dst start on 16 bytes (16-bit types) or 8 bytes (E4M3)
        const bool vec = aligned(J.dst, 8 * esz) && J.ld_dst % 8 == 0;
        hj[j] = {J.src, J.dst, J.rows, J.cols, J.ld_src, J.ld_dst, J.transpose ? 1 : 0, vec ? 1 : 0,
                 dt == TC_E4M3 ? scale_out[j] : nullptr, 0u, 0u};
        if (J.rows == 0 || J.cols == 0) {
            if (dt == TC_E4M3) ht[t++] = {j, 0, 0, 0};
            continue;
        }
        for (int64_t r = 0; r < J.rows; r += tcg::kQuantTileRows)
            for (int64_t c = 0; c < J.cols; c += tcg::kQuantTileCols) ht[t++] = {j, 0, r, c};
    }
    *desc_bytes_out = desc_bytes;
    *ntiles_out = ntiles;
    return TC_OK;
}

// Shared body of tc_quantize_batch and tc_quantize_batch_e4m3: the host table, one upload, the
// launches.
tc_status quantize_batch_impl(const char* name, int32_t dt, int32_t count, const tc_quantize_job* jobs,
                              float* const* scale_out, void* workspace, size_t workspace_bytes, void* stream) {
    std::vector<unsigned char> host;
    size_t desc_bytes = 0;
    int64_t ntiles = 0;
    tc_status s = quantize_batch_build(name, dt, count, jobs, scale_out, host, &desc_bytes, &ntiles);
    if (s != TC_OK || count == 0) return s;
    if (!workspace || !aligned(workspace, 256))
        return fail(TC_ERR_INVALID, "%s: workspace must be a 256-byte aligned device pointer", name);
    if (workspace_bytes < host.size())
        return fail(TC_ERR_INVALID, "%s: workspace of %zu bytes, need %zu", name, workspace_bytes, host.size());
    if ((s = refuse_capture(name, as_stream(stream))) != TC_OK) return s;
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    cudaStream_t st = as_stream(stream);
    cudaError_t e = cudaMemcpyAsync(workspace, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, name);
    auto* dev = static_cast<unsigned char*>(workspace);
    return enqueue(tcg::launch_quantize_jobs(dt, reinterpret_cast<tcg::QuantJobDev*>(dev),
                                             reinterpret_cast<const tcg::QuantTileDev*>(dev + desc_bytes),
                                             static_cast<int32_t>(ntiles), st),
                   name);
}

}  // namespace

namespace tcgserve {

tc_status round_and_grouped_ws(int32_t dt, int32_t njobs, const tc_quantize_job* jobs, int32_t count,
                               const tc_problem* problems, const void* ab_base, float* c_base, float alpha,
                               float beta, void* desc, size_t desc_bytes, void* stream) {
    const char* name = "serve batch";
    if (dt != TC_F16 && dt != TC_BF16) return fail(TC_ERR_UNSUPPORTED, "%s: F16 or BF16 only", name);
    std::vector<unsigned char> q;
    size_t q_table = 0;
    int64_t q_tiles = 0;
    tc_status s = quantize_batch_build(name, dt, njobs, jobs, nullptr, q, &q_table, &q_tiles);
    if (s != TC_OK) return s;
    const size_t q_bytes = (q.size() + 255) / 256 * 256;
    std::vector<unsigned char> g;
    size_t g_table = 0;
    int64_t g_tiles = 0;
    const bool tc = grouped_use_tensor_cores(TC_ROW_MAJOR);
    if ((s = grouped_mma_host(name, dt, count, problems, ab_base, TC_ROW_MAJOR, ab_base, TC_ROW_MAJOR, c_base, g,
                              &g_table, &g_tiles, !tc)) != TC_OK)
        return s;
    int32_t tc_tiles = 0;
    if (tc && count > 0) {
        bool fits = false;
        if ((s = grouped_tc_host(dt, count, problems, ab_base, ab_base, TC_ROW_MAJOR,
                                 desc_bytes > q_bytes ? desc_bytes - q_bytes : 0, g, &g_table, &tc_tiles, &fits)) !=
            TC_OK)
            return s;
        if (!fits) return fail(TC_ERR_INVALID, "%s: descriptor space of %zu bytes is too small", name, desc_bytes);
    }
    if (!desc || !aligned(desc, 256) || q_bytes + g.size() > desc_bytes)
        return fail(TC_ERR_INVALID, "%s: descriptor space of %zu bytes is too small", name, desc_bytes);
    cudaStream_t st = as_stream(stream);
    if ((s = refuse_capture(name, st)) != TC_OK) return s;
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    // both tables in one upload: the rounding's at desc, the grouped GEMM's 256-byte aligned after it
    q.resize(q_bytes, 0);
    q.insert(q.end(), g.begin(), g.end());
    cudaError_t e = cudaMemcpyAsync(desc, q.data(), q.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, name);
    auto* dev = static_cast<unsigned char*>(desc);
    if (q_tiles > 0 &&
        (s = enqueue(tcg::launch_quantize_jobs(dt, reinterpret_cast<tcg::QuantJobDev*>(dev),
                                               reinterpret_cast<const tcg::QuantTileDev*>(dev + q_table),
                                               static_cast<int32_t>(q_tiles), st),
                     name)) != TC_OK)
        return s;
    if (count == 0) return TC_OK;
    unsigned char* gdev = dev + q_bytes;
    if (tc)
        return enqueue(tcg::launch_grouped_tc(dt, reinterpret_cast<const tcg::GroupedTcTile*>(gdev + g_table),
                                              tc_tiles, reinterpret_cast<const CUtensorMap*>(gdev), c_base, alpha,
                                              beta, d->status, d->sm_count, st, -1, true),
                       name);
    return enqueue(tcg::launch_grouped(dt, TC_ROW_MAJOR, reinterpret_cast<const tcg::GroupedProblemDev*>(gdev),
                                       reinterpret_cast<const tcg::GroupedTileDev*>(gdev + g_table),
                                       static_cast<int32_t>(g_tiles), ab_base, ab_base, c_base, alpha, beta,
                                       d->sm_count, st),
                   name);
}

}  // namespace tcgserve

extern "C" tc_status tc_quantize_batch(int32_t dt, int32_t count, const tc_quantize_job* jobs, void* workspace,
                                       size_t workspace_bytes, void* stream) {
    if (dt != TC_F16 && dt != TC_BF16)
        return fail(TC_ERR_UNSUPPORTED, "tc_quantize_batch: F16 or BF16 only (E4M3: tc_quantize_batch_e4m3)");
    return quantize_batch_impl("tc_quantize_batch", dt, count, jobs, nullptr, workspace, workspace_bytes, stream);
}

extern "C" tc_status tc_quantize_batch_e4m3(int32_t count, const tc_quantize_job* jobs, float* const* scale_out,
                                            void* workspace, size_t workspace_bytes, void* stream) {
    return quantize_batch_impl("tc_quantize_batch_e4m3", TC_E4M3, count, jobs, scale_out, workspace,
                               workspace_bytes, stream);
}

// ------------------------------------------------------------ autotuning

namespace {

// Mean time of `iters` launches after `warm`, with CUDA events on `st`.
template <typename F>
tc_status time_ms(F&& launch, cudaStream_t st, int warm, int iters, double* ms_out) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return cuda_fail(e, "autotune: event");
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(e, "autotune: event");
    }
    tc_status s = TC_OK;
    for (int i = 0; i < warm && s == TC_OK; ++i) s = launch();
    cudaEventRecord(e0, st);
    for (int i = 0; i < iters && s == TC_OK; ++i) s = launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (s == TC_OK && e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != TC_OK) return s;
    if (e != cudaSuccess) return cuda_fail(e, "autotune: synchronize");
    *ms_out = ms / iters;
    return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_autotune_gemm(int32_t dt, int64_t m, int64_t n, int64_t k, void* stream, double* best_ms) {
    if (dt != TC_F16 && dt != TC_BF16 && dt != TC_E4M3) return fail(TC_ERR_INVALID, "tc_autotune_gemm: bad dtype");
    tc_status s = check_dims(m, n, k);
    if (s != TC_OK) return s;
    if (m < 1 || n < 1 || k < 1) return fail(TC_ERR_INVALID, "tc_autotune_gemm: empty problem");
    Device* d;
    if ((s = get_device(&d)) != TC_OK) return s;
    cudaStream_t st = as_stream(stream);
    const int esz = elem_size(dt);
    const int64_t kp = (k + 15) / 16 * 16;
    const size_t a_bytes = size_t(m) * kp * esz, b_bytes = size_t(n) * kp * esz, c_bytes = size_t(m) * n * 4;
    void* buf = nullptr;
    cudaError_t e = cudaMallocAsync(&buf, a_bytes + b_bytes + c_bytes + 256 * 3 + 8, st);
    if (e != cudaSuccess) return fail(TC_ERR_OOM, "tc_autotune_gemm: scratch: %s", cudaGetErrorString(e));
    uint8_t* A = static_cast<uint8_t*>(buf);
    uint8_t* B = A + (a_bytes + 255) / 256 * 256;
    float* C = reinterpret_cast<float*>(B + (b_bytes + 255) / 256 * 256);
    float* scales = reinterpret_cast<float*>(reinterpret_cast<uint8_t*>(C) + (c_bytes + 255) / 256 * 256);
    // operands of moderate magnitude (byte 0x3C: 1.05 in FP16, 0.0117 in BF16, 1.5 in E4M3)
    cudaMemsetAsync(A, 0x3C, a_bytes, st);
    cudaMemsetAsync(B, 0x3C, b_bytes, st);
    cudaMemsetAsync(C, 0, c_bytes, st);
    const float ones[2] = {1.0f, 1.0f};
    cudaMemcpyAsync(scales, ones, sizeof(ones), cudaMemcpyHostToDevice, st);
    // candidates are passed to the launch explicitly: nothing another thread's calls see changes
    // until the winner is stored in the table at the end
    auto time_cfg = [&](const GemmCfg& c, double* ms) {
        return time_ms([&] {
            return gemm_mixed_impl(dt, m, n, k, 1.0f, A, kp, TC_ROW_MAJOR, B, kp, TC_COL_MAJOR, 0.0f, C, n,
                                   dt == TC_E4M3 ? scales : nullptr, dt == TC_E4M3 ? scales + 1 : nullptr, st, &c);
        }, st, 2, 5, ms);
    };
    // The untuned configuration is timed first and stays unless a candidate beats it by more than
    // 2 %: single timings of one configuration scatter by about that much, and a pick made on noise
    // would trade the default's lower DRAM traffic (serpentine K order) for nothing.
    const GemmCfg dflt = default_gemm_cfg(m, n, d->sm_count);
    TuneCfg best{dflt, 1e30};
    auto same = [](const GemmCfg& x, const GemmCfg& y) {
        return x.pair == y.pair && x.group_m == y.group_m && x.tail == y.tail && x.korder == y.korder &&
               x.cluster == y.cluster && (x.pair || x.bn == y.bn);
    };
    auto consider = [&](const GemmCfg& c) {
        if (s != TC_OK || (best.ms < 1e30 && same(c, dflt))) return;
        double ms = 0;
        s = time_cfg(c, &ms);
        if (s == TC_OK && (same(c, dflt) ? ms < best.ms : ms < 0.98 * best.ms)) best = {c, ms};
    };
    consider(dflt);
    // tile kind and width (single CTAs 128 x 64 / 128 x 128 / 128 x 256, or pairs), then the raster
    // band of the best of those; for pairs then clusters of four (A multicast between two pairs,
    // whole tiles only) with each band, and the tail split; last the K order
    for (int bn : {64, 128, 256}) consider(GemmCfg{0, 8, 2, 1, 2, bn});
    if (m > 128) consider(GemmCfg{1, 8, 2, 1, 2, 256});  // a pair tile would leave half of it empty
    for (int g : {4, 8, 16, 32}) consider(GemmCfg{best.cfg.pair, g, 2, 1, 2, best.cfg.bn});
    if (best.cfg.pair) {
        for (int g : {4, 8, 16, 32}) consider(GemmCfg{1, g, 1, 1, 4, 256});
        if (best.cfg.cluster == 2)
            for (int tail : {0, 1, 2}) consider(GemmCfg{1, best.cfg.group_m, tail, best.cfg.korder, 2, 256});
    }
    consider(GemmCfg{best.cfg.pair, best.cfg.group_m, best.cfg.tail, 0, best.cfg.cluster, best.cfg.bn});
    cudaFreeAsync(buf, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (s != TC_OK) return s;
    if (e2 != cudaSuccess) return cuda_fail(e2, "tc_autotune_gemm: synchronize");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[tune_key(dt, m, n, k)] = best;
    }
    if (best_ms) *best_ms = best.ms;
    return TC_OK;
}

tc_status gemm_grouped_plan_autotune(tc_grouped_plan* plan, const void* a_base, const void* b_base, float* c_base,
                                     void* stream, double* best_ms) {
    if (!plan) return fail(TC_ERR_INVALID, "grouped autotune: null plan");
    cudaStream_t st = as_stream(stream);
    const int variants[3] = {0, 1, 2};
    const int nvar = plan->use_tc ? 3 : 1;
    double best = 1e30;
    int best_v = plan->use_tc ? 0 : 2;
    for (int i = 0; i < nvar; ++i) {
        plan->variant = plan->use_tc ? variants[i] : 2;
        double ms = 0;
        tc_status s = time_ms([&] { return gemm_grouped_plan_run(plan, a_base, b_base, c_base, 1.0f, 0.0f, 0, stream); },
                              st, 1, 3, &ms);
        if (s != TC_OK) {
            plan->variant = -1;
            return s;
        }
        if (ms < best) {
            best = ms;
            best_v = plan->variant;
        }
    }
    plan->variant = best_v;
    if (plan->exec) {  // a recorded graph holds the previous variant
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
    }
    if (best_ms) *best_ms = best;
    return TC_OK;
}

tc_status tc_autotune_save(const char* path) {
    if (!path) return fail(TC_ERR_INVALID, "tc_autotune_save: null path");
    FILE* f = fopen(path, "w");
    if (!f) return fail(TC_ERR_INVALID, "tc_autotune_save: cannot open %s", path);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    fprintf(f, "# tcgemm autotune: dt log2m log2n log2k pair group_m tail korder cluster bn ms\n");
    for (const auto& kv : g_tune)
        fprintf(f, "%d %d %d %d %d %d %d %d %d %d %.6f\n", kv.first.dt, kv.first.lm, kv.first.ln, kv.first.lk,
                kv.second.cfg.pair, kv.second.cfg.group_m, kv.second.cfg.tail, kv.second.cfg.korder,
                kv.second.cfg.cluster, kv.second.cfg.bn, kv.second.ms);
    fclose(f);
    return TC_OK;
}

tc_status tc_autotune_load(const char* path) {
    if (!path) return fail(TC_ERR_INVALID, "tc_autotune_load: null path");
    FILE* f = fopen(path, "r");
    if (!f) return fail(TC_ERR_INVALID, "tc_autotune_load: cannot open %s", path);
    char line[256];
    int n = 0;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    while (fgets(line, sizeof(line), f)) {
        if (line[0] == '#') continue;
        TuneKey key;
        TuneCfg t{{0, 8, 1, 1, 2, 256}, 0.0};
        // whitespace-separated fields: integers, then the time; eleven of them, ten in a table
        // without the tile width (256), seven in one without the tail, K-order, cluster and
        // tile-width columns
        int v[10];
        int nf = 0;
        bool bad = false;
        char* save = nullptr;
        for (char* tok = strtok_r(line, " \t\r\n", &save); tok; tok = strtok_r(nullptr, " \t\r\n", &save)) {
            if (nf < 10 && strchr(tok, '.') == nullptr) {
                char* end = nullptr;
                const long x = strtol(tok, &end, 10);
                if (*end != '\0' || x < -1000000 || x > 1000000) bad = true;
                v[nf++] = static_cast<int>(x);
            } else {
                char* end = nullptr;
                t.ms = strtod(tok, &end);
                if (*end != '\0' || strtok_r(nullptr, " \t\r\n", &save) != nullptr) bad = true;
                ++nf;
                break;
            }
        }
        if (bad) continue;
        if (nf == 11) {
            t.cfg = {v[4], v[5], v[6], v[7], v[8], v[9]};
        } else if (nf == 10) {
            t.cfg = {v[4], v[5], v[6], v[7], v[8], 256};
        } else if (nf == 7) {
            t.cfg = {v[4], v[5], 1, 1, 2, 256};
        } else {
            continue;
        }
        key = {v[0], v[1], v[2], v[3]};
        const GemmCfg& c = t.cfg;
        if ((c.pair == 0 || c.pair == 1) && c.group_m >= 1 && c.group_m <= 1024 && (c.tail >= 0 && c.tail <= 2) &&
            (c.korder == 0 || c.korder == 1) && (c.cluster == 2 || c.cluster == 4) &&
            (c.bn == 64 || c.bn == 128 || c.bn == 256)) {
            g_tune[key] = t;
            ++n;
        }
    }
    fclose(f);
    return n > 0 ? TC_OK : fail(TC_ERR_INVALID, "tc_autotune_load: no entries in %s", path);
}

}  // extern "C"
