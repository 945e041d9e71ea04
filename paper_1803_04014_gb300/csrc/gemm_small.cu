// Batched and grouped small GEMM (Sec. IV-B; Sec. VI: the paper's batched
// kernel runs one 16x16x16 product per warp, 16 problems per 512-thread block).
//
// Both workloads move far more bytes than they compute (4 FLOP/byte for the
// 16^3 batch, about 34 for the grouped sizes), so they are built around the
// memory system: the 16^3 batch streams whole chunks of problems into shared
// memory with bulk TMA copies (one thread issues them, an mbarrier tracks the
// bytes) and the grouped kernel runs a 3-stage cp.async pipeline per 64 x 64
// output tile.  The multiply itself is the warp-level mma.sync m16n8k16 with
// FP32 accumulation: a 16x16 problem is two of them, far below the 64- and
// 128-row shapes of tcgen05.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "launch.h"
#include "tc_ptx.cuh"

namespace tcg {
namespace {

// ------------------------------------------------------------ warp MMA helpers

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

template <int DT>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (DT == 0) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// ------------------------------------------------------------ 16^3 batch

constexpr int kBatchProbs = 32;     // problems per stage (16 KB of A + 16 KB of B)
constexpr int kBatchStages = 3;
constexpr int kBatchThreads = 256;  // 8 warps, 4 problems each per stage
constexpr int kProbBytes = 512;     // 16 x 16 x 2 bytes
constexpr int kBatchSmem = kBatchStages * 2 * kBatchProbs * kProbBytes + 64;

template <int DT, int LB>
__global__ void __launch_bounds__(kBatchThreads, 2)
    k_batched16(int64_t batch, float alpha, const uint16_t* __restrict__ A, int64_t sa,
                const uint16_t* __restrict__ B, int64_t sb, float beta, float* __restrict__ C, int64_t sc,
                int* status) {
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t sbase = smem_addr(smem);
    const uint32_t bars = sbase + kBatchStages * 2 * kBatchProbs * kProbBytes;
    __shared__ int abort_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nchunks = (batch + kBatchProbs - 1) / kBatchProbs;
    const bool dense_a = (sa == 256), dense_b = (sb == 256);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kBatchStages; ++s) mbar_init(bars + 8 * s, 1);
        abort_s = 0;
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int64_t chunk, int s) {
        const int64_t p0 = chunk * kBatchProbs;
        const int np = static_cast<int>((batch - p0) < kBatchProbs ? (batch - p0) : kBatchProbs);
        const uint32_t bar = bars + 8 * s;
        const uint32_t dA = sbase + s * 2 * kBatchProbs * kProbBytes;
        const uint32_t dB = dA + kBatchProbs * kProbBytes;
        mbar_arrive_expect_tx(bar, static_cast<uint32_t>(np) * 2 * kProbBytes);
        if (dense_a) bulk_load(dA, A + p0 * 256, np * kProbBytes, bar);
        else
            for (int i = 0; i < np; ++i) bulk_load(dA + i * kProbBytes, A + (p0 + i) * sa, kProbBytes, bar);
        if (dense_b) bulk_load(dB, B + p0 * 256, np * kProbBytes, bar);
        else
            for (int i = 0; i < np; ++i) bulk_load(dB + i * kProbBytes, B + (p0 + i) * sb, kProbBytes, bar);
    };

    // chunks of this block: blockIdx.x + j * gridDim.x
    if (threadIdx.x == 0) {
        for (int s = 0; s < kBatchStages; ++s) {
            const int64_t c = blockIdx.x + (int64_t)s * gridDim.x;
            if (c < nchunks) issue(c, s);
        }
    }
    int64_t j = 0;
    for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x, ++j) {
        const int s = static_cast<int>(j % kBatchStages);
        const uint32_t parity = static_cast<uint32_t>((j / kBatchStages) & 1);
        const bool ok = mbar_wait(bars + 8 * s, parity, &abort_s, status);
        if (__syncthreads_or(!ok)) break;
        const int64_t p0 = c * kBatchProbs;
        const int np = static_cast<int>((batch - p0) < kBatchProbs ? (batch - p0) : kBatchProbs);
        const uint32_t sA = sbase + s * 2 * kBatchProbs * kProbBytes;
        const uint32_t sB = sA + kBatchProbs * kProbBytes;
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {
            const int p = warp * 4 + q;
            if (p >= np) break;
            uint32_t a[4];
            // A row-major 16 x 16: lanes 0-15 rows 0-15 at k 0, lanes 16-31 at k 8
            ldsm_x4(sA + p * kProbBytes + (lane & 15) * 32 + (lane >> 4) * 16, a[0], a[1], a[2], a[3]);
            uint32_t b[4];
            if (LB == 0) {
                // B row-major [k][n]: transposed 8x8 loads; lane -> k row, n column block
                const int kr = (lane & 7) + ((lane >> 3) & 1) * 8;
                ldsm_x4_t(sB + p * kProbBytes + kr * 32 + (lane >> 4) * 16, b[0], b[1], b[2], b[3]);
            } else {
                // B column-major [n][k]: lane -> n row, k column block
                const int nr = (lane & 7) + (lane >> 4) * 8;
                ldsm_x4(sB + p * kProbBytes + nr * 32 + ((lane >> 3) & 1) * 16, b[0], b[1], b[2], b[3]);
            }
            float d0[4] = {0.f, 0.f, 0.f, 0.f}, d1[4] = {0.f, 0.f, 0.f, 0.f};
            mma16816<DT>(d0, a, b[0], b[1]);
            mma16816<DT>(d1, a, b[2], b[3]);
            const int g = lane >> 2, cc = (lane & 3) * 2;
            float* cp = C + (p0 + p) * sc;
            float2* r0a = reinterpret_cast<float2*>(cp + g * 16 + cc);
            float2* r1a = reinterpret_cast<float2*>(cp + (g + 8) * 16 + cc);
            float2* r0b = reinterpret_cast<float2*>(cp + g * 16 + 8 + cc);
            float2* r1b = reinterpret_cast<float2*>(cp + (g + 8) * 16 + 8 + cc);
            float2 o0 = make_float2(alpha * d0[0], alpha * d0[1]), o1 = make_float2(alpha * d0[2], alpha * d0[3]);
            float2 o2 = make_float2(alpha * d1[0], alpha * d1[1]), o3 = make_float2(alpha * d1[2], alpha * d1[3]);
            if (beta != 0.0f) {
                const float2 c0 = *r0a, c1 = *r1a, c2 = *r0b, c3 = *r1b;
                o0.x += beta * c0.x; o0.y += beta * c0.y; o1.x += beta * c1.x; o1.y += beta * c1.y;
                o2.x += beta * c2.x; o2.y += beta * c2.y; o3.x += beta * c3.x; o3.y += beta * c3.y;
            }
            __stcs(r0a, o0);
            __stcs(r1a, o1);
            __stcs(r0b, o2);
            __stcs(r1b, o3);
        }
        __syncthreads();  // every warp is done with stage s
        if (threadIdx.x == 0) {
            const int64_t nc = c + (int64_t)kBatchStages * gridDim.x;
            if (nc < nchunks) issue(nc, s);
        }
    }
    if (abort_s && threadIdx.x == 0) {
        // leaving early: let issued copies land before the block exits
        for (int s = 0; s < kBatchStages; ++s) mbar_wait_bounded(bars + 8 * s, 0, 100000000ull);
    }
}

// ------------------------------------------------------------ grouped GEMM

constexpr int GT_M = kGroupedTileM, GT_N = kGroupedTileN, GT_K = 32, GT_STAGES = 3;
constexpr int kGThreads = 128;  // 4 warps as 2 x 2, each 32 x 32 of the tile
constexpr int kGStageA = GT_M * GT_K * 2;  // 4 KB
constexpr int kGStageB = GT_K * GT_N * 2;  // 4 KB

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int DT, int LB>
__global__ void __launch_bounds__(kGThreads) k_grouped(const GroupedProblemDev* __restrict__ probs,
                                                       const GroupedTileDev* __restrict__ tiles, int32_t num_tiles,
                                                       const uint16_t* __restrict__ a_base,
                                                       const uint16_t* __restrict__ b_base, float* __restrict__ c_base,
                                                       float alpha, float beta) {
    __shared__ __align__(128) uint8_t sm[GT_STAGES * (kGStageA + kGStageB)];
    const uint32_t s0 = smem_addr(sm);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int wm = warp >> 1, wn = warp & 1;

    for (int t = blockIdx.x; t < num_tiles; t += gridDim.x) {
        const GroupedTileDev tile = tiles[t];
        const GroupedProblemDev P = probs[tile.prob];
        const int m0 = tile.tm * GT_M, n0 = tile.tn * GT_N;
        const uint16_t* Ag = a_base + P.off_a;
        const uint16_t* Bg = b_base + P.off_b;
        const int nk = (P.k + GT_K - 1) / GT_K;

        auto load_stage = [&](int kc, int s) {
            const int k0 = kc * GT_K;
            const uint32_t dA = s0 + s * (kGStageA + kGStageB);
            const uint32_t dB = dA + kGStageA;
#pragma unroll
            for (int i = 0; i < 2; ++i) {  // A: 64 rows x 4 chunks of 16 B
                const int q = tid + i * kGThreads;
                const int row = q >> 2, kc8 = q & 3;
                const int gk = k0 + kc8 * 8;
                int bytes = 0;
                const uint16_t* src = Ag;
                if (m0 + row < P.m && gk < P.k) {
                    bytes = min(8, P.k - gk) * 2;
                    src = Ag + (int64_t)(m0 + row) * P.lda + gk;
                }
                cp_async16(dA + row * 64 + ((kc8 ^ ((row >> 1) & 3)) << 4), src, bytes);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int q = tid + i * kGThreads;
                int bytes = 0;
                const uint16_t* src = Bg;
                if (LB == 0) {  // B row-major [k][n]: 32 rows x 8 chunks
                    const int kr = q >> 3, nc = q & 7;
                    const int gn = n0 + nc * 8;
                    if (k0 + kr < P.k && gn < P.n) {
                        bytes = min(8, P.n - gn) * 2;
                        src = Bg + (int64_t)(k0 + kr) * P.ldb + gn;
                    }
                    cp_async16(dB + kr * 128 + ((nc ^ (kr & 7)) << 4), src, bytes);
                } else {  // B column-major [n][k]: 64 rows x 4 chunks
                    const int nr = q >> 2, kc8 = q & 3;
                    const int gk = k0 + kc8 * 8;
                    if (n0 + nr < P.n && gk < P.k) {
                        bytes = min(8, P.k - gk) * 2;
                        src = Bg + (int64_t)(n0 + nr) * P.ldb + gk;
                    }
                    cp_async16(dB + nr * 64 + ((kc8 ^ ((nr >> 1) & 3)) << 4), src, bytes);
                }
            }
        };

        float acc[2][4][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

#pragma unroll
        for (int s = 0; s < GT_STAGES - 1; ++s) {
            if (s < nk) load_stage(s, s);
            cp_async_commit();
        }
        for (int kc = 0; kc < nk; ++kc) {
            cp_async_wait<GT_STAGES - 2>();
            __syncthreads();
            const int s = kc % GT_STAGES;
            const uint32_t sA = s0 + s * (kGStageA + kGStageB);
            const uint32_t sB = sA + kGStageA;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                uint32_t af[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int row = wm * 32 + mt * 16 + (lane & 15);
                    const int kc8 = ks * 2 + (lane >> 4);
                    ldsm_x4(sA + row * 64 + ((kc8 ^ ((row >> 1) & 3)) << 4), af[mt][0], af[mt][1], af[mt][2],
                            af[mt][3]);
                }
                uint32_t bf[4][2];
#pragma unroll
                for (int np = 0; np < 2; ++np) {
                    uint32_t r0, r1, r2, r3;
                    if (LB == 0) {
                        const int kr = ks * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                        const int nc = (wn * 32 + np * 16) / 8 + (lane >> 4);
                        ldsm_x4_t(sB + kr * 128 + ((nc ^ (kr & 7)) << 4), r0, r1, r2, r3);
                    } else {
                        const int nr = wn * 32 + np * 16 + (lane & 7) + (lane >> 4) * 8;
                        const int kc8 = ks * 2 + ((lane >> 3) & 1);
                        ldsm_x4(sB + nr * 64 + ((kc8 ^ ((nr >> 1) & 3)) << 4), r0, r1, r2, r3);
                    }
                    bf[np * 2][0] = r0;
                    bf[np * 2][1] = r1;
                    bf[np * 2 + 1][0] = r2;
                    bf[np * 2 + 1][1] = r3;
                }
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt) mma16816<DT>(acc[mt][nt], af[mt], bf[nt][0], bf[nt][1]);
            }
            const int nxt = kc + GT_STAGES - 1;
            if (nxt < nk) load_stage(nxt, nxt % GT_STAGES);
            cp_async_commit();
        }
        cp_async_wait<0>();
        __syncthreads();  // shared memory is reused by the next tile

        float* Cg = c_base + P.off_c;
        const int g = lane >> 2, cc = (lane & 3) * 2;
        const bool vec2 = ((P.ldc & 1) == 0) && ((P.off_c & 1) == 0);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int r = m0 + wm * 32 + mt * 16 + g + h * 8;
                if (r >= P.m) continue;
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    const int c = n0 + wn * 32 + nt * 8 + cc;
                    float* p = Cg + (int64_t)r * P.ldc + c;
                    const float v0 = alpha * acc[mt][nt][h * 2 + 0], v1 = alpha * acc[mt][nt][h * 2 + 1];
                    if (vec2 && c + 1 < P.n) {
                        float2 o = make_float2(v0, v1);
                        if (beta != 0.0f) {
                            const float2 old = *reinterpret_cast<const float2*>(p);
                            o.x += beta * old.x;
                            o.y += beta * old.y;
                        }
                        *reinterpret_cast<float2*>(p) = o;
                    } else {
                        if (c < P.n) p[0] = (beta != 0.0f) ? v0 + beta * p[0] : v0;
                        if (c + 1 < P.n) p[1] = (beta != 0.0f) ? v1 + beta * p[1] : v1;
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_batched16(int dt, int64_t batch, float alpha, const void* A, int64_t sa, const void* B, int64_t sb,
                             int lb, float beta, float* C, int64_t sc, int* status, int sm_count, cudaStream_t st) {
    if (batch <= 0) return cudaSuccess;
    const int64_t nchunks = (batch + kBatchProbs - 1) / kBatchProbs;
    const int64_t want = static_cast<int64_t>(sm_count) * 2;
    const int grid = static_cast<int>(nchunks < want ? nchunks : want);
    auto* a = static_cast<const uint16_t*>(A);
    auto* b = static_cast<const uint16_t*>(B);
    void (*kern)(int64_t, float, const uint16_t*, int64_t, const uint16_t*, int64_t, float, float*, int64_t, int*);
    if (dt == 0) kern = (lb == 0) ? k_batched16<0, 0> : k_batched16<0, 1>;
    else kern = (lb == 0) ? k_batched16<1, 0> : k_batched16<1, 1>;
    cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), kBatchSmem, nullptr, 0, nullptr);
    if (e != cudaSuccess) return e;
    kern<<<grid, kBatchThreads, kBatchSmem, st>>>(batch, alpha, a, sa, b, sb, beta, C, sc, status);
    return cudaGetLastError();
}

cudaError_t launch_grouped(int dt, int lb, const GroupedProblemDev* probs, const GroupedTileDev* tiles,
                           int32_t num_tiles, const void* a_base, const void* b_base, float* c_base, float alpha,
                           float beta, int sm_count, cudaStream_t st) {
    if (num_tiles <= 0) return cudaSuccess;
    auto* a = static_cast<const uint16_t*>(a_base);
    auto* b = static_cast<const uint16_t*>(b_base);
    void (*kern)(const GroupedProblemDev*, const GroupedTileDev*, int32_t, const uint16_t*, const uint16_t*, float*,
                 float, float);
    if (dt == 0) kern = (lb == 0) ? k_grouped<0, 0> : k_grouped<0, 1>;
    else kern = (lb == 0) ? k_grouped<1, 0> : k_grouped<1, 1>;
    // persistent grid of exactly the CTAs that can be resident, so the static tile stride has no tail wave
    int per_sm = 0;
    const cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), 0, nullptr, kGThreads, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int want = sm_count * per_sm;
    const int grid = num_tiles < want ? num_tiles : want;
    kern<<<grid, kGThreads, 0, st>>>(probs, tiles, num_tiles, a, b, c_base, alpha, beta);
    return cudaGetLastError();
}

}  // namespace tcg
