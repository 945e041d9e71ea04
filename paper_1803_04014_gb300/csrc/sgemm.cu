// FP32 GEMM on the CUDA cores: the paper's "sgemm" comparison (Sec. VII-A:
// GEMM without tensor cores; Sec. VII-B: the refined tensor-core GEMM is
// weighed against it in time and error).  No tensor cores are involved.
//
// A block of 256 threads (16 x 16) computes a (RM*16) x (RN*16) output tile;
// thread (ty, tx) = (tid / 16, tid % 16) holds an RM x RN register block: rows
// ty*4 + 64*i + {0..3} (i < RM/4) and columns tx*4 + 64*j + {0..3} (j < RN/4).
// K advances SK at a time through double-buffered shared memory, As[k][m] and
// Bs[k][n]; the next step's operands are loaded into registers while the
// current one is used.  Interior tiles whose rows are 16-byte aligned load 16
// bytes per access; the edge of the matrix and unaligned operands load element
// by element.
//
// Every output element is the FP32 FMA chain acc = fma(a_k, b_k, acc) over k
// in increasing order, then alpha * acc (+ beta * C).  The accumulators of two
// adjacent columns are updated by one packed FP32 FMA (__ffma2_rn: two
// independent round-to-nearest FMAs), which halves the FMA instructions issued.
#include "launch.h"

namespace tcg {
namespace {

constexpr int kThreads = 256;

// Staging of one operand's SK x BX slice of a K step, NV 16-byte groups per thread.
//   "k-contiguous" operand (row-major A, column-major B: rows of K): group f = tid + 256 h covers
//   row f / (SK/4), k-group f % (SK/4); stored transposed into rows of pitch BX + 4.
//   "mn-contiguous" operand (column-major A, row-major B: rows of M or N): group f covers k-row
//   f / (BX/4), elements 4 (f % (BX/4)) ... + 3, stored as they are.
template <bool KCONT, int BX, int SK>
struct Stage {
    static constexpr int NV = BX * SK / 4 / kThreads;
    static constexpr int SP = BX + 4;
    float4 v[NV];

    __device__ __forceinline__ static void coords(int f, int& r, int& kk) {
        if (KCONT) {
            r = f / (SK / 4);
            kk = (f % (SK / 4)) * 4;
        } else {
            kk = f / (BX / 4);
            r = (f % (BX / 4)) * 4;
        }
    }

    __device__ __forceinline__ void load(const float* __restrict__ X, int64_t ld, int rows, int k, int r0, int k0,
                                         bool fast, int tid) {
#pragma unroll
        for (int h = 0; h < NV; ++h) {
            int r, kk;
            coords(tid + kThreads * h, r, kk);
            const int gr = r0 + r, gk = k0 + kk;
            if (fast) {
                const float* p = KCONT ? X + static_cast<int64_t>(gr) * ld + gk : X + static_cast<int64_t>(gk) * ld + gr;
                v[h] = *reinterpret_cast<const float4*>(p);
            } else {
                float e[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int rr = KCONT ? gr : gr + i, kq = KCONT ? gk + i : gk;
                    e[i] = (rr < rows && kq < k) ? (KCONT ? X[static_cast<int64_t>(rr) * ld + kq]
                                                          : X[static_cast<int64_t>(kq) * ld + rr])
                                                 : 0.0f;
                }
                v[h] = make_float4(e[0], e[1], e[2], e[3]);
            }
        }
    }

    __device__ __forceinline__ void store(float (*S)[SP], int tid) const {
#pragma unroll
        for (int h = 0; h < NV; ++h) {
            int r, kk;
            coords(tid + kThreads * h, r, kk);
            if (KCONT) {
                S[kk + 0][r] = v[h].x;
                S[kk + 1][r] = v[h].y;
                S[kk + 2][r] = v[h].z;
                S[kk + 3][r] = v[h].w;
            } else {
                *reinterpret_cast<float4*>(&S[kk][r]) = v[h];
            }
        }
    }
};

template <int LA, int LB, int RM, int RN, int SK, int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
    k_sgemm(int m, int n, int k, float alpha, const float* __restrict__ A, int64_t lda, const float* __restrict__ B,
            int64_t ldb, float beta, float* __restrict__ C, int64_t ldc, int vec_a, int vec_b) {
    constexpr int BM = RM * 16, BN = RN * 16;
    // A is k-contiguous when row-major (LA = 0), B when column-major (LB = 1)
    using SA = Stage<LA == 0, BM, SK>;
    using SB = Stage<LB == 1, BN, SK>;
    __shared__ __align__(16) float As[2][SK][SA::SP];
    __shared__ __align__(16) float Bs[2][SK][SB::SP];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    SA sa;
    SB sb;
    const bool full_m = m0 + BM <= m, full_n = n0 + BN <= n;
    auto load = [&](int k0) {
        const bool kfull = k0 + SK <= k;
        sa.load(A, lda, m, k, m0, k0, vec_a && full_m && kfull, tid);
        sb.load(B, ldb, n, k, n0, k0, vec_b && full_n && kfull, tid);
    };

    // accumulators in column pairs: one packed FP32 FMA (two lanes of RN FMA) per pair and k
    float2 acc[RM][RN / 2];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN / 2; ++j) acc[i][j] = make_float2(0.0f, 0.0f);

    const int nk = (k + SK - 1) / SK;
    load(0);
    sa.store(As[0], tid);
    sb.store(Bs[0], tid);
    __syncthreads();
    for (int s = 0; s < nk; ++s) {
        const int buf = s & 1;
        if (s + 1 < nk) load((s + 1) * SK);
#pragma unroll
        for (int kk = 0; kk < SK; ++kk) {
            float av[RM];
            float2 bv[RN / 2];
#pragma unroll
            for (int i = 0; i < RM / 4; ++i) {
                const float4 a4 = *reinterpret_cast<const float4*>(&As[buf][kk][64 * i + ty * 4]);
                av[4 * i + 0] = a4.x;
                av[4 * i + 1] = a4.y;
                av[4 * i + 2] = a4.z;
                av[4 * i + 3] = a4.w;
            }
#pragma unroll
            for (int j = 0; j < RN / 4; ++j) {
                const float4 b4 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 * j + tx * 4]);
                bv[2 * j + 0] = make_float2(b4.x, b4.y);
                bv[2 * j + 1] = make_float2(b4.z, b4.w);
            }
#pragma unroll
            for (int i = 0; i < RM; ++i) {
                const float2 a2 = make_float2(av[i], av[i]);
#pragma unroll
                for (int j = 0; j < RN / 2; ++j) acc[i][j] = __ffma2_rn(a2, bv[j], acc[i][j]);
            }
        }
        if (s + 1 < nk) {
            sa.store(As[buf ^ 1], tid);
            sb.store(Bs[buf ^ 1], tid);
        }
        __syncthreads();
    }

    const bool vec_c = (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
    auto el = [&](int i, int j) { return (j & 1) ? acc[i][j >> 1].y : acc[i][j >> 1].x; };
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int r = m0 + 64 * (i / 4) + ty * 4 + (i % 4);
        if (r >= m) continue;
#pragma unroll
        for (int jh = 0; jh < RN / 4; ++jh) {
            const int c = n0 + jh * 64 + tx * 4;
            float* p = C + static_cast<int64_t>(r) * ldc + c;
            if (vec_c && c + 4 <= n) {
                float4 o = make_float4(alpha * el(i, 4 * jh + 0), alpha * el(i, 4 * jh + 1),
                                       alpha * el(i, 4 * jh + 2), alpha * el(i, 4 * jh + 3));
                if (beta != 0.0f) {
                    const float4 old = *reinterpret_cast<const float4*>(p);
                    o.x = fmaf(alpha, el(i, 4 * jh + 0), beta * old.x);
                    o.y = fmaf(alpha, el(i, 4 * jh + 1), beta * old.y);
                    o.z = fmaf(alpha, el(i, 4 * jh + 2), beta * old.z);
                    o.w = fmaf(alpha, el(i, 4 * jh + 3), beta * old.w);
                }
                *reinterpret_cast<float4*>(p) = o;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (c + j >= n) continue;
                    p[j] = (beta != 0.0f) ? fmaf(alpha, el(i, 4 * jh + j), beta * p[j]) : alpha * el(i, 4 * jh + j);
                }
            }
        }
    }
}

template <int RM, int RN, int SK, int MINB>
cudaError_t run_sgemm(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int la,
                      const float* B, int64_t ldb, int lb, float beta, float* C, int64_t ldc, cudaStream_t st) {
    constexpr int BM = RM * 16, BN = RN * 16;
    dim3 grid(static_cast<unsigned>((n + BN - 1) / BN), static_cast<unsigned>((m + BM - 1) / BM));
    const int im = static_cast<int>(m), in = static_cast<int>(n), ik = static_cast<int>(k);
    // 16-byte loads need 16-byte aligned rows
    const int va = ((lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) ? 1 : 0;
    const int vb = ((ldb & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0) ? 1 : 0;
    if (la == 0 && lb == 0)
        k_sgemm<0, 0, RM, RN, SK, MINB><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    else if (la == 0)
        k_sgemm<0, 1, RM, RN, SK, MINB><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    else if (lb == 0)
        k_sgemm<1, 0, RM, RN, SK, MINB><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    else
        k_sgemm<1, 1, RM, RN, SK, MINB><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    return cudaGetLastError();
}

}  // namespace

// 128 x 128 tiles, 8 x 8 per thread, two blocks per SM (128 registers); K steps of 16, or of 8 for
// row-major A with row-major B, whose staging at 16 spills (140 bytes).  Measured at N = 8192 over
// the four layouts with packed FMAs (TFLOP/s): K steps of 16 53.1 / 60.3 / 60.6 / 61.5 (A, B
// row/row, row/col, col/row, col/col), of 8 57.4 / 59.8 / 61.4 / 57.5; with one FMA per instruction
// 51.7-54.4, and 128 x 256, 256 x 128 tiles or one block per SM were within 2 % of that.  All are
// bit-identical (the same FMA chain per element).
cudaError_t launch_sgemm(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int la,
                         const float* B, int64_t ldb, int lb, float beta, float* C, int64_t ldc, cudaStream_t st) {
    if (la == 0 && lb == 0) return run_sgemm<8, 8, 8, 2>(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, st);
    return run_sgemm<8, 8, 16, 2>(m, n, k, alpha, A, lda, la, B, ldb, lb, beta, C, ldc, st);
}

}  // namespace tcg
