// FP32 GEMM on the CUDA cores: the paper's "sgemm" comparison (Sec. VII-A:
// GEMM without tensor cores; Sec. VII-B: the refined tensor-core GEMM is
// weighed against it in time and error).  No tensor cores are involved.
//
// 128 x 128 output tile per block of 256 threads (two blocks per SM), each
// thread an 8 x 8 register block (rows ty*4 + {0..3} and 64 + ty*4 + {0..3},
// same for columns, ty, tx = thread / 16, thread % 16).  K advances 16 at a
// time through double-buffered shared memory, As[k][m] and Bs[k][n]; the next
// step's operands are loaded into registers while the current one is used.
// Interior tiles whose rows are 16-byte aligned load 16 bytes per access; the
// edge of the matrix and unaligned operands load element by element.
//
// Every output element is the FP32 FMA chain acc = fma(a_k, b_k, acc) over k
// in increasing order, then alpha * acc (+ beta * C).
#include "launch.h"

namespace tcg {
namespace {

constexpr int SB = 128;
constexpr int SK = 16;
constexpr int SP = SB + 4;  // shared row pitch: k-rows of the transposed operand land on different banks
constexpr int kThreads = 256;

// Staging of one operand's 16 x 128 slice of a K step: two 16-byte groups per thread.
//   "k-contiguous" operand (row-major A, column-major B: rows of K): thread t takes rows
//   t / 4 and t / 4 + 64, k-group t % 4 (4 elements), so four lanes read a row's 64 bytes
//   together; stored transposed into rows of pitch SP (at most two-way bank conflicts).
//   "mn-contiguous" operand (column-major A, row-major B: rows of M or N): thread t takes
//   k-row t / 32 and t / 32 + 8, elements 4 (t % 32) ... + 3, stored as they are.
template <bool KCONT>
struct Stage {
    float4 v[2];

    __device__ __forceinline__ void load(const float* __restrict__ X, int64_t ld, int rows, int k, int r0, int k0,
                                         bool fast, int tid) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            int r, kk;
            if (KCONT) {
                r = (tid >> 2) + 64 * h;
                kk = (tid & 3) * 4;
            } else {
                kk = (tid >> 5) + 8 * h;
                r = (tid & 31) * 4;
            }
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
        for (int h = 0; h < 2; ++h) {
            if (KCONT) {
                const int r = (tid >> 2) + 64 * h, kk = (tid & 3) * 4;
                S[kk + 0][r] = v[h].x;
                S[kk + 1][r] = v[h].y;
                S[kk + 2][r] = v[h].z;
                S[kk + 3][r] = v[h].w;
            } else {
                const int kk = (tid >> 5) + 8 * h, r = (tid & 31) * 4;
                *reinterpret_cast<float4*>(&S[kk][r]) = v[h];
            }
        }
    }
};

template <int LA, int LB>
__global__ void __launch_bounds__(kThreads, 2) k_sgemm(int m, int n, int k, float alpha, const float* __restrict__ A,
                                                       int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                       float beta, float* __restrict__ C, int64_t ldc, int vec_a,
                                                       int vec_b) {
    __shared__ __align__(16) float As[2][SK][SP];
    __shared__ __align__(16) float Bs[2][SK][SP];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * SB, n0 = blockIdx.x * SB;
    // A is k-contiguous when row-major (LA = 0), B when column-major (LB = 1)
    Stage<LA == 0> sa;
    Stage<LB == 1> sb;
    const bool full_m = m0 + SB <= m, full_n = n0 + SB <= n;
    auto load = [&](int k0) {
        const bool kfull = k0 + SK <= k;
        sa.load(A, lda, m, k, m0, k0, vec_a && full_m && kfull, tid);
        sb.load(B, ldb, n, k, n0, k0, vec_b && full_n && kfull, tid);
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

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
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (s + 1 < nk) {
            sa.store(As[buf ^ 1], tid);
            sb.store(Bs[buf ^ 1], tid);
        }
        __syncthreads();
    }

    const bool vec_c = (ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(C) & 15) == 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= m) continue;
#pragma unroll
        for (int jh = 0; jh < 2; ++jh) {
            const int c = n0 + jh * 64 + tx * 4;
            float* p = C + static_cast<int64_t>(r) * ldc + c;
            if (vec_c && c + 4 <= n) {
                float4 o = make_float4(alpha * acc[i][4 * jh + 0], alpha * acc[i][4 * jh + 1],
                                       alpha * acc[i][4 * jh + 2], alpha * acc[i][4 * jh + 3]);
                if (beta != 0.0f) {
                    const float4 old = *reinterpret_cast<const float4*>(p);
                    o.x = fmaf(alpha, acc[i][4 * jh + 0], beta * old.x);
                    o.y = fmaf(alpha, acc[i][4 * jh + 1], beta * old.y);
                    o.z = fmaf(alpha, acc[i][4 * jh + 2], beta * old.z);
                    o.w = fmaf(alpha, acc[i][4 * jh + 3], beta * old.w);
                }
                *reinterpret_cast<float4*>(p) = o;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if (c + j >= n) continue;
                    p[j] = (beta != 0.0f) ? fmaf(alpha, acc[i][4 * jh + j], beta * p[j]) : alpha * acc[i][4 * jh + j];
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_sgemm(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int la,
                         const float* B, int64_t ldb, int lb, float beta, float* C, int64_t ldc, cudaStream_t st) {
    dim3 grid(static_cast<unsigned>((n + SB - 1) / SB), static_cast<unsigned>((m + SB - 1) / SB));
    const int im = static_cast<int>(m), in = static_cast<int>(n), ik = static_cast<int>(k);
    // 16-byte loads need 16-byte aligned rows
    const int va = ((lda & 3) == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0) ? 1 : 0;
    const int vb = ((ldb & 3) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0) ? 1 : 0;
    if (la == 0 && lb == 0)
        k_sgemm<0, 0><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    else if (la == 0)
        k_sgemm<0, 1><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    else if (lb == 0)
        k_sgemm<1, 0><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    else
        k_sgemm<1, 1><<<grid, kThreads, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc, va, vb);
    return cudaGetLastError();
}

}  // namespace tcg
