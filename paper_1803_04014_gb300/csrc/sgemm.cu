// FP32 GEMM on the CUDA cores: the paper's "sgemm" comparison (Sec. VII-A:
// GEMM without tensor cores; Sec. VII-B: the refined tensor-core GEMM is
// weighed against it in time and error).  No tensor cores are involved.
//
// 128 x 128 output tile per block of 256 threads, each thread an 8 x 8
// register block (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, same for
// columns), K in steps of 8 through double-buffered shared memory; the next
// step's operands are loaded into registers while the current one is used.
#include "launch.h"

namespace tcg {
namespace {

constexpr int SB = 128;
constexpr int SK = 8;

template <int LA, int LB>
__global__ void __launch_bounds__(256) k_sgemm(int m, int n, int k, float alpha, const float* __restrict__ A,
                                               int64_t lda, const float* __restrict__ B, int64_t ldb, float beta,
                                               float* __restrict__ C, int64_t ldc) {
    __shared__ __align__(16) float As[2][SK][SB];
    __shared__ __align__(16) float Bs[2][SK][SB];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * SB, n0 = blockIdx.x * SB;

    // Each thread loads 4 elements of A (128 x 8) and 4 of B (8 x 128) per step.
    float ra[4], rb[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int mm, kk;
            if (LA == 0) { mm = tid >> 1; kk = (tid & 1) * 4 + i; }   // row-major: 4 consecutive k
            else { kk = tid >> 5; mm = (tid & 31) * 4 + i; }           // col-major: 4 consecutive m
            const int gm = m0 + mm, gk = k0 + kk;
            ra[i] = (gm < m && gk < k) ? (LA == 0 ? A[(int64_t)gm * lda + gk] : A[(int64_t)gk * lda + gm]) : 0.0f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int nn, kk;
            if (LB == 0) { kk = tid >> 5; nn = (tid & 31) * 4 + i; }   // row-major: 4 consecutive n
            else { nn = tid >> 1; kk = (tid & 1) * 4 + i; }           // col-major: 4 consecutive k
            const int gn = n0 + nn, gk = k0 + kk;
            rb[i] = (gn < n && gk < k) ? (LB == 0 ? B[(int64_t)gk * ldb + gn] : B[(int64_t)gn * ldb + gk]) : 0.0f;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (LA == 0) As[buf][(tid & 1) * 4 + i][tid >> 1] = ra[i];
            else As[buf][tid >> 5][(tid & 31) * 4 + i] = ra[i];
            if (LB == 0) Bs[buf][tid >> 5][(tid & 31) * 4 + i] = rb[i];
            else Bs[buf][(tid & 1) * 4 + i][tid >> 1] = rb[i];
        }
    };

    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    const int nk = (k + SK - 1) / SK;
    load(0);
    store(0);
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
        if (s + 1 < nk) store(buf ^ 1);
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int c = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
            if (c >= n) continue;
            float* p = C + (int64_t)r * ldc + c;
            *p = (beta != 0.0f) ? fmaf(alpha, acc[i][j], beta * *p) : alpha * acc[i][j];
        }
    }
}

}  // namespace

cudaError_t launch_sgemm(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int la,
                         const float* B, int64_t ldb, int lb, float beta, float* C, int64_t ldc, cudaStream_t st) {
    dim3 grid(static_cast<unsigned>((n + SB - 1) / SB), static_cast<unsigned>((m + SB - 1) / SB));
    const int im = static_cast<int>(m), in = static_cast<int>(n), ik = static_cast<int>(k);
    if (la == 0 && lb == 0) k_sgemm<0, 0><<<grid, 256, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (la == 0) k_sgemm<0, 1><<<grid, 256, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc);
    else if (lb == 0) k_sgemm<1, 0><<<grid, 256, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc);
    else k_sgemm<1, 1><<<grid, 256, 0, st>>>(im, in, ik, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

}  // namespace tcg
