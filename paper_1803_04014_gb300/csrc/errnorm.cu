// FP64 error reduction (Sec. VI: e = C_half - C_single and its max norm; the
// normwise error ||C - C64||_F / (||A||_F ||B||_F) against an FP64 truth).
//
// The only FP64 arithmetic on the GPU.  Two passes with a fixed grid of
// kErrBlocks blocks: each block reduces a fixed strided subset of the
// elements into partial sums, then one block adds the partials in a fixed
// tree order, so the result is bit-for-bit repeatable and independent of the
// GPU's SM count.  Memory-bound: 4 + 8 bytes read per element of C.
#include "launch.h"

namespace tcg {
namespace {

constexpr int kErrThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    }
    return s;  // valid in thread 0
}

__device__ __forceinline__ double block_max(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        s = (l < (int)(blockDim.x >> 5)) ? red[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
    }
    return s;
}

// Fixed assignment of a rows x cols matrix to the kErrBlocks x kErrThreads
// threads: thread (b, t) visits rows b, b + kErrBlocks, ... and in each row the
// columns t, t + kErrThreads, ...  No division per element, coalesced rows, and
// the same order on every GPU.
template <typename F>
__device__ __forceinline__ void for_each_mine(int64_t rows, int64_t cols, F&& f) {
    for (int64_t r = blockIdx.x; r < rows; r += kErrBlocks)
        for (int64_t c = threadIdx.x; c < cols; c += kErrThreads) f(r, c);
}

// partial layout: [3][kErrBlocks][2] = (sum, max) for (C - ref), A, B
__global__ void __launch_bounds__(kErrThreads) k_err_partials(int64_t m, int64_t n, const float* __restrict__ C,
                                                              int64_t ldc, const void* __restrict__ ref, int64_t ldr,
                                                              int ref_f64, const float* __restrict__ A, int64_t ar,
                                                              int64_t ac, int64_t lda, const float* __restrict__ B,
                                                              int64_t br, int64_t bc, int64_t ldb,
                                                              double* __restrict__ partial) {
    __shared__ double red[32];
    double s = 0.0, mx = 0.0;
    if (ref_f64) {
        const double* R = static_cast<const double*>(ref);
        for_each_mine(m, n, [&](int64_t r, int64_t c) {
            const double d = static_cast<double>(C[r * ldc + c]) - R[r * ldr + c];
            s += d * d;
            mx = fmax(mx, fabs(d));
        });
    } else {
        const float* R = static_cast<const float*>(ref);
        for_each_mine(m, n, [&](int64_t r, int64_t c) {
            const double d = static_cast<double>(C[r * ldc + c]) - static_cast<double>(R[r * ldr + c]);
            s += d * d;
            mx = fmax(mx, fabs(d));
        });
    }
    double bs = block_sum(s, red);
    double bm = block_max(mx, red);
    if (threadIdx.x == 0) {
        partial[(0 * kErrBlocks + blockIdx.x) * 2 + 0] = bs;
        partial[(0 * kErrBlocks + blockIdx.x) * 2 + 1] = bm;
    }

    const float* mats[2] = {A, B};
    const int64_t rows[2] = {ar, br}, cols[2] = {ac, bc}, lds[2] = {lda, ldb};
#pragma unroll
    for (int w = 0; w < 2; ++w) {
        double t = 0.0;
        if (mats[w] != nullptr) {
            const float* X = mats[w];
            const int64_t ld = lds[w];
            for_each_mine(rows[w], cols[w], [&](int64_t r, int64_t c) {
                const double x = static_cast<double>(X[r * ld + c]);
                t += x * x;
            });
        }
        const double bt = block_sum(t, red);
        if (threadIdx.x == 0) {
            partial[((1 + w) * kErrBlocks + blockIdx.x) * 2 + 0] = bt;
            partial[((1 + w) * kErrBlocks + blockIdx.x) * 2 + 1] = 0.0;
        }
    }
}

__global__ void __launch_bounds__(kErrBlocks) k_err_final(const double* __restrict__ partial, double* out4) {
    __shared__ double red[32];
    const int t = threadIdx.x;
    double v[3], mx;
#pragma unroll
    for (int w = 0; w < 3; ++w) v[w] = partial[(w * kErrBlocks + t) * 2 + 0];
    mx = partial[(0 * kErrBlocks + t) * 2 + 1];
    double r[3];
#pragma unroll
    for (int w = 0; w < 3; ++w) r[w] = block_sum(v[w], red);
    const double rm = block_max(mx, red);
    if (t == 0) {
        out4[0] = r[0];
        out4[1] = r[1];
        out4[2] = r[2];
        out4[3] = rm;
    }
}

}  // namespace

cudaError_t launch_error_norm(int64_t m, int64_t n, const float* C, int64_t ldc, const void* ref, int64_t ldr,
                              bool ref_f64, const float* A, int64_t ar, int64_t ac, int64_t lda, const float* B,
                              int64_t br, int64_t bc, int64_t ldb, double* partial, double* out4_dev,
                              cudaStream_t st) {
    k_err_partials<<<kErrBlocks, kErrThreads, 0, st>>>(m, n, C, ldc, ref, ldr, ref_f64 ? 1 : 0, A, ar, ac, lda, B, br,
                                                       bc, ldb, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_err_final<<<1, kErrBlocks, 0, st>>>(partial, out4_dev);
    return cudaGetLastError();
}

}  // namespace tcg
