// FP64 error reduction (Sec. VI: e = C_half - C_single and its max norm; the
// normwise error ||C - C64||_F / (||A||_F ||B||_F) against an FP64 truth).
//
// The only FP64 arithmetic on the GPU.  Two passes with a fixed grid of
// kErrBlocks blocks: each block reduces a fixed strided subset of the
// elements into partial sums, then one block adds the partials in a fixed
// tree order, so the result is bit-for-bit repeatable and independent of the
// GPU's SM count.  Memory-bound: 4 + 8 bytes read per element of C (FP64
// reference), 4 per element of A and B; streamed with 16-byte loads.
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
// column groups t, t + kErrThreads, ... of VEC consecutive elements, kUnroll
// groups per step so that several loads are in flight.  No division per
// element, coalesced rows, and the same order on every GPU.
constexpr int kUnroll = 4;

template <int VEC, typename F>
__device__ __forceinline__ void for_each_mine(int64_t rows, int64_t cols, F&& f) {
    const int64_t groups = cols / VEC;
    for (int64_t r = blockIdx.x; r < rows; r += kErrBlocks)
        for (int64_t g0 = threadIdx.x; g0 < groups; g0 += kErrThreads * kUnroll) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                const int64_t g = g0 + u * kErrThreads;
                if (g < groups) f(r, g * VEC);
            }
        }
}

// GB300 runs FP64 arithmetic at about 1/64 of the FP32 rate, so this kernel
// is bound by its FP64 instructions before HBM.  Two changes keep the results
// bit-identical while halving that count (the sums of squares of A and B then
// move to the FP32 pipe, above, which changes their last bits, not their
// accuracy): FP32 -> FP64 conversion of normal
// values by integer bit assembly (IEEE 754 binary32 -> binary64: same sign,
// exponent rebiased by 1023 - 127, significand shifted up by 29 bits), and
// the running max of |d| compared as integer bit patterns (the order of
// non-negative IEEE values is the order of their patterns).  The difference
// c - c64 of an FP64 reference is taken on integers where that is exact
// (abs_diff_bits, below), so what remains on the FP64 unit is, per group of 4
// elements of C and of 8 of A and of B, the two additions that merge the
// group's float-float sum of squares (FP32 pipe, below) into the FP64 sum.
// Launch bounds hold the kernel at 32 registers: 8 of the fixed grid's 1024
// blocks per SM, so the grid runs as one wave.
__device__ __forceinline__ double to_f64(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xFFu;
    const uint64_t sign = static_cast<uint64_t>(u & 0x80000000u) << 32;
    if (e != 0u && e != 0xFFu)
        return __longlong_as_double(static_cast<long long>(sign | (static_cast<uint64_t>(e + (1023u - 127u)) << 52) |
                                                           (static_cast<uint64_t>(u & 0x7FFFFFu) << 29)));
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double(static_cast<long long>(sign));  // signed zero
    return static_cast<double>(x);  // subnormal, infinity, NaN
}

__device__ __forceinline__ void acc_diff(double d, double& s, unsigned long long& mx_bits) {
    s = fma(d, d, s);
    const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(d)) & 0x7FFFFFFFFFFFFFFFull;
    mx_bits = a > mx_bits ? a : mx_bits;
}

// Sums of squares of FP32 values on the FP32 pipe.  Each square a*a is split
// exactly into p = RN(a*a) and e = a*a - p (a fused multiply-add), and the
// p are added with Knuth's error-free two-sum into (hi, lo): hi collects the
// rounded sums, lo their exact rounding errors and the e terms.  A group of
// 8 values costs two FP64 additions when it is merged into the FP64 sum,
// instead of 8 FP64 fused multiply-adds.  The group's only roundings are
// those of lo (|lo| <= 16 * 2^-24 of the group's sum), below 2^-40 of it in
// all.  Exactness needs every square and partial sum inside FP32's normal
// range: 2^-50 <= |a| < 2^60 (or a = 0); any other value (subnormal, huge,
// infinite, NaN) sends its group of 4 to the FP64 path.  The intrinsics keep
// the compiler from fusing the steps, which would break the two-sum.
__device__ __forceinline__ bool square_fits_f32(float a) {
    const uint32_t u = __float_as_uint(a);
    const uint32_t eb = (u >> 23) & 0xFFu;
    return (u & 0x7FFFFFFFu) == 0u || (eb >= 127u - 50u && eb <= 127u + 59u);
}

__device__ __forceinline__ void add_square_ff(float a, float& hi, float& lo) {
    const float p = __fmul_rn(a, a);
    const float e = __fmaf_rn(a, a, -p);              // a*a - p, exact
    const float s = __fadd_rn(hi, p);
    const float bv = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bv)), __fsub_rn(p, bv));   // hi + p - s, exact
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
}

// The square of a difference d = c - c64 (an FP64 value) on the FP32 pipe: d
// splits exactly into hi, its leading 24 significand bits (an FP32 value
// made by integer bit assembly), and the remaining 29 bits, rounded once to
// FP32 as lo (|lo| < 2^-23 |hi|, error below 2^-47 |d|).  hi*hi goes into
// the float-float sum exactly (add_square_ff) and 2*hi*lo is added to its
// low part; lo*lo (below 2^-46 d^2) is dropped.  Needs 2^-50 <= |d| < 2^60;
// false (nothing added) for any other d, which the caller sums in FP64.
__device__ __forceinline__ bool add_diff_square_ff(double d, float& hi_sum, float& lo_sum) {
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(d)) & 0x7FFFFFFFFFFFFFFFull;
    const uint32_t eb = static_cast<uint32_t>(bits >> 52);
    if (eb < 1023u - 50u || eb > 1023u + 59u) return false;
    const uint32_t fe = eb - 1023u + 127u;                                    // FP32 biased exponent of hi
    const float hi = __uint_as_float((fe << 23) | static_cast<uint32_t>((bits >> 29) & 0x7FFFFFu));
    const float scale = __uint_as_float((eb - 1075u + 127u) << 23);          // 2^(exponent of d - 52), normal
    const float lo = __fmul_rn(__uint2float_rn(static_cast<uint32_t>(bits & 0x1FFFFFFFull)), scale);
    add_square_ff(hi, hi_sum, lo_sum);
    lo_sum = __fadd_rn(lo_sum, __fmul_rn(__fadd_rn(hi, hi), lo));
    return true;
}

// The same split from the bit pattern of |d| (sign bit clear): hi*hi and 2*hi*lo into the float-float
// sum exactly as add_diff_square_ff does for d.  The caller has checked 2^-50 <= |d| < 2^60.
__device__ __forceinline__ void add_diff_square_ff_bits(unsigned long long bits, float& hi_sum, float& lo_sum) {
    const uint32_t eb = static_cast<uint32_t>(bits >> 52);
    const uint32_t fe = eb - 1023u + 127u;
    const float hi = __uint_as_float((fe << 23) | static_cast<uint32_t>((bits >> 29) & 0x7FFFFFu));
    const float scale = __uint_as_float((eb - 1075u + 127u) << 23);
    const float lo = __fmul_rn(__uint2float_rn(static_cast<uint32_t>(bits & 0x1FFFFFFFull)), scale);
    add_square_ff(hi, hi_sum, lo_sum);
    lo_sum = __fadd_rn(lo_sum, __fmul_rn(__fadd_rn(hi, hi), lo));
}

// |c - r| for an FP32 c and an FP64 r without FP64 arithmetic (the FP64 unit is the scarce one):
// the two significands, aligned to the smaller exponent, are subtracted as 64-bit integers, which
// is exact; the result is the bit pattern of |c - r| when both are normal with the same sign and
// exponents at most 1 apart, the difference has at most 53 significant bits (so the FP64
// subtraction would have been exact and gives the same bits) and 2^-50 <= |c - r| < 2^60 or
// c == r.  Returns false otherwise; the caller then takes the FP64 path.
__device__ __forceinline__ bool abs_diff_bits(float c, double r, unsigned long long& out) {
    const uint32_t cu = __float_as_uint(c);
    const unsigned long long ru = static_cast<unsigned long long>(__double_as_longlong(r));
    const uint32_t ce = (cu >> 23) & 0xFFu;
    const uint32_t re = static_cast<uint32_t>(ru >> 52) & 0x7FFu;
    if (ce == 0u || ce == 0xFFu || re == 0u || re == 0x7FFu || (cu >> 31) != static_cast<uint32_t>(ru >> 63))
        return false;
    const int ec = static_cast<int>(ce) + (1023 - 127);   // c's exponent with the FP64 bias
    const int em = min(ec, static_cast<int>(re));
    if (ec - em > 1 || static_cast<int>(re) - em > 1) return false;
    const long long mc = static_cast<long long>((1ull << 52) | (static_cast<unsigned long long>(cu & 0x7FFFFFu) << 29))
                         << (ec - em);
    const long long mr = static_cast<long long>((1ull << 52) | (ru & 0xFFFFFFFFFFFFFull)) << (static_cast<int>(re) - em);
    const long long diff = mc - mr;   // |c - r| = |diff| * 2^(em - 1075), exactly
    if (diff == 0) {
        out = 0ull;
        return true;
    }
    const unsigned long long ad = static_cast<unsigned long long>(diff < 0 ? -diff : diff);
    const int p = 63 - __clzll(static_cast<long long>(ad));   // leading bit, at most 54
    if (p > 52) return false;
    const int e = p + em - 1075;                              // exponent of |c - r|
    if (e < -50 || e > 59) return false;
    out = (static_cast<unsigned long long>(e + 1023) << 52) | ((ad << (52 - p)) & 0xFFFFFFFFFFFFFull);
    return true;
}

// Four differences of C against an FP64 reference: the integer path for all four when each allows
// it (the same max and the same float-float terms as acc_diff4 below, bit for bit, with no FP64
// subtraction), else acc_diff4 on the FP64 differences.
__device__ __forceinline__ void acc_diff4_f64ref(float4 x, double2 y0, double2 y1, double& s,
                                                 unsigned long long& mx_bits);

// Four differences of C against its reference: the max norm on bit patterns, and
// their squares through the float-float path when all four allow it (two FP64
// additions for the four), else in FP64.
__device__ __forceinline__ void acc_diff4(double d0, double d1, double d2, double d3, double& s,
                                          unsigned long long& mx_bits) {
    const double d[4] = {d0, d1, d2, d3};
    bool fits = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const unsigned long long a = static_cast<unsigned long long>(__double_as_longlong(d[i])) & 0x7FFFFFFFFFFFFFFFull;
        mx_bits = a > mx_bits ? a : mx_bits;
        const uint32_t eb = static_cast<uint32_t>(a >> 52);
        fits = fits && (a == 0ull || (eb >= 1023u - 50u && eb <= 1023u + 59u));
    }
    if (fits) {
        float hi = 0.0f, lo = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) add_diff_square_ff(d[i], hi, lo);   // zeros add nothing
        s += to_f64(hi);
        s += to_f64(lo);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) s = fma(d[i], d[i], s);
    }
}

__device__ __forceinline__ void acc_diff4_f64ref(float4 x, double2 y0, double2 y1, double& s,
                                                 unsigned long long& mx_bits) {
    unsigned long long a0, a1, a2, a3;
    if (abs_diff_bits(x.x, y0.x, a0) && abs_diff_bits(x.y, y0.y, a1) && abs_diff_bits(x.z, y1.x, a2) &&
        abs_diff_bits(x.w, y1.y, a3)) {
        const unsigned long long a[4] = {a0, a1, a2, a3};
        float hi = 0.0f, lo = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            mx_bits = a[i] > mx_bits ? a[i] : mx_bits;
            if (a[i] != 0ull) add_diff_square_ff_bits(a[i], hi, lo);
        }
        s += to_f64(hi);
        s += to_f64(lo);
        return;
    }
    acc_diff4(to_f64(x.x) - y0.x, to_f64(x.y) - y0.y, to_f64(x.z) - y1.x, to_f64(x.w) - y1.y, s, mx_bits);
}

// partial layout: [3][kErrBlocks][2] = (sum, max) for (C - ref), A, B.
// vec: every row of C, ref, A and B starts on a 16-byte boundary and n, the
// column counts of A and B are multiples of 4 (4-wide loads); else scalar.
__global__ void __launch_bounds__(kErrThreads, 8) k_err_partials(int64_t m, int64_t n, const float* __restrict__ C,
                                                              int64_t ldc, const void* __restrict__ ref, int64_t ldr,
                                                              int ref_f64, const float* __restrict__ A, int64_t ar,
                                                              int64_t ac, int64_t lda, const float* __restrict__ B,
                                                              int64_t br, int64_t bc, int64_t ldb, int vec,
                                                              double* __restrict__ partial) {
    __shared__ double red[32];
    double s = 0.0;
    unsigned long long mx = 0ull;
    if (vec) {
        if (ref_f64) {
            const double* R = static_cast<const double*>(ref);
            for_each_mine<4>(m, n, [&](int64_t r, int64_t c) {
                const float4 x = __ldcs(reinterpret_cast<const float4*>(C + r * ldc + c));
                const double2 y0 = __ldcs(reinterpret_cast<const double2*>(R + r * ldr + c));
                const double2 y1 = __ldcs(reinterpret_cast<const double2*>(R + r * ldr + c + 2));
                acc_diff4_f64ref(x, y0, y1, s, mx);
            });
        } else {
            const float* R = static_cast<const float*>(ref);
            for_each_mine<4>(m, n, [&](int64_t r, int64_t c) {
                const float4 x = __ldcs(reinterpret_cast<const float4*>(C + r * ldc + c));
                const float4 y = __ldcs(reinterpret_cast<const float4*>(R + r * ldr + c));
                acc_diff4(to_f64(x.x) - to_f64(y.x), to_f64(x.y) - to_f64(y.y), to_f64(x.z) - to_f64(y.z),
                          to_f64(x.w) - to_f64(y.w), s, mx);
            });
        }
    } else if (ref_f64) {
        const double* R = static_cast<const double*>(ref);
        for_each_mine<1>(m, n, [&](int64_t r, int64_t c) {
            acc_diff(to_f64(C[r * ldc + c]) - R[r * ldr + c], s, mx);
        });
    } else {
        const float* R = static_cast<const float*>(ref);
        for_each_mine<1>(m, n, [&](int64_t r, int64_t c) {
            acc_diff(to_f64(C[r * ldc + c]) - to_f64(R[r * ldr + c]), s, mx);
        });
    }
    double bs = block_sum(s, red);
    double bm = block_max(__longlong_as_double(static_cast<long long>(mx)), red);
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
            if (vec) {
                float hi = 0.0f, lo = 0.0f;   // float-float sum of the current group
                int in_group = 0;             // groups of 4 values in it
                for_each_mine<4>(rows[w], cols[w], [&](int64_t r, int64_t c) {
                    const float4 x = __ldcs(reinterpret_cast<const float4*>(X + r * ld + c));
                    if (square_fits_f32(x.x) && square_fits_f32(x.y) && square_fits_f32(x.z) &&
                        square_fits_f32(x.w)) {
                        add_square_ff(x.x, hi, lo);
                        add_square_ff(x.y, hi, lo);
                        add_square_ff(x.z, hi, lo);
                        add_square_ff(x.w, hi, lo);
                        if (++in_group == 2) {   // 8 values: merge into the FP64 sum
                            t += to_f64(hi);
                            t += to_f64(lo);
                            hi = lo = 0.0f;
                            in_group = 0;
                        }
                    } else {
                        double v = to_f64(x.x);
                        t = fma(v, v, t);
                        v = to_f64(x.y);
                        t = fma(v, v, t);
                        v = to_f64(x.z);
                        t = fma(v, v, t);
                        v = to_f64(x.w);
                        t = fma(v, v, t);
                    }
                });
                t += to_f64(hi);
                t += to_f64(lo);
            } else {
                for_each_mine<1>(rows[w], cols[w], [&](int64_t r, int64_t c) {
                    const double x = to_f64(X[r * ld + c]);
                    t = fma(x, x, t);
                });
            }
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
    auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    const bool vec = (n % 4 == 0) && (ldc % 4 == 0) && al16(C) && al16(ref) &&
                     (ref_f64 ? (ldr % 2 == 0) : (ldr % 4 == 0)) &&
                     (A == nullptr || ((ac % 4 == 0) && (lda % 4 == 0) && al16(A))) &&
                     (B == nullptr || ((bc % 4 == 0) && (ldb % 4 == 0) && al16(B)));
    k_err_partials<<<kErrBlocks, kErrThreads, 0, st>>>(m, n, C, ldc, ref, ldr, ref_f64 ? 1 : 0, A, ar, ac, lda, B, br,
                                                       bc, ldb, vec ? 1 : 0, partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_err_final<<<1, kErrBlocks, 0, st>>>(partial, out4_dev);
    return cudaGetLastError();
}

}  // namespace tcg
