// Input rounding and residual split (Sec. V; Sec. VI rounds A and B to half
// precision before the GEMM).
//
//   quantize: dst = RNE(src) to F16 / BF16, or RNE_satfinite(src * s) to E4M3
//             with s = 2^j the largest power of two with max|src| * s <= 448.
//   split:    hi = RNE16(x), lo = RNE16(x - hi) (the residual R of Sec. V,
//             stored in 16 bits as Eq. 1 / Eq. 2 multiply it on tensor cores);
//             the scaled variant rounds (x - hi) * 2^s instead (Ootomo and
//             Yokota, 2022), the BF16x3 variant adds a third BF16 piece
//             RNE16(x - hi - lo) (Henry, Tang and Heinecke, 2019).
//
// All of these are HBM-bound streams (4 bytes in, 1-4 bytes out per element):
// the row kernels move 8 elements per thread with 16-byte loads, the
// transposing kernels stage tiles of 64 source rows in shared memory so that
// the FP32 reads are coalesced and every thread writes one 16-byte chunk.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "launch.h"

namespace tcg {
namespace {

constexpr int kDtF16 = 0, kDtBF16 = 1, kDtE4M3 = 2;

// Exponent j of the E4M3 scale: the largest j with amax * 2^j <= 448, capped
// at 127; amax = 0 or non-finite gives 0.  With amax = m * 2^E, m in [0.5, 1):
// amax * 2^j <= 0.875 * 2^9  <=>  E + j <= 9 (m <= 0.875) or E + j <= 8.
__device__ __forceinline__ int e4m3_scale_exp(float amax) {
    if (!(amax > 0.0f) || !isfinite(amax)) return 0;
    int E;
    const float m = frexpf(amax, &E);
    const int j = (m <= 0.875f) ? (9 - E) : (8 - E);
    return j > 127 ? 127 : j;
}

__device__ __forceinline__ float e4m3_scale_from_amax_word(const float* scale_word) {
    const float amax = __uint_as_float(*reinterpret_cast<const volatile unsigned*>(scale_word));
    return ldexpf(1.0f, e4m3_scale_exp(amax));
}

template <int DT>
struct Narrow;
template <>
struct Narrow<kDtF16> {
    using T = unsigned short;
    __device__ static T cvt(float x, float) { return __half_as_ushort(__float2half_rn(x)); }
};
template <>
struct Narrow<kDtBF16> {
    using T = unsigned short;
    __device__ static T cvt(float x, float) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
};
template <>
struct Narrow<kDtE4M3> {
    using T = unsigned char;
    __device__ static T cvt(float x, float s) {
        return static_cast<T>(__nv_cvt_float_to_fp8(x * s, __NV_SATFINITE, __NV_E4M3));
    }
};

// max |x| over a rows x cols matrix into the word at scale_word (as FP32 bits;
// non-negative floats order like their bit patterns).  Grid: x over column
// chunks of 4 * blockDim.x, y over rows (grid-stride); no divisions per element.
__global__ void __launch_bounds__(256) k_absmax(int64_t rows, int64_t cols, const float* __restrict__ src, int64_t ld,
                                                float* scale_word, int vec4) {
    float m = 0.0f;
    const int64_t chunk = 4 * (int64_t)blockDim.x;
    for (int64_t r = blockIdx.y; r < rows; r += gridDim.y) {
        const float* row = src + r * ld;
        for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < cols; c0 += (int64_t)gridDim.x * chunk) {
            const int64_t c = c0 + 4 * (int64_t)threadIdx.x;
            if (vec4 && c + 3 < cols) {
                const float4 v = __ldcs(reinterpret_cast<const float4*>(row + c));
                m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            } else {
                for (int j = 0; j < 4; ++j)
                    if (c + j < cols) m = fmaxf(m, fabsf(row[c + j]));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        m = (threadIdx.x < (blockDim.x >> 5)) ? wmax[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned*>(scale_word), __float_as_uint(m));
    }
}

__global__ void k_e4m3_finalize(float* scale_word) {
    *scale_word = e4m3_scale_from_amax_word(scale_word);
}

__global__ void k_store_one(float* p) { *p = 1.0f; }

// 8 consecutive elements per thread; requires cols % 8 == 0 and 16-byte
// aligned rows of src and dst.
template <int DT>
__global__ void __launch_bounds__(256) k_quantize_vec8(int64_t rows, int64_t cols, const float* __restrict__ src,
                                                       int64_t ld_src, typename Narrow<DT>::T* __restrict__ dst,
                                                       int64_t ld_dst, const float* scale_word) {
    using T = typename Narrow<DT>::T;
    const float s = (DT == kDtE4M3) ? e4m3_scale_from_amax_word(scale_word) : 1.0f;
    const int64_t vpr = cols / 8;
    const int64_t total = rows * vpr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / vpr, c = (i - r * vpr) * 8;
        const float4* p = reinterpret_cast<const float4*>(src + r * ld_src + c);
        const float4 a = __ldcs(p), b = __ldcs(p + 1);
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        T o[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) o[j] = Narrow<DT>::cvt(v[j], s);
        if constexpr (sizeof(T) == 2) {
            uint4 w;
            w.x = o[0] | (uint32_t(o[1]) << 16);
            w.y = o[2] | (uint32_t(o[3]) << 16);
            w.z = o[4] | (uint32_t(o[5]) << 16);
            w.w = o[6] | (uint32_t(o[7]) << 16);
            *reinterpret_cast<uint4*>(dst + r * ld_dst + c) = w;
        } else {
            uint2 w;
            w.x = o[0] | (uint32_t(o[1]) << 8) | (uint32_t(o[2]) << 16) | (uint32_t(o[3]) << 24);
            w.y = o[4] | (uint32_t(o[5]) << 8) | (uint32_t(o[6]) << 16) | (uint32_t(o[7]) << 24);
            *reinterpret_cast<uint2*>(dst + r * ld_dst + c) = w;
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(256) k_quantize_scalar(int64_t rows, int64_t cols, const float* __restrict__ src,
                                                         int64_t ld_src, typename Narrow<DT>::T* __restrict__ dst,
                                                         int64_t ld_dst, const float* scale_word) {
    const float s = (DT == kDtE4M3) ? e4m3_scale_from_amax_word(scale_word) : 1.0f;
    const int64_t total = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i - r * cols;
        dst[r * ld_dst + c] = Narrow<DT>::cvt(src[r * ld_src + c], s);
    }
}

// dst[c * ld_dst + r] = cvt(src[r * ld_src + c]).  One tile of 64 source rows x
// TC source columns per block of 256 threads: the FP32 tile is read along its
// rows (coalesced) into shared memory, then every thread converts
// 16 / sizeof(T) consecutive source rows of one source column and writes them
// as one 16-byte chunk of a destination row (TC = 32 for 2-byte outputs, 64 for
// 1-byte outputs, so the tile's chunks are exactly the block's 256 threads).
// The aligned path needs ld_dst * sizeof(T) and dst to be 16-byte aligned.
// Load a TR x TC tile of the FP32 source (rows r0.., columns c0..) into shared memory, zero
// outside the matrix; all loads are issued before any is stored.  vec4: every source row
// starts on 16 bytes, so a thread loads 4 consecutive columns at once (fewer, wider loads).
template <int TR, int TC>
__device__ __forceinline__ void load_tile_t(float (&tile)[TR][TC + 1], const float* __restrict__ src, int64_t rows,
                                            int64_t cols, int64_t ld_src, int64_t r0, int64_t c0, int vec4) {
    const int t = threadIdx.x;
    if (vec4) {
        constexpr int C4 = TC / 4;
        constexpr int NL4 = TR * C4 / 256;
        float4 v[NL4];
#pragma unroll
        for (int q = 0; q < NL4; ++q) {
            const int i = t + q * 256;
            const int rr = i / C4, c4 = i - rr * C4;
            const int64_t r = r0 + rr, c = c0 + 4 * c4;
            if (r < rows && c + 3 < cols) {
                v[q] = __ldcs(reinterpret_cast<const float4*>(src + r * ld_src + c));
            } else {
                const float* p = src + r * ld_src + c;
                v[q].x = (r < rows && c + 0 < cols) ? __ldcs(p + 0) : 0.0f;
                v[q].y = (r < rows && c + 1 < cols) ? __ldcs(p + 1) : 0.0f;
                v[q].z = (r < rows && c + 2 < cols) ? __ldcs(p + 2) : 0.0f;
                v[q].w = (r < rows && c + 3 < cols) ? __ldcs(p + 3) : 0.0f;
            }
        }
#pragma unroll
        for (int q = 0; q < NL4; ++q) {
            const int i = t + q * 256;
            const int rr = i / C4, c4 = i - rr * C4;
            tile[rr][4 * c4 + 0] = v[q].x;
            tile[rr][4 * c4 + 1] = v[q].y;
            tile[rr][4 * c4 + 2] = v[q].z;
            tile[rr][4 * c4 + 3] = v[q].w;
        }
    } else {
        constexpr int NL = TR * TC / 256;
        float v[NL];
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int i = t + q * 256;
            const int rr = i / TC, cc = i - rr * TC;
            const int64_t r = r0 + rr, c = c0 + cc;
            v[q] = (r < rows && c < cols) ? __ldcs(src + r * ld_src + c) : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < NL; ++q) {
            const int i = t + q * 256;
            tile[i / TC][i % TC] = v[q];
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(256) k_quantize_transpose(int64_t rows, int64_t cols, const float* __restrict__ src,
                                                            int64_t ld_src, typename Narrow<DT>::T* __restrict__ dst,
                                                            int64_t ld_dst, const float* scale_word, int aligned,
                                                            int vec4) {
    using T = typename Narrow<DT>::T;
    constexpr int TR = 64;
    constexpr int PER = 16 / sizeof(T);          // source rows per output chunk
    constexpr int TC = 256 * PER / TR;           // source columns per tile
    __shared__ float tile[TR][TC + 1];
    const float s = (DT == kDtE4M3) ? e4m3_scale_from_amax_word(scale_word) : 1.0f;
    const int64_t r0 = (int64_t)blockIdx.y * TR, c0 = (int64_t)blockIdx.x * TC;
    const int t = threadIdx.x;
    // load: TR x TC floats, coalesced along the source row
    load_tile_t<TR, TC>(tile, src, rows, cols, ld_src, r0, c0, vec4);
    __syncthreads();
    const int cc = t / (TR / PER);               // destination row within the tile
    const int j = t - cc * (TR / PER);           // chunk within the destination row
    const int64_t c = c0 + cc;
    if (c >= cols) return;
    const int64_t rbase = r0 + j * PER;
    T o[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) o[q] = Narrow<DT>::cvt(tile[j * PER + q][cc], s);
    T* d = dst + c * ld_dst + rbase;
    if (aligned && rbase + PER <= rows) {
        uint4 w;
        uint32_t* wp = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t v = 0;
#pragma unroll
            for (int e = 0; e < 4 / (int)sizeof(T); ++e)
                v |= uint32_t(o[q * (4 / sizeof(T)) + e]) << (8 * sizeof(T) * e);
            wp[q] = v;
        }
        *reinterpret_cast<uint4*>(d) = w;
    } else {
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (rbase + q < rows) d[q] = o[q];
    }
}

// Split schemes: 0 = hi, lo (Eq. 1 / Eq. 2); 1 = hi, lo scaled by 2^s before
// rounding (s = 11 for FP16 pieces, 8 for BF16); 2 = three BF16 pieces.
constexpr int kSplitPlain = 0, kSplitScaled = 1, kSplitBf16x3 = 2;

template <int PIECE>
struct Piece16;
template <>
struct Piece16<kDtF16> {
    __device__ static unsigned short rn(float x) { return __half_as_ushort(__float2half_rn(x)); }
    __device__ static float back(unsigned short h) { return __half2float(__ushort_as_half(h)); }
    static constexpr float kScale = 2048.0f;  // 2^11
};
template <>
struct Piece16<kDtBF16> {
    __device__ static unsigned short rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    __device__ static float back(unsigned short h) { return __bfloat162float(__ushort_as_bfloat16(h)); }
    static constexpr float kScale = 256.0f;  // 2^8
};

template <int SCHEME>
constexpr int pieces_of() {
    return SCHEME == kSplitBf16x3 ? 3 : 2;
}

// x - p0 and (x - p0) - p1 are exact in FP32 (the residual of a rounding to a
// shorter significand is representable), and so is the scaling by 2^s.
template <int PIECE, int SCHEME>
__device__ __forceinline__ void split_one(float x, unsigned short (&o)[3]) {
    using P = Piece16<PIECE>;
    o[0] = P::rn(x);
    const float r = x - P::back(o[0]);
    if constexpr (SCHEME == kSplitPlain) {
        o[1] = P::rn(r);
    } else if constexpr (SCHEME == kSplitScaled) {
        o[1] = P::rn(r * P::kScale);
    } else {
        o[1] = P::rn(r);
        o[2] = P::rn(r - P::back(o[1]));
    }
}

struct SplitOut {
    unsigned short* p[3];
};

__device__ __forceinline__ uint4 pack8(const unsigned short* h) {
    uint4 w;
    w.x = h[0] | (uint32_t(h[1]) << 16);
    w.y = h[2] | (uint32_t(h[3]) << 16);
    w.z = h[4] | (uint32_t(h[5]) << 16);
    w.w = h[6] | (uint32_t(h[7]) << 16);
    return w;
}

template <int PIECE, int SCHEME>
__global__ void __launch_bounds__(256) k_split_vec8(int64_t rows, int64_t cols, const float* __restrict__ src,
                                                    int64_t ld_src, SplitOut out, int64_t ld_dst) {
    constexpr int NP = pieces_of<SCHEME>();
    const int64_t vpr = cols / 8;
    const int64_t total = rows * vpr;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / vpr, c = (i - r * vpr) * 8;
        const float4* p = reinterpret_cast<const float4*>(src + r * ld_src + c);
        const float4 a = __ldcs(p), b = __ldcs(p + 1);
        const float v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
        unsigned short o[3][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            unsigned short t[3];
            split_one<PIECE, SCHEME>(v[j], t);
#pragma unroll
            for (int q = 0; q < NP; ++q) o[q][j] = t[q];
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) *reinterpret_cast<uint4*>(out.p[q] + r * ld_dst + c) = pack8(o[q]);
    }
}

template <int PIECE, int SCHEME>
__global__ void __launch_bounds__(256) k_split_scalar(int64_t rows, int64_t cols, const float* __restrict__ src,
                                                      int64_t ld_src, SplitOut out, int64_t ld_dst) {
    constexpr int NP = pieces_of<SCHEME>();
    const int64_t total = rows * cols;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / cols, c = i - r * cols;
        unsigned short t[3];
        split_one<PIECE, SCHEME>(src[r * ld_src + c], t);
#pragma unroll
        for (int q = 0; q < NP; ++q) out.p[q][r * ld_dst + c] = t[q];
    }
}

template <int PIECE, int SCHEME>
__global__ void __launch_bounds__(256) k_split_transpose(int64_t rows, int64_t cols, const float* __restrict__ src,
                                                         int64_t ld_src, SplitOut out, int64_t ld_dst, int aligned,
                                                         int vec4) {
    constexpr int NP = pieces_of<SCHEME>();
    constexpr int TR = 64, PER = 8, TC = 32;
    __shared__ float tile[TR][TC + 1];
    const int64_t r0 = (int64_t)blockIdx.y * TR, c0 = (int64_t)blockIdx.x * TC;
    const int t = threadIdx.x;
    load_tile_t<TR, TC>(tile, src, rows, cols, ld_src, r0, c0, vec4);
    __syncthreads();
    const int cc = t / (TR / PER);
    const int j = t - cc * (TR / PER);
    const int64_t c = c0 + cc;
    if (c >= cols) return;
    const int64_t rbase = r0 + j * PER;
    unsigned short o[3][PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        unsigned short w[3];
        split_one<PIECE, SCHEME>(tile[j * PER + q][cc], w);
#pragma unroll
        for (int z = 0; z < NP; ++z) o[z][q] = w[z];
    }
    if (aligned && rbase + PER <= rows) {
#pragma unroll
        for (int z = 0; z < NP; ++z) *reinterpret_cast<uint4*>(out.p[z] + c * ld_dst + rbase) = pack8(o[z]);
    } else {
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (rbase + q < rows) {
#pragma unroll
                for (int z = 0; z < NP; ++z) out.p[z][c * ld_dst + rbase + q] = o[z][q];
            }
    }
}

// max |x| of every tile of a batch of E4M3 jobs into the job's amax word (FP32 bits; the words
// are uploaded as 0, and non-negative floats order like their bit patterns).  fmaxf drops NaN, as
// k_absmax does, so a job's scale is the one tc_quantize gives it.
__global__ void __launch_bounds__(256) k_absmax_jobs(QuantJobDev* __restrict__ jobs,
                                                     const QuantTileDev* __restrict__ tiles, int32_t ntiles) {
    constexpr int TC = 32;
    __shared__ float wmax[8];
    for (int32_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const QuantTileDev td = tiles[ti];
        const QuantJobDev J = jobs[td.job];
        float m = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = threadIdx.x + q * 256;
            const int rr = i / TC, cc = i - rr * TC;
            const int64_t r = td.r0 + rr, c = td.c0 + cc;
            if (r < J.rows && c < J.cols) m = fmaxf(m, fabsf(__ldg(J.src + r * J.ld_src + c)));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        __syncthreads();  // the previous tile's wmax readers are done
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x < 32) {
            m = threadIdx.x < 8 ? wmax[threadIdx.x] : 0.0f;
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (threadIdx.x == 0 && m > 0.0f) atomicMax(&jobs[td.job].amax, __float_as_uint(m));
        }
    }
}

// Many independent FP32 -> FP16/BF16/E4M3 conversions in one launch (a batch
// of small operands, where one launch per operand would cost more than the
// conversion).  The host cuts every job into 64 x 32 tiles of its source; a
// block converts one tile through shared memory and writes it either in the
// source's layout (rows of 32 elements, four chunks of 8 each) or transposed
// (rows of 64 elements, eight chunks each).  E4M3 jobs take the scale from
// the job's amax word (k_absmax_jobs ran before), and the job's first tile
// stores it.
template <int DT>
__global__ void __launch_bounds__(256) k_quantize_jobs(const QuantJobDev* __restrict__ jobs,
                                                       const QuantTileDev* __restrict__ tiles, int32_t ntiles) {
    using T = typename Narrow<DT>::T;
    constexpr int TR = 64, TC = 32;
    __shared__ float tile[TR][TC + 1];
    for (int32_t ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const QuantTileDev td = tiles[ti];
        const QuantJobDev J = jobs[td.job];
        float s = 1.0f;
        if constexpr (DT == kDtE4M3) {
            s = ldexpf(1.0f, e4m3_scale_exp(__uint_as_float(J.amax)));
            if (td.r0 == 0 && td.c0 == 0 && threadIdx.x == 0) *J.scale = s;
        }
        const float* __restrict__ src = J.src;
        T* __restrict__ dst = static_cast<T*>(J.dst);
        const int64_t r0 = td.r0, c0 = td.c0;
        const int t = threadIdx.x;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = t + q * 256;
            const int rr = i / TC, cc = i - rr * TC;
            const int64_t r = r0 + rr, c = c0 + cc;
            v[q] = (r < J.rows && c < J.cols) ? __ldcs(src + r * J.ld_src + c) : 0.0f;
        }
        __syncthreads();  // the previous tile's readers are done
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int i = t + q * 256;
            tile[i / TC][i % TC] = v[q];
        }
        __syncthreads();
        T o[8];
        T* d;
        int64_t avail;  // destination elements of this chunk inside the job
        if (J.transpose) {
            const int cc = t >> 3, j = t & 7;  // destination row c0 + cc, elements r0 + 8j ..
            const int64_t c = c0 + cc;
            avail = (c < J.cols) ? J.rows - (r0 + j * 8) : 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) o[q] = Narrow<DT>::cvt(tile[j * 8 + q][cc], s);
            d = dst + c * J.ld_dst + r0 + j * 8;
        } else {
            const int rr = t >> 2, q4 = t & 3;  // destination row r0 + rr, elements c0 + 8 q4 ..
            const int64_t r = r0 + rr;
            avail = (r < J.rows) ? J.cols - (c0 + q4 * 8) : 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) o[q] = Narrow<DT>::cvt(tile[rr][q4 * 8 + q], s);
            d = dst + r * J.ld_dst + c0 + q4 * 8;
        }
        if (avail >= 8 && J.vec) {
            if constexpr (sizeof(T) == 2) {
                uint4 w;
                w.x = o[0] | (uint32_t(o[1]) << 16);
                w.y = o[2] | (uint32_t(o[3]) << 16);
                w.z = o[4] | (uint32_t(o[5]) << 16);
                w.w = o[6] | (uint32_t(o[7]) << 16);
                *reinterpret_cast<uint4*>(d) = w;
            } else {
                uint2 w;
                w.x = o[0] | (uint32_t(o[1]) << 8) | (uint32_t(o[2]) << 16) | (uint32_t(o[3]) << 24);
                w.y = o[4] | (uint32_t(o[5]) << 8) | (uint32_t(o[6]) << 16) | (uint32_t(o[7]) << 24);
                *reinterpret_cast<uint2*>(d) = w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q < avail) d[q] = o[q];
        }
    }
}

__global__ void __launch_bounds__(256) k_scale_c(int64_t m, int64_t n, float beta, float* C, int64_t ldc) {
    const int64_t total = m * n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / n, c = i - r * n;
        float* p = C + r * ldc + c;
        *p = (beta == 0.0f) ? 0.0f : beta * *p;
    }
}

inline unsigned grid_for(int64_t work, int64_t per_block) {
    int64_t g = (work + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;  // grid-stride beyond this
    return static_cast<unsigned>(g);
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

template <int DT>
cudaError_t quantize_dt(int64_t rows, int64_t cols, const float* src, int64_t ld_src, void* dst, int64_t ld_dst,
                        bool transpose, const float* scale, cudaStream_t st) {
    using T = typename Narrow<DT>::T;
    T* d = static_cast<T*>(dst);
    if (transpose) {
        constexpr int TC = 256 * (16 / sizeof(T)) / 64;
        dim3 grid(static_cast<unsigned>((cols + TC - 1) / TC), static_cast<unsigned>((rows + 63) / 64));
        const int al = ((ld_dst * sizeof(T)) % 16 == 0) && aligned16(dst);
        const int v4 = (ld_src % 4 == 0) && aligned16(src);
        k_quantize_transpose<DT><<<grid, 256, 0, st>>>(rows, cols, src, ld_src, d, ld_dst, scale, al, v4);
    } else {
        const bool vec = (cols % 8 == 0) && (ld_src % 4 == 0) && ((ld_dst * sizeof(T)) % (8 * sizeof(T)) == 0) &&
                         aligned16(src) && ((reinterpret_cast<uintptr_t>(dst) % (8 * sizeof(T))) == 0);
        if (vec) {
            k_quantize_vec8<DT><<<grid_for(rows * (cols / 8), 256), 256, 0, st>>>(rows, cols, src, ld_src, d, ld_dst,
                                                                              scale);
        } else {
            k_quantize_scalar<DT><<<grid_for(rows * cols, 256), 256, 0, st>>>(rows, cols, src, ld_src, d, ld_dst,
                                                                           scale);
        }
    }
    return cudaGetLastError();
}

template <int PIECE, int SCHEME>
cudaError_t split_piece(int64_t rows, int64_t cols, const float* src, int64_t ld_src, bool transpose,
                        void* const* dst, int64_t ld_dst, cudaStream_t st) {
    constexpr int NP = pieces_of<SCHEME>();
    SplitOut out{};
    bool all_aligned = true;
    for (int q = 0; q < NP; ++q) {
        out.p[q] = static_cast<unsigned short*>(dst[q]);
        all_aligned = all_aligned && aligned16(dst[q]);
    }
    if (transpose) {
        dim3 grid(static_cast<unsigned>((cols + 31) / 32), static_cast<unsigned>((rows + 63) / 64));
        const int al = (ld_dst % 8 == 0) && all_aligned;
        const int v4 = (ld_src % 4 == 0) && aligned16(src);
        k_split_transpose<PIECE, SCHEME><<<grid, 256, 0, st>>>(rows, cols, src, ld_src, out, ld_dst, al, v4);
    } else {
        const bool vec = (cols % 8 == 0) && (ld_src % 4 == 0) && (ld_dst % 8 == 0) && aligned16(src) && all_aligned;
        if (vec)
            k_split_vec8<PIECE, SCHEME><<<grid_for(rows * (cols / 8), 256), 256, 0, st>>>(rows, cols, src, ld_src, out,
                                                                                       ld_dst);
        else
            k_split_scalar<PIECE, SCHEME><<<grid_for(rows * cols, 256), 256, 0, st>>>(rows, cols, src, ld_src, out,
                                                                                   ld_dst);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_quantize(int dt, int64_t rows, int64_t cols, const float* src, int64_t ld_src, void* dst,
                            int64_t ld_dst, bool transpose, float* scale, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (dt == kDtE4M3) {
        e = cudaMemsetAsync(scale, 0, sizeof(float), st);
        if (e != cudaSuccess) return e;
        if (rows > 0 && cols > 0) {
            const int64_t xblocks = (cols + 1023) / 1024;
            const unsigned gx = static_cast<unsigned>(xblocks < 64 ? xblocks : 64);
            const int64_t want_y = (152 * 16 + gx - 1) / gx;
            const unsigned gy = static_cast<unsigned>(rows < want_y ? rows : (want_y < 65535 ? want_y : 65535));
            const int v4 = (ld_src % 4 == 0) && aligned16(src);
            k_absmax<<<dim3(gx, gy), 256, 0, st>>>(rows, cols, src, ld_src, scale, v4);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if ((e = quantize_dt<kDtE4M3>(rows, cols, src, ld_src, dst, ld_dst, transpose, scale, st)) != cudaSuccess)
                return e;
        }
        k_e4m3_finalize<<<1, 1, 0, st>>>(scale);
        return cudaGetLastError();
    }
    if (rows > 0 && cols > 0) {
        e = (dt == kDtF16) ? quantize_dt<kDtF16>(rows, cols, src, ld_src, dst, ld_dst, transpose, nullptr, st)
                           : quantize_dt<kDtBF16>(rows, cols, src, ld_src, dst, ld_dst, transpose, nullptr, st);
        if (e != cudaSuccess) return e;
    }
    if (scale) {
        k_store_one<<<1, 1, 0, st>>>(scale);
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_split(int scheme, int piece, int64_t rows, int64_t cols, const float* src, int64_t ld_src,
                         bool transpose, void* const* dst, int64_t ld_dst, cudaStream_t st) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    if (scheme == kSplitBf16x3)
        return split_piece<kDtBF16, kSplitBf16x3>(rows, cols, src, ld_src, transpose, dst, ld_dst, st);
    if (scheme == kSplitScaled)
        return piece == kDtF16 ? split_piece<kDtF16, kSplitScaled>(rows, cols, src, ld_src, transpose, dst, ld_dst, st)
                               : split_piece<kDtBF16, kSplitScaled>(rows, cols, src, ld_src, transpose, dst, ld_dst, st);
    return piece == kDtF16 ? split_piece<kDtF16, kSplitPlain>(rows, cols, src, ld_src, transpose, dst, ld_dst, st)
                           : split_piece<kDtBF16, kSplitPlain>(rows, cols, src, ld_src, transpose, dst, ld_dst, st);
}

cudaError_t launch_quantize_jobs(int dt, QuantJobDev* jobs, const QuantTileDev* tiles, int32_t ntiles,
                                 cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    const unsigned grid = static_cast<unsigned>(ntiles < 152 * 16 ? ntiles : 152 * 16);
    if (dt == kDtF16) {
        k_quantize_jobs<kDtF16><<<grid, 256, 0, st>>>(jobs, tiles, ntiles);
    } else if (dt == kDtBF16) {
        k_quantize_jobs<kDtBF16><<<grid, 256, 0, st>>>(jobs, tiles, ntiles);
    } else {
        k_absmax_jobs<<<grid, 256, 0, st>>>(jobs, tiles, ntiles);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_quantize_jobs<kDtE4M3><<<grid, 256, 0, st>>>(jobs, tiles, ntiles);
    }
    return cudaGetLastError();
}

cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t st) {
    if (m == 0 || n == 0) return cudaSuccess;
    k_scale_c<<<grid_for(m * n, 256), 256, 0, st>>>(m, n, beta, C, ldc);
    return cudaGetLastError();
}

}  // namespace tcg
