// Refined GEMM with the split formed on chip (Sec. V: R_A = A_single - A_half;
// Eq. 1 / Eq. 2: the products of the pieces summed into one FP32 result).
//
// The kernel reads the FP32 operands A and B directly.  For every k-block of
// 64 it forms their 16-bit pieces (hi = RN(x), lo = RN(x - hi); the scaled
// residual RN((x - hi) 2^s); or three BF16 pieces) in registers and writes them
// into shared memory in the 128-byte-swizzled layout that the tensor cores
// read, so a refined GEMM is a single launch that needs no workspace: the
// pieces never reach HBM.  The paper instead stores R_A and R_B in memory and
// chains four GEMMs (Sec. VI); the two-pass path of this library (a split
// pass, then the promoted pair kernel of gemm_tc.cu) is kept beside it.
//
// The CUDA cores form the pieces of the next k-blocks while the tensor cores
// multiply the current ones (Sec. VIII proposes running both kinds of core
// concurrently): the conversion is hidden behind the MMAs.
//
// CTA pairs (cluster of 2, tcgen05.mma.cta_group::2), 256 x 256 output tiles,
// persistent over tiles; 640 threads = five warpgroups:
//   warpgroup 0  warp 0 allocates TMEM and (even CTA, one thread) issues the
//                MMAs; warp 1 (one thread) streams FP32 tiles in by TMA
//   warpgroups 1, 2  eight epilogue warps: promote each chunk's partial sums
//                out of TMEM into FP32 registers with round-to-nearest (the
//                tensor cores' internal accumulation is not RN), store C
//   warpgroups 3, 4  eight warps forming the pieces
// The epilogue warps hold 128 FP32 sums each, so registers are rebalanced with
// setmaxnreg: warpgroup 0 and the piece warps drop to 48 per thread, the
// epilogue rises to 168 (384 x 48 + 256 x 168 = 640 x 96, the launch's registers).
//
// Data path of one k-block (64 of K) in each CTA: TMA copies its FP32 rows of
// A and B in two halves of 32 k (32 KB per half) into a three-slot ring,
// zero-filling outside the matrix; the piece warps read each half from shared
// memory, round it and store the 16-bit pieces into a two-slot ring of piece
// tiles.  A K-major piece tile is 128 rows of 128 bytes (64 k); an MN-major one
// (column-major A, row-major B) two 8 KB slabs of 64 k-rows x 64 elements,
// read by the MMA through the transpose bits of the instruction descriptor.
// After its stores each lane fences the generic-to-async proxy and one lane
// per warp arrives (release, cluster scope) on the even CTA's "full" barrier,
// which expects the 16 piece warps of both CTAs; the MMA thread waits on it
// with cluster-scope acquire.  Loading by TMA rather than per-thread loads
// matters: a thread's loads keep too few bytes in flight per SM to stream
// 64 KB per k-block at the tensor cores' pace.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "launch.h"
#include "pair_sched.cuh"
#include "tc_ptx.cuh"

namespace tcg {
namespace {

constexpr int kFusedThreads = 640;
constexpr int kPieceTile = 128 * 128;   // one piece tile: 128 rows x 128 bytes (or two 64 x 64 slabs)
constexpr int kXformWarps = 8;          // piece-forming warps per CTA
constexpr int kHalfBytes = 2 * 128 * 32 * 4;  // FP32 A and B rows of one CTA, 32 k: 32 KB
constexpr int kPStages = 2;             // piece slots
constexpr int kPrefetchHalves = 8;      // L2 prefetch distance of the FP32 halves (4 k-blocks)
constexpr uint32_t kCtlRegs = 48, kXformRegs = 48, kEpiRegs = 168;
static_assert(128 * kCtlRegs + 256 * kXformRegs + 256 * kEpiRegs <= kFusedThreads * 96,
              "register split of the fused kernel");

constexpr int kSchemePlain = 0, kSchemeScaled = 1, kSchemeBf16x3 = 2;

struct FusedArgs {
    int m, n, k;
    int num_kb, tiles_m, tiles_n, num_tiles, group_m;
    float alpha, beta, corr_scale;
    int a_mn, b_mn;  // 1: the operand is MN-major in memory (column-major A, row-major B)
    int bf16;        // pieces are BF16 (else FP16)
    float* C;
    int64_t ldc;
    int* status;
    uint32_t idesc;
    int stall_kb;  // test hook: >= 0 makes the even CTA of the first pair withhold this k-block
    int serpentine;  // odd rounds of tiles of a CTA pair walk K downwards (as the two-pass kernel)
    // work units (chunk_unit): tiles, then two parts of K of each tile of a cut last round; the
    // second part's epilogue warp waits for the first part's flag in kflags (8 per CTA and tile) to
    // hold ktoken
    int full_units, num_units, chunk_split;
    unsigned long long* kflags;
    unsigned long long ktoken;
};

template <int NA, int NB>
struct FusedLayout {
    static constexpr int kPStageBytes = (NA + NB) * kPieceTile;
    // FP32 half-k-block slots: as many as fit beside the piece ring (they set how far the loads
    // run ahead of the conversion)
    static constexpr int kFStages = NB == 1 ? 4 : 3;
    static constexpr int kFOffset = kPStages * kPStageBytes;           // FP32 ring after the piece ring
    static constexpr int kBarOffset = kFOffset + kFStages * kHalfBytes;
    // full[P], empty[P], ffull[F], fempty[F], cfull[2], cempty[2], drain
    static constexpr int kNumBars = 2 * kPStages + 2 * kFStages + 5;
    static constexpr int kSlotOffset = kBarOffset + 8 * kNumBars;
    static constexpr int kBytes = kSlotOffset + 16 + 1024;
    static constexpr int kTmemCols = 512;
};

__device__ __forceinline__ uint32_t pack_rn(float lo, float hi, bool bf16) {
    if (bf16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<const uint32_t*>(&h);
    }
    const __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float2 unpack(uint32_t w, bool bf16) {
    if (bf16) return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
}

// Pieces of four consecutive elements, two packed 16-bit values per word.
// x - p0 and (x - p0) - p1 are exact in FP32 (the residual of a rounding to a
// shorter significand is representable), and so is the scaling by 2^s.
template <int SCHEME>
__device__ __forceinline__ void split4(const float4 x, bool bf16, uint2 (&o)[3]) {
    o[0].x = pack_rn(x.x, x.y, bf16);
    o[0].y = pack_rn(x.z, x.w, bf16);
    const float2 b0 = unpack(o[0].x, bf16), b1 = unpack(o[0].y, bf16);
    float r0 = x.x - b0.x, r1 = x.y - b0.y, r2 = x.z - b1.x, r3 = x.w - b1.y;
    if constexpr (SCHEME == kSchemeScaled) {
        const float s = bf16 ? 256.0f : 2048.0f;  // 2^8, 2^11
        r0 *= s;
        r1 *= s;
        r2 *= s;
        r3 *= s;
    }
    o[1].x = pack_rn(r0, r1, bf16);
    o[1].y = pack_rn(r2, r3, bf16);
    if constexpr (SCHEME == kSchemeBf16x3) {
        const float2 c0 = unpack(o[1].x, true), c1 = unpack(o[1].y, true);
        o[2].x = pack_rn(r0 - c0.x, r1 - c0.y, true);
        o[2].y = pack_rn(r2 - c1.x, r3 - c1.y, true);
    }
}

__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint2 v) {
    asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(v.x), "r"(v.y) : "memory");
}

// FP32 ring slot of a half k-block: A rows at +0 (16 KB), B rows at +16 KB.
// A K-major operand half is one TMA box of 128 rows x 32 k (128-byte rows,
// swizzled); an MN-major one four boxes of 32 k-rows x 32 elements (4 KB each).
__device__ __forceinline__ void load_half(const CUtensorMap* map, bool mn, uint32_t dst, uint32_t bar, int row0, int k0) {
    if (!mn) {
        tma_load_3d(dst, map, bar, k0, row0, 0);
    } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) tma_load_3d(dst + b * 4096, map, bar, row0 + 32 * b, k0, 0);
    }
}

// L2 prefetch of the same half: lets the loads a few k-blocks later hit L2.
__device__ __forceinline__ void prefetch_half(const CUtensorMap* map, bool mn, int row0, int k0) {
    if (!mn) {
        tma_prefetch_3d(map, k0, row0, 0);
    } else {
#pragma unroll
        for (int b = 0; b < 4; ++b) tma_prefetch_3d(map, row0 + 32 * b, k0, 0);
    }
}

template <int OFF>
__device__ __forceinline__ float4 ld_shared_f4(uint32_t addr) {
    float4 x;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
                 : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w)
                 : "r"(addr), "n"(OFF)
                 : "memory");
    return x;
}

template <int OFF>
__device__ __forceinline__ void st_shared_v2_at(uint32_t addr, uint2 v) {
    asm volatile("st.shared.v2.u32 [%0+%1], {%2, %3};" ::"r"(addr), "n"(OFF), "r"(v.x), "r"(v.y) : "memory");
}

// Where lane `lane` of piece warp w reads and writes within one operand half
// (32 k) of an FP32 slot and the piece tiles.  Step `it` (0..3) of the lane
// adds 1024 bytes to both (eight rows further on); the lane's swizzle phase is
// the same at every step, so its offsets are a base plus a constant.
//   K-major operand (rows of k): step it covers row r = 32 (w >> 1) + 8 it +
//   rho, rho = 2 (w & 1) + 4 (g & 1) + (g >> 1), g = lane / 8, and 16-byte
//   chunk c = lane % 8 of the row (k = 4c ... 4c+3 of the half).  In the piece
//   tile those four k are 8 bytes of 16-byte chunk 4 kh + c / 2 of row r.
//   MN-major operand (k-rows of 32-element boxes): step it covers k-row
//   kk = 8 it + w of box g, chunk c; in the piece tile, slab g / 2, k-row
//   32 kh + kk, 16-byte chunk 4 (g & 1) + c / 2.
// Eight lanes (one g) read one whole 128-byte row of the swizzled FP32 tile
// and the two g of a half-warp write one whole 128-byte row of a piece tile:
// neither access has a bank conflict.
struct LaneOffsets {
    uint32_t src;  // FP32 half
    uint32_t dst;  // piece tile, kh = 0 (kh = 1: dst ^ 64 for K-major, dst + 4096 for MN-major)
};

template <bool MN>
__device__ __forceinline__ LaneOffsets lane_offsets(int w, int lane) {
    const int g = lane >> 3, c = lane & 7;
    LaneOffsets o;
    if (!MN) {
        const int rho = 2 * (w & 1) + 4 * (g & 1) + (g >> 1);
        const int r0 = 32 * (w >> 1) + rho;
        o.src = static_cast<uint32_t>(r0 * 128 + ((c ^ rho) << 4));
        o.dst = static_cast<uint32_t>(r0 * 128 + (((c >> 1) ^ rho) << 4) + (c & 1) * 8);
    } else {
        o.src = static_cast<uint32_t>(g * 4096 + w * 128 + ((c ^ w) << 4));
        const int ch = (g & 1) * 4 + (c >> 1);
        o.dst = static_cast<uint32_t>((g >> 1) * 8192 + w * 128 + ((ch ^ w) << 4) + (c & 1) * 8);
    }
    return o;
}

// Pieces of one operand half: four 16-byte shared loads first, so their
// latencies overlap, then the roundings and the 8-byte stores of every piece.
template <int SCHEME, int NPIECE, bool MN>
__device__ __forceinline__ void convert_half(uint32_t src_base, uint32_t dst_base, LaneOffsets o, int kh, bool bf16) {
    const uint32_t src = src_base + o.src;
    const uint32_t dst = dst_base + (MN ? o.dst + kh * 4096 : (o.dst ^ (kh << 6)));
    const float4 x0 = ld_shared_f4<0>(src), x1 = ld_shared_f4<1024>(src), x2 = ld_shared_f4<2048>(src),
                 x3 = ld_shared_f4<3072>(src);
    auto put = [&](const float4& x, auto off) {
        constexpr int OFF = decltype(off)::value;
        uint2 pc[3];
        split4<SCHEME>(x, bf16, pc);
        st_shared_v2_at<OFF>(dst, pc[0]);
        if constexpr (NPIECE > 1) st_shared_v2_at<OFF + kPieceTile>(dst, pc[1]);
        if constexpr (NPIECE > 2) st_shared_v2_at<OFF + 2 * kPieceTile>(dst, pc[2]);
    };
    put(x0, std::integral_constant<int, 0>{});
    put(x1, std::integral_constant<int, 1024>{});
    put(x2, std::integral_constant<int, 2048>{});
    put(x3, std::integral_constant<int, 3072>{});
}

// The piece warps' loop over this cluster's k-blocks.
template <int SCHEME, int NA, int NB, int STAGES, int FSTAGES, int PSTAGE_BYTES, int FOFFSET, bool A_MN, bool B_MN>
__device__ __forceinline__ void form_pieces(const FusedArgs& a, int xw, int lane, uint32_t rank, int cid, int ncl,
                                            uint32_t base, uint32_t bars, volatile int* abort_flag,
                                            uint32_t peer_abort, int64_t total_kb) {
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
    auto ffull_bar = [&](int s) { return bars + 8u * (2 * STAGES + s); };
    auto fempty_bar = [&](int s) { return bars + 8u * (2 * STAGES + FSTAGES + s); };
    auto wait = [&](uint32_t bar, uint32_t parity) {
        const bool ok = mbar_wait(bar, parity, abort_flag, a.status);
        if (!ok) st_shared_cluster_u32(peer_abort, 1u);
        return ok;
    };
    const bool bf16 = a.bf16 != 0;
    const LaneOffsets oa = lane_offsets<A_MN>(xw, lane);
    const LaneOffsets ob = lane_offsets<B_MN>(xw, lane);
    int ps = 0, fs = 0;
    uint32_t pph = 0, fph = 0;
    const uint32_t fbase = base + FOFFSET;
    for (int64_t done_kb = 0; done_kb < total_kb; ++done_kb) {
        if (!wait(empty_bar(ps), pph ^ 1u)) return;
        const uint32_t pbase = base + ps * PSTAGE_BYTES;
        for (int kh = 0; kh < 2; ++kh) {
            if (!wait(ffull_bar(fs), fph)) return;
            const uint32_t src = fbase + fs * kHalfBytes;
            convert_half<SCHEME, NA, A_MN>(src, pbase, oa, kh, bf16);
            convert_half<SCHEME, NB, B_MN>(src + kHalfBytes / 2, pbase + NA * kPieceTile, ob, kh, bf16);
            __syncwarp();
            if (lane == 0) mbar_arrive(fempty_bar(fs));
            if (++fs == FSTAGES) {
                fs = 0;
                fph ^= 1u;
            }
        }
        // the stage's stores become visible to the tensor cores' (async) proxy, then one arrival
        // per warp on the even CTA's full barrier
        fence_async_shared();
        __syncwarp();
        const bool withhold = a.stall_kb >= 0 && done_kb == a.stall_kb && cid == 0 && rank == 0 && xw == 0;
        if (lane == 0 && !withhold) mbar_arrive_cluster(mapa_shared(full_bar(ps), 0));
        if (++ps == STAGES) {
            ps = 0;
            pph ^= 1u;
        }
    }
}

template <int SCHEME, int NPROD, int CHUNK_KB>
__global__ void __launch_bounds__(kFusedThreads, 1)
    k_split_fused(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const FusedArgs a) {
    constexpr int NA = SCHEME == kSchemeBf16x3 ? 3 : 2;
    constexpr int NB = NPROD == 2 ? 1 : NA;
    constexpr bool SCALED = SCHEME != kSchemePlain;  // corrections in a second accumulator
    constexpr int STAGES = kPStages;
    using L = FusedLayout<NA, NB>;
    static_assert(L::kBytes <= 227 * 1024, "shared memory of the fused kernel");
    constexpr int kSteps = 4;  // MMA K = 16 elements per step, 64 per k-block
    constexpr int PM = 256, PN = 256;

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + L::kBarOffset;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
    auto ffull_bar = [&](int s) { return bars + 8u * (2 * STAGES + s); };
    auto fempty_bar = [&](int s) { return bars + 8u * (2 * STAGES + L::kFStages + s); };
    auto cfull_bar = [&](int i) { return bars + 8u * (2 * STAGES + 2 * L::kFStages + i); };
    auto cempty_bar = [&](int i) { return bars + 8u * (2 * STAGES + 2 * L::kFStages + 2 + i); };
    const uint32_t drain_bar = bars + 8u * (2 * STAGES + 2 * L::kFStages + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + L::kSlotOffset);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base_ptr + L::kSlotOffset + 4);
    const uint32_t abort_addr = base + L::kSlotOffset + 4;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const uint32_t peer_abort = mapa_shared(abort_addr, rank ^ 1u);
    const int cid = static_cast<int>(cluster_id_x());
    const int ncl = static_cast<int>(num_clusters_x());
    const int nchunks = (a.num_kb + CHUNK_KB - 1) / CHUNK_KB;

    auto wait = [&](uint32_t bar, uint32_t parity) {
        const bool ok = mbar_wait(bar, parity, abort_flag, a.status);
        if (!ok) st_shared_cluster_u32(peer_abort, 1u);
        return ok;
    };
    auto wait_full = [&](uint32_t bar, uint32_t parity) {
        const bool ok = mbar_wait_acq_cluster(bar, parity, abort_flag, a.status);
        if (!ok) st_shared_cluster_u32(peer_abort, 1u);
        return ok;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 2 * kXformWarps);  // the piece warps of both CTAs
            mbar_init(empty_bar(s), 1);
        }
        for (int s = 0; s < L::kFStages; ++s) {
            mbar_init(ffull_bar(s), 1);
            mbar_init(fempty_bar(s), kXformWarps);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(cfull_bar(i), 1);
            mbar_init(cempty_bar(i), 16);  // eight epilogue warps in each CTA
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 0) {
        tmem_alloc_pair(smem_addr(tmem_slot), L::kTmemCols);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the set-up above overlaps the previous kernel of the stream; operands and C only from here on
    griddep_wait();
    griddep_launch_dependents();

    const int wg = warp >> 2;
    if (wg == 1 || wg == 2) {
        setmaxnreg_inc<kEpiRegs>();
        // ---------------- epilogue: drain every chunk into FP32 registers, store at the end of the tile
        const int e = warp - 4;
        const int quarter = warp & 3;  // TMEM lanes [32*quarter, +32)
        const int half = e >> 2;       // columns [128*half, +128)
        const float alpha = a.alpha;
        const float beta_in = a.beta;
        const bool vec_ok = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15u) == 0);
        auto part_flag = [&](int u) {
            const int j = (u - a.full_units) >> 1;
            return a.kflags + (j * 2 + static_cast<int>(rank)) * 8 + e;
        };
        const uint32_t leader_cempty0 = mapa_shared(cempty_bar(0), 0);
        const uint32_t leader_cempty1 = mapa_shared(cempty_bar(1), 0);
        int buf = 0;
        uint32_t buf_phase = 0;
        for (int u = cid; u < a.num_units; u += ncl) {
            const ChunkUnit pu = chunk_unit(a.full_units, a.chunk_split, nchunks, u);
            int mb, nb;
            tile_coords(pu.t, a.tiles_m, a.tiles_n, a.group_m, mb, nb);
            // the second part of K adds its sum to what the first part's warp stored (beta = 1)
            const float beta = pu.kpart == 2 ? 1.0f : beta_in;
            const int row = mb * PM + static_cast<int>(rank) * 128 + quarter * 32 + lane;
            const int col0 = nb * PN + half * 128;
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.0f;
            bool ok = true;
            for (int c = pu.c0; c < pu.c1; ++c) {
                const int cb = SCALED ? 0 : buf;
                const bool w = wait(cfull_bar(cb), buf_phase);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                       static_cast<uint32_t>(cb * PN + half * 128);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float v[32];
                    tmem_load_32(taddr + q * 32, v);
#pragma unroll
                    for (int j = 0; j < 32; ++j) acc[q * 32 + j] += v[j];
                }
                if (SCALED && c == pu.c1 - 1) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float v[32];
                        tmem_load_32(taddr + PN + q * 32, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[q * 32 + j] = fmaf(v[j], a.corr_scale, acc[q * 32 + j]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(cb == 0 ? leader_cempty0 : leader_cempty1);
                if (SCALED) {
                    buf_phase ^= 1u;
                } else {
                    buf ^= 1;
                    if (buf == 0) buf_phase ^= 1u;
                }
            }
            if (!ok) break;
            if (pu.kpart == 2) {
                const bool fl = poll_flag_acquire(part_flag(u), a.ktoken, abort_flag, a.status);
                if (!fl) st_shared_cluster_u32(peer_abort, 1u);
                if (!__all_sync(0xffffffffu, fl)) break;
            }
            if (row < a.m && col0 < a.n) {
                float* p = a.C + static_cast<int64_t>(row) * a.ldc + col0;
                const int ncols = min(128, a.n - col0);
                if (ncols == 128 && vec_ok) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float4 o;
                        if (beta != 0.0f) {
                            const float4 old = __ldcg(reinterpret_cast<const float4*>(p + 4 * j));
                            o.x = fmaf(alpha, acc[4 * j + 0], beta * old.x);
                            o.y = fmaf(alpha, acc[4 * j + 1], beta * old.y);
                            o.z = fmaf(alpha, acc[4 * j + 2], beta * old.z);
                            o.w = fmaf(alpha, acc[4 * j + 3], beta * old.w);
                        } else {
                            o.x = alpha * acc[4 * j + 0];
                            o.y = alpha * acc[4 * j + 1];
                            o.z = alpha * acc[4 * j + 2];
                            o.w = alpha * acc[4 * j + 3];
                        }
                        *reinterpret_cast<float4*>(p + 4 * j) = o;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 128; ++j) {
                        if (j < ncols) p[j] = (beta != 0.0f) ? fmaf(alpha, acc[j], beta * __ldcg(p + j)) : alpha * acc[j];
                    }
                }
            }
            if (pu.kpart == 1) {   // this warp's stores are visible before its flag is raised
                __threadfence();
                __syncwarp();
                if (lane == 0) st_release_gpu(part_flag(u), a.ktoken);
            }
        }
    } else if (wg == 0) {
        setmaxnreg_dec<kCtlRegs>();
        if (warp == 0) {
            if (lane == 0 && rank == 0) {
                // ---------------- MMA issuer (even CTA only)
                const uint32_t idesc = a.idesc;
                auto adesc = [&](uint32_t sbase, int piece, int ks) -> uint64_t {
                    const uint32_t t = sbase + piece * kPieceTile;
                    return a.a_mn ? sw128_mnmajor_desc(t + ks * 2048, 8192, 1024) : sw128_kmajor_desc(t + ks * 32);
                };
                auto bdesc = [&](uint32_t sbase, int piece, int ks) -> uint64_t {
                    const uint32_t t = sbase + (NA + piece) * kPieceTile;
                    return a.b_mn ? sw128_mnmajor_desc(t + ks * 2048, 8192, 1024) : sw128_kmajor_desc(t + ks * 32);
                };
                auto advance = [&](int& s_, uint32_t& ph_) {
                    if (++s_ == STAGES) {
                        s_ = 0;
                        ph_ ^= 1u;
                    }
                };
                int stage = 0;
                uint32_t phase = 0;
                bool ok = true;
                bool issued_any = false;
                if constexpr (SCALED) {
                    // the corrections of the first kAhead k-blocks of a chunk are issued before the wait
                    // for H (the hi x hi chunk accumulator), so its drain overlaps them
                    constexpr int kAhead = (CHUNK_KB < STAGES - 1) ? CHUNK_KB : (STAGES - 1);
                    static_assert(kAhead >= 1, "SCALED needs at least two stages");
                    uint32_t h_phase = 0;
                    const uint32_t h_tmem = tmem_base;
                    const uint32_t y_tmem = tmem_base + static_cast<uint32_t>(PN);
                    int ukb0 = 0;  // first k-block of the unit: the correction accumulator restarts there
                    auto corrections = [&](int kb, int s_) {
                        const uint32_t sbase = base + s_ * L::kPStageBytes;
#pragma unroll
                        for (int ks = 0; ks < kSteps; ++ks) {
#pragma unroll
                            for (int p = 1; p < NPROD; ++p) {
                                const uint32_t accumulate = (kb != ukb0 || ks != 0 || p != 1) ? 1u : 0u;
                                mma_pair_f16(y_tmem, adesc(sbase, prod_a<NA>(p), ks), bdesc(sbase, prod_b<NA>(p), ks),
                                             idesc, accumulate);
                            }
                        }
                    };
                    auto hi_hi = [&](int kb, int kb0, int s_) {
                        const uint32_t sbase = base + s_ * L::kPStageBytes;
#pragma unroll
                        for (int ks = 0; ks < kSteps; ++ks) {
                            const uint32_t accumulate = (kb != kb0 || ks != 0) ? 1u : 0u;
                            mma_pair_f16(h_tmem, adesc(sbase, 0, ks), bdesc(sbase, 0, ks), idesc, accumulate);
                        }
                        mma_commit_pair_mc(empty_bar(s_), 0x3);
                    };
                    for (int u = cid; ok && u < a.num_units; u += ncl) {
                        const ChunkUnit w = chunk_unit(a.full_units, a.chunk_split, nchunks, u);
                        ukb0 = w.c0 * CHUNK_KB;
                        for (int c = w.c0; ok && c < w.c1; ++c) {
                            const int kb0 = c * CHUNK_KB;
                            const int kb_end = min(a.num_kb, kb0 + CHUNK_KB);
                            const int ahead = min(kb_end - kb0, kAhead);
                            if (c == w.c0) {
                                // Y restarts with this unit: the previous unit's Y and H must be drained
                                if (!wait(cempty_bar(0), h_phase ^ 1u)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                            }
                            int s2 = stage;
                            uint32_t ph2 = phase;
                            for (int kb = kb0; kb < kb0 + ahead; ++kb) {
                                if (!wait_full(full_bar(stage), phase)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                corrections(kb, stage);
                                issued_any = true;
                                advance(stage, phase);
                            }
                            if (!ok) break;
                            if (c != 0) {
                                if (!wait(cempty_bar(0), h_phase ^ 1u)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                            }
                            for (int kb = kb0; kb < kb0 + ahead; ++kb) {
                                hi_hi(kb, kb0, s2);
                                advance(s2, ph2);
                            }
                            for (int kb = kb0 + ahead; kb < kb_end; ++kb) {
                                if (!wait_full(full_bar(stage), phase)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                corrections(kb, stage);
                                hi_hi(kb, kb0, stage);
                                advance(stage, phase);
                            }
                            if (!ok) break;
                            mma_commit_pair_mc(cfull_bar(0), 0x3);
                            h_phase ^= 1u;
                        }
                    }
                } else {
                    int buf = 0;
                    uint32_t buf_phase = 0;
                    for (int u = cid; ok && u < a.num_units; u += ncl) {
                        const ChunkUnit w = chunk_unit(a.full_units, a.chunk_split, nchunks, u);
                        for (int c = w.c0; ok && c < w.c1; ++c) {
                            if (!wait(cempty_bar(buf), buf_phase ^ 1u)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(buf * PN);
                            const int kb_end = min(a.num_kb, (c + 1) * CHUNK_KB);
                            for (int kb = c * CHUNK_KB; kb < kb_end; ++kb) {
                                if (!wait_full(full_bar(stage), phase)) {
                                    ok = false;
                                    break;
                                }
                                tc_fence_after();
                                const uint32_t sbase = base + stage * L::kPStageBytes;
#pragma unroll
                                for (int ks = 0; ks < kSteps; ++ks) {
#pragma unroll
                                    for (int p = 0; p < NPROD; ++p) {
                                        const uint32_t accumulate =
                                            (kb != c * CHUNK_KB || ks != 0 || p != 0) ? 1u : 0u;
                                        mma_pair_f16(d_tmem, adesc(sbase, prod_a<NA>(p), ks),
                                                     bdesc(sbase, prod_b<NA>(p), ks), idesc, accumulate);
                                    }
                                }
                                issued_any = true;
                                mma_commit_pair_mc(empty_bar(stage), 0x3);
                                advance(stage, phase);
                            }
                            if (!ok) break;
                            mma_commit_pair_mc(cfull_bar(buf), 0x3);
                            buf ^= 1;
                            if (buf == 0) buf_phase ^= 1u;
                        }
                    }
                }
                if (!ok && issued_any) {
                    mma_commit_pair_mc(drain_bar, 0x1);
                    mbar_wait_bounded(drain_bar, 0, 100000000ull);
                }
            }
            __syncwarp();
        } else if (warp == 1) {
            if (lane == 0) {
                // ---------------- TMA producer (each CTA): its FP32 rows of A and B, half a k-block at a time
                int fs = 0;
                uint32_t fph = 0;
                int issued_phase[L::kFStages];
#pragma unroll
                for (int s = 0; s < L::kFStages; ++s) issued_phase[s] = -1;
                bool ok = true;
                const uint32_t fbase = base + L::kFOffset;
                // half i (0 <= i < 2 (kb1 - kb0)) of a unit with k-blocks [kb0, kb1) covers k from
                // 64 kb0 + 32 i, or, in the odd rounds of whole tiles that walk K downwards, half i % 2
                // of k-block kb1 - 1 - i / 2
                auto half_k = [&](const ChunkUnit& w_, int i, bool down) {
                    const int kb0 = w_.c0 * CHUNK_KB, kb1 = min(a.num_kb, w_.c1 * CHUNK_KB);
                    const int kb = down ? kb1 - 1 - (i >> 1) : kb0 + (i >> 1);
                    return 64 * kb + 32 * (i & 1);
                };
                auto unit_down = [&](const ChunkUnit& w_, int u_) {
                    return a.serpentine && w_.kpart == 0 && (((u_ - cid) / ncl) & 1);
                };
                for (int u = cid; ok && u < a.num_units; u += ncl) {
                    const ChunkUnit w = chunk_unit(a.full_units, a.chunk_split, nchunks, u);
                    int mb, nb;
                    tile_coords(w.t, a.tiles_m, a.tiles_n, a.group_m, mb, nb);
                    const bool down = unit_down(w, u);
                    const int nhalf = 2 * (min(a.num_kb, w.c1 * CHUNK_KB) - w.c0 * CHUNK_KB);
                    const int arow = mb * PM + static_cast<int>(rank) * 128;
                    const int brow = nb * PN + static_cast<int>(rank) * 128;
                    // the next unit of this cluster, whose first halves are prefetched near the end of this one
                    int mb2 = -1, nb2 = -1;
                    ChunkUnit w2{0, 0, 0, 0};
                    bool down2 = false;
                    if (u + ncl < a.num_units) {
                        w2 = chunk_unit(a.full_units, a.chunk_split, nchunks, u + ncl);
                        tile_coords(w2.t, a.tiles_m, a.tiles_n, a.group_m, mb2, nb2);
                        down2 = unit_down(w2, u + ncl);
                    }
                    for (int h = 0; h < nhalf; ++h) {
                        // L2 prefetch kPrefetchHalves ahead: the ring of three halves alone keeps too few
                        // bytes in flight to cover the latency of loads that miss L2
                        const int hp = h + kPrefetchHalves;
                        if (hp < nhalf) {
                            prefetch_half(&tmA, a.a_mn != 0, arow, half_k(w, hp, down));
                            prefetch_half(&tmB, a.b_mn != 0, brow, half_k(w, hp, down));
                        } else if (mb2 >= 0 && hp - nhalf < 2 * (min(a.num_kb, w2.c1 * CHUNK_KB) - w2.c0 * CHUNK_KB)) {
                            const int k2 = half_k(w2, hp - nhalf, down2);
                            prefetch_half(&tmA, a.a_mn != 0, mb2 * PM + static_cast<int>(rank) * 128, k2);
                            prefetch_half(&tmB, a.b_mn != 0, nb2 * PN + static_cast<int>(rank) * 128, k2);
                        }
                        if (!wait(fempty_bar(fs), fph ^ 1u)) {
                            ok = false;
                            break;
                        }
                        const uint32_t dst = fbase + fs * kHalfBytes;
                        mbar_arrive_expect_tx(ffull_bar(fs), kHalfBytes);
                        load_half(&tmA, a.a_mn != 0, dst, ffull_bar(fs), arow, half_k(w, h, down));
                        load_half(&tmB, a.b_mn != 0, dst + kHalfBytes / 2, ffull_bar(fs), brow, half_k(w, h, down));
                        issued_phase[fs] = static_cast<int>(fph);
                        if (++fs == L::kFStages) {
                            fs = 0;
                            fph ^= 1u;
                        }
                    }
                }
                if (!ok) {
                    // leaving early: let the copies already issued land before the CTA exits
                    for (int s = 0; s < L::kFStages; ++s)
                        if (issued_phase[s] >= 0)
                            mbar_wait_bounded(ffull_bar(s), static_cast<uint32_t>(issued_phase[s]), 100000000ull);
                }
            }
            __syncwarp();
        }
    } else {
        setmaxnreg_dec<kXformRegs>();
        // ---------------- piece formation (warps 12-19)
        const int xw = warp - 12;
        int64_t total_kb = 0;   // k-blocks of this cluster's units
        for (int u = cid; u < a.num_units; u += ncl) {
            const ChunkUnit w = chunk_unit(a.full_units, a.chunk_split, nchunks, u);
            total_kb += min(a.num_kb, w.c1 * CHUNK_KB) - w.c0 * CHUNK_KB;
        }
        constexpr int FS = L::kFStages, PB = L::kPStageBytes, FO = L::kFOffset;
        if (!a.a_mn && !a.b_mn)
            form_pieces<SCHEME, NA, NB, STAGES, FS, PB, FO, false, false>(a, xw, lane, rank, cid, ncl, base, bars,
                                                                         abort_flag, peer_abort, total_kb);
        else if (!a.a_mn && a.b_mn)
            form_pieces<SCHEME, NA, NB, STAGES, FS, PB, FO, false, true>(a, xw, lane, rank, cid, ncl, base, bars,
                                                                        abort_flag, peer_abort, total_kb);
        else if (a.a_mn && !a.b_mn)
            form_pieces<SCHEME, NA, NB, STAGES, FS, PB, FO, true, false>(a, xw, lane, rank, cid, ncl, base, bars,
                                                                        abort_flag, peer_abort, total_kb);
        else
            form_pieces<SCHEME, NA, NB, STAGES, FS, PB, FO, true, true>(a, xw, lane, rank, cid, ncl, base, bars,
                                                                       abort_flag, peer_abort, total_kb);
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();  // neither CTA leaves while the other may still touch its shared memory or TMEM
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, L::kTmemCols);
    }
}

template <int SCHEME, int NPROD, int CHUNK_KB>
cudaError_t run_fused(const CUtensorMap& tmA, const CUtensorMap& tmB, const FusedArgs& args, int clusters,
                      cudaStream_t st) {
    constexpr int NA = SCHEME == kSchemeBf16x3 ? 3 : 2;
    constexpr int NB = NPROD == 2 ? 1 : NA;
    using L = FusedLayout<NA, NB>;
    auto kern = k_split_fused<SCHEME, NPROD, CHUNK_KB>;
    FusedArgs a = args;
    // the same cut as the two-pass kernel's (decided on the nominal grid)
    const ChunkPlan cp = plan_chunk_parts(a.num_tiles, clusters, (a.num_kb + CHUNK_KB - 1) / CHUNK_KB,
                                          a.kflags != nullptr, kKpartFlags / 16);
    a.full_units = cp.full_units;
    a.num_units = cp.num_units;
    a.chunk_split = cp.chunk_split;
    // the setmaxnreg split assumes the launch's 96 registers per thread; refuse anything less
    static int checked_regs = 0;
    if (checked_regs == 0) {
        cudaFuncAttributes fa{};
        cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void*>(kern));
        if (e != cudaSuccess) return e;
        checked_regs = fa.numRegs;
    }
    if (checked_regs < 96) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int resident = 0;
    const cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), L::kBytes, &cfg, 0, &resident);
    if (e != cudaSuccess) return e;
    if (resident > 0 && clusters > resident) {
        clusters = resident;
        cfg.gridDim = dim3(2 * clusters, 1, 1);
    }
    if (clusters > a.num_units) {
        clusters = a.num_units;
        cfg.gridDim = dim3(2 * clusters, 1, 1);
    }
    add_pdl(cfg);
    return cudaLaunchKernelEx(&cfg, kern, tmA, tmB, a);
}

}  // namespace

bool split_fused_supported(int scheme, int nprod) { return scheme == kSchemePlain || scheme == kSchemeScaled; }

cudaError_t launch_split_fused(const CUtensorMap& tmA, const CUtensorMap& tmB, const SplitFusedLaunch& p,
                               cudaStream_t st) {
    FusedArgs a{};
    a.m = static_cast<int>(p.m);
    a.n = static_cast<int>(p.n);
    a.k = static_cast<int>(p.k);
    a.num_kb = static_cast<int>((p.k + 63) / 64);
    a.tiles_m = static_cast<int>((p.m + 255) / 256);
    a.tiles_n = static_cast<int>((p.n + 255) / 256);
    a.num_tiles = a.tiles_m * a.tiles_n;
    a.group_m = p.group_m > 0 ? p.group_m : 8;
    a.alpha = p.alpha;
    a.beta = p.beta;
    a.a_mn = p.a_mn;
    a.b_mn = p.b_mn;
    a.bf16 = p.bf16;
    a.C = p.C;
    a.ldc = p.ldc;
    a.status = p.status;
    a.stall_kb = p.stall_at - 1;
    a.serpentine = p.serpentine;
    a.kflags = p.split_tail == 2 ? p.kpart_flags : nullptr;
    a.ktoken = p.kpart_token;
    a.idesc = make_idesc(256, 256, p.bf16 ? 1u : 0u) | (p.a_mn ? kIdescTransposeA : 0u) |
              (p.b_mn ? kIdescTransposeB : 0u);
    a.corr_scale = 1.0f;
    if (p.scheme == kSchemeScaled) a.corr_scale = p.bf16 ? 1.0f / 256.0f : 1.0f / 2048.0f;
    const int max_clusters = p.sm_count / 2;
    const int clusters = a.num_tiles < max_clusters ? a.num_tiles : max_clusters;
    if (clusters <= 0) return cudaSuccess;
    if (p.scheme == kSchemePlain) {
        if (p.nprod == 2) return run_fused<kSchemePlain, 2, 2>(tmA, tmB, a, clusters, st);
        if (p.nprod == 3) return run_fused<kSchemePlain, 3, 2>(tmA, tmB, a, clusters, st);
        if (p.nprod == 4) return run_fused<kSchemePlain, 4, 2>(tmA, tmB, a, clusters, st);
    } else if (p.scheme == kSchemeScaled) {
        if (p.nprod == 2) return run_fused<kSchemeScaled, 2, 4>(tmA, tmB, a, clusters, st);
        if (p.nprod == 3) return run_fused<kSchemeScaled, 3, 4>(tmA, tmB, a, clusters, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace tcg
