// Persistent tcgen05 GEMM for sm_103a: C = alpha * descale * sum_p X_p Y_p + beta * C.
//
// Mixed precision (Sec. IV, one product of FP16/BF16/E4M3 operands with FP32
// accumulation) and the precision refinement of Sec. V (Eq. 1: 2 products,
// Eq. 2: 4 products, or 3 without R_A R_B) share this kernel: the operands are
// stacks of "pieces" (A: NA pieces of m x k, B: NB pieces of n x k, all K-major)
// and every product of the list accumulates into the same TMEM accumulator, so
// a refined GEMM is one launch instead of the paper's four chained GEMMs.
//
// Block of 192 threads, one CTA per SM, persistent over output tiles of
// 128 x BN:
//   warp 0     one thread issues TMA loads of every piece's k-block into a
//              STAGES-deep shared-memory ring (full/empty mbarriers);
//   warp 1     allocates 2*BN TMEM columns (two accumulators); one thread
//              issues tcgen05.mma (128 x BN x 16 for 16-bit inputs, x 32 for
//              E4M3) and commits each stage back to the producer and each
//              finished accumulator to the epilogue;
//   warps 2-5  epilogue: tcgen05.ld of the accumulator (each warp owns 32 TMEM
//              lanes = 32 rows), alpha/beta in FP32, stores to C, then frees
//              the accumulator so the MMA of tile i+1 overlaps the epilogue of
//              tile i.
// Shared-memory tiles use the 128-byte swizzle written by TMA and read by the
// UMMA descriptors (rows of 128 bytes = one k-block).
//
// Three kernels follow: k_tc_gemm (above, single CTA, used for m <= 128),
// k_tc_gemm_pair (256 x 256 tiles on CTA pairs, the default) and
// k_tc_gemm_pair_promote (the refined products with their partial sums
// promoted to FP32 registers; SCALED keeps the correction products in a second
// accumulator for the scaled split and the three-piece BF16 split).
#include <cstdlib>
#include <cstring>

#include "launch.h"
#include "pair_sched.cuh"
#include "tc_ptx.cuh"

namespace tcg {
namespace {

constexpr int BM = 128;
constexpr int kRowBytes = 128;
constexpr int kATileBytes = BM * kRowBytes;
constexpr int kThreads = 192;

struct Args {
    int m, n, k;
    int num_kb, tiles_m, tiles_n, num_tiles;
    float alpha, beta;
    float* C;
    int64_t ldc;
    const float* scale_a;
    const float* scale_b;
    int* status;
    uint32_t idesc;
    int group_m;  // raster: bands of group_m M-tiles, N-tiles swept inside a band (L2 reuse)
    int stall_kb;  // test hook: >= 0 makes the first CTA (pair) withhold this k-block of its first tile
    int staged_epilogue;  // pair kernel: transpose 32 x 32 chunks through shared memory before storing
    float corr_scale;     // scaled split: 2^-s applied to the correction accumulator
    // pair kernel: work units are the first full_units tiles of the raster (256 x 256) followed by
    // the remaining tiles cut in two each, num_units in all.  Cutting the last, partial round of
    // tiles in two lets twice as many CTA pairs share it.
    //   split_tail 1: two 256 x 128 halves (idesc_half is the half-width MMA's descriptor);
    //   split_tail 2: two parts of K, k-blocks [0, kb_split) and [kb_split, num_kb).  The first
    //     part's epilogue stores alpha * P_1 + beta * C into C and sets one flag per epilogue warp
    //     in kflags to ktoken; the second part's warp waits for that value and stores
    //     alpha * P_2 + C.
    //     An MMA takes about as long at N = 128 as at N = 256, so halves of N take as long as
    //     whole tiles, and parts of K less.
    int full_units, num_units;
    uint32_t idesc_half;
    int split_tail;  // 0 keeps every unit whole (TCGEMM_PAIR_TAIL=full)
    int kb_split;
    unsigned long long* kflags;
    unsigned long long ktoken;  // the value this launch's first parts store in their flags
    // pair kernel with promotion: parts of K only (split_tail 2), cut between chunks: the first part
    // takes chunks [0, chunk_split)
    int chunk_split;
    int serpentine;  // pair kernel: every other unit of a CTA pair walks K from the end (L2 reuse)
};

// Work unit u of the pair kernel: its tile (mb, nb), the column offset inside the 256-wide tile,
// the unit's width (256, or 128 for the halves of the last tiles), its k-blocks [kb0, kb1) and its
// part of K (0: all of it; 1, 2: the first or second part of a tile of the last round).
struct Unit {
    int mb, nb, coff, width, kb0, kb1, kpart;
};
__device__ __forceinline__ Unit unit_coords(const Args& a, int u) {
    Unit w{0, 0, 0, 256, 0, a.num_kb, 0};
    int t = u;
    if (u >= a.full_units) {
        const int h = u - a.full_units;
        t = a.full_units + (h >> 1);
        if (a.split_tail == 2) {
            w.kpart = 1 + (h & 1);
            if (h & 1) w.kb0 = a.kb_split;
            else w.kb1 = a.kb_split;
        } else {
            w.coff = (h & 1) * 128;
            w.width = 128;
        }
    }
    tile_coords(t, a.tiles_m, a.tiles_n, a.group_m, w.mb, w.nb);
    return w;
}

// Flag of epilogue warp (rank, quarter) of the unit's tile, for parts of K of the pair kernel.
__device__ __forceinline__ unsigned long long* kpart_flag(const Args& a, int u, uint32_t rank, int quarter) {
    const int j = (u - a.full_units) >> 1;
    return a.kflags + (j * 2 + static_cast<int>(rank)) * 4 + quarter;
}

template <int BN, int STAGES, int NA, int NB>
struct Layout {
    static constexpr int kBTileBytes = BN * kRowBytes;
    static constexpr int kStageBytes = NA * kATileBytes + NB * kBTileBytes;
    static constexpr int kBarOffset = STAGES * kStageBytes;
    // full[S], empty[S], tfull[2], tempty[2], drain
    static constexpr int kNumBars = 2 * STAGES + 5;
    static constexpr int kSlotOffset = kBarOffset + 8 * kNumBars;
    static constexpr int kBytes = kSlotOffset + 16 + 1024;  // + alignment slack
    static constexpr int kTmemCols = 2 * BN;
};

template <int KIND, int BN, int STAGES, int NA, int NB, int NPROD>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Args a) {
    using L = Layout<BN, STAGES, NA, NB>;
    static_assert(L::kTmemCols == 128 || L::kTmemCols == 256 || L::kTmemCols == 512,
                  "TMEM columns must be a power of two");
    constexpr int kElemBytes = (KIND == 1) ? 1 : 2;
    constexpr int BK = kRowBytes / kElemBytes;  // elements per k-block
    constexpr int kSteps = 4;                   // 4 MMAs of 32 bytes of K per k-block

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + L::kBarOffset;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
    auto tfull_bar = [&](int i) { return bars + 8u * (2 * STAGES + i); };
    auto tempty_bar = [&](int i) { return bars + 8u * (2 * STAGES + 2 + i); };
    const uint32_t drain_bar = bars + 8u * (2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + L::kSlotOffset);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base_ptr + L::kSlotOffset + 4);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull_bar(i), 1);
            mbar_init(tempty_bar(i), 4);  // one arrival per epilogue warp
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(smem_addr(tmem_slot), L::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    // the set-up above overlaps the previous kernel of the stream; operands and C only from here on
    griddep_wait();
    griddep_launch_dependents();

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int t = blockIdx.x; ok && t < a.num_tiles; t += gridDim.x) {
                int mb, nb;
                tile_coords(t, a.tiles_m, a.tiles_n, a.group_m, mb, nb);
                for (int kb = 0; kb < a.num_kb; ++kb) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    if (kb == a.stall_kb && t == static_cast<int>(blockIdx.x) && blockIdx.x == 0) {
                        // test hook: this stage's barrier is never completed
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                        continue;
                    }
                    const uint32_t sbase = base + stage * L::kStageBytes;
                    mbar_arrive_expect_tx(full_bar(stage), L::kStageBytes);
#pragma unroll
                    for (int p = 0; p < NA; ++p)
                        tma_load_3d(sbase + p * kATileBytes, &tmA, full_bar(stage), kb * BK, mb * BM, p);
#pragma unroll
                    for (int p = 0; p < NB; ++p)
                        tma_load_3d(sbase + NA * kATileBytes + p * L::kBTileBytes, &tmB, full_bar(stage), kb * BK,
                                    nb * BN, p);
                    issued_phase[stage] = static_cast<int>(phase);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // leaving early: let the copies already issued land before the CTA exits
                for (int s = 0; s < STAGES; ++s)
                    if (issued_phase[s] >= 0)
                        mbar_wait_bounded(full_bar(s), static_cast<uint32_t>(issued_phase[s]), 100000000ull);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            bool issued_any = false;
            for (int t = blockIdx.x; ok && t < a.num_tiles; t += gridDim.x) {
                if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * BN);
                for (int kb = 0; kb < a.num_kb; ++kb) {
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sbase = base + stage * L::kStageBytes;
#pragma unroll
                    for (int ks = 0; ks < kSteps; ++ks) {
#pragma unroll
                        for (int p = 0; p < NPROD; ++p) {
                            const uint32_t a_addr = sbase + prod_a<NA>(p) * kATileBytes + ks * 32;
                            const uint32_t b_addr = sbase + NA * kATileBytes + prod_b<NA>(p) * L::kBTileBytes + ks * 32;
                            const uint32_t accumulate = (kb | ks | p) != 0 ? 1u : 0u;
                            if constexpr (KIND == 1)
                                mma_f8(d_tmem, sw128_kmajor_desc(a_addr), sw128_kmajor_desc(b_addr), a.idesc,
                                       accumulate);
                            else
                                mma_f16(d_tmem, sw128_kmajor_desc(a_addr), sw128_kmajor_desc(b_addr), a.idesc,
                                        accumulate);
                        }
                    }
                    issued_any = true;
                    mma_commit(empty_bar(stage));  // the stage is free once these MMAs read it
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit(tfull_bar(acc));
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (!ok && issued_any) {
                // leaving early: wait for the MMAs in flight before TMEM is freed
                mma_commit(drain_bar);
                mbar_wait_bounded(drain_bar, 0, 100000000ull);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..5)
        const int quarter = warp & 3;  // TMEM lanes [32*quarter, 32*quarter + 32)
        float alpha = a.alpha;
        if constexpr (KIND == 1) alpha = alpha * (1.0f / *a.scale_a) * (1.0f / *a.scale_b);
        const float beta = a.beta;
        const bool vec_ok = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15u) == 0);
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < a.num_tiles; t += gridDim.x) {
            int mb, nb;
            tile_coords(t, a.tiles_m, a.tiles_n, a.group_m, mb, nb);
            const int row = mb * BM + quarter * 32 + lane;
            const int col0 = nb * BN;
            float* crow = a.C + static_cast<int64_t>(row) * a.ldc + col0;
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                   static_cast<uint32_t>(acc * BN);
            // old C of a whole 32-column chunk of this thread's row (the vector path's chunks only);
            // the first two chunks are read before the accumulator is waited for, so their latency
            // hides behind the main loop, and each later one two chunks ahead of its use
            auto load_old = [&](int c, float4 (&o)[8]) {
                if (c < BN && beta != 0.0f && vec_ok && row < a.m && col0 + c + 32 <= a.n) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) o[j] = *reinterpret_cast<const float4*>(crow + c + 4 * j);
                }
            };
            auto store_chunk = [&](int c, const float4 (&o)[8]) {
                float v[32];
                tmem_load_32(taddr + c, v);
                if (row < a.m) {
                    const int ncols = min(32, a.n - (col0 + c));
                    float* p = crow + c;
                    if (ncols == 32 && vec_ok) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float4 r;
                            if (beta != 0.0f) {
                                r.x = fmaf(alpha, v[4 * j + 0], beta * o[j].x);
                                r.y = fmaf(alpha, v[4 * j + 1], beta * o[j].y);
                                r.z = fmaf(alpha, v[4 * j + 2], beta * o[j].z);
                                r.w = fmaf(alpha, v[4 * j + 3], beta * o[j].w);
                            } else {
                                r.x = alpha * v[4 * j + 0];
                                r.y = alpha * v[4 * j + 1];
                                r.z = alpha * v[4 * j + 2];
                                r.w = alpha * v[4 * j + 3];
                            }
                            *reinterpret_cast<float4*>(p + 4 * j) = r;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (j < ncols) p[j] = (beta != 0.0f) ? fmaf(alpha, v[j], beta * p[j]) : alpha * v[j];
                        }
                    }
                }
            };
            float4 o0[8], o1[8];
            load_old(0, o0);
            load_old(32, o1);
            const bool ok = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, a.status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
#pragma unroll
            for (int c = 0; c < BN; c += 64) {
                if (col0 + c >= a.n) break;  // uniform across the warp
                store_chunk(c, o0);
                load_old(c + 64, o0);
                if (c + 32 >= BN || col0 + c + 32 >= a.n) break;
                store_chunk(c + 32, o1);
                load_old(c + 96, o1);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty_bar(acc));
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, L::kTmemCols);
    }
}

template <int KIND, int BN, int STAGES, int NA, int NB, int NPROD>
cudaError_t run(const CUtensorMap& tmA, const CUtensorMap& tmB, const Args& args, int grid, cudaStream_t st) {
    using L = Layout<BN, STAGES, NA, NB>;
    auto kern = k_tc_gemm<KIND, BN, STAGES, NA, NB, NPROD>;
    cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), L::kBytes, nullptr, 0, nullptr);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    cfg.attrs = attr;
    cfg.numAttrs = 0;
    add_pdl(cfg);
    return cudaLaunchKernelEx(&cfg, kern, tmA, tmB, args);
}


// ====================================================================== CTA-pair kernel
//
// Same computation with 256 x 256 output tiles on a cluster of two CTAs that
// share one tcgen05.mma.cta_group::2: each CTA loads 128 rows of A and 128
// rows (its half of N) of B per k-block (32 KB instead of 48 KB per SM), the
// even CTA issues the MMAs for both and every CTA keeps its 128 rows x 256
// columns of the accumulator in its own TMEM.  Both CTAs' TMA loads complete
// on the even CTA's "full" barrier; the MMA commits are multicast to the
// "empty"/"accumulator full" barriers of both CTAs; both epilogues arrive on
// the even CTA's "accumulator empty" barrier.  A last round of tiles that would
// leave more than half of the pairs idle runs as two units per tile
// (unit_coords): two parts of K, the second adding to what the first stored
// once the first's epilogue warps have raised their flags, or, for a short K,
// two 256 x 128 halves.

template <int STAGES, int NA, int NB>
struct PairLayout {
    static constexpr int kHalfTile = 128 * kRowBytes;  // 128 rows x 128 bytes
    static constexpr int kStageBytes = (NA + NB) * kHalfTile;
    static constexpr int kBarOffset = STAGES * kStageBytes;
    static constexpr int kNumBars = 2 * STAGES + 5;
    static constexpr int kSlotOffset = kBarOffset + 8 * kNumBars;
    static constexpr int kEpiOffset = (kSlotOffset + 16 + 127) / 128 * 128;  // 4 warps x 4 KB of store staging
    static constexpr int kBytes = kEpiOffset + 4 * kChunkSlotBytes + 1024;
    static constexpr int kTmemCols = 512;  // two 256-column accumulators
};

template <int KIND, int STAGES, int NA, int NB, int NPROD, bool B_MN = false>
__global__ void __launch_bounds__(kThreads, 1)
    k_tc_gemm_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const Args a) {
    using L = PairLayout<STAGES, NA, NB>;
    constexpr int kElemBytes = (KIND == 1) ? 1 : 2;
    constexpr int BK = kRowBytes / kElemBytes;
    constexpr int kSteps = 4;
    constexpr int PM = 256, PN = 256;  // pair tile

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + L::kBarOffset;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
    auto tfull_bar = [&](int i) { return bars + 8u * (2 * STAGES + i); };
    auto tempty_bar = [&](int i) { return bars + 8u * (2 * STAGES + 2 + i); };
    const uint32_t drain_bar = bars + 8u * (2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + L::kSlotOffset);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base_ptr + L::kSlotOffset + 4);
    const uint32_t abort_addr = base + L::kSlotOffset + 4;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();
    const uint32_t peer_abort = mapa_shared(abort_addr, rank ^ 1u);
    const int cid = static_cast<int>(cluster_id_x());
    const int ncl = static_cast<int>(num_clusters_x());

    // a failed wait stops this CTA and its peer
    auto wait = [&](uint32_t bar, uint32_t parity) {
        const bool ok = mbar_wait(bar, parity, abort_flag, a.status);
        if (!ok) st_shared_cluster_u32(peer_abort, 1u);
        return ok;
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull_bar(i), 1);
            mbar_init(tempty_bar(i), 8);  // four epilogue warps in each CTA
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
    }
    if (warp == 1) {
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

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer (both CTAs): own half of A and B, completing on the even CTA's barrier
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int u = cid; ok && u < a.num_units; u += ncl) {
                const Unit w = unit_coords(a, u);
                const int mb = w.mb;
                // this CTA's half of the unit's B rows (a half-width unit uses the first 64 of the 128 loaded)
                const int brow = w.nb * PN + w.coff + static_cast<int>(rank) * (w.width >> 1);
                // odd rounds of units walk K downwards: a round of units shares A panels with the round
                // before it (same raster band), and starts on the k-blocks that round left in L2
                const bool down = a.serpentine && (((u - cid) / ncl) & 1);
                for (int kb_i = 0; kb_i < w.kb1 - w.kb0; ++kb_i) {
                    const int kb = down ? w.kb1 - 1 - kb_i : w.kb0 + kb_i;
                    if (!wait(empty_bar(stage), phase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    if (kb_i == a.stall_kb && u == cid && cid == 0 && rank == 0) {
                        // test hook: the even CTA never arms this stage's barrier
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                        continue;
                    }
                    const uint32_t sbase = base + stage * L::kStageBytes;
                    const uint32_t leader_full = mapa_shared(full_bar(stage), 0);
                    if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * L::kStageBytes);
#pragma unroll
                    for (int p = 0; p < NA; ++p)
                        tma_load_3d_pair(sbase + p * L::kHalfTile, &tmA, leader_full, kb * BK,
                                         mb * PM + static_cast<int>(rank) * 128, p);
#pragma unroll
                    for (int p = 0; p < NB; ++p) {
                        if constexpr (B_MN) {
                            // B row-major (k x n): two boxes of 64 k-rows x 64 n (128 bytes) per CTA
                            tma_load_3d_pair(sbase + (NA + p) * L::kHalfTile, &tmB, leader_full, brow, kb * BK, p);
                            tma_load_3d_pair(sbase + (NA + p) * L::kHalfTile + L::kHalfTile / 2, &tmB, leader_full,
                                             brow + 64, kb * BK, p);
                        } else {
                            tma_load_3d_pair(sbase + (NA + p) * L::kHalfTile, &tmB, leader_full, kb * BK, brow, p);
                        }
                    }
                    issued_phase[stage] = static_cast<int>(phase);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                if (rank == 0) {
                    for (int s = 0; s < STAGES; ++s)
                        if (issued_phase[s] >= 0)
                            mbar_wait_bounded(full_bar(s), static_cast<uint32_t>(issued_phase[s]), 100000000ull);
                } else {
                    // the peer cannot observe its copies (they complete on the even CTA): give them time to land
                    const uint64_t t0 = global_timer_ns();
                    while (global_timer_ns() - t0 < 2000000ull) __nanosleep(1000);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // ---------------- MMA issuer (even CTA only)
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool ok = true;
            bool issued_any = false;
            for (int u = cid; ok && u < a.num_units; u += ncl) {
                if (!wait(tempty_bar(acc), acc_phase ^ 1u)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * PN);
                const Unit w = unit_coords(a, u);
                const uint32_t idesc = w.width == 256 ? a.idesc : a.idesc_half;
                for (int kb = 0; kb < w.kb1 - w.kb0; ++kb) {
                    if (!wait(full_bar(stage), phase)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sbase = base + stage * L::kStageBytes;
#pragma unroll
                    for (int ks = 0; ks < kSteps; ++ks) {
#pragma unroll
                        for (int p = 0; p < NPROD; ++p) {
                            const uint32_t a_addr = sbase + prod_a<NA>(p) * L::kHalfTile + ks * 32;
                            const uint32_t accumulate = (kb | ks | p) != 0 ? 1u : 0u;
                            uint64_t bdesc;
                            if constexpr (B_MN) {
                                // 16 k-rows of 128 bytes per MMA step; slabs of 64 n are 8 KB apart
                                const uint32_t b_addr = sbase + (NA + prod_b<NA>(p)) * L::kHalfTile + ks * 2048;
                                bdesc = sw128_mnmajor_desc(b_addr, L::kHalfTile / 2, 1024);
                            } else {
                                const uint32_t b_addr = sbase + (NA + prod_b<NA>(p)) * L::kHalfTile + ks * 32;
                                bdesc = sw128_kmajor_desc(b_addr);
                            }
                            if constexpr (KIND == 1)
                                mma_pair_f8(d_tmem, sw128_kmajor_desc(a_addr), bdesc, idesc, accumulate);
                            else
                                mma_pair_f16(d_tmem, sw128_kmajor_desc(a_addr), bdesc, idesc, accumulate);
                        }
                    }
                    issued_any = true;
                    mma_commit_pair_mc(empty_bar(stage), 0x3);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_pair_mc(tfull_bar(acc), 0x3);
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (!ok && issued_any) {
                mma_commit_pair_mc(drain_bar, 0x1);
                mbar_wait_bounded(drain_bar, 0, 100000000ull);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..5 of both CTAs): this CTA's 128 rows of the pair tile
        const int quarter = warp & 3;
        float alpha = a.alpha;
        if constexpr (KIND == 1) alpha = alpha * (1.0f / *a.scale_a) * (1.0f / *a.scale_b);
        const float beta_in = a.beta;
        // flag of the first part of K set: a bounded poll with acquire by every lane
        auto wait_flag = [&](const unsigned long long* f) {
            const bool ok = poll_flag_acquire(f, a.ktoken, abort_flag, a.status);
            if (!ok) st_shared_cluster_u32(peer_abort, 1u);
            return __all_sync(0xffffffffu, ok);
        };
        // this warp's stores of the first part of K are visible before its flag is raised
        auto raise_flag = [&](int u) {
            __threadfence();
            __syncwarp();
            if (lane == 0) st_release_gpu(kpart_flag(a, u, rank, quarter), a.ktoken);
        };
        const bool vec_ok = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15u) == 0);
        const uint32_t leader_tempty0 = mapa_shared(tempty_bar(0), 0);
        const uint32_t leader_tempty1 = mapa_shared(tempty_bar(1), 0);
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int u = cid; u < a.num_units; u += ncl) {
            const Unit w = unit_coords(a, u);
            const int width = w.width;
            const int row = w.mb * PM + static_cast<int>(rank) * 128 + quarter * 32 + lane;
            const int col0 = w.nb * PN + w.coff;
            // the second part of K adds its product to what the first part's warp stored: wait for
            // that warp's flag before reading C (beta = 1 for this unit)
            const float beta = w.kpart == 2 ? 1.0f : beta_in;
            if (w.kpart == 2 && !wait_flag(kpart_flag(a, u, rank, quarter))) break;
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                   static_cast<uint32_t>(acc * PN);
            float* crow = a.C + static_cast<int64_t>(row) * a.ldc + col0;
            if (a.staged_epilogue) {
                // rows r0..r0+31 of this warp: each 32 x 32 chunk goes through shared memory and is
                // written as four 128-byte row segments per store instruction
                uint8_t* slot = base_ptr + L::kEpiOffset + (warp - 2) * kChunkSlotBytes;
                const int r0 = row - lane;
                const int g = lane & 7;
                const int cc = g * 4;
                // old C of chunk c, in the store pattern (rows r0 + 4q + lane / 8, columns cc..cc+3):
                // the first two chunks are read before the accumulator is waited for, so their latency
                // hides behind the main loop, and each later one two chunks ahead of its use
                auto load_old = [&](int c, float4 (&o)[8]) {
                    if (beta == 0.0f || c >= width || col0 + c >= a.n) return;
                    const int nc = min(32, a.n - (col0 + c));
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int grow = r0 + q * 4 + (lane >> 3);
                        o[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (grow < a.m && vec_ok && cc + 4 <= nc)
                            o[q] = __ldcg(reinterpret_cast<const float4*>(a.C + static_cast<int64_t>(grow) * a.ldc +
                                                                          col0 + c + cc));
                    }
                };
                auto store_chunk = [&](int c, const float4 (&old)[8]) {
                    const int nc = min(32, a.n - (col0 + c));
                    float v[32];
                    tmem_load_32(taddr + c, v);
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        *reinterpret_cast<float4*>(slot + chunk_slot_off(lane, q)) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int rr = q * 4 + (lane >> 3);
                        const int grow = r0 + rr;
                        if (grow < a.m) {
                            float* p = a.C + static_cast<int64_t>(grow) * a.ldc + col0 + c + cc;
                            const float4 s4 = *reinterpret_cast<const float4*>(slot + chunk_slot_off(rr, g));
                            const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
                            if (vec_ok && cc + 4 <= nc) {
                                float4 o = make_float4(alpha * sv[0], alpha * sv[1], alpha * sv[2], alpha * sv[3]);
                                if (beta != 0.0f) {
                                    o.x = fmaf(beta, old[q].x, o.x);
                                    o.y = fmaf(beta, old[q].y, o.y);
                                    o.z = fmaf(beta, old[q].z, o.z);
                                    o.w = fmaf(beta, old[q].w, o.w);
                                }
                                *reinterpret_cast<float4*>(p) = o;
                            } else {
                                for (int e = 0; e < 4; ++e)
                                    if (cc + e < nc)
                                        p[e] = (beta != 0.0f) ? fmaf(alpha, sv[e], beta * __ldcg(p + e)) : alpha * sv[e];
                            }
                        }
                    }
                    __syncwarp();
                };
                float4 o0[8], o1[8];
                load_old(0, o0);
                load_old(32, o1);
                const bool ok = wait(tfull_bar(acc), acc_phase);
                if (!__all_sync(0xffffffffu, ok)) break;
                tc_fence_after();
#pragma unroll 1
                for (int c = 0; c < width; c += 64) {
                    if (col0 + c >= a.n) break;
                    store_chunk(c, o0);
                    load_old(c + 64, o0);
                    if (c + 32 >= width || col0 + c + 32 >= a.n) break;
                    store_chunk(c + 32, o1);
                    load_old(c + 96, o1);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(acc == 0 ? leader_tempty0 : leader_tempty1);
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
                if (w.kpart == 1) raise_flag(u);
                continue;
            }
            const bool ok = wait(tfull_bar(acc), acc_phase);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
#pragma unroll 1
            for (int c = 0; c < width; c += 32) {
                if (col0 + c >= a.n) break;
                float v[32];
                tmem_load_32(taddr + c, v);
                if (row < a.m) {
                    const int ncols = min(32, a.n - (col0 + c));
                    float* p = crow + c;
                    if (ncols == 32 && vec_ok) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float4 o;
                            if (beta != 0.0f) {
                                const float4 old = __ldcg(reinterpret_cast<const float4*>(p + 4 * j));
                                o.x = fmaf(alpha, v[4 * j + 0], beta * old.x);
                                o.y = fmaf(alpha, v[4 * j + 1], beta * old.y);
                                o.z = fmaf(alpha, v[4 * j + 2], beta * old.z);
                                o.w = fmaf(alpha, v[4 * j + 3], beta * old.w);
                            } else {
                                o.x = alpha * v[4 * j + 0];
                                o.y = alpha * v[4 * j + 1];
                                o.z = alpha * v[4 * j + 2];
                                o.w = alpha * v[4 * j + 3];
                            }
                            *reinterpret_cast<float4*>(p + 4 * j) = o;
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (j < ncols) p[j] = (beta != 0.0f) ? fmaf(alpha, v[j], beta * __ldcg(p + j)) : alpha * v[j];
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc == 0 ? leader_tempty0 : leader_tempty1);
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
            if (w.kpart == 1) raise_flag(u);
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();  // neither CTA leaves while the other may still touch its shared memory or TMEM
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, L::kTmemCols);
    }
}

template <int KIND, int STAGES, int NA, int NB, int NPROD, bool B_MN = false>
cudaError_t run_pair(const CUtensorMap& tmA, const CUtensorMap& tmB, const Args& args, int clusters,
                     cudaStream_t st) {
    if (clusters <= 0) return cudaSuccess;
    using L = PairLayout<STAGES, NA, NB>;
    auto kern = k_tc_gemm_pair<KIND, STAGES, NA, NB, NPROD, B_MN>;
    Args a = args;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    cfg.blockDim = dim3(kThreads, 1, 1);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // no more clusters than can be resident at once (persistent tiles)
    int resident = 0;
    const cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), L::kBytes, &cfg, 0, &resident);
    if (e != cudaSuccess) return e;
    if (resident > 0 && clusters > resident) {
        clusters = resident;
        cfg.gridDim = dim3(2 * clusters, 1, 1);
    }
    // a last round that would leave more than half of the pairs idle (or a grid of fewer tiles than
    // half the pairs) is cut into two units per tile
    const int rem = a.num_tiles % clusters;
    a.full_units = a.num_tiles;
    // parts of K need a flag per epilogue warp of each cut tile and a K long enough that the first
    // part's epilogue (about 16 k-blocks' time) ends before the second part's main loop; else halves
    // of N (a short K would chain the two parts' epilogues: 23 us against 11.5 us at m = n = k = 1024)
    if (a.split_tail == 2 && (a.num_kb < kKpartMinKb || !a.kflags || 8 * rem > kKpartFlags)) a.split_tail = 1;
    if (rem > 0 && 2 * rem <= clusters && a.split_tail) a.full_units = a.num_tiles - rem;
    a.num_units = a.full_units + 2 * (a.num_tiles - a.full_units);
    if (clusters > a.num_units) {
        clusters = a.num_units;
        cfg.gridDim = dim3(2 * clusters, 1, 1);
    }
    add_pdl(cfg);
    return cudaLaunchKernelEx(&cfg, kern, tmA, tmB, a);
}

// ====================================================================== CTA-pair kernel with promotion
//
// For the refined (split) products: the tensor cores' internal FP32
// accumulation loses accuracy as K grows (its error grows like sqrt(K) where a
// round-to-nearest FP32 sum's does not), which would waste the precision the
// residual products win back.  This variant restarts the TMEM accumulator
// every CHUNK_KB k-blocks and lets the epilogue warps add each chunk's partial
// sums into FP32 registers with round-to-nearest ("promotion" of the partial
// sums out of the tensor core).  Chunk accumulators are double-buffered in
// TMEM (2 x 256 columns) so the MMAs of chunk c+1 overlap the draining of
// chunk c.  Eight epilogue warps: warp w drains TMEM lanes 32*(w%4).. and
// columns [128*((w-2)/4), +128) into 128 registers per thread.
//
// SCALED (corrections apart; the scaled-residual split of Ootomo and Yokota,
// 2022, and the three-piece BF16 split): product 0 (hi x hi) goes to a
// single-buffered chunk accumulator H (columns 0-255) and is promoted as
// above; the correction products (for the scaled split lo' x hi and hi x lo',
// whose residuals were multiplied by 2^s before rounding) accumulate over the
// whole of K in a second accumulator Y (columns 256-511), which the epilogue
// adds once per tile times corr_scale (2^-s, or 1 for BF16 pieces).  Kept
// apart, the small products are not truncated against the large partial sums
// of hi x hi inside the tensor core.  The correction MMAs of the first
// k-blocks of a chunk (up to STAGES - 1 of them) are issued before the MMA
// warp waits for H to be drained, so the drain of chunk c overlaps the
// corrections of chunk c+1.

constexpr int kPromoteThreads = 320;  // TMA warp, MMA warp, 8 epilogue warps

template <int KIND, int STAGES, int NA, int NB, int NPROD, int CHUNK_KB, bool SCALED>
__global__ void __launch_bounds__(kPromoteThreads, 1)
    k_tc_gemm_pair_promote(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                           const Args a) {
    using L = PairLayout<STAGES, NA, NB>;
    constexpr int kElemBytes = (KIND == 1) ? 1 : 2;
    constexpr int BK = kRowBytes / kElemBytes;
    constexpr int kSteps = 4;
    constexpr int PM = 256, PN = 256;

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + L::kBarOffset;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (STAGES + s); };
    auto cfull_bar = [&](int i) { return bars + 8u * (2 * STAGES + i); };   // chunk accumulator ready
    auto cempty_bar = [&](int i) { return bars + 8u * (2 * STAGES + 2 + i); };  // chunk accumulator drained
    const uint32_t drain_bar = bars + 8u * (2 * STAGES + 4);
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

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
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
    if (warp == 1) {
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

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int u = cid; ok && u < a.num_units; u += ncl) {
                const ChunkUnit w = chunk_unit(a.full_units, a.chunk_split, nchunks, u);
                int mb, nb;
                tile_coords(w.t, a.tiles_m, a.tiles_n, a.group_m, mb, nb);
                // odd rounds of tiles walk K downwards (L2 reuse, as in the pair kernel); a part of K
                // walks its own k-blocks
                const bool down = a.serpentine && w.kpart == 0 && (((u - cid) / ncl) & 1);
                const int ukb0 = w.c0 * CHUNK_KB, ukb1 = min(a.num_kb, w.c1 * CHUNK_KB);
                for (int kb_i = 0; kb_i < ukb1 - ukb0; ++kb_i) {
                    const int kb = down ? ukb1 - 1 - kb_i : ukb0 + kb_i;
                    if (!wait(empty_bar(stage), phase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    if (kb_i == a.stall_kb && u == cid && cid == 0 && rank == 0) {
                        // test hook: the even CTA never arms this stage's barrier
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                        continue;
                    }
                    const uint32_t sbase = base + stage * L::kStageBytes;
                    const uint32_t leader_full = mapa_shared(full_bar(stage), 0);
                    if (rank == 0) mbar_arrive_expect_tx(full_bar(stage), 2 * L::kStageBytes);
#pragma unroll
                    for (int p = 0; p < NA; ++p)
                        tma_load_3d_pair(sbase + p * L::kHalfTile, &tmA, leader_full, kb * BK,
                                         mb * PM + static_cast<int>(rank) * 128, p);
#pragma unroll
                    for (int p = 0; p < NB; ++p)
                        tma_load_3d_pair(sbase + (NA + p) * L::kHalfTile, &tmB, leader_full, kb * BK,
                                         nb * PN + static_cast<int>(rank) * 128, p);
                    issued_phase[stage] = static_cast<int>(phase);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                if (rank == 0) {
                    for (int s = 0; s < STAGES; ++s)
                        if (issued_phase[s] >= 0)
                            mbar_wait_bounded(full_bar(s), static_cast<uint32_t>(issued_phase[s]), 100000000ull);
                } else {
                    const uint64_t t0 = global_timer_ns();
                    while (global_timer_ns() - t0 < 2000000ull) __nanosleep(1000);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0 && SCALED) {
            // the corrections of the first kAhead k-blocks of a chunk are issued before the wait for H,
            // so the drain of the previous chunk overlaps them; one stage stays free for the producer
            constexpr int kAhead = (CHUNK_KB < STAGES - 1) ? CHUNK_KB : (STAGES - 1);
            static_assert(kAhead >= 1, "SCALED needs at least two stages");
            int stage = 0;
            uint32_t phase = 0;
            uint32_t h_phase = 0;
            bool ok = true;
            bool issued_any = false;
            const uint32_t h_tmem = tmem_base;
            const uint32_t y_tmem = tmem_base + static_cast<uint32_t>(PN);
            int ukb0 = 0;  // first k-block of the unit: the correction accumulator restarts there
            auto advance = [&](int& s_, uint32_t& ph_) {
                if (++s_ == STAGES) {
                    s_ = 0;
                    ph_ ^= 1u;
                }
            };
            auto corrections = [&](int kb, int s_) {
                const uint32_t sbase = base + s_ * L::kStageBytes;
#pragma unroll
                for (int ks = 0; ks < kSteps; ++ks) {
#pragma unroll
                    for (int p = 1; p < NPROD; ++p) {
                        const uint32_t a_addr = sbase + prod_a<NA>(p) * L::kHalfTile + ks * 32;
                        const uint32_t b_addr = sbase + (NA + prod_b<NA>(p)) * L::kHalfTile + ks * 32;
                        const uint32_t accumulate = (kb != ukb0 || ks != 0 || p != 1) ? 1u : 0u;
                        mma_pair_f16(y_tmem, sw128_kmajor_desc(a_addr), sw128_kmajor_desc(b_addr), a.idesc,
                                     accumulate);
                    }
                }
            };
            auto hi_hi = [&](int kb, int kb0, int s_) {
                const uint32_t sbase = base + s_ * L::kStageBytes;
#pragma unroll
                for (int ks = 0; ks < kSteps; ++ks) {
                    const uint32_t accumulate = (kb != kb0 || ks != 0) ? 1u : 0u;
                    mma_pair_f16(h_tmem, sw128_kmajor_desc(sbase + ks * 32),
                                 sw128_kmajor_desc(sbase + NA * L::kHalfTile + ks * 32), a.idesc, accumulate);
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
                        // Y restarts with this unit: wait until the previous unit's Y and H are drained
                        if (!wait(cempty_bar(0), h_phase ^ 1u)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    int s2 = stage;
                    uint32_t ph2 = phase;
                    for (int kb = kb0; kb < kb0 + ahead; ++kb) {
                        if (!wait(full_bar(stage), phase)) {
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
                        if (!wait(full_bar(stage), phase)) {
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
            if (!ok && issued_any) {
                mma_commit_pair_mc(drain_bar, 0x1);
                mbar_wait_bounded(drain_bar, 0, 100000000ull);
            }
        } else if (lane == 0 && rank == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int buf = 0;
            uint32_t buf_phase = 0;
            bool ok = true;
            bool issued_any = false;
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
                        if (!wait(full_bar(stage), phase)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sbase = base + stage * L::kStageBytes;
#pragma unroll
                        for (int ks = 0; ks < kSteps; ++ks) {
#pragma unroll
                            for (int p = 0; p < NPROD; ++p) {
                                const uint32_t a_addr = sbase + prod_a<NA>(p) * L::kHalfTile + ks * 32;
                                const uint32_t b_addr = sbase + (NA + prod_b<NA>(p)) * L::kHalfTile + ks * 32;
                                const uint32_t accumulate = (kb != c * CHUNK_KB || ks != 0 || p != 0) ? 1u : 0u;
                                if constexpr (KIND == 1)
                                    mma_pair_f8(d_tmem, sw128_kmajor_desc(a_addr), sw128_kmajor_desc(b_addr), a.idesc,
                                                accumulate);
                                else
                                    mma_pair_f16(d_tmem, sw128_kmajor_desc(a_addr), sw128_kmajor_desc(b_addr),
                                                 a.idesc, accumulate);
                            }
                        }
                        issued_any = true;
                        mma_commit_pair_mc(empty_bar(stage), 0x3);
                        if (++stage == STAGES) {
                            stage = 0;
                            phase ^= 1u;
                        }
                    }
                    if (!ok) break;
                    mma_commit_pair_mc(cfull_bar(buf), 0x3);
                    buf ^= 1;
                    if (buf == 0) buf_phase ^= 1u;
                }
            }
            if (!ok && issued_any) {
                mma_commit_pair_mc(drain_bar, 0x1);
                mbar_wait_bounded(drain_bar, 0, 100000000ull);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: drain every chunk into FP32 registers, store at the end of the tile
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;  // columns [128*half, 128*half + 128)
        float alpha = a.alpha;
        if constexpr (KIND == 1) alpha = alpha * (1.0f / *a.scale_a) * (1.0f / *a.scale_b);
        const float beta_in = a.beta;
        const bool vec_ok = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15u) == 0);
        // flags of parts of K: one per epilogue warp of each cut tile (as in the pair kernel)
        auto part_flag = [&](int u) {
            const int j = (u - a.full_units) >> 1;
            return a.kflags + (j * 2 + static_cast<int>(rank)) * 8 + (warp - 2);
        };
        const uint32_t leader_cempty0 = mapa_shared(cempty_bar(0), 0);
        const uint32_t leader_cempty1 = mapa_shared(cempty_bar(1), 0);
        int buf = 0;
        uint32_t buf_phase = 0;
        bool ok = true;
        for (int u = cid; ok && u < a.num_units; u += ncl) {
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
            for (int c = pu.c0; c < pu.c1; ++c) {
                // SCALED: one H buffer whose phase flips every chunk; else two buffers in turn
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
                    // the correction accumulator, complete with the unit's last chunk
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
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, L::kTmemCols);
    }
}

template <int KIND, int STAGES, int NA, int NB, int NPROD, int CHUNK_KB, bool SCALED = false>
cudaError_t run_pair_promote(const CUtensorMap& tmA, const CUtensorMap& tmB, const Args& args, int clusters,
                             cudaStream_t st) {
    if (clusters <= 0) return cudaSuccess;
    using L = PairLayout<STAGES, NA, NB>;
    static_assert(L::kBytes <= 227 * 1024, "shared memory of the promoted pair kernel");
    auto kern = k_tc_gemm_pair_promote<KIND, STAGES, NA, NB, NPROD, CHUNK_KB, SCALED>;
    Args a = args;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * clusters, 1, 1);
    cfg.blockDim = dim3(kPromoteThreads, 1, 1);
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
    // a last round that would keep at most half of the pairs busy runs as two parts of K per tile,
    // cut between chunks as the one-launch kernel cuts them (decided on the nominal grid, so that
    // both paths give the same bits)
    const ChunkPlan cp = plan_chunk_parts(a.num_tiles, clusters, (a.num_kb + CHUNK_KB - 1) / CHUNK_KB,
                                          a.split_tail == 2 && a.kflags != nullptr, kKpartFlags / 16);
    a.full_units = cp.full_units;
    a.num_units = cp.num_units;
    a.chunk_split = cp.chunk_split;
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

size_t tc_gemm_smem_bytes(int na, int nb, int bn, int* stages_out) {
    const int stage = na * kATileBytes + nb * bn * kRowBytes;
    int stages = (192 * 1024) / stage;
    if (stages > 4) stages = 4;
    if (stages_out) *stages_out = stages;
    return static_cast<size_t>(stages) * stage + 8 * (2 * stages + 5) + 16 + 1024;
}

cudaError_t launch_tc_gemm(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmLaunch& p, cudaStream_t st) {
    Args a{};
    a.m = static_cast<int>(p.m);
    a.n = static_cast<int>(p.n);
    a.k = static_cast<int>(p.k);
    const int bk = (p.kind == 1) ? 128 : 64;
    a.num_kb = static_cast<int>((p.k + bk - 1) / bk);
    a.tiles_m = static_cast<int>((p.m + BM - 1) / BM);
    a.tiles_n = static_cast<int>((p.n + p.bn - 1) / p.bn);
    a.num_tiles = a.tiles_m * a.tiles_n;
    a.alpha = p.alpha;
    a.beta = p.beta;
    a.C = p.C;
    a.ldc = p.ldc;
    a.scale_a = p.scale_a;
    a.scale_b = p.scale_b;
    a.status = p.status;
    a.idesc = make_idesc(BM, p.bn, static_cast<uint32_t>(p.ab_format));
    a.group_m = p.group_m > 0 ? p.group_m : 16;
    a.stall_kb = p.stall_at - 1;
    a.staged_epilogue = p.staged_epilogue;
    a.corr_scale = 1.0f;
    if (p.pair) {
        // 256 x 256 tiles on CTA pairs
        a.tiles_m = static_cast<int>((p.m + 255) / 256);
        a.tiles_n = static_cast<int>((p.n + 255) / 256);
        a.num_tiles = a.tiles_m * a.tiles_n;
        a.idesc = make_idesc(256, 256, static_cast<uint32_t>(p.ab_format));
        a.idesc_half = make_idesc(256, 128, static_cast<uint32_t>(p.ab_format));
        a.full_units = a.num_units = a.num_tiles;
        a.split_tail = p.split_tail;
        a.serpentine = p.serpentine;
        // the first part of K is 16 k-blocks shorter, so that its epilogue overlaps the second's main loop
        a.kb_split = (a.num_kb - 16) / 2 > 0 ? (a.num_kb - 16) / 2 : 1;
        a.kflags = p.kpart_flags;
        a.ktoken = p.kpart_token;
        const int max_clusters = p.sm_count / 2;
        const int clusters = a.num_tiles < max_clusters ? a.num_tiles : max_clusters;
        if (clusters <= 0) return cudaSuccess;
        if (p.quad && p.na == 1 && p.nb == 1 && !p.b_mn_major) return launch_tc_gemm_quad(tmA, tmB, p, st);
        if (p.kind == 1) {
            if (p.na == 1 && p.nb == 1) return run_pair<1, 6, 1, 1, 1>(tmA, tmB, a, max_clusters, st);
            return cudaErrorInvalidValue;
        }
        if (p.corr_exp > 0 || p.na == 3) {
            // corrections apart from hi x hi: the scaled split (16-bit pieces, 2 or 3 products,
            // corrections times 2^-s) and the three BF16 pieces (6 products, corrections times 1)
            a.corr_scale = ldexpf(1.0f, -p.corr_exp);
            const bool long_chunk = p.promote_kb == 4;
            if (p.na == 2 && p.nb == 1 && p.nprod == 2)
                return long_chunk ? run_pair_promote<0, 4, 2, 1, 2, 4, true>(tmA, tmB, a, clusters, st)
                                  : run_pair_promote<0, 4, 2, 1, 2, 2, true>(tmA, tmB, a, clusters, st);
            if (p.na == 2 && p.nb == 2 && p.nprod == 3)
                return long_chunk ? run_pair_promote<0, 3, 2, 2, 3, 4, true>(tmA, tmB, a, clusters, st)
                                  : run_pair_promote<0, 3, 2, 2, 3, 2, true>(tmA, tmB, a, clusters, st);
            if (p.na == 3 && p.nb == 3 && p.nprod == 6)
                return long_chunk ? run_pair_promote<0, 2, 3, 3, 6, 4, true>(tmA, tmB, a, clusters, st)
                                  : run_pair_promote<0, 2, 3, 3, 6, 2, true>(tmA, tmB, a, clusters, st);
            return cudaErrorInvalidValue;
        }
        if (p.promote_kb > 0) {
            // split products with promoted partial sums
            if (p.na == 2 && p.nb == 1 && p.nprod == 2) {
                if (p.promote_kb == 1) return run_pair_promote<0, 4, 2, 1, 2, 1>(tmA, tmB, a, clusters, st);
                if (p.promote_kb == 2) return run_pair_promote<0, 4, 2, 1, 2, 2>(tmA, tmB, a, clusters, st);
                return run_pair_promote<0, 4, 2, 1, 2, 4>(tmA, tmB, a, clusters, st);
            }
            if (p.na == 2 && p.nb == 2 && p.nprod == 3) {
                if (p.promote_kb == 1) return run_pair_promote<0, 3, 2, 2, 3, 1>(tmA, tmB, a, clusters, st);
                if (p.promote_kb == 2) return run_pair_promote<0, 3, 2, 2, 3, 2>(tmA, tmB, a, clusters, st);
                return run_pair_promote<0, 3, 2, 2, 3, 4>(tmA, tmB, a, clusters, st);
            }
            if (p.na == 2 && p.nb == 2 && p.nprod == 4) {
                if (p.promote_kb == 1) return run_pair_promote<0, 3, 2, 2, 4, 1>(tmA, tmB, a, clusters, st);
                if (p.promote_kb == 2) return run_pair_promote<0, 3, 2, 2, 4, 2>(tmA, tmB, a, clusters, st);
                return run_pair_promote<0, 3, 2, 2, 4, 4>(tmA, tmB, a, clusters, st);
            }
            return cudaErrorInvalidValue;
        }
        if (p.na == 1 && p.nb == 1) {
            if (p.b_mn_major) {
                a.idesc |= kIdescTransposeB;
                a.idesc_half |= kIdescTransposeB;
                return run_pair<0, 6, 1, 1, 1, true>(tmA, tmB, a, max_clusters, st);
            }
            return run_pair<0, 6, 1, 1, 1>(tmA, tmB, a, max_clusters, st);
        }
        if (p.na == 2 && p.nb == 1 && p.nprod == 2) return run_pair<0, 4, 2, 1, 2>(tmA, tmB, a, max_clusters, st);
        if (p.na == 2 && p.nb == 2 && p.nprod == 3) return run_pair<0, 3, 2, 2, 3>(tmA, tmB, a, max_clusters, st);
        if (p.na == 2 && p.nb == 2 && p.nprod == 4) return run_pair<0, 3, 2, 2, 4>(tmA, tmB, a, max_clusters, st);
        return cudaErrorInvalidValue;
    }
    const int grid = a.num_tiles < p.sm_count ? a.num_tiles : p.sm_count;
    if (grid <= 0) return cudaSuccess;

    // one product: 128 x 256 tiles, or 128 x 128 / 128 x 64 for problems too small to fill the SMs
    // with wide tiles (same 192 KB of stages, deeper rings)
    if (p.kind == 1) {
        if (p.na == 1 && p.nb == 1 && p.bn == 256) return run<1, 256, 4, 1, 1, 1>(tmA, tmB, a, grid, st);
        if (p.na == 1 && p.nb == 1 && p.bn == 128) return run<1, 128, 6, 1, 1, 1>(tmA, tmB, a, grid, st);
        if (p.na == 1 && p.nb == 1 && p.bn == 64) return run<1, 64, 8, 1, 1, 1>(tmA, tmB, a, grid, st);
        return cudaErrorInvalidValue;
    }
    if (p.na == 1 && p.nb == 1 && p.bn == 256) return run<0, 256, 4, 1, 1, 1>(tmA, tmB, a, grid, st);
    if (p.na == 1 && p.nb == 1 && p.bn == 128) return run<0, 128, 6, 1, 1, 1>(tmA, tmB, a, grid, st);
    if (p.na == 1 && p.nb == 1 && p.bn == 64) return run<0, 64, 8, 1, 1, 1>(tmA, tmB, a, grid, st);
    if (p.na == 2 && p.nb == 1 && p.nprod == 2 && p.bn == 256) return run<0, 256, 3, 2, 1, 2>(tmA, tmB, a, grid, st);
    if (p.na == 2 && p.nb == 2 && p.nprod == 3 && p.bn == 128) return run<0, 128, 3, 2, 2, 3>(tmA, tmB, a, grid, st);
    if (p.na == 2 && p.nb == 2 && p.nprod == 4 && p.bn == 128) return run<0, 128, 3, 2, 2, 4>(tmA, tmB, a, grid, st);
    if (p.na == 2 && p.nb == 2 && p.nprod == 3 && p.bn == 256) return run<0, 256, 2, 2, 2, 3>(tmA, tmB, a, grid, st);
    if (p.na == 2 && p.nb == 2 && p.nprod == 4 && p.bn == 256) return run<0, 256, 2, 2, 2, 4>(tmA, tmB, a, grid, st);
    return cudaErrorInvalidValue;
}

}  // namespace tcg
