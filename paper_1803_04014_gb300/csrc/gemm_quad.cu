// Persistent tcgen05 GEMM on clusters of four CTAs fed by TMA multicast:
// C = alpha * descale * A B + beta * C with one product of FP16/BF16/E4M3
// operands (Sec. IV), both K-major, FP32 accumulation.
//
// A cluster holds two CTA pairs (cluster ranks 0-1 and 2-3; each pair issues
// tcgen05.mma.cta_group::2 for a 256 x 256 tile, as the pair kernel of
// gemm_tc.cu).  The two pairs take horizontally adjacent tiles of the same
// row band, (mb, 2j) and (mb, 2j + 1), so they need the same 256 rows of A in
// every k-block.  Rank r = 0, 1 of pair q = 0, 1 needs A rows mb*256 + 128 r
// ... + 127; it loads the 64-row quarter 64 q of them and multicasts it to
// the CTAs of both pairs that need those rows (cluster ranks r and r + 2), so
// A crosses from L2 into the SMs once per cluster instead of once per pair:
// per CTA and k-block 8 KB of A and 16 KB of B are requested instead of
// 16 KB + 16 KB.
//
// Synchronisation of a stage (a k-block's A and B in every CTA):
//   - the copies are 2-SM copies (.cta_group::2): the multicast A quarters
//     complete on the "full" barrier of each destination's pair leader, the
//     B half on this pair's leader, so a leader's "full" barrier expects the
//     64 KB that land in its pair (four A quarters, two B halves), armed by
//     the leader's expect-tx alone;
//   - every CTA's "empty" barrier takes one tcgen05.commit arrival from each
//     pair leader (multicast to all four CTAs), because a stage's A quarter
//     lands in both pairs: it is refilled only when both pairs are done.
// (A first version multicast with plain per-CTA completion and relayed each
// CTA's "A landed" to its leader: the quarters took 4.4 us to land and the
// kernel ran 2.7x slower than the pair kernel.)
// Every wait is bounded; on a timeout the CTA raises the abort flags of all
// four CTAs.  Block of 192 threads: warp 0 TMA, warp 1 TMEM + MMA, warps 2-5
// epilogue (32 x 32 chunks staged through shared memory).
#include "launch.h"
#include "pair_sched.cuh"
#include "tc_ptx.cuh"

namespace tcg {
namespace {

constexpr int kQuadThreads = 192;
constexpr int kRowBytes = 128;

struct QuadArgs {
    int m, n, k;
    int num_kb, tiles_m, tiles_n, units_n, num_units, group_m;
    float alpha, beta;
    float* C;
    int64_t ldc;
    const float* scale_a;
    const float* scale_b;
    int* status;
    uint32_t idesc;
    int stall_kb;
    int serpentine;
};

template <int STAGES>
struct QuadLayout {
    static constexpr int kHalfTile = 128 * kRowBytes;  // 128 rows x 128 bytes
    static constexpr int kStageBytes = 2 * kHalfTile;  // A rows and B rows of this CTA
    static constexpr int kBarOffset = STAGES * kStageBytes;
    // full[S], empty[S], tfull[2], tempty[2], drain
    static constexpr int kNumBars = 2 * STAGES + 5;
    static constexpr int kSlotOffset = kBarOffset + 8 * kNumBars;
    static constexpr int kEpiOffset = kSlotOffset + 16;
    static constexpr int kBytes = kEpiOffset + 4 * 32 * 33 * 4 + 1024;
    static constexpr int kTmemCols = 512;
};

// 2-SM tiled load multicast to the CTAs of `mask`: lands at the same offset in each and completes
// on the mbarrier at offset `bar` in each destination's pair leader (bar: this pair's leader's
// barrier as a shared::cluster address).
__device__ __forceinline__ void tma_load_3d_mc(uint32_t dst, const CUtensorMap* map, uint32_t bar, int32_t x,
                                               int32_t y, int32_t z, uint16_t mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar), "h"(mask)
        : "memory");
}

template <int KIND, int STAGES>
__global__ void __launch_bounds__(kQuadThreads, 1)
    k_tc_gemm_quad(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const QuadArgs a) {
    using L = QuadLayout<STAGES>;
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
    auto tfull_bar = [&](int i) { return bars + 8u * (2 * STAGES + i); };
    auto tempty_bar = [&](int i) { return bars + 8u * (2 * STAGES + 2 + i); };
    const uint32_t drain_bar = bars + 8u * (2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + L::kSlotOffset);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base_ptr + L::kSlotOffset + 4);
    const uint32_t abort_addr = base + L::kSlotOffset + 4;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();  // 0..3
    const uint32_t q = rank >> 1;             // CTA pair of the cluster
    const uint32_t r = rank & 1;              // rank inside the pair
    const uint32_t leader = rank & ~1u;
    const int cid = static_cast<int>(cluster_id_x());
    const int ncl = static_cast<int>(num_clusters_x());

    // a failed wait stops all four CTAs
    auto wait = [&](uint32_t bar, uint32_t parity) {
        const bool ok = mbar_wait(bar, parity, abort_flag, a.status);
        if (!ok) {
            for (uint32_t o = 1; o < 4; ++o) st_shared_cluster_u32(mapa_shared(abort_addr, rank ^ o), 1u);
        }
        return ok;
    };
    // unit u: the cluster's two tiles (mb, 2 nbp) and (mb, 2 nbp + 1); this pair takes the second
    auto unit_tile = [&](int u, int& mb, int& nb) {
        int nbp;
        tile_coords(u, a.tiles_m, a.units_n, a.group_m, mb, nbp);
        nb = 2 * nbp + static_cast<int>(q);
    };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);   // the leader's expect-tx
            mbar_init(empty_bar(s), 2);  // a commit from each pair leader
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull_bar(i), 1);
            mbar_init(tempty_bar(i), 8);  // four epilogue warps in each CTA of the pair
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
            // ---------------- TMA producer: a multicast quarter of A, this CTA's half of B
            const uint16_t a_mask = static_cast<uint16_t>((1u << r) | (1u << (r + 2)));
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[STAGES];
#pragma unroll
            for (int s = 0; s < STAGES; ++s) issued_phase[s] = -1;
            bool ok = true;
            for (int u = cid; ok && u < a.num_units; u += ncl) {
                int mb, nb;
                unit_tile(u, mb, nb);
                const int arow = mb * PM + static_cast<int>(r) * 128 + static_cast<int>(q) * 64;
                const int brow = nb * PN + static_cast<int>(r) * 128;
                const bool down = a.serpentine && (((u - cid) / ncl) & 1);
                for (int kb_i = 0; kb_i < a.num_kb; ++kb_i) {
                    const int kb = down ? a.num_kb - 1 - kb_i : kb_i;
                    if (!wait(empty_bar(stage), phase ^ 1u)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sbase = base + stage * L::kStageBytes;
                    const uint32_t leader_full = mapa_shared(full_bar(stage), leader);
                    // test hook: the first pair's leader never arms this stage's full barrier (the copies
                    // still run)
                    const bool withhold = kb_i == a.stall_kb && u == cid && cid == 0 && rank == 0;
                    if (r == 0 && !withhold) mbar_arrive_expect_tx(full_bar(stage), 4 * L::kHalfTile);
                    tma_load_3d_mc(sbase + q * (L::kHalfTile / 2), &tmA, leader_full, kb * BK, arow, 0, a_mask);
                    tma_load_3d_pair(sbase + L::kHalfTile, &tmB, leader_full, kb * BK, brow, 0);
                    issued_phase[stage] = static_cast<int>(phase);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // leaving early: let the copies in flight land (they complete on the pair leaders)
                if (r == 0) {
                    for (int s = 0; s < STAGES; ++s)
                        if (issued_phase[s] >= 0)
                            mbar_wait_bounded(full_bar(s), static_cast<uint32_t>(issued_phase[s]), 100000000ull);
                }
                const uint64_t t0 = global_timer_ns();
                while (global_timer_ns() - t0 < 2000000ull) __nanosleep(1000);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && r == 0) {
            // ---------------- MMA issuer (the even CTA of each pair)
            const uint16_t pair_mask = static_cast<uint16_t>(0x3u << (2 * q));
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
                for (int kb = 0; kb < a.num_kb; ++kb) {
                    if (!wait(full_bar(stage), phase)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sbase = base + stage * L::kStageBytes;
#pragma unroll
                    for (int ks = 0; ks < kSteps; ++ks) {
                        const uint64_t adesc = sw128_kmajor_desc(sbase + ks * 32);
                        const uint64_t bdesc = sw128_kmajor_desc(sbase + L::kHalfTile + ks * 32);
                        const uint32_t accumulate = (kb | ks) != 0 ? 1u : 0u;
                        if constexpr (KIND == 1)
                            mma_pair_f8(d_tmem, adesc, bdesc, a.idesc, accumulate);
                        else
                            mma_pair_f16(d_tmem, adesc, bdesc, a.idesc, accumulate);
                    }
                    issued_any = true;
                    mma_commit_pair_mc(empty_bar(stage), 0xF);  // both pairs read the A quarters of this stage
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
                if (!ok) break;
                mma_commit_pair_mc(tfull_bar(acc), pair_mask);
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
            }
            if (!ok && issued_any) {
                mma_commit_pair_mc(drain_bar, static_cast<uint16_t>(1u << rank));
                mbar_wait_bounded(drain_bar, 0, 100000000ull);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..5 of every CTA): this CTA's 128 rows of its pair's tile
        const int quarter = warp & 3;
        float alpha = a.alpha;
        if constexpr (KIND == 1) alpha = alpha * (1.0f / *a.scale_a) * (1.0f / *a.scale_b);
        const float beta = a.beta;
        const bool vec_ok = ((a.ldc & 3) == 0) && ((reinterpret_cast<uintptr_t>(a.C) & 15u) == 0);
        const uint32_t leader_tempty0 = mapa_shared(tempty_bar(0), leader);
        const uint32_t leader_tempty1 = mapa_shared(tempty_bar(1), leader);
        float* stg = reinterpret_cast<float*>(base_ptr + L::kEpiOffset) + (warp - 2) * (32 * 33);
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int u = cid; u < a.num_units; u += ncl) {
            int mb, nb;
            unit_tile(u, mb, nb);
            const bool ok = wait(tfull_bar(acc), acc_phase);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int r0 = mb * PM + static_cast<int>(r) * 128 + quarter * 32;
            const int col0 = nb * PN;
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                   static_cast<uint32_t>(acc * PN);
            const int cc = (lane & 7) * 4;
            // each 32 x 32 chunk goes through shared memory and is written as four 128-byte row
            // segments per store instruction
#pragma unroll 1
            for (int c = 0; c < PN; c += 32) {
                if (col0 + c >= a.n) break;
                const int nc = min(32, a.n - (col0 + c));
                float4 old[8];
                if (beta != 0.0f) {
#pragma unroll
                    for (int qq = 0; qq < 8; ++qq) {
                        const int grow = r0 + qq * 4 + (lane >> 3);
                        old[qq] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (grow < a.m && vec_ok && cc + 4 <= nc)
                            old[qq] = *reinterpret_cast<const float4*>(a.C + static_cast<int64_t>(grow) * a.ldc +
                                                                       col0 + c + cc);
                    }
                }
                float v[32];
                tmem_load_32(taddr + c, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
                __syncwarp();
#pragma unroll
                for (int qq = 0; qq < 8; ++qq) {
                    const int rr = qq * 4 + (lane >> 3);
                    const int grow = r0 + rr;
                    if (grow < a.m) {
                        float* p = a.C + static_cast<int64_t>(grow) * a.ldc + col0 + c + cc;
                        const float* sv = stg + rr * 33 + cc;
                        if (vec_ok && cc + 4 <= nc) {
                            float4 o = make_float4(alpha * sv[0], alpha * sv[1], alpha * sv[2], alpha * sv[3]);
                            if (beta != 0.0f) {
                                o.x = fmaf(beta, old[qq].x, o.x);
                                o.y = fmaf(beta, old[qq].y, o.y);
                                o.z = fmaf(beta, old[qq].z, o.z);
                                o.w = fmaf(beta, old[qq].w, o.w);
                            }
                            *reinterpret_cast<float4*>(p) = o;
                        } else {
                            for (int e = 0; e < 4; ++e)
                                if (cc + e < nc)
                                    p[e] = (beta != 0.0f) ? fmaf(alpha, sv[e], beta * p[e]) : alpha * sv[e];
                        }
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive_cluster(acc == 0 ? leader_tempty0 : leader_tempty1);
            acc ^= 1;
            if (acc == 0) acc_phase ^= 1u;
        }
    }

    tc_fence_before();
    __syncthreads();
    cluster_sync();  // no CTA leaves while another may still touch its shared memory or TMEM
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, L::kTmemCols);
    }
}

template <int KIND, int STAGES>
cudaError_t run_quad(const CUtensorMap& tmA, const CUtensorMap& tmB, const QuadArgs& args, int sm_count,
                     cudaStream_t st) {
    using L = QuadLayout<STAGES>;
    static_assert(L::kBytes <= 227 * 1024, "shared memory of the quad kernel");
    auto kern = k_tc_gemm_quad<KIND, STAGES>;
    int clusters = sm_count / 4;
    if (clusters > args.num_units) clusters = args.num_units;
    if (clusters <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(4 * clusters, 1, 1);
    cfg.blockDim = dim3(kQuadThreads, 1, 1);
    cfg.dynamicSmemBytes = L::kBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 4;
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
        cfg.gridDim = dim3(4 * clusters, 1, 1);
    }
    add_pdl(cfg);
    return cudaLaunchKernelEx(&cfg, kern, tmA, tmB, args);
}

}  // namespace

cudaError_t launch_tc_gemm_quad(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmLaunch& p,
                                cudaStream_t st) {
    QuadArgs a{};
    a.m = static_cast<int>(p.m);
    a.n = static_cast<int>(p.n);
    a.k = static_cast<int>(p.k);
    const int bk = (p.kind == 1) ? 128 : 64;
    a.num_kb = static_cast<int>((p.k + bk - 1) / bk);
    a.tiles_m = static_cast<int>((p.m + 255) / 256);
    a.tiles_n = static_cast<int>((p.n + 255) / 256);
    a.units_n = (a.tiles_n + 1) / 2;
    a.num_units = a.tiles_m * a.units_n;
    a.group_m = p.group_m > 0 ? p.group_m : 8;
    a.alpha = p.alpha;
    a.beta = p.beta;
    a.C = p.C;
    a.ldc = p.ldc;
    a.scale_a = p.scale_a;
    a.scale_b = p.scale_b;
    a.status = p.status;
    a.idesc = make_idesc(256, 256, static_cast<uint32_t>(p.ab_format));
    a.stall_kb = p.stall_at - 1;
    a.serpentine = p.serpentine;
    if (a.num_units <= 0) return cudaSuccess;
    return p.kind == 1 ? run_quad<1, 6>(tmA, tmB, a, p.sm_count, st) : run_quad<0, 6>(tmA, tmB, a, p.sm_count, st);
}

}  // namespace tcg
