// Grouped GEMM on the tensor cores (Sec. IV-B generalised to uneven sizes):
// C_g = alpha * A_g B_g + beta * C_g for every problem g of a plan.
//
// The workload moves far more bytes than it computes (about 34 FLOP/byte for
// m, n, k <= 256), so the kernel is built to keep HBM streaming:
//   * one persistent CTA per SM walks a longest-first list of output tiles of
//     128 x 256, or 256 x n for a problem with n <= 128 (a "tall" tile: both
//     128-row blocks against one B tile, so B is fetched once and the tile
//     pays one round of pipeline and epilogue latency instead of two; every
//     problem of the benchmark is one or two tiles);
//   * every problem has its own pair of TMA tensor maps (A: k x m, B: k x n,
//     K-major) in device memory, so each tile is fetched by TMA with the box
//     cut to the problem (rows beyond m or n are zero-filled, not read);
//   * one thread issues the TMA loads into a 4-stage ring and runs ahead across
//     tile boundaries, so the loads of the next tile overlap the MMAs and the
//     epilogue of the current one;
//   * one thread issues tcgen05.mma 128 x N x 16 (N = the problem's n rounded up
//     to 16, at most 256) into a double-buffered TMEM accumulator (a tall
//     tile: two MMAs per step, rows 128-255 into columns 128... of the buffer);
//   * eight epilogue warps read the accumulator and store C with alpha/beta,
//     the two warps of each TMEM lane quarter taking alternate 32-column chunks
//     (of a tall tile: one warp rows 0-127, the other rows 128-255);
//     each chunk (32 rows x 32 columns) is transposed through a 4 KB swizzled
//     shared-memory slot of the warp so that C leaves as whole row segments;
//   * a problem with m < n <= 256 runs transposed, C^T = B^T A^T (B's map in
//     the A operand's place; a row-major B then reads as an MN-major A): a
//     warp reads only its quarter of the accumulator's lanes, so the n rows of
//     the transposed tile keep all eight warps busy where m rows would keep a
//     few.  Its chunks are written into the slots transposed and leave as C
//     row segments all the same.
//     (Storing the chunks by TMA instead was measured slower: the stores queue
//     behind the operand loads in the SM's one TMA unit.)
#include <cstdlib>
#include <cstring>

#include "launch.h"
#include "tc_ptx.cuh"

namespace tcg {
namespace {

constexpr int GM = 128;
constexpr int GN = 256;
constexpr int kRow = 128;                    // bytes per k-block row (64 x 16-bit)
constexpr int kABytes = GM * kRow;           // 16 KB
constexpr int kBBytes = GN * kRow;           // 32 KB (largest B box)
constexpr int kStages = 4;
// A stage holds a 128-row tile's A box and B box (B at kABytes), or a tall tile's two A boxes
// (rows tm * 128 ... and (tm + 1) * 128 ...) and a B box of at most 128 rows (B at 2 * kABytes).
constexpr int kStage = kABytes + kBBytes;
constexpr int kBarOff = kStages * kStage;
constexpr int kNumBars = 2 * kStages + 5;
constexpr int kSlotOff = kBarOff + 8 * kNumBars;
constexpr int kEpiWarps = 8;                         // two warps per TMEM lane quarter, 128 columns each
constexpr int kEpiWarpBytes = kChunkSlotBytes;       // one 32 x 32 FP32 chunk, 128-byte rows
constexpr int kEpiOff = (kSlotOff + 16 + 127) / 128 * 128;
constexpr int kSmem = kEpiOff + kEpiWarps * kEpiWarpBytes + 1024;
static_assert(kSmem <= 232448, "shared memory per CTA");

constexpr int kThreads = 64 + 32 * kEpiWarps;

struct Args {
    const GroupedTcTile* tiles;
    const CUtensorMap* maps;  // [2 * problems]: A map, B map
    int num_tiles;
    float* c_base;
    float alpha, beta;
    uint32_t ab_format;
    int* status;
    int staged_epilogue;  // 1: transpose each 32 x 32 chunk through shared memory for row-contiguous stores
};

__device__ __forceinline__ GroupedTcTile load_tile(const GroupedTcTile* tiles, int t, int num_tiles) {
    GroupedTcTile r;
    if (t < num_tiles) {
        const int4* p = reinterpret_cast<const int4*>(tiles + t);
        const int4 x = __ldg(p), y = __ldg(p + 1), z = __ldg(p + 2);
        r.prob = x.x; r.tm = x.y; r.tn = x.z; r.m = x.w;
        r.n = y.x; r.k = y.y; r.ldc = y.z; r.nk = y.w;
        r.off_c = (static_cast<int64_t>(static_cast<uint32_t>(z.y)) << 32) | static_cast<uint32_t>(z.x);
        r.rows = z.z;
        r.flags = z.w;
    } else {
        r = GroupedTcTile{};
    }
    return r;
}

// N of the MMA (and rows of the B box) for a problem: n rounded up to 16, capped at 256.
__host__ __device__ __forceinline__ int mma_n(int n) {
    const int r = (n + 15) / 16 * 16;
    return r < GN ? r : GN;
}

// With a row-major (MN-major) B the N of the MMA is a whole number of 64-wide swizzle slabs.
__host__ __device__ __forceinline__ int mma_n_mn(int n) {
    const int r = (n + 63) / 64 * 64;
    return r < GN ? r : GN;
}

// A tall tile (256 rows: M-blocks tm and tm + 1 against one B tile) is taken as one only when its
// MMA N is at most 128: its B box then fits beside the two A boxes in a stage, and its two 128-row
// accumulators share one 256-column buffer (rows 128-255 in columns 128...).  Any other tile
// record is a 128-row tile.
__device__ __forceinline__ bool tall_tile(const GroupedTcTile& t, bool b_mn) {
    return t.rows > GM && (b_mn ? mma_n_mn(t.n) : mma_n(t.n)) <= GN / 2;
}

// B_MN: B_g is row-major (k x n, maps[2g+1] dims {n, k}, boxes of 64 n x 64 k) and is read by
// the MMA as MN-major; otherwise B_g is K-major (n x k).
template <bool B_MN>
__global__ void __launch_bounds__(kThreads, 1) k_grouped_tc(const Args a) {
    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = smem_addr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* base_ptr = smem_raw + (base - raw);
    const uint32_t bars = base + kBarOff;
    auto full_bar = [&](int s) { return bars + 8u * s; };
    auto empty_bar = [&](int s) { return bars + 8u * (kStages + s); };
    auto tfull_bar = [&](int i) { return bars + 8u * (2 * kStages + i); };
    auto tempty_bar = [&](int i) { return bars + 8u * (2 * kStages + 2 + i); };
    const uint32_t drain_bar = bars + 8u * (2 * kStages + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(base_ptr + kSlotOff);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(base_ptr + kSlotOff + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(tfull_bar(i), 1);
            mbar_init(tempty_bar(i), kEpiWarps);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(smem_addr(tmem_slot), 2 * GN);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer, running ahead across tiles
            int stage = 0;
            uint32_t phase = 0;
            int issued_phase[kStages];
#pragma unroll
            for (int s = 0; s < kStages; ++s) issued_phase[s] = -1;
            bool ok = true;
            GroupedTcTile nxt = load_tile(a.tiles, blockIdx.x, a.num_tiles);
            if (static_cast<int>(blockIdx.x) < a.num_tiles) {
                tmap_acquire(a.maps + 2 * nxt.prob);
                tmap_acquire(a.maps + 2 * nxt.prob + 1);
            }
            for (int t = blockIdx.x; ok && t < a.num_tiles; t += gridDim.x) {
                const GroupedTcTile tile = nxt;
                const CUtensorMap* mA = a.maps + 2 * tile.prob;
                const CUtensorMap* mB = mA + 1;
                // fetch the next tile's record and warm its tensor maps while this tile streams
                nxt = load_tile(a.tiles, t + gridDim.x, a.num_tiles);
                if (t + static_cast<int>(gridDim.x) < a.num_tiles) {
                    tmap_acquire(a.maps + 2 * nxt.prob);
                    tmap_acquire(a.maps + 2 * nxt.prob + 1);
                    prefetch_tmap(a.maps + 2 * nxt.prob);
                    prefetch_tmap(a.maps + 2 * nxt.prob + 1);
                }
                const int nk = tile.nk;
                // a transposed problem with a row-major B_g: its A operand (B_g^T) is MN-major, its
                // B operand (A_g) K-major
                const bool a_mn = B_MN && (tile.flags & kGroupedTcSwapped);
                const bool b_mn = B_MN && !a_mn;
                const bool tall = tall_tile(tile, b_mn);
                const int boff = tall ? 2 * kABytes : kABytes;
                const int nslabs = b_mn ? mma_n_mn(tile.n) / 64 : 0;
                const uint32_t bytes = static_cast<uint32_t>((tall ? 2 : 1) * kABytes +
                                                             (b_mn ? nslabs * 64 : mma_n(tile.n)) * kRow);
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sbase = base + stage * kStage;
                    mbar_arrive_expect_tx(full_bar(stage), bytes);
                    for (int blk = 0; blk < (tall ? 2 : 1); ++blk) {
                        const int row_a = (tile.tm + blk) * GM;
                        if (a_mn) {   // 128 rows of A as two slabs of 64 (rows of B_g^T) x 64 k
                            tma_load_3d(sbase + blk * kABytes, mA, full_bar(stage), row_a, kb * 64, 0);
                            tma_load_3d(sbase + blk * kABytes + 64 * kRow, mA, full_bar(stage), row_a + 64, kb * 64, 0);
                        } else {
                            tma_load_3d(sbase + blk * kABytes, mA, full_bar(stage), kb * 64, row_a, 0);
                        }
                    }
                    if (b_mn) {
                        for (int sl = 0; sl < nslabs; ++sl)
                            tma_load_3d(sbase + boff + sl * 64 * kRow, mB, full_bar(stage), tile.tn * GN + sl * 64,
                                        kb * 64, 0);
                    } else {
                        tma_load_3d(sbase + boff, mB, full_bar(stage), kb * 64, tile.tn * GN, 0);
                    }
                    issued_phase[stage] = static_cast<int>(phase);
                    if (++stage == kStages) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                for (int s = 0; s < kStages; ++s)
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
            bool ok = true, issued_any = false;
            GroupedTcTile nxt = load_tile(a.tiles, blockIdx.x, a.num_tiles);
            for (int t = blockIdx.x; ok && t < a.num_tiles; t += gridDim.x) {
                const GroupedTcTile tile = nxt;
                nxt = load_tile(a.tiles, t + gridDim.x, a.num_tiles);
                const int nk = tile.nk;
                const bool a_mn = B_MN && (tile.flags & kGroupedTcSwapped);
                const bool b_mn = B_MN && !a_mn;
                // bit 15 of the instruction descriptor: A MN-major; bit 16: B MN-major
                const uint32_t idesc = b_mn ? (make_idesc(GM, mma_n_mn(tile.n), a.ab_format) | (1u << 16))
                                            : (make_idesc(GM, mma_n(tile.n), a.ab_format) | (a_mn ? (1u << 15) : 0u));
                const bool tall = tall_tile(tile, b_mn);
                const int boff = tall ? 2 * kABytes : kABytes;
                if (!mbar_wait(tempty_bar(acc), acc_phase ^ 1u, abort_flag, a.status)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * GN);
                for (int kb = 0; kb < nk; ++kb) {
                    if (!mbar_wait(full_bar(stage), phase, abort_flag, a.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sbase = base + stage * kStage;
#pragma unroll
                    for (int ks = 0; ks < 4; ++ks) {
                        // MN-major operand: 16 k-rows of 128 bytes per step, 64-row slabs 8 KB apart
                        const uint64_t bdesc = b_mn ? sw128_mnmajor_desc(sbase + boff + ks * 2048, 64 * kRow, 1024)
                                                    : sw128_kmajor_desc(sbase + boff + ks * 32);
                        auto adesc = [&](int blk) {
                            const uint32_t at = sbase + blk * kABytes;
                            return a_mn ? sw128_mnmajor_desc(at + ks * 2048, 64 * kRow, 1024)
                                        : sw128_kmajor_desc(at + ks * 32);
                        };
                        mma_f16(d_tmem, adesc(0), bdesc, idesc, (kb | ks) != 0 ? 1u : 0u);
                        if (tall)   // rows 128-255 against the same B, into columns 128... of the buffer
                            mma_f16(d_tmem + static_cast<uint32_t>(GN / 2), adesc(1), bdesc, idesc,
                                    (kb | ks) != 0 ? 1u : 0u);
                    }
                    issued_any = true;
                    mma_commit(empty_bar(stage));
                    if (++stage == kStages) {
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
                mma_commit(drain_bar);
                mbar_wait_bounded(drain_bar, 0, 100000000ull);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue (warps 2..9): lanes 32*(warp%4).., every other 32-column chunk
        // (chunks half, half + 2, ...), so both warps of a lane quarter share any width of tile
        // A tall tile's rows go to the halves: half h stores rows 128 h .. 128 h + 127, every chunk.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const float alpha = a.alpha, beta = a.beta;
        int acc = 0;
        uint32_t acc_phase = 0;
        GroupedTcTile nxt = load_tile(a.tiles, blockIdx.x, a.num_tiles);
        for (int t = blockIdx.x; t < a.num_tiles; t += gridDim.x) {
            const GroupedTcTile P = nxt;
            const GroupedTcTile& tile = P;
            nxt = load_tile(a.tiles, t + gridDim.x, a.num_tiles);
            const bool ok = mbar_wait(tfull_bar(acc), acc_phase, abort_flag, a.status);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const bool tall = tall_tile(P, B_MN && !(P.flags & kGroupedTcSwapped));
            const int c_first = tall ? 0 : half * 32, c_step = tall ? 32 : 64;
            const int row0 = tile.tm * GM + (tall ? half * GM : 0);
            const int row = row0 + quarter * 32 + lane;
            const int col0 = tile.tn * GN;
            const int ncols_tile = max(0, min(GN, P.n - col0));
            const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                                   static_cast<uint32_t>(acc * GN + (tall ? half * (GN / 2) : 0));
            float* crow = a.c_base + P.off_c + static_cast<int64_t>(row) * P.ldc + col0;
            // a transposed problem (C^T = B^T A^T): tile row r is column r of C_g, tile column c its
            // row c; the chunks are staged transposed, so the stores are C_g row segments again
            const bool swapped = (P.flags & kGroupedTcSwapped) != 0;
            const bool vec_ok = ((P.ldc & 3) == 0) && (((P.off_c + (swapped ? 0 : col0)) & 3) == 0) &&
                                ((reinterpret_cast<uintptr_t>(a.c_base) & 15u) == 0);
            uint8_t* slot_ptr = base_ptr + kEpiOff + (warp - 2) * kEpiWarpBytes;
            const int r0 = row0 + quarter * 32;
            // a warp whose 32 rows all lie past the last row of C_g has nothing to read or store
            const int ncols_warp = r0 < P.m ? ncols_tile : 0;
            if (a.staged_epilogue) {
                // each warp owns rows r0..r0+31 of the tile; stage 32 x 32 chunks and store whole row segments
#pragma unroll 1
                for (int c = c_first; c < ncols_warp; c += c_step) {
                    // the chunk as C_g rows: rows crow0 + 0..31, columns ccol0 + 0..31, of which nrows
                    // and nc exist (a transposed tile's chunk is 32 of its columns by 32 of its rows)
                    const int crow0 = swapped ? col0 + c : r0;
                    const int ccol0 = swapped ? r0 : col0 + c;
                    const int nrows = swapped ? min(32, P.n - (col0 + c)) : min(32, P.m - r0);
                    const int nc = swapped ? min(32, P.m - r0) : min(32, ncols_tile - c);
                    // lane l writes 16-byte group g = l % 8 (columns 4g..4g+3) of rows q*4 + l/8, q = 0..7
                    const int g = lane & 7;
                    const int cc = g * 4;
                    // old C of this chunk first: its global-memory latency overlaps the TMEM load
                    float4 old[8];
                    if (beta != 0.0f) {
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int rr = q * 4 + (lane >> 3);
                            old[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (rr < nrows && vec_ok && cc + 4 <= nc)
                                old[q] = *reinterpret_cast<const float4*>(
                                    a.c_base + P.off_c + static_cast<int64_t>(crow0 + rr) * P.ldc + ccol0 + cc);
                        }
                    }
                    float v[32];
                    tmem_load_32(taddr + c, v);
                    if (swapped) {
                        // lane l holds column l of the C chunk: value i goes to row i, column l
#pragma unroll
                        for (int i = 0; i < 32; ++i)
                            *reinterpret_cast<float*>(slot_ptr + chunk_slot_off(i, lane >> 2) + (lane & 3) * 4) = v[i];
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q)
                            *reinterpret_cast<float4*>(slot_ptr + chunk_slot_off(lane, q)) =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                    __syncwarp();
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int rr = q * 4 + (lane >> 3);
                        if (rr < nrows) {
                            float* p = a.c_base + P.off_c + static_cast<int64_t>(crow0 + rr) * P.ldc + ccol0 + cc;
                            const float4 sv = *reinterpret_cast<const float4*>(slot_ptr + chunk_slot_off(rr, g));
                            if (vec_ok && cc + 4 <= nc) {
                                float4 o = make_float4(alpha * sv.x, alpha * sv.y, alpha * sv.z, alpha * sv.w);
                                if (beta != 0.0f) {
                                    o.x = fmaf(beta, old[q].x, o.x);
                                    o.y = fmaf(beta, old[q].y, o.y);
                                    o.z = fmaf(beta, old[q].z, o.z);
                                    o.w = fmaf(beta, old[q].w, o.w);
                                }
                                __stcs(reinterpret_cast<float4*>(p), o);
                            } else {
                                const float e4[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (cc + e < nc)
                                        p[e] = (beta != 0.0f) ? fmaf(alpha, e4[e], beta * p[e]) : alpha * e4[e];
                            }
                        }
                    }
                    __syncwarp();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty_bar(acc));
                acc ^= 1;
                if (acc == 0) acc_phase ^= 1u;
                continue;
            }
#pragma unroll 1
            for (int c = c_first; c < ncols_warp; c += c_step) {
                float v[32];
                tmem_load_32(taddr + c, v);
                if (swapped) {
                    // lane l holds C_g column `row` for the chunk's 32 rows: one row per step, the
                    // warp's 32 lanes writing 32 consecutive columns of it
                    if (row < P.m) {
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            if (col0 + c + j < P.n) {
                                float* q = a.c_base + P.off_c + static_cast<int64_t>(col0 + c + j) * P.ldc + row;
                                *q = (beta != 0.0f) ? fmaf(alpha, v[j], beta * *q) : alpha * v[j];
                            }
                        }
                    }
                    continue;
                }
                if (row < P.m) {
                    const int nc = min(32, ncols_tile - c);
                    float* p = crow + c;
                    if (nc == 32 && vec_ok) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            float4 o;
                            if (beta != 0.0f) {
                                const float4 old = *reinterpret_cast<const float4*>(p + 4 * j);
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
                            __stcs(reinterpret_cast<float4*>(p + 4 * j), o);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            if (j < nc) p[j] = (beta != 0.0f) ? fmaf(alpha, v[j], beta * p[j]) : alpha * v[j];
                    }
                }
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
        tmem_dealloc(tmem_base, 2 * GN);
    }
}

}  // namespace

int grouped_tc_box_rows(int n) { return mma_n(n); }

cudaError_t launch_grouped_tc(int dt, const GroupedTcTile* tiles, int32_t num_tiles, const CUtensorMap* maps,
                              float* c_base, float alpha, float beta, int* status, int sm_count, cudaStream_t st,
                              int staged, bool b_mn) {
    if (num_tiles <= 0) return cudaSuccess;
    auto kern = b_mn ? k_grouped_tc<true> : k_grouped_tc<false>;
    cudaError_t e = kernel_setup(reinterpret_cast<const void*>(kern), kSmem, nullptr, 0, nullptr);
    if (e != cudaSuccess) return e;
    Args a;
    a.tiles = tiles;
    a.maps = maps;
    a.num_tiles = num_tiles;
    a.c_base = c_base;
    a.alpha = alpha;
    a.beta = beta;
    a.ab_format = dt == 1 ? 1u : 0u;
    a.status = status;
    if (staged >= 0) {
        a.staged_epilogue = staged;
    } else {
        const char* env = getenv("TCGEMM_GROUPED_EPI");
        a.staged_epilogue = (env && strcmp(env, "direct") == 0) ? 0 : 1;
    }
    const int grid = num_tiles < sm_count ? num_tiles : sm_count;
    kern<<<grid, kThreads, kSmem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tcg
