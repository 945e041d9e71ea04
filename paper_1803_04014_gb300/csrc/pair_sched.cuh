// Tile schedule and product tables shared by the CTA-pair GEMM kernels
// (gemm_tc.cu: operands staged by TMA; split_fused.cu: refinement pieces
// formed on chip from FP32 tiles).
#pragma once

#include <stdint.h>

namespace tcg {

// product p multiplies A piece prod_a(p) with B piece prod_b(p).  Two pieces:
// (hi,hi), (lo,hi), (hi,lo), (lo,lo) -- Eq. 1 is the first two, Eq. 2 all
// four, three products drop R_A R_B.  Three BF16 pieces (NA = 3): the six
// products with piece orders adding up to at most 2, largest first:
// (0,0), (1,0), (0,1), (2,0), (1,1), (0,2).
template <int NA = 2>
__host__ __device__ constexpr int prod_a(int p) {
    return NA == 3 ? (p == 1 || p == 4 ? 1 : (p == 3 ? 2 : 0)) : (p & 1);
}
template <int NA = 2>
__host__ __device__ constexpr int prod_b(int p) {
    return NA == 3 ? (p == 2 || p == 4 ? 1 : (p == 5 ? 2 : 0)) : (p >> 1);
}
static_assert(prod_a<3>(3) == 2 && prod_b<3>(3) == 0 && prod_a<3>(5) == 0 && prod_b<3>(5) == 2 &&
                  prod_a<3>(4) == 1 && prod_b<3>(4) == 1 && prod_a<3>(2) == 0 && prod_b<3>(2) == 1,
              "three-piece product table");

// Raster of output tiles: bands of group_m M-tiles, N-tiles swept inside a
// band, so the tiles in flight share A rows and B columns in L2.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group_m, int& mb, int& nb) {
    const int band = group_m * tiles_n;
    const int g = t / band;
    const int first = g * group_m;
    const int gm = min(tiles_m - first, group_m);
    const int r = t - g * band;
    mb = first + r % gm;
    nb = r / gm;
}

// Work units of the refined (promoting) pair kernels.  The two-pass kernel (gemm_tc.cu) and the
// one-launch kernel (split_fused.cu) cut the same tiles at the same chunk, so that they give the
// same bits: units u < full_units are tiles u with every chunk; unit full_units + 2 j + h is part
// h + 1 of tile full_units + j, chunks [0, chunk_split) (h = 0) or [chunk_split, nchunks) (h = 1).
// A part walks its k-blocks upwards; the second part adds its sum to what the first stored.
struct ChunkUnit {
    int t, c0, c1, kpart;
};
__host__ __device__ __forceinline__ ChunkUnit chunk_unit(int full_units, int chunk_split, int nchunks, int u) {
    ChunkUnit w{u, 0, nchunks, 0};
    if (u >= full_units) {
        const int h = u - full_units;
        w.t = full_units + (h >> 1);
        w.kpart = 1 + (h & 1);
        if (h & 1) w.c0 = chunk_split;
        else w.c1 = chunk_split;
    }
    return w;
}

// The cut: a last round of tiles that would keep at most half of `clusters` CTA pairs busy (or a
// grid of fewer tiles than half of them), at most max_cut tiles, K at least 16 chunks.  The first
// part is 4 chunks shorter, so that its epilogue (a few k-blocks' time at three or more products
// per k-step) ends before the second part's main loop; with a shorter K the two parts' epilogues
// would follow one another.
struct ChunkPlan {
    int full_units, num_units, chunk_split;
};
inline ChunkPlan plan_chunk_parts(int num_tiles, int clusters, int nchunks, bool enabled, int max_cut) {
    ChunkPlan p{num_tiles, num_tiles, 0};
    const int rem = clusters > 0 ? num_tiles % clusters : 0;
    if (enabled && nchunks >= 16 && rem > 0 && 2 * rem <= clusters && rem <= max_cut) {
        p.full_units = num_tiles - rem;
        p.num_units = p.full_units + 2 * rem;
        p.chunk_split = (nchunks - 4) / 2;
    }
    return p;
}

// Instruction-descriptor bits that read A (bit 15) or B (bit 16) as MN-major
// (rows of the shared-memory tile run along M or N instead of K).
constexpr uint32_t kIdescTransposeA = 1u << 15;
constexpr uint32_t kIdescTransposeB = 1u << 16;

__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t num_clusters_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}

}  // namespace tcg
