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
