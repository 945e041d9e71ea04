// Host side of the grouped tensor-core GEMM's schedule (grouped_tc.cu runs it): which problems run
// transposed, the output tiles of each problem, and a bound on their number that holds under every
// setting.  Included by api.cu; compiles for the host alone.
#pragma once

#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "launch.h"
#include "tcgemm.h"

namespace tcg {

// Problems with m < n <= 256 run transposed on the tensor cores: C_g^T = B_g^T A_g^T, so that the n
// rows of the transposed tile fill the accumulator's lanes (and the epilogue warps that read them)
// where the m rows would fill a few.  B_g (K-major, or row-major and then read as an MN-major A
// operand) takes the A operand's place and A_g the K-major B operand's; with tall tiles the tile count
// does not grow (one tile, or two for m > 128), without them a problem with m <= 128 < n takes two
// 128-row tiles instead of one.  Unless TCGEMM_GROUPED_SWAP=0.  (10 000-problem mix with m, n, k
// uniform over 16..256: 2-3 % faster; problems with m <= 48 and n >= 128 alone: 3.3 -> 3.9 TB/s.)
inline bool grouped_swap(const tc_problem& p, int32_t lb) {
    (void)lb;
    if (!(p.m < p.n && p.n <= kGroupedTcTileN)) return false;
    const char* env = getenv("TCGEMM_GROUPED_SWAP");
    return !(env && strcmp(env, "0") == 0);
}

// Tensor-core tiles of one problem: 128 x 256, or, for n <= 128, tall 256-row tiles that cover
// M-blocks tm and tm + 1 with one B tile (an odd last M-block stays 128 rows high).  Tall tiles
// unless TCGEMM_GROUPED_TALL=0.
inline bool grouped_tall_tiles() {
    const char* env = getenv("TCGEMM_GROUPED_TALL");
    return !(env && strcmp(env, "0") == 0);
}

// Rows and columns of the problem's tiled output: m x n, or n x m when it runs transposed.
inline int64_t grouped_tc_tile_count(const tc_problem& p, bool tall_on, int32_t lb) {
    const bool sw = grouped_swap(p, lb);
    const int64_t rm = sw ? p.n : p.m, rn = sw ? p.m : p.n;
    const int64_t tm = (rm + kGroupedTcTileM - 1) / kGroupedTcTileM;
    const int64_t tn = (rn + kGroupedTcTileN - 1) / kGroupedTcTileN;
    return (tall_on && rn <= kGroupedTcTileN / 2 ? (tm + 1) / 2 : tm) * tn;
}

template <class Emit>
inline void grouped_tc_tiles(const tc_problem& p, int32_t g, bool tall_on, int32_t lb, Emit&& emit) {
    const bool sw = grouped_swap(p, lb);
    const int32_t rm = sw ? p.n : p.m, rn = sw ? p.m : p.n;
    const bool tall = tall_on && rn <= kGroupedTcTileN / 2;
    const int tm = (rm + kGroupedTcTileM - 1) / kGroupedTcTileM;
    const int tn = (rn + kGroupedTcTileN - 1) / kGroupedTcTileN;
    for (int i = 0; i < tm;) {
        const int rows = (tall && i + 1 < tm) ? 2 * kGroupedTcTileM : kGroupedTcTileM;
        for (int j = 0; j < tn; ++j)
            emit(GroupedTcTile{g, i, j, rm, rn, p.k, p.ldc, (p.k + 63) / 64, p.off_c, rows,
                               sw ? kGroupedTcSwapped : 0});
        i += rows / kGroupedTcTileM;
    }
}

// At least grouped_tc_tile_count(p, tall, lb) under every setting (tall tiles on or off, problems
// transposed or not): 128 x 256 tiles of C_g, or of C_g^T for a problem that may run transposed
// (m < n <= 256: n rows in one or two tiles); tall tiles only ever take fewer.
inline int64_t grouped_tc_tile_bound(const tc_problem& p) {
    int64_t t = int64_t((p.m + kGroupedTcTileM - 1) / kGroupedTcTileM) *
                ((p.n + kGroupedTcTileN - 1) / kGroupedTcTileN);
    if (p.m < p.n && p.n <= kGroupedTcTileN) {
        const int64_t tt = (p.n + kGroupedTcTileM - 1) / kGroupedTcTileM;
        if (tt > t) t = tt;
    }
    return t;
}

}  // namespace tcg
