// Host build of the CTA-pair kernels' schedule (paper_1803_04014_gb300/csrc/pair_sched.cuh),
// checked without a GPU: the output-tile raster, the cut of a last round into parts of K, and
// that the persistent grid's waits (the second part of a tile waits for the first) always end.
// Prints "ok" and exits 0, or prints the first failed case and exits 1.
#define __host__
#define __device__
#define __forceinline__ inline
#include <algorithm>
#include <cstdio>
#include <vector>
using std::min;
#include "../paper_1803_04014_gb300/csrc/pair_sched.cuh"

using namespace tcg;

static int fail(const char* what, int a, int b, int c, int d) {
    std::printf("FAIL %s (%d %d %d %d)\n", what, a, b, c, d);
    return 1;
}

// every tile index maps to a distinct (mb, nb) in range, and a band of group_m M-tiles is
// swept down each column before moving to the next
static int check_raster(int tiles_m, int tiles_n, int group_m) {
    std::vector<int> seen(static_cast<size_t>(tiles_m) * tiles_n, 0);
    for (int t = 0; t < tiles_m * tiles_n; ++t) {
        int mb = -1, nb = -1;
        tile_coords(t, tiles_m, tiles_n, group_m, mb, nb);
        if (mb < 0 || mb >= tiles_m || nb < 0 || nb >= tiles_n) return fail("raster range", tiles_m, tiles_n, group_m, t);
        if (seen[static_cast<size_t>(mb) * tiles_n + nb]++) return fail("raster repeat", tiles_m, tiles_n, group_m, t);
        if (mb / group_m != t / (group_m * tiles_n)) return fail("raster band", tiles_m, tiles_n, group_m, t);
    }
    return 0;
}

// the units of one plan cover chunks [0, nchunks) of every tile exactly once; a tile that is cut
// has part 1 at unit u and part 2 at u + 1, part 1 the shorter; the cut units fit in one round of
// the nominal grid; and the persistent schedule ends on every grid of at most `clusters` pairs
static int check_plan(int num_tiles, int clusters, int nchunks, bool enabled, int max_cut) {
    const ChunkPlan p = plan_chunk_parts(num_tiles, clusters, nchunks, enabled, max_cut);
    const bool cut = p.num_units != num_tiles;
    if (cut) {
        const int rem = num_tiles - p.full_units;
        if (!enabled || nchunks < 16 || rem <= 0 || rem > max_cut || 2 * rem > clusters)
            return fail("cut outside its rule", num_tiles, clusters, nchunks, max_cut);
        if (p.full_units % clusters != 0 || p.num_units != p.full_units + 2 * rem ||
            p.num_units - p.full_units > clusters)
            return fail("cut units not one round", num_tiles, clusters, nchunks, max_cut);
        if (p.chunk_split <= 0 || p.chunk_split >= nchunks || 2 * p.chunk_split + 4 > nchunks)
            return fail("chunk split", num_tiles, clusters, nchunks, p.chunk_split);
    } else if (p.full_units != num_tiles) {
        return fail("uncut plan", num_tiles, clusters, nchunks, p.full_units);
    }
    std::vector<int> covered(static_cast<size_t>(num_tiles) * nchunks, 0);
    for (int u = 0; u < p.num_units; ++u) {
        const ChunkUnit w = chunk_unit(p.full_units, p.chunk_split, nchunks, u);
        if (w.t < 0 || w.t >= num_tiles || w.c0 < 0 || w.c0 >= w.c1 || w.c1 > nchunks)
            return fail("unit range", num_tiles, clusters, nchunks, u);
        if ((w.kpart != 0) != (u >= p.full_units)) return fail("unit kind", num_tiles, clusters, nchunks, u);
        if (w.kpart == 2) {
            const ChunkUnit f = chunk_unit(p.full_units, p.chunk_split, nchunks, u - 1);
            if (f.kpart != 1 || f.t != w.t || f.c1 != w.c0) return fail("part pairing", num_tiles, clusters, nchunks, u);
            if (f.c1 - f.c0 > w.c1 - w.c0) return fail("first part longer", num_tiles, clusters, nchunks, u);
        }
        for (int c = w.c0; c < w.c1; ++c) covered[static_cast<size_t>(w.t) * nchunks + c]++;
    }
    for (size_t i = 0; i < covered.size(); ++i)
        if (covered[i] != 1) return fail("chunk coverage", num_tiles, clusters, nchunks, static_cast<int>(i));
    // the kernels may run on fewer pairs than the nominal grid (fewer resident, or fewer units):
    // pair c takes units c, c + g, c + 2g, ... in order, and a second part waits for its first
    for (int g = 1; g <= clusters; ++g) {
        std::vector<int> next(g), done(p.num_units, 0);
        for (int c = 0; c < g; ++c) next[c] = c;
        int left = p.num_units;
        for (bool moved = true; moved && left > 0;) {
            moved = false;
            for (int c = 0; c < g; ++c) {
                const int u = next[c];
                if (u >= p.num_units) continue;
                const ChunkUnit w = chunk_unit(p.full_units, p.chunk_split, nchunks, u);
                if (w.kpart == 2 && !done[u - 1]) continue;
                done[u] = 1;
                next[c] += g;
                --left;
                moved = true;
            }
        }
        if (left) return fail("schedule does not end", num_tiles, clusters, nchunks, g);
    }
    return 0;
}

int main() {
    static_assert(prod_a<2>(0) == 0 && prod_b<2>(0) == 0 && prod_a<2>(1) == 1 && prod_b<2>(1) == 0 &&
                      prod_a<2>(2) == 0 && prod_b<2>(2) == 1 && prod_a<2>(3) == 1 && prod_b<2>(3) == 1,
                  "two-piece product table");
    // the six three-piece products are distinct and have piece orders adding up to at most 2
    for (int p = 0; p < 6; ++p) {
        if (prod_a<3>(p) + prod_b<3>(p) > 2) return fail("bf16x3 order", p, prod_a<3>(p), prod_b<3>(p), 0);
        for (int q = 0; q < p; ++q)
            if (prod_a<3>(p) == prod_a<3>(q) && prod_b<3>(p) == prod_b<3>(q)) return fail("bf16x3 repeat", p, q, 0, 0);
    }
    for (int tm = 1; tm <= 40; tm += 3)
        for (int tn = 1; tn <= 40; tn += 5)
            for (int gm : {1, 2, 8, 16, 32})
                if (check_raster(tm, tn, gm)) return 1;
    // 76 CTA pairs on 152 SMs, and a few other grids
    for (int clusters : {1, 2, 7, 64, 74, 76})
        for (int tiles : {1, 2, 3, 37, 38, 39, 76, 100, 113, 256, 1024})
            for (int nchunks : {1, 15, 16, 17, 32, 64})
                for (bool en : {false, true})
                    for (int max_cut : {0, 1, 64})
                        if (check_plan(tiles, clusters, nchunks, en, max_cut)) return 1;
    std::printf("ok\n");
    return 0;
}
