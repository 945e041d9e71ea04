// Host build of the grouped tensor-core GEMM's schedule (paper_1803_04014_gb300/csrc/grouped_sched.h),
// checked without a GPU under each setting (tall tiles on and off, transposed problems on and off):
// every element of every problem's output lies in exactly one tile, a tile's record carries the
// problem as the kernel reads it (transposed where it runs transposed), the count the host sizes its
// buffers by equals the tiles emitted, and the setting-free bound covers them.
// Prints "ok" and exits 0, or prints the first failed case and exits 1.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_1803_04014_gb300/csrc/grouped_sched.h"

using namespace tcg;

static int fail(const char* what, const tc_problem& p, bool tall, bool swap_on, int extra) {
    std::printf("FAIL %s (m %d n %d k %d, tall %d, swap %d, %d)\n", what, p.m, p.n, p.k, int(tall), int(swap_on),
                extra);
    return 1;
}

static int check(const tc_problem& p, int32_t g, bool tall_on, bool swap_on, int32_t lb) {
    const bool want_swap = swap_on && p.m < p.n && p.n <= kGroupedTcTileN;
    if (grouped_swap(p, lb) != want_swap) return fail("transposed or not", p, tall_on, swap_on, 0);
    const int rm = want_swap ? p.n : p.m, rn = want_swap ? p.m : p.n;
    std::vector<GroupedTcTile> tiles;
    grouped_tc_tiles(p, g, tall_on, lb, [&](const GroupedTcTile& t) { tiles.push_back(t); });
    if (int64_t(tiles.size()) != grouped_tc_tile_count(p, tall_on, lb))
        return fail("count", p, tall_on, swap_on, static_cast<int>(tiles.size()));
    if (int64_t(tiles.size()) > grouped_tc_tile_bound(p)) return fail("bound", p, tall_on, swap_on, 0);
    std::vector<unsigned char> cover(size_t(rm) * rn, 0);
    for (const GroupedTcTile& t : tiles) {
        if (t.prob != g || t.m != rm || t.n != rn || t.k != p.k || t.ldc != p.ldc || t.off_c != p.off_c ||
            t.nk != (p.k + 63) / 64 || t.flags != (want_swap ? kGroupedTcSwapped : 0))
            return fail("record", p, tall_on, swap_on, t.tm);
        if (t.rows != kGroupedTcTileM && t.rows != 2 * kGroupedTcTileM) return fail("rows", p, tall_on, swap_on, t.rows);
        if (t.rows == 2 * kGroupedTcTileM && !(tall_on && rn <= kGroupedTcTileN / 2))
            return fail("tall tile where none belongs", p, tall_on, swap_on, t.tm);
        const int r0 = t.tm * kGroupedTcTileM, c0 = t.tn * kGroupedTcTileN;
        if (t.tm < 0 || t.tn < 0 || r0 >= rm || c0 >= rn) return fail("tile outside", p, tall_on, swap_on, t.tm);
        // a tall tile's second half may be empty only if it is the last M-block pair's (it is not
        // emitted then: an odd last M-block stays 128 rows high)
        if (t.rows == 2 * kGroupedTcTileM && r0 + kGroupedTcTileM >= rm)
            return fail("empty tall half", p, tall_on, swap_on, t.tm);
        for (int r = r0; r < r0 + t.rows && r < rm; ++r)
            for (int c = c0; c < c0 + kGroupedTcTileN && c < rn; ++c) cover[size_t(r) * rn + c]++;
    }
    for (size_t i = 0; i < cover.size(); ++i)
        if (cover[i] != 1) return fail("coverage", p, tall_on, swap_on, static_cast<int>(i));
    return 0;
}

int main() {
    const int sizes[] = {1, 8, 16, 63, 64, 100, 127, 128, 129, 200, 255, 256, 257, 300, 383, 384, 385, 513, 700};
    int32_t g = 0;
    for (int swap_on = 0; swap_on < 2; ++swap_on) {
        if (swap_on) unsetenv("TCGEMM_GROUPED_SWAP");
        else setenv("TCGEMM_GROUPED_SWAP", "0", 1);
        for (int tall = 0; tall < 2; ++tall)
            for (int32_t lb : {TC_ROW_MAJOR, TC_COL_MAJOR})
                for (int m : sizes)
                    for (int n : sizes) {
                        tc_problem p{};
                        p.m = m;
                        p.n = n;
                        p.k = 16 + (m * 7 + n * 3) % 300;
                        p.ldc = n + (m % 3);
                        p.off_c = int64_t(g) * 1000 + 5;
                        p.lda = p.k;
                        p.ldb = lb == TC_ROW_MAJOR ? n : p.k;
                        if (check(p, g, tall != 0, swap_on != 0, lb)) return 1;
                        ++g;
                    }
    }
    // the settings are read from the environment as documented
    unsetenv("TCGEMM_GROUPED_TALL");
    if (!grouped_tall_tiles()) return std::printf("FAIL tall tiles default\n"), 1;
    setenv("TCGEMM_GROUPED_TALL", "0", 1);
    if (grouped_tall_tiles()) return std::printf("FAIL TCGEMM_GROUPED_TALL=0\n"), 1;
    std::printf("ok\n");
    return 0;
}
