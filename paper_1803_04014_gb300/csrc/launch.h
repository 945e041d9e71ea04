// Internal launchers: each kernel file exposes host functions that enqueue its
// kernels; api.cu validates arguments and calls them.  Not part of the C ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tcg {

// ---- quantize.cu
// Round rows x cols FP32 (row-major, ld_src) to dt; transpose writes cols x rows.
// For E4M3 `scale` is the device word used first as the max|x| accumulator and
// finally holding the scale.
cudaError_t launch_quantize(int dt, int64_t rows, int64_t cols, const float* src, int64_t ld_src, void* dst,
                            int64_t ld_dst, bool transpose, float* scale, cudaStream_t st);
// scheme 0: (hi, lo); 1: (hi, lo * 2^s); 2: three BF16 pieces.  dst holds 2 or 3 piece pointers.
cudaError_t launch_split(int scheme, int piece, int64_t rows, int64_t cols, const float* src, int64_t ld_src,
                         bool transpose, void* const* dst, int64_t ld_dst, cudaStream_t st);
cudaError_t launch_scale_c(int64_t m, int64_t n, float beta, float* C, int64_t ldc, cudaStream_t st);
// A batch of conversions: job j converts rows x cols FP32 at src (ld_src) into dst (ld_dst),
// transposed if asked; vec = every 8-element chunk of dst starts on 8 elements' worth of aligned
// bytes (16 for FP16/BF16, 8 for E4M3).  E4M3 jobs: amax (uploaded as 0) gathers max |x| as FP32
// bits, and scale receives the job's power-of-two scale.
struct QuantJobDev {
    const float* src;
    void* dst;
    int64_t rows, cols, ld_src, ld_dst;
    int32_t transpose, vec;
    float* scale;
    uint32_t amax, pad;
};
struct QuantTileDev {  // 64 source rows x 32 source columns of one job
    int32_t job, pad;
    int64_t r0, c0;
};
static_assert(sizeof(QuantJobDev) <= 80 && sizeof(QuantTileDev) <= 32, "the serving loop's descriptor bound");
constexpr int kQuantTileRows = 64, kQuantTileCols = 32;
// dt F16 / BF16: one launch.  E4M3: a max-|x| pass over every tile into the jobs' amax words, then
// the rounding (which also writes each job's scale); every job needs at least one tile.
cudaError_t launch_quantize_jobs(int dt, QuantJobDev* jobs, const QuantTileDev* tiles, int32_t ntiles,
                                 cudaStream_t st);

// ---- kernel_setup.cu
// Raises `kern`'s dynamic shared-memory limit to smem_bytes (if > 0) and, with
// cluster_cfg, returns the resident clusters (cudaOccupancyMaxActiveClusters),
// else with block_threads > 0 the resident blocks per SM; 0 if unknown.  Done
// once per (kernel, device), then answered from a cache.
cudaError_t kernel_setup(const void* kern, int smem_bytes, const cudaLaunchConfig_t* cluster_cfg, int block_threads,
                         int* resident);

// Programmatic stream serialization for a GEMM launch: the kernel may be placed on SMs and run its
// set-up (barriers, TMEM allocation, tensor-map prefetch) while the kernel before it in the stream
// finishes; it waits for that kernel (griddepcontrol.wait) before touching any operand.  On unless
// TCGEMM_PDL=0.  add_pdl appends the attribute to cfg.attrs, which must have room for one more.
bool pdl_enabled();
inline void add_pdl(cudaLaunchConfig_t& cfg) {
    if (!pdl_enabled()) return;
    cudaLaunchAttribute& at = cfg.attrs[cfg.numAttrs];
    at.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at.val.programmaticStreamSerializationAllowed = 1;
    ++cfg.numAttrs;
}

// ---- gemm_tc.cu
struct TcGemmLaunch {
    int kind;           // 0: 16-bit inputs (F16/BF16), 1: E4M3
    int ab_format;      // instruction-descriptor operand format
    int na, nb, nprod;  // pieces of A and B, number of products
    int64_t m, n, k;
    float alpha, beta;
    float* C;
    int64_t ldc;
    const float* scale_a;
    const float* scale_b;
    int* status;
    int sm_count;
    int bn;             // tile width of the single-CTA kernel (128 or 256)
    int pair;           // 1: 256 x 256 tiles on CTA pairs (B box of 128 rows per CTA)
    int group_m;        // tile raster band height in M-tiles (0: default)
    int staged_epilogue;  // pair kernel: store C through shared memory in row segments
    int stall_at;       // test hook: k-block + 1 to withhold, 0 = off (tc_debug_stall_next_gemm)
    int promote_kb;     // pair kernel only: >0 adds the partial sums of every promote_kb k-blocks
                        // into FP32 registers with round-to-nearest (1, 2 or 4); 0 keeps them in TMEM
    int b_mn_major;     // pair kernel, one 16-bit product: B is row-major k x n (tmB dims {n, k, 1},
                        // box 64 x 64), read by the MMA as MN-major
    int corr_exp;       // pair kernel with promotion, s > 0: products 1.. (the corrections of a scaled
                        // split) accumulate apart and are multiplied by 2^-s in the epilogue
    int serpentine;     // pair kernels: every other round of tiles of a CTA pair walks K downwards
    int split_tail;     // pair kernel: a last round of tiles keeping at most half of the pairs busy runs
                        // as two units per tile: 1 = 256 x 128 halves, 2 = two parts of K (which need
                        // kpart_flags; else halves)
    unsigned long long* kpart_flags;  // kKpartFlags 64-bit flags of device memory no other launch uses while
                                      // this one runs (see kpart_token)
    unsigned long long kpart_token;   // this launch's flag value: nonzero, never used by another launch
    int quad;           // one product, K-major B: clusters of four CTAs (two pairs) sharing A by TMA
                        // multicast (gemm_quad.cu); tmA then has a 64-row box
};
// Flags of one launch of the pair kernels with parts of K: 8 (16 with promotion) per cut tile.
constexpr int kKpartFlags = 1024;
// Shortest K (in k-blocks) the pair kernel cuts into parts; the promoting kernels cut from 16 chunks
// (32 k-blocks at the shortest chunk).
constexpr int kKpartMinKb = 48;
constexpr int kKpartMinKbPromoted = 32;
// tmA: 3-D map {k, m, na} with a 128 x (128 bytes) box; tmB: {k, n, nb} with a bn x (128 bytes) box.
cudaError_t launch_tc_gemm(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmLaunch& p, cudaStream_t st);
// ---- gemm_quad.cu: the pair GEMM on clusters of four CTAs, A multicast between the two pairs.
cudaError_t launch_tc_gemm_quad(const CUtensorMap& tmA, const CUtensorMap& tmB, const TcGemmLaunch& p,
                                cudaStream_t st);
size_t tc_gemm_smem_bytes(int na, int nb, int bn, int* stages_out);

// ---- split_fused.cu: refined GEMM reading FP32 A and B, pieces formed on chip (one launch).
struct SplitFusedLaunch {
    int scheme;      // 0: hi, lo (Eq. 1 / Eq. 2); 1: scaled residuals
    int nprod;       // 2, 3, 4 (scheme 0); 2, 3 (scheme 1)
    int bf16;        // pieces are BF16 (else FP16)
    int64_t m, n, k;
    float alpha, beta;
    int a_mn;        // 1: A column-major (k x m in memory)
    int b_mn;        // 1: B row-major (k x n in memory)
    float* C;
    int64_t ldc;
    int* status;
    int sm_count;
    int group_m;
    int stall_at;    // test hook: k-block + 1 to withhold, 0 = off
    int serpentine;  // every other round of tiles of a CTA pair walks K downwards
    int split_tail;  // 2: a partial last round of tiles runs as two parts of K (as the two-pass kernel)
    unsigned long long* kpart_flags;  // as in TcGemmLaunch
    unsigned long long kpart_token;
};
// Schemes the one-launch kernel runs (the three-piece BF16 split does not: its pieces and the
// FP32 staging do not fit in shared memory together).
bool split_fused_supported(int scheme, int nprod);
// tmA / tmB: FP32 maps, 128-byte swizzle.  K-major operand: dims {k, rows, 1}, box 32 x 128;
// MN-major operand: dims {rows, k, 1}, box 32 x 32.
cudaError_t launch_split_fused(const CUtensorMap& tmA, const CUtensorMap& tmB, const SplitFusedLaunch& p,
                               cudaStream_t st);

// ---- sgemm.cu
cudaError_t launch_sgemm(int64_t m, int64_t n, int64_t k, float alpha, const float* A, int64_t lda, int la,
                         const float* B, int64_t ldb, int lb, float beta, float* C, int64_t ldc, cudaStream_t st);

// ---- gemm_small.cu
cudaError_t launch_batched16(int dt, int64_t batch, float alpha, const void* A, int64_t sa, const void* B, int64_t sb,
                             int lb, float beta, float* C, int64_t sc, int* status, int sm_count, cudaStream_t st);

struct GroupedProblemDev {   // device copy of one problem
    int32_t m, n, k, pad;
    int64_t off_a, off_b, off_c;
    int32_t lda, ldb, ldc, pad2;
};
struct GroupedTileDev {      // one output tile of one problem
    int32_t prob, tm, tn, pad;
};
cudaError_t launch_grouped(int dt, int lb, const GroupedProblemDev* probs, const GroupedTileDev* tiles,
                           int32_t num_tiles, const void* a_base, const void* b_base, float* c_base, float alpha,
                           float beta, int sm_count, cudaStream_t st);
constexpr int kGroupedTileM = 64;
constexpr int kGroupedTileN = 64;

// ---- grouped_tc.cu: tcgen05 grouped GEMM, K-major A and B, 128 x 256 output tiles (256 x n tall
// tiles for n <= 128).
// maps: per problem g, maps[2g] = A (dims {k, m, 1}, box 64 x 128) and maps[2g+1] =
// B (dims {k, n, 1}, box 64 x grouped_tc_box_rows(n)), both 128-byte swizzled.
constexpr int kGroupedTcTileM = 128;
constexpr int kGroupedTcTileN = 256;
// Everything a role needs about one output tile, in one 48-byte record (no dependent loads).
struct alignas(16) GroupedTcTile {
    int32_t prob, tm, tn, m;  // problem, tile coordinates, problem rows
    int32_t n, k, ldc, nk;    // problem columns, depth, C row stride, k-blocks of 64
    int64_t off_c;            // element offset of C_g
    int32_t rows, flags;      // rows of the tile: 128, or 256 for a tall tile (M-blocks tm and tm + 1); 0 = 128
};
// flags bit 0: the problem runs transposed, C_g^T = B_g^T A_g^T (maps[2g] is then B_g's, maps[2g+1]
// A_g's; m and n of the record are n_g and m_g), its tiles stored to C_g transposed.
constexpr int32_t kGroupedTcSwapped = 1;
int grouped_tc_box_rows(int n);
constexpr int kGroupedTcMapsPerProblem = 2;
// staged: 1 = epilogue through shared memory, 0 = direct row stores, -1 = TCGEMM_GROUPED_EPI or staged
// b_mn: every B_g is row-major (k x n) and maps[2g+1] has dims {n, k, 1} with 64 x 64 boxes.
cudaError_t launch_grouped_tc(int dt, const GroupedTcTile* tiles, int32_t num_tiles, const CUtensorMap* maps,
                              float* c_base, float alpha, float beta, int* status, int sm_count, cudaStream_t st,
                              int staged = -1, bool b_mn = false);

// ---- errnorm.cu
constexpr int kErrBlocks = 1024;  // fixed grid: the reduction order does not depend on the GPU
// partial: 3 * kErrBlocks * 2 doubles of scratch.
cudaError_t launch_error_norm(int64_t m, int64_t n, const float* C, int64_t ldc, const void* ref, int64_t ldr,
                              bool ref_f64, const float* A, int64_t ar, int64_t ac, int64_t lda, const float* B,
                              int64_t br, int64_t bc, int64_t ldb, double* partial, double* out4_dev,
                              cudaStream_t st);

}  // namespace tcg
