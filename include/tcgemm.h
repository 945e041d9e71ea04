/*
 * tcgemm: mixed-precision GEMM on tensor cores for one NVIDIA GB300 (sm_103a).
 *
 * C ABI of the library built from paper_1803_04014_gb300/csrc.  The method is
 * the one of "NVIDIA Tensor Core Programmability, Performance & Precision"
 * (Markidis et al., arXiv 1803.04014):
 *   - GEMM C = alpha*A*B + beta*C with low-precision inputs and FP32
 *     accumulation (Sec. IV, Sec. VI);
 *   - precision refinement: A = A_hi + R_A, B = B_hi + R_B and the sum of the
 *     residual products (Sec. V, Eq. 1 and Eq. 2);
 *   - batched small GEMM (Sec. IV-B);
 *   - the error measures of Sec. VI.
 *
 * Conventions shared by every call
 *   - Matrix pointers are device pointers owned by the caller unless stated;
 *     the library never frees caller memory.
 *   - Sizes and leading dimensions are in elements.  A is m x k, B is k x n,
 *     C is m x n.  TC_ROW_MAJOR: element (i, j) at p[i*ld + j];
 *     TC_COL_MAJOR: at p[j*ld + i].  C and C0 are always row-major.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue work on it and return without synchronising,
 *     except where a host result is returned (tc_error_norm, tc_sync_status).
 *   - Errors found on the host are returned at once and nothing is enqueued.
 *     A kernel that gives up on a bounded wait records TC_ERR_TIMEOUT in a
 *     per-device status word, frees what it holds and returns; the next
 *     tc_sync_status() reports and clears it.
 *   - tc_last_error() gives a message for the last failing call of the
 *     calling thread.  No C++ exception crosses this interface.
 */
#ifndef TCGEMM_H
#define TCGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tc_status;
#define TC_OK 0
#define TC_PENDING 1            /* serve_poll: request not finished yet        */
#define TC_ERR_INVALID (-1)     /* bad size, pointer, alignment or argument    */
#define TC_ERR_UNSUPPORTED (-2) /* valid request this build does not implement */
#define TC_ERR_OOM (-3)         /* device allocation or HBM budget exhausted   */
#define TC_ERR_CUDA (-4)        /* a CUDA runtime/driver call failed           */
#define TC_ERR_TIMEOUT (-5)     /* a kernel gave up on a bounded wait          */
#define TC_ERR_BUSY (-6)        /* serve_submit: queue full, retry later       */

/* input formats of the tensor-core products */
#define TC_F16 0   /* IEEE binary16 (the paper's half precision)        */
#define TC_BF16 1  /* bfloat16                                           */
#define TC_E4M3 2  /* FP8 E4M3 with a per-tensor power-of-two scale     */

#define TC_ROW_MAJOR 0
#define TC_COL_MAJOR 1

/* ------------------------------------------------------------------------ */
/* library / device                                                          */
/* ------------------------------------------------------------------------ */

/* Version string of the library (static storage). */
const char* tc_version(void);

/* Message of the last failing call of this thread ("" if none). */
const char* tc_last_error(void);

/* SM count and compute capability of the current device (host pointers). */
tc_status tc_device_info(int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor);

/* Synchronise `stream`, then read and clear the current device's status
 * word.  Returns TC_ERR_TIMEOUT if a kernel gave up on a wait since the last
 * call, TC_ERR_CUDA if the synchronisation failed, TC_OK otherwise. */
tc_status tc_sync_status(void* stream);

/* ------------------------------------------------------------------------ */
/* Input rounding (Sec. V "rounded" single -> half; Sec. VI: A and B are first
 * rounded to half precision, untimed in the paper)                           */
/* ------------------------------------------------------------------------ */

/* dst = round(src) to `dt` with round-to-nearest-even.
 *   src: rows x cols FP32, row-major with ld_src (device).
 *   dst: `dt` elements (2 bytes for F16/BF16, 1 byte for E4M3), row-major;
 *        transpose = 0: rows x cols with ld_dst; transpose = 1: cols x rows
 *        (dst[c*ld_dst + r] = round(src[r*ld_src + c])) -- used to make a
 *        K-major copy of a row-major K x N operand.
 *   scale_out (device float): for E4M3 required; receives s = 2^j, the largest
 *        power of two with max|src| * s <= 448, and dst = round(src * s) with
 *        saturation to +-448.  The word is used as the max|src| accumulator
 *        while the call runs.  For F16/BF16 it may be NULL; if given it
 *        receives 1.0.
 * Overflow follows IEEE for F16/BF16 (to +-inf).  rows or cols == 0 is a
 * no-op (for E4M3 the scale becomes 1). */
tc_status tc_quantize(int32_t dt, int64_t rows, int64_t cols, const float* src, int64_t ld_src,
                      void* dst, int64_t ld_dst, int32_t transpose, float* scale_out, void* stream);

/* Residual split (Sec. V: R_A = A_single - A_half, stored in 16 bits):
 *   hi = round(x), lo = round(x - hi) in `piece` (TC_F16 or TC_BF16), RNE.
 *   src: rows x cols FP32 row-major (ld_src).  dst_hi / dst_lo: 16-bit,
 *   row-major rows x cols (transpose = 0) or cols x rows (transpose = 1),
 *   leading dimension ld_dst.  Values |x| >= 65520 overflow the F16 hi piece. */
tc_status tc_split(int32_t piece, int64_t rows, int64_t cols, const float* src, int64_t ld_src,
                   int32_t transpose, void* dst_hi, void* dst_lo, int64_t ld_dst, void* stream);

/* Many FP32 -> FP16/BF16 roundings (as tc_quantize) in one launch: job j
 * rounds the rows x cols FP32 matrix at src (row-major, ld_src) into dst
 * (ld_dst), transposed (dst cols x rows) if transpose != 0.  For a batch of
 * small operands, where a launch per operand costs more than the rounding.
 *   dt: TC_F16 or TC_BF16 (E4M3 needs a scale per tensor: tc_quantize_batch_e4m3).
 *   workspace: 256-byte aligned device memory of at least
 *   tc_quantize_batch_workspace_bytes(count, jobs) bytes for the job table
 *   and the tile list, not touched by other work until the kernel has
 *   finished on `stream`.  The job array itself is read on the host, and the
 *   job table is uploaded from host memory that the call frees on return: on
 *   a stream that is being captured the call returns TC_ERR_UNSUPPORTED. */
typedef struct tc_quantize_job {
    int64_t rows, cols;
    const float* src;
    int64_t ld_src;
    void* dst;
    int64_t ld_dst;
    int32_t transpose, reserved;
} tc_quantize_job;
size_t tc_quantize_batch_workspace_bytes(int32_t count, const tc_quantize_job* jobs);
tc_status tc_quantize_batch(int32_t dt, int32_t count, const tc_quantize_job* jobs,
                            void* workspace, size_t workspace_bytes, void* stream);

/* Many FP32 -> E4M3 roundings (as tc_quantize with dt = TC_E4M3, each job
 * with its own per-tensor scale): job j's scale s_j is the largest power of
 * two with max|src_j| * s_j <= 448 (1 for an empty or all-zero job), stored
 * as a device float at scale_out[j] (a host array of count device pointers,
 * 4-byte aligned), and dst_j = RNE_satfinite(src_j * s_j).  Two launches: a
 * max-|x| pass over every job, then the rounding.  Codes and scales equal
 * tc_quantize's bit for bit.  Jobs, workspace (same size function) and the
 * capture rule as tc_quantize_batch; dst needs 1-byte alignment only. */
tc_status tc_quantize_batch_e4m3(int32_t count, const tc_quantize_job* jobs, float* const* scale_out,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* Scaled residual split (Ootomo and Yokota, 2022, refining Sec. V):
 *   hi = RNE(x), lo = RNE((x - hi) * 2^s), s = 11 for TC_F16, 8 for TC_BF16.
 *   The scaling keeps residuals of small |x| in the normal range of the
 *   16-bit format (an FP16 residual below 2^-14 would lose bits).  Arguments,
 *   layouts and errors as tc_split. */
tc_status tc_split_scaled(int32_t piece, int64_t rows, int64_t cols, const float* src, int64_t ld_src,
                          int32_t transpose, void* dst_hi, void* dst_lo, int64_t ld_dst, void* stream);

/* Three BF16 pieces (Sec. V's split carried one piece further, as Henry, Tang
 * and Heinecke, 2019): p0 = RNE(x), p1 = RNE(x - p0), p2 = RNE(x - p0 - p1);
 * p0 + p1 + p2 == x for FP32 x whose pieces stay in the normal range.
 *   dst0, dst1, dst2: BF16 outputs, 2-byte aligned; otherwise as tc_split. */
tc_status tc_split_bf16x3(int64_t rows, int64_t cols, const float* src, int64_t ld_src, int32_t transpose,
                          void* dst0, void* dst1, void* dst2, int64_t ld_dst, void* stream);

/* ------------------------------------------------------------------------ */
/* GEMM on tensor cores (Sec. IV: C = alpha*A*B + beta*C; FP32 accumulation) */
/* ------------------------------------------------------------------------ */

/* C = alpha * descale * (A B) + beta * C, A and B already in format `dt`.
 *   Layout: A row-major (la = TC_ROW_MAJOR, m x k, lda >= k).  B column-
 *   major (lb = TC_COL_MAJOR, i.e. stored n x k, ldb >= k: K-major) or, for
 *   TC_F16 and TC_BF16, row-major (lb = TC_ROW_MAJOR, k x n, ldb >= n: read
 *   by the tensor cores as MN-major, on the CTA-pair kernel).  A column-major
 *   A and a row-major E4M3 B return TC_ERR_UNSUPPORTED; tc_quantize with
 *   transpose = 1 makes a K-major copy.
 *   Alignment: A, B 16-byte aligned, lda*size and ldb*size multiples of 16.
 *   scale_a / scale_b: E4M3 only, device floats from tc_quantize; descale =
 *   1/(scale_a*scale_b).  NULL for F16/BF16.
 *   beta == 0: C is not read.  k == 0: C = beta*C.
 * Runs a persistent tcgen05 kernel: TMA-fed shared-memory ring, one thread
 * issuing the MMAs into a double-buffered TMEM accumulator, four epilogue
 * warps.  Untuned tiles: 256 x 256 on CTA pairs; 128 x 64 (else 128 x 128)
 * on single CTAs when that many tiles fit on the SMs at once; single CTAs
 * whenever m <= 128.  On CTA pairs, a last round of tiles that would keep at
 * most half of the pairs busy runs as two units per tile: with K of at least
 * 48 k-blocks (3072 FP16/BF16, 6144 E4M3 elements) two parts of K, the first
 * storing alpha*P1 + beta*C, the second, once the first has signalled
 * through a device flag, alpha*P2 + C (a fixed order: the same bits every
 * run); with a shorter K two 256 x 128 halves.  The flags of an eager
 * launch are 8 KB of device memory per stream handle (per host thread for
 * cudaStreamPerThread), allocated on the stream's first such launch and kept
 * for the process; a launch being captured into a graph takes a block the
 * graph allocates, zeroes and frees at each replay.  No two launches in
 * flight at once share flags, with one exception: a stream destroyed while
 * such a launch still runs, whose handle a new stream takes over at once.
 * The earlier launch's second parts may then wait in vain; they give up
 * after 2 s with an error status (tc_sync_status) rather than hang.  So
 * synchronise a stream before destroying it.  TCGEMM_PAIR_TAIL=full keeps
 * whole tiles, =halves always cuts halves.  The kernel is launched with
 * programmatic stream
 * serialization: it may run its set-up while the previous kernel of the
 * stream finishes and waits for it before touching A, B, C or the scales
 * (TCGEMM_PDL=0 turns this off). */
tc_status gemm_mixed(int32_t dt, int64_t m, int64_t n, int64_t k, float alpha,
                     const void* A, int64_t lda, int32_t la,
                     const void* B, int64_t ldb, int32_t lb,
                     float beta, float* C, int64_t ldc,
                     const float* scale_a, const float* scale_b, void* stream);

/* Bytes of workspace gemm_split, gemm_split_scaled (nprod 2-4: two pieces per
 * operand) or gemm_split_bf16x3 (nprod = 6: three pieces) needs. */
size_t gemm_split_workspace_bytes(int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k);

/* Precision refinement (Sec. V, Eq. 1 and Eq. 2) in one accumulator:
 *   C = alpha * sum_{(p,q)} X_p Y_q + beta * C, X_0 = hi(A), X_1 = lo(A),
 *   Y_0 = hi(B), Y_1 = lo(B), products
 *     nprod = 2: A_hi B_hi + A_lo B_hi                (Eq. 1)
 *     nprod = 3: + A_hi B_lo                          (Eq. 2 without R_A R_B)
 *     nprod = 4: + A_lo B_lo                          (Eq. 2)
 *   A: m x k FP32, B: k x n FP32, any layout (la, lb), 4-byte aligned.
 *   piece: TC_F16 or TC_BF16.
 * Two paths, the same C bit for bit:
 *   - workspace == NULL: one launch that allocates nothing.  TMA streams the
 *     FP32 rows of A and B into shared memory, the CUDA cores form the pieces
 *     of every k-block there while the tensor cores multiply the previous
 *     ones; the pieces never reach HBM.  Needs A and B 16-byte aligned with
 *     lda, ldb multiples of 4; other operands fall back to the second path
 *     with its workspace taken from the stream-ordered pool (cudaMallocAsync
 *     on `stream`, freed on `stream`).
 *   - workspace != NULL (device memory of gemm_split_workspace_bytes() bytes
 *     owned by the caller, 256-byte aligned): a split pass writes the pieces
 *     there and a second launch multiplies them.  About 1.7x faster than the
 *     one-launch kernel at m = n = k = 8192 on GB300, whose shared memory then
 *     carries 288 KB per k-block and CTA against 160 KB here.
 *   The environment variable TCGEMM_SPLIT=fused or =twopass forces a path.
 * All products accumulate in TMEM, with partial sums promoted to
 * round-to-nearest FP32 registers every 128 of K. */
tc_status gemm_split(int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, int32_t la,
                     const float* B, int64_t ldb, int32_t lb,
                     float beta, float* C, int64_t ldc,
                     void* workspace, size_t workspace_bytes, void* stream);

/* Refinement with scaled residuals (Ootomo and Yokota, 2022):
 *   C = alpha * (A_hi B_hi + 2^-s (A_lo' B_hi [+ A_hi B_lo'])) + beta * C,
 *   lo' = RNE((x - hi) * 2^s) as tc_split_scaled; nprod = 2 keeps Eq. 1's
 *   pair of products, nprod = 3 Eq. 2 without R_A R_B.
 * A_hi B_hi accumulates in one TMEM accumulator whose partial sums are added
 * into round-to-nearest FP32 registers every 256 of K; the correction
 * products accumulate in a second TMEM accumulator over all of K and are
 * scaled by 2^-s once per output tile.  piece: TC_F16 or TC_BF16.
 * Arguments, workspace and errors otherwise as gemm_split. */
tc_status gemm_split_scaled(int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k, float alpha,
                            const float* A, int64_t lda, int32_t la,
                            const float* B, int64_t ldb, int32_t lb,
                            float beta, float* C, int64_t ldc,
                            void* workspace, size_t workspace_bytes, void* stream);

/* Refinement with three BF16 pieces per operand (tc_split_bf16x3):
 *   C = alpha * sum_{i + j <= 2} A_i B_j + beta * C  (six products),
 * FP32-level accuracy over the whole FP32 exponent range, where FP16 pieces
 * overflow or underflow.  A_0 B_0 is promoted to round-to-nearest FP32
 * registers every 128 of K; the five correction products accumulate in a
 * second TMEM accumulator, as in gemm_split_scaled.  Workspace:
 * gemm_split_workspace_bytes(TC_BF16, 6, m, n, k).  Arguments and errors
 * otherwise as gemm_split. */
tc_status gemm_split_bf16x3(int64_t m, int64_t n, int64_t k, float alpha,
                            const float* A, int64_t lda, int32_t la,
                            const float* B, int64_t ldb, int32_t lb,
                            float beta, float* C, int64_t ldc,
                            void* workspace, size_t workspace_bytes, void* stream);

/* The two halves of gemm_split, gemm_split_scaled and gemm_split_bf16x3, so that
 * the HBM-bound forming of the next product's pieces (CUDA cores) can run on a
 * second stream while the tensor cores run the current refined GEMM: the
 * concurrent CUDA-core / tensor-core use of streams that Sec. VIII proposes.
 *   scheme: 0 = gemm_split (nprod 2, 3 or 4), 1 = gemm_split_scaled (nprod 2
 *   or 3), 2 = gemm_split_bf16x3 (piece TC_BF16, nprod 6).
 *   gemm_split_prepare forms the pieces of A and B (arguments as gemm_split)
 *   in `workspace`: device memory of gemm_split_workspace_bytes(piece, nprod,
 *   m, n, k) bytes, 256-byte aligned, owned by the caller; NULL is refused.
 *   gemm_split_run computes C = alpha * (the scheme's products) + beta * C
 *   from the pieces a gemm_split_prepare with the same scheme, piece, nprod,
 *   m, n and k left in `workspace`.
 * prepare then run on one stream is the one-call entry point, bit for bit.
 * Ordering across streams is the caller's: a run must start after its prepare
 * has finished, and a workspace may be prepared again only after the run that
 * reads it has finished (cudaEventRecord / cudaStreamWaitEvent). */
tc_status gemm_split_prepare(int32_t scheme, int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k,
                             const float* A, int64_t lda, int32_t la,
                             const float* B, int64_t ldb, int32_t lb,
                             void* workspace, size_t workspace_bytes, void* stream);
tc_status gemm_split_run(int32_t scheme, int32_t piece, int32_t nprod, int64_t m, int64_t n, int64_t k,
                         float alpha, float beta, float* C, int64_t ldc,
                         const void* workspace, size_t workspace_bytes, void* stream);

/* FP32 GEMM on the CUDA cores (no tensor cores): the paper's sgemm
 * comparison (Sec. VII-A, VII-B).  Any layouts; C row-major. */
tc_status gemm_sgemm(int64_t m, int64_t n, int64_t k, float alpha,
                     const float* A, int64_t lda, int32_t la,
                     const float* B, int64_t ldb, int32_t lb,
                     float beta, float* C, int64_t ldc, void* stream);

/* ------------------------------------------------------------------------ */
/* Batched and grouped GEMM (Sec. IV-B; Sec. VI: 16x16 problems, one warp per
 * problem in the paper's WMMA kernel)                                        */
/* ------------------------------------------------------------------------ */

/* batch independent 16 x 16 x 16 products, C_i = alpha*A_i B_i + beta*C_i.
 *   dt: TC_F16 or TC_BF16.  m = n = k = 16 (others: TC_ERR_UNSUPPORTED).
 *   A_i at A + i*stride_a, row-major 16 x 16 (la must be TC_ROW_MAJOR);
 *   B_i at B + i*stride_b, 16 x 16, row-major (lb = TC_ROW_MAJOR) or
 *   column-major (TC_COL_MAJOR); C_i at C + i*stride_c, FP32 row-major.
 *   Strides in elements, multiples of 8 (16 bytes) for A and B, of 2 for C;
 *   pointers 16-byte aligned. */
tc_status gemm_batched_strided(int32_t dt, int64_t batch, int32_t m, int32_t n, int32_t k, float alpha,
                               const void* A, int64_t stride_a, int32_t la,
                               const void* B, int64_t stride_b, int32_t lb,
                               float beta, float* C, int64_t stride_c, void* stream);

/* One problem of a grouped GEMM.  Offsets are in elements from the bases
 * passed at run time; A_g is m x k (row-major, lda), B_g is k x n (layout of
 * the group, ldb), C_g is m x n FP32 row-major (ldc). */
typedef struct tc_problem {
    int32_t m, n, k, reserved;
    int64_t off_a, off_b, off_c;
    int32_t lda, ldb, ldc, reserved2;
} tc_problem;

typedef struct tc_grouped_plan tc_grouped_plan;

/* Validate `count` problems (host array) and build a schedule: every problem
 * is cut into output tiles, the tiles are ordered longest-first and stored
 * on the device (on the tensor cores a problem with m < n <= 256 is computed
 * as C^T = B^T A^T and stored to C transposed; n <= 128 takes 256-row
 * tiles).  dt: TC_F16 or TC_BF16.  la must be TC_ROW_MAJOR; lb either.
 * Constraints: m, n, k >= 1; lda, ldb multiples of 8 and offsets of A and B
 * multiples of 8 (16-byte rows); ldc >= n.  The plan owns its device memory. */
tc_status gemm_grouped_plan_create(int32_t dt, int32_t count, const tc_problem* problems,
                                   int32_t la, int32_t lb, tc_grouped_plan** plan_out);

/* One persistent launch over every tile of the plan:
 * C_g = alpha*A_g B_g + beta*C_g for all g.  use_graph = 1 records the launch
 * in a CUDA graph on the first call and replays it while the arguments stay
 * the same.  Runs on the tensor cores (tcgen05, 128 x 256 tiles, one TMA map
 * pair per problem) for both B layouts: a row-major B_g is read as MN-major.
 * TCGEMM_GROUPED=mma selects the mma.sync kernel (64 x 64 tiles) instead. */
tc_status gemm_grouped_plan_run(tc_grouped_plan* plan, const void* a_base, const void* b_base,
                                float* c_base, float alpha, float beta, int32_t use_graph, void* stream);

/* Free the plan (synchronises with its last run). */
tc_status gemm_grouped_plan_destroy(tc_grouped_plan* plan);

/* One-shot convenience: plan, run once, destroy. */
tc_status gemm_grouped(int32_t dt, int32_t count, const tc_problem* problems,
                       const void* a_base, int32_t la, const void* b_base, int32_t lb,
                       float* c_base, float alpha, float beta, void* stream);

/* Grouped GEMM that allocates nothing.  The paper has no counterpart: this
 * entry exists for callers that may not call cudaMalloc -- code running inside
 * a memory budget owned by someone else (a framework's caching allocator or a
 * serving engine that reserved the GPU's memory up front, where a fresh
 * allocation can fail or fragment the pool), and latency-critical loops that
 * cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * Same arguments and result as gemm_grouped (host problem array, device
 * operands and outputs owned by the caller), but what the kernel reads besides
 * the operands is copied into a static device array of 8 MiB that every GPU
 * loading the library holds until the process exits: for the tcgen05 kernel
 * (the default) two TMA tensor maps per problem (256 bytes) and 48 bytes per
 * 128 x 256 output tile; for a group whose maps do not fit, or with
 * TCGEMM_GROUPED=mma, the mma.sync kernel's problem table (48 bytes per
 * problem) and 16 bytes per 64 x 64 tile.  A group that fits neither returns
 * TC_ERR_INVALID with the byte counts in tc_last_error().
 *   - The first call on a device looks up the array's device address and the
 *     status word's (cudaGetSymbolAddress, once per device, with that device
 *     current).  It changes no setting of the device or of its memory pools.
 *   - The schedule is uploaded from pageable host memory, so the call waits on
 *     the host for earlier work on `stream` before it enqueues the kernel;
 *     it does not wait for the kernel.
 *   - That upload reads host memory the call frees on return, so the call
 *     cannot be recorded in a CUDA graph: on a stream that is being captured
 *     it returns TC_ERR_UNSUPPORTED and enqueues nothing.  Use
 *     gemm_grouped_plan_run for graphs.
 *   - Every call reuses the same array, which keeps the last call's contents
 *     (nothing in it needs to start at zero).  Calls whose work overlaps on
 *     the GPU (different streams, or another thread) race on it: order them
 *     on one stream. */
tc_status gemm_grouped_noalloc(int32_t dt, int32_t count, const tc_problem* problems,
                               const void* a_base, int32_t la, const void* b_base, int32_t lb,
                               float* c_base, float alpha, float beta, void* stream);

/* The grouped GEMM of gemm_grouped_noalloc, with its problem table and tile
 * schedule in caller-owned device memory instead of the library's static
 * array: calls on different streams with different workspaces may overlap.
 *   workspace: 256-byte aligned device memory of at least
 *   gemm_grouped_workspace_bytes(count, problems) bytes, not touched by other
 *   work until this call's kernel has finished on `stream`.
 * Runs the tcgen05 kernel of gemm_grouped (maps and tiles in the workspace;
 * the mma.sync kernel with TCGEMM_GROUPED=mma); arguments and errors otherwise
 * as gemm_grouped.  Like gemm_grouped_noalloc it uploads the schedule from
 * host memory that it frees on return, so on a stream that is being captured
 * it returns TC_ERR_UNSUPPORTED and enqueues nothing.
 * gemm_grouped_workspace_bytes: a size that holds either kernel's schedule
 * under every tile setting (tall tiles on or off, transposed problems);
 * 0 for count <= 0 or a null array.  Host only. */
size_t gemm_grouped_workspace_bytes(int32_t count, const tc_problem* problems);
tc_status gemm_grouped_ws(int32_t dt, int32_t count, const tc_problem* problems,
                          const void* a_base, int32_t la, const void* b_base, int32_t lb,
                          float* c_base, float alpha, float beta,
                          void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Autotuning (the paper picked the best CUTLASS tiling per size, Sec. VI)    */
/* ------------------------------------------------------------------------ */

/* Time gemm_mixed's kernel configurations for this shape on scratch operands
 * and remember the fastest for every later call of the same shape class in
 * this process.  Candidates: 128 x 64, 128 x 128 and 128 x 256 tiles on single
 * CTAs and 256 x 256 tiles on CTA pairs (cluster of 2), then raster bands of 4,
 * 8, 16 or 32 M-tiles for the best of those; if pairs win, clusters of four
 * CTAs (two pairs sharing A by TMA multicast) with each band height, and a
 * last partial round of pair tiles kept whole (tail 0) or cut into 256 x 128
 * halves (tail 1) instead of two parts of K (tail 2); last, K walked upwards
 * in every round of tiles instead of downwards in odd rounds.  The untuned configuration (see gemm_mixed) is timed first
 * and a candidate replaces it only if more than 2 % faster.  A shape class is
 * (dt, m, n, k) with each size rounded up to a power of two.  The candidates
 * are passed to the launches explicitly: calls of other threads keep their
 * configuration until the winner is stored at the end.  Allocates and frees
 * stream-ordered scratch (cudaMallocAsync) and synchronises `stream`.
 * *best_ms (host, may be NULL) receives the winner's time.  TCGEMM_TILE,
 * TCGEMM_BN, TCGEMM_GROUP_M, TCGEMM_PAIR_TAIL, TCGEMM_K_ORDER and
 * TCGEMM_CLUSTER, when set, still override the table. */
tc_status tc_autotune_gemm(int32_t dt, int64_t m, int64_t n, int64_t k, void* stream, double* best_ms);

/* Time the variants of a grouped plan on its own operands (the tensor-core
 * path with a shared-memory-staged or a direct epilogue, and the mma.sync
 * path) and keep the fastest in the plan.  C is overwritten (alpha = 1,
 * beta = 0).  Synchronises `stream`.  A plan with row-major B has one variant. */
tc_status gemm_grouped_plan_autotune(tc_grouped_plan* plan, const void* a_base, const void* b_base, float* c_base,
                                     void* stream, double* best_ms);

/* Write / read the gemm_mixed autotune table (text, one shape class per line:
 * dt log2m log2n log2k pair group_m tail korder cluster bn ms, tail 0, 1 or 2
 * as in tc_autotune_gemm; lines without
 * the bn field are read with bn = 256, lines of the older form
 * "dt log2m log2n log2k pair group_m ms" with tail = korder = 1, cluster = 2
 * and bn = 256). */
tc_status tc_autotune_save(const char* path);
tc_status tc_autotune_load(const char* path);

/* ------------------------------------------------------------------------ */
/* Error measures (Sec. VI: e = C_half - C_single, ||e||_max; normwise
 * error ||C - C64||_F / (||A||_F ||B||_F) against an FP64 truth)           */
/* ------------------------------------------------------------------------ */

/* out[0] = sum (C - Cref)^2, out[1] = sum A^2, out[2] = sum B^2,
 * out[3] = max |C - Cref|, all accumulated in FP64 in a fixed order
 * (deterministic for the same sizes).  out is a HOST array of 4 doubles;
 * the call synchronises `stream`.
 *   C: m x n FP32 row-major (ldc).  Cref: m x n row-major (ldr), FP64 if
 *   ref_is_f64 = 1, FP32 if 0.  A: a_rows x a_cols FP32 row-major (lda);
 *   B: b_rows x b_cols FP32 row-major (ldb); either may be NULL (sum 0).
 * Uses stream-ordered scratch (cudaMallocAsync) for the partial sums. */
tc_status tc_error_norm(int64_t m, int64_t n, const float* C, int64_t ldc,
                        const void* Cref, int64_t ldr, int32_t ref_is_f64,
                        const float* A, int64_t a_rows, int64_t a_cols, int64_t lda,
                        const float* B, int64_t b_rows, int64_t b_cols, int64_t ldb,
                        double* out, void* stream);

/* The same reduction enqueued on `stream` without synchronising: the four
 * sums land in out_dev, a DEVICE array of 4 doubles (8-byte aligned), and the
 * per-block partial sums in `workspace`, caller-owned device memory of
 * tc_error_norm_workspace_bytes() bytes (8-byte aligned).  Nothing is
 * allocated; the result is bit for bit that of tc_error_norm.  Arguments and
 * errors otherwise as tc_error_norm. */
size_t tc_error_norm_workspace_bytes(void);
tc_status tc_error_norm_dev(int64_t m, int64_t n, const float* C, int64_t ldc,
                            const void* Cref, int64_t ldr, int32_t ref_is_f64,
                            const float* A, int64_t a_rows, int64_t a_cols, int64_t lda,
                            const float* B, int64_t b_rows, int64_t b_cols, int64_t ldb,
                            double* out_dev, void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of GEMM requests (beyond the paper)          */
/* ------------------------------------------------------------------------ */

#define TC_MODE_F16 0
#define TC_MODE_BF16 1
#define TC_MODE_E4M3 2
#define TC_MODE_SPLIT3 3

typedef struct tc_serve_cfg {
    int64_t hbm_budget_bytes; /* device workspace the server may hold at once */
    int32_t max_inflight;     /* requests on the GPU at once                 */
    int32_t num_streams;      /* CUDA streams the server launches on         */
    int32_t queue_capacity;   /* pending requests before serve_submit is BUSY */
    int32_t reserved;
} tc_serve_cfg;

/* One request: C = alpha*A*B + beta*C computed in `mode` from FP32 operands
 * resident on the device.  A: m x k FP32 row-major (lda), B: k x n FP32
 * row-major (ldb), C: m x n FP32 row-major (ldc).  The caller keeps A, B and
 * C alive and untouched until serve_poll reports completion. */
typedef struct tc_request {
    int32_t mode, reserved;
    int64_t m, n, k;
    const float* A; int64_t lda;
    const float* B; int64_t ldb;
    float* C; int64_t ldc;
    float alpha, beta;
} tc_request;

typedef struct tc_result {
    int32_t status, reserved;  /* TC_OK or an error of the request            */
    double t_submit_us;        /* host clock (steady, microseconds)           */
    double t_start_us;         /* admitted and launched                       */
    double t_done_us;          /* completion observed (event)                 */
} tc_result;

typedef struct tc_server tc_server;

/* Start a server on the current device: allocates the budget arena and the
 * streams, starts the scheduler thread.  The scheduler admits queued requests
 * in arrival order while the in-flight count and the budget allow, batches
 * small FP16/BF16 requests (rounding + grouped GEMM) and small E4M3 requests
 * (rounding) admitted together, runs small split-3 requests as the one-launch
 * refined GEMM, and gives each launch group the stream with the least
 * admitted, unretired tensor-core work.  A request's kernels depend only on
 * its mode, sizes and pointer alignment, so its result is bitwise the same
 * alone and in any mix. */
tc_status serve_open(const tc_serve_cfg* cfg, tc_server** out);

/* Queue a request (non-blocking).  TC_ERR_BUSY if the queue is full,
 * TC_ERR_INVALID for a malformed request or one whose workspace exceeds the
 * whole budget.  *ticket identifies it for serve_poll. */
tc_status serve_submit(tc_server* s, const tc_request* req, uint64_t* ticket);

/* TC_PENDING while the request is queued or running; otherwise fills *out
 * (if not NULL), forgets the ticket and returns TC_OK (out->status holds the
 * request's own status).  TC_ERR_INVALID for an unknown ticket. */
tc_status serve_poll(tc_server* s, uint64_t ticket, tc_result* out);

/* Block until every submitted request finished or `timeout_ms` elapsed
 * (TC_ERR_TIMEOUT). */
tc_status serve_drain(tc_server* s, int64_t timeout_ms);

/* Counters: out[0] submitted, out[1] completed, out[2] peak bytes in use,
 * out[3] peak requests in flight, out[4] times admission waited for budget. */
tc_status serve_stats(tc_server* s, int64_t* out5);

/* Where the scheduler thread's time went, cumulative since serve_open: out6 =
 * {retire ns (completion-event queries and arena release), admit ns (queue to
 * workspace, event and stream), launch ns (the library calls that enqueue the
 * kernels), launch groups (single requests and batches), event queries,
 * completed requests}.  out6: host array of 6. */
tc_status serve_timing(tc_server* s, int64_t* out6);

/* Drain, stop the scheduler, free the arena and streams. */
tc_status serve_close(tc_server* s);

#ifdef __cplusplus
}
#endif

#endif /* TCGEMM_H */
