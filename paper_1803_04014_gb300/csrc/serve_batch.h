// Internal entry of the serving loop (not part of the C ABI).
#pragma once

#include "tcgemm.h"

namespace tcgserve {

// tc_quantize_batch of `jobs` followed by gemm_grouped_ws of `problems` (A and B row-major at
// offsets from ab_base, C at offsets from c_base), with both schedules uploaded from host memory in
// one copy into `desc` (256-byte aligned device memory of desc_bytes, free once the kernels have run
// on `stream`).  The same kernels and results as the two calls.
tc_status round_and_grouped_ws(int32_t dt, int32_t njobs, const tc_quantize_job* jobs, int32_t count,
                               const tc_problem* problems, const void* ab_base, float* c_base, float alpha,
                               float beta, void* desc, size_t desc_bytes, void* stream);

}  // namespace tcgserve
