/*
 * tcgemm failure-injection hook (test use only; no counterpart in the paper).
 *
 * The tensor-core GEMM kernels bound every wait on an mbarrier (2 s of
 * %globaltimer); a wait that runs out records TC_ERR_TIMEOUT in the device
 * status word, stops the CTA (and its CTA-pair peer), waits for the copies and
 * MMAs it already issued, frees its TMEM and returns.  This hook makes that
 * path run without any fault: it is the "flag that nothing sets".
 */
#ifndef TCGEMM_DEBUG_H
#define TCGEMM_DEBUG_H

#include <stdint.h>

#include "tcgemm.h"

#ifdef __cplusplus
extern "C" {
#endif

/* The next gemm_mixed or gemm_split call made by this thread launches its
 * kernel with the TMA producer of the first CTA (pair) withholding k-block
 * `k_block` of its first tile: the MMA issuer then waits on a barrier that
 * nothing completes, gives up after the time limit and the call's stream
 * reports TC_ERR_TIMEOUT through tc_sync_status().  k_block < 0 clears a
 * pending request.  Returns TC_OK. */
tc_status tc_debug_stall_next_gemm(int32_t k_block);

#ifdef __cplusplus
}
#endif

#endif /* TCGEMM_DEBUG_H */
