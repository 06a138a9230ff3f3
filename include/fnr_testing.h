/*
 * fnr_testing.h -- failure-injection hooks of libfnr, for tests only.
 *
 * The paper has no counterpart to these calls. They let a test make the
 * library's error paths run without faulting a GPU: a device allocation that
 * fails, and a bounded wait inside the tensor-core cache-build kernel that runs
 * out. Production code never calls them; with no hook armed the library
 * behaves exactly as without them. Hooks are process-wide and not
 * thread-safe against concurrent builds: arm one, run the call under test,
 * and check its status.
 */
#ifndef FNR_TESTING_H
#define FNR_TESTING_H

#include "fnr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Device allocations made by the library (caches, staging, MLP weights,
 * scratch): the next `skip` succeed, the `count` after them fail as if the
 * device were out of memory (the calling entry point returns FNR_ERR_OOM and
 * releases whatever it had allocated and charged to the budget). count = 0
 * disarms the hook. Errors: INVALID_ARG for negative arguments. */
FNR_API fnr_status fnr_testing_fail_allocations(int32_t skip, int32_t count);

/* Arms a fault for the next tensor-core cache-build launch (fnr_build_cache
 * with FNR_SRC_MLP, or fnr_render_mlp): every mbarrier wait in the kernel
 * gives up after wait_limit polls (instead of 2^22), and, if withhold_chunk is
 * >= 0, each CTA's weight producer withholds that chunk (counted from 0 in
 * the CTA's stream of 64-column weight chunks), so the MMA issuer's wait for
 * it runs out. The kernel then sets its error word, drains the copies and
 * tensor-core operations it has in flight, frees its tensor memory and
 * returns; the entry point returns FNR_ERR_DEVICE and releases the cache. The
 * hook disarms itself after one launch. Errors: INVALID_ARG for
 * wait_limit < 1. */
FNR_API fnr_status fnr_testing_mlp_fault(int64_t wait_limit, int64_t withhold_chunk);

#ifdef __cplusplus
}
#endif
#endif /* FNR_TESTING_H */
