/*
 * fnr_testing.h -- test hooks of libfnr, for tests only.
 *
 * The paper has no counterpart to these calls. Two of them let a test make the
 * library's error paths run without faulting a GPU: a device allocation that
 * fails, and a bounded wait inside the tensor-core cache-build kernel that runs
 * out. The third selects an alternative form of that kernel so that a test can
 * check it against the default one. Production code never calls them; with no
 * hook armed the library behaves exactly as without them. Hooks are
 * process-wide and not thread-safe against concurrent builds: arm one, run the
 * call under test, and check its status.
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

/* Selects the form of the tensor-core cache-build kernel for the builds that
 * follow (fnr_build_cache with FNR_SRC_MLP, fnr_render_mlp), until called
 * again: on != 0 the CTA-pair form -- clusters of two CTAs on an SM pair, M =
 * 256 MMAs issued for both (tcgen05 cta_group::2), each SM holding half of every
 * weight chunk; on = 0 (the default) the single-CTA form, M = 128 per SM. Both
 * compute the same products in the same order: their caches are bit-identical.
 * The pair form measured slower on the 512^3 build. Never fails. */
FNR_API fnr_status fnr_testing_mlp_cta_pair(int32_t on);

#ifdef __cplusplus
}
#endif
#endif /* FNR_TESTING_H */
