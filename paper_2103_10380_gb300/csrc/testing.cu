// testing.cu -- test hooks (fnr_testing.h): failure injection and the choice
// of the cache-build kernel's form; and the one device allocation helper every
// library allocation goes through.
#include <atomic>

#include "fnr_internal.h"
#include "fnr_testing.h"

namespace fnr {

fnr_status fail(fnr_status st, const char *fmt, ...);
void clear_error();

namespace {
std::atomic<int> g_alloc_skip{0}, g_alloc_fail{0};
std::atomic<long long> g_mlp_wait_limit{0}, g_mlp_withhold{-1};
std::atomic<int> g_mlp_cta_pair{0};
}  // namespace

bool mlp_cta_pair() { return g_mlp_cta_pair.load() != 0; }

cudaError_t dev_malloc(void **p, size_t bytes) {
    if (g_alloc_fail.load() > 0) {
        if (g_alloc_skip.load() > 0) {
            g_alloc_skip.fetch_sub(1);
        } else {
            g_alloc_fail.fetch_sub(1);
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

void take_mlp_fault(long long *wait_limit, long long *withhold) {
    const long long w = g_mlp_wait_limit.exchange(0);
    const long long h = g_mlp_withhold.exchange(-1);
    if (w > 0) {
        *wait_limit = w;
        *withhold = h;
    }
}

}  // namespace fnr

using namespace fnr;

extern "C" fnr_status fnr_testing_fail_allocations(int32_t skip, int32_t count) {
    clear_error();
    if (skip < 0 || count < 0) return fail(FNR_ERR_INVALID_ARG, "negative skip or count");
    g_alloc_fail.store(0);
    g_alloc_skip.store(skip);
    g_alloc_fail.store(count);
    return FNR_OK;
}

extern "C" fnr_status fnr_testing_mlp_fault(int64_t wait_limit, int64_t withhold_chunk) {
    clear_error();
    if (wait_limit < 1) return fail(FNR_ERR_INVALID_ARG, "wait_limit must be >= 1");
    g_mlp_withhold.store(withhold_chunk);
    g_mlp_wait_limit.store(wait_limit);
    return FNR_OK;
}

extern "C" fnr_status fnr_testing_mlp_cta_pair(int32_t on) {
    clear_error();
    g_mlp_cta_pair.store(on != 0 ? 1 : 0);
    return FNR_OK;
}
