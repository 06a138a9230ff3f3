// march.cu -- the cached ray-march kernel (Sections 3.1-3.3 and 4 of FastNeRF).
//
// One warp renders one 8 x 4 pixel tile, one lane per ray. Neighbouring rays
// sample neighbouring cells at the same depth, so one load instruction of the
// warp touches a handful of 32-byte sectors instead of 32. Per ray:
//   a1 ray generation (binary32, fixed op sequence, see fnr.h)
//   a2 direction cell: a count of passed bin boundaries against the cache's
//      binary32 tables; beta (D values) staged in shared memory for the warp
//   a3-a5 U samples at a time: positions, cells, and U independent density
//      loads in flight before any is used
//   a6-a8 occupied samples queued per warp and shaded 32 at a time: the
//      (u, v, w) record with 16-byte loads, Eq. 5 + activation, Eq. 1
//      compositing in sample order, exact integer termination
//   a9 RGBA (+ optional per-ray counters and per-sample cells)
//
// The kernels for FNR_RENDER_SKIP_EMPTY (density loads only in occupied
// bricks) and for FNR_LAYOUT_BRICKS caches are the same template with SKIP
// (and BRICKS) set, compiled in march_skip.cu / march_bricks.cu so the kernel
// sets build in parallel.
#include "march_device.cuh"

namespace fnr {

namespace {

using namespace dev;

template <int PREC, int D, bool SKIP, bool BRICKS>
__global__ void __launch_bounds__(FNR_BLOCK, dev::min_blocks(PREC)) march_kernel(const __grid_constant__ MarchArgs A) {
    allow_next_grid();  // the next render launch may be scheduled as SMs free up
    const int tile = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (tile >= A.total_tiles) return;  // whole warp
    int f = 0;
    while (f + 1 < A.n_frames && tile >= A.f[f + 1].tile_begin) ++f;
    const FrameDesc &F = A.f[f];
    const int t = tile - F.tile_begin;
    int x0, y0;
    tile_origin(F, t, x0, y0);
    const int lane = threadIdx.x & 31;
    const int px = x0 + (lane & (kTileW - 1)), py = y0 + lane / kTileW;
    __shared__ QueueFor<PREC, D> queues[FNR_BLOCK / 32];
    march_tile_queued<PREC, D, SKIP, BRICKS>(A.c, A.r, F, px, py, px < F.W && py < F.H, queues[threadIdx.x >> 5]);
}

template <int PREC, int D, bool SKIP, bool BRICKS>
cudaError_t launch_t(const MarchArgs &a, cudaStream_t s) {
    const int threads = FNR_BLOCK;
    const int warps_per_block = threads / 32;
    const unsigned blocks = static_cast<unsigned>((a.total_tiles + warps_per_block - 1) / warps_per_block);
    // programmatic stream serialization: overlaps this launch's start with the
    // previous render launch's tail (see wait_prior_grid)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, march_kernel<PREC, D, SKIP, BRICKS>, a);
}

template <int PREC, bool SKIP, bool BRICKS>
cudaError_t launch_p(const MarchArgs &a, cudaStream_t s) {
#ifdef FNR_TUNING_D8_ONLY  // faster builds for launch-shape sweeps: D = 8 only
    return a.c.D == 8 ? launch_t<PREC, 8, SKIP, BRICKS>(a, s) : cudaErrorInvalidValue;
#endif
    switch (a.c.D) {
        case 1: return launch_t<PREC, 1, SKIP, BRICKS>(a, s);
        case 2: return launch_t<PREC, 2, SKIP, BRICKS>(a, s);
        case 3: return launch_t<PREC, 3, SKIP, BRICKS>(a, s);
        case 4: return launch_t<PREC, 4, SKIP, BRICKS>(a, s);
        case 5: return launch_t<PREC, 5, SKIP, BRICKS>(a, s);
        case 6: return launch_t<PREC, 6, SKIP, BRICKS>(a, s);
        case 7: return launch_t<PREC, 7, SKIP, BRICKS>(a, s);
        case 8: return launch_t<PREC, 8, SKIP, BRICKS>(a, s);
        case 9: return launch_t<PREC, 9, SKIP, BRICKS>(a, s);
        case 10: return launch_t<PREC, 10, SKIP, BRICKS>(a, s);
        case 11: return launch_t<PREC, 11, SKIP, BRICKS>(a, s);
        case 12: return launch_t<PREC, 12, SKIP, BRICKS>(a, s);
        case 13: return launch_t<PREC, 13, SKIP, BRICKS>(a, s);
        case 14: return launch_t<PREC, 14, SKIP, BRICKS>(a, s);
        case 15: return launch_t<PREC, 15, SKIP, BRICKS>(a, s);
        case 16: return launch_t<PREC, 16, SKIP, BRICKS>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <bool SKIP, bool BRICKS>
cudaError_t launch_all(const MarchArgs &a, cudaStream_t s) {
    switch (a.c.pos_prec) {
        case FNR_PREC_FP32: return launch_p<FNR_PREC_FP32, SKIP, BRICKS>(a, s);
        case FNR_PREC_FP16: return launch_p<FNR_PREC_FP16, SKIP, BRICKS>(a, s);
        case FNR_PREC_FP8_E4M3: return launch_p<FNR_PREC_FP8_E4M3, SKIP, BRICKS>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

#if defined(FNR_MARCH_SKIP_UNIT)
cudaError_t launch_march_skip(const MarchArgs &a, cudaStream_t s) { return launch_all<true, false>(a, s); }
#elif defined(FNR_MARCH_BRICKS_UNIT)
cudaError_t launch_march_bricks(const MarchArgs &a, cudaStream_t s) { return launch_all<true, true>(a, s); }
#else
cudaError_t launch_march_skip(const MarchArgs &a, cudaStream_t s);    // march_skip.cu
cudaError_t launch_march_bricks(const MarchArgs &a, cudaStream_t s);  // march_bricks.cu

cudaError_t launch_march(const MarchArgs &a, cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    if (a.c.layout == FNR_LAYOUT_BRICKS) return launch_march_bricks(a, s);  // always skipping
    if (a.r.flags & FNR_RENDER_SKIP_EMPTY) return launch_march_skip(a, s);
    return launch_all<false, false>(a, s);
}
#endif

}  // namespace fnr
