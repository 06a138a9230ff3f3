// march.cu -- the cached ray-march kernel (Sections 3.1-3.3 and 4 of FastNeRF).
//
// One warp renders one 8 x 4 pixel tile, one lane per ray. Neighbouring rays
// sample neighbouring cells at the same depth, so one load instruction of the
// warp touches a handful of 32-byte sectors instead of 32. Per ray:
//   a1 ray generation (binary32, fixed op sequence, see fnr.h)
//   a2 direction cell: estimate from acosf/atan2f, corrected exactly against
//      the cache's binary32 boundary tables; beta (D values) kept in registers
//   a3-a5 U samples at a time: positions, cells, and U independent density
//      loads in flight before any is used
//   a6-a8 per occupied sample: the (u, v, w) record with 16-byte loads,
//      Eq. 5 + activation, Eq. 1 compositing, exact integer termination
//   a9 RGBA (+ optional per-ray counters and per-sample cells)
#include "march_device.cuh"

namespace fnr {

namespace {

using namespace dev;

template <int PREC, int D>
__global__ void __launch_bounds__(FNR_BLOCK, dev::min_blocks(PREC)) march_kernel(const __grid_constant__ MarchArgs A) {
    const int tile = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (tile >= A.total_tiles) return;  // whole warp
    int f = 0;
    while (f + 1 < A.n_frames && tile >= A.f[f + 1].tile_begin) ++f;
    const FrameDesc &F = A.f[f];
    const int t = tile - F.tile_begin;
    const int ty = t / F.tiles_x, tx = t - ty * F.tiles_x;
    const int lane = threadIdx.x & 31;
    const int px = tx * kTileW + (lane & (kTileW - 1)), py = ty * kTileH + lane / kTileW;
#if FNR_QUEUE
    __shared__ WarpQueue<D> queues[FNR_BLOCK / 32];
    march_tile_queued<PREC, D>(A.c, A.r, F, px, py, px < F.W && py < F.H, queues[threadIdx.x >> 5]);
#else
    if (px >= F.W || py >= F.H) return;
    march_ray<PREC, D>(A.c, A.r, F, px, py);
#endif
}

template <int PREC, int D>
cudaError_t launch_t(const MarchArgs &a, cudaStream_t s) {
    const int threads = FNR_BLOCK;
    const int warps_per_block = threads / 32;
    const unsigned blocks = static_cast<unsigned>((a.total_tiles + warps_per_block - 1) / warps_per_block);
    march_kernel<PREC, D><<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_p(const MarchArgs &a, cudaStream_t s) {
#ifdef FNR_TUNING_D8_ONLY  // faster builds for launch-shape sweeps: D = 8 only
    return a.c.D == 8 ? launch_t<PREC, 8>(a, s) : cudaErrorInvalidValue;
#endif
    switch (a.c.D) {
        case 1: return launch_t<PREC, 1>(a, s);
        case 2: return launch_t<PREC, 2>(a, s);
        case 3: return launch_t<PREC, 3>(a, s);
        case 4: return launch_t<PREC, 4>(a, s);
        case 5: return launch_t<PREC, 5>(a, s);
        case 6: return launch_t<PREC, 6>(a, s);
        case 7: return launch_t<PREC, 7>(a, s);
        case 8: return launch_t<PREC, 8>(a, s);
        case 9: return launch_t<PREC, 9>(a, s);
        case 10: return launch_t<PREC, 10>(a, s);
        case 11: return launch_t<PREC, 11>(a, s);
        case 12: return launch_t<PREC, 12>(a, s);
        case 13: return launch_t<PREC, 13>(a, s);
        case 14: return launch_t<PREC, 14>(a, s);
        case 15: return launch_t<PREC, 15>(a, s);
        case 16: return launch_t<PREC, 16>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_march(const MarchArgs &a, cudaStream_t s) {
    if (a.total_tiles <= 0) return cudaSuccess;
    switch (a.c.pos_prec) {
        case FNR_PREC_FP32: return launch_p<FNR_PREC_FP32>(a, s);
        case FNR_PREC_FP16: return launch_p<FNR_PREC_FP16>(a, s);
        case FNR_PREC_FP8_E4M3: return launch_p<FNR_PREC_FP8_E4M3>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fnr
