// noalloc.cu -- fnr_render_noalloc: a render entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc (or anything that does): a process whose
// device memory is owned by another allocator that has already reserved almost
// all of HBM, a render loop that must never stall on cudaMalloc / cudaFree
// (cudaFree synchronises the whole device), or a host that plans every byte of
// device memory at start-up. For them this entry point runs the persistent,
// tile-popping variant of the march kernel (the kernel the request loop uses)
// with its scratch -- the tile counter and one finished-tile counter per view
// -- in a file-scope static __device__ array instead of allocated memory. The
// views are passed to the kernel by value, so there is no table to upload.
//
// The static array: every GPU that loads this library holds these 256 bytes
// until the process exits. All calls share it and it keeps the last call's
// contents; each call clears the counters it uses (cudaMemsetAsync on its own
// stream) before its launch. Calls whose launches overlap on the GPU therefore
// race on the counters: keep such calls on one stream, or order them.
#include <string.h>

#include <mutex>

#include "march_device.cuh"

namespace fnr {

fnr_status fail(fnr_status st, const char *fmt, ...);
fnr_status cuda_fail(cudaError_t e, const char *what);
void clear_error();
fnr_status make_render_const(const fnr_render_params *p, RenderConst *rc);
fnr_status check_camera(const fnr_camera *c);
void fill_frame(FrameDesc *f, const fnr_camera *cam, float *rgba, fnr_ray_stats *stats, int32_t *cells,
                int tile_begin);
int frame_tiles(const fnr_camera *cam);
bool cache_belongs(fnr_context *ctx, const fnr_cache *c);

namespace {

constexpr int kNoAllocMaxViews = 32;     // views per call (also the kernel-parameter limit)
constexpr int kNoAllocScratchWords = 64;  // word 0: next tile; words 1..32: finished tiles per view
constexpr int kMaxDevices = 64;

static_assert(1 + kNoAllocMaxViews <= kNoAllocScratchWords, "scratch too small");
static_assert(kNoAllocMaxViews <= kMaxFramesPerLaunch, "views are passed by value");

static __device__ __align__(256) unsigned int g_noalloc_scratch[kNoAllocScratchWords];

std::mutex g_setup_mu;
int g_grid[kMaxDevices][3][17] = {};

template <int PREC, int D>
__global__ void __launch_bounds__(FNR_BLOCK, dev::min_blocks(PREC))
    noalloc_kernel(const __grid_constant__ MarchArgs A, unsigned int *scratch, uint32_t *done_words) {
    __shared__ dev::QueueFor<PREC, D> queues[FNR_BLOCK / 32];
    const int lane = threadIdx.x & 31;
    for (;;) {
        int t = 0;
        if (lane == 0) t = static_cast<int>(atomicAdd(&scratch[0], 1u));
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= A.total_tiles) break;
        int f = 0;
        while (f + 1 < A.n_frames && t >= A.f[f + 1].tile_begin) ++f;
        const FrameDesc &F = A.f[f];
        const int lt = t - F.tile_begin;
        int x0, y0;
        tile_origin(F, lt, x0, y0);
        const int px = x0 + (lane & (kTileW - 1)), py = y0 + lane / kTileW;
        dev::march_tile_queued<PREC, D, false>(A.c, A.r, F, px, py, px < F.W && py < F.H, queues[threadIdx.x >> 5]);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            const int end = f + 1 < A.n_frames ? A.f[f + 1].tile_begin : A.total_tiles;
            const unsigned prev = atomicAdd(&scratch[1 + f], 1u);
            if (done_words && prev + 1u == static_cast<unsigned>(end - F.tile_begin)) {
                __threadfence_system();
                *reinterpret_cast<volatile uint32_t *>(done_words + f) = 1u;
            }
        }
    }
}

using NoAllocFn = void (*)(MarchArgs, unsigned int *, uint32_t *);

template <int PREC>
NoAllocFn noalloc_fn_p(int D) {
    switch (D) {
        case 1: return noalloc_kernel<PREC, 1>;
        case 2: return noalloc_kernel<PREC, 2>;
        case 3: return noalloc_kernel<PREC, 3>;
        case 4: return noalloc_kernel<PREC, 4>;
        case 6: return noalloc_kernel<PREC, 6>;
        case 8: return noalloc_kernel<PREC, 8>;
        case 12: return noalloc_kernel<PREC, 12>;
        case 16: return noalloc_kernel<PREC, 16>;
        default: return nullptr;
    }
}

NoAllocFn noalloc_fn(int prec, int D) {
    switch (prec) {
        case FNR_PREC_FP32: return noalloc_fn_p<FNR_PREC_FP32>(D);
        case FNR_PREC_FP16: return noalloc_fn_p<FNR_PREC_FP16>(D);
        case FNR_PREC_FP8_E4M3: return noalloc_fn_p<FNR_PREC_FP8_E4M3>(D);
        default: return nullptr;
    }
}

}  // namespace
}  // namespace fnr

using namespace fnr;

extern "C" fnr_status fnr_render_noalloc(const fnr_cache *cache, const fnr_camera *cams, int32_t n_cams,
                                         const fnr_render_params *params, float *rgba_dev,
                                         fnr_ray_stats *stats_dev, uint32_t *done_words, fnr_stream_t stream) {
    clear_error();
    if (!cache || !cams || !rgba_dev) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    if (n_cams < 1) return fail(FNR_ERR_INVALID_ARG, "n_cams must be >= 1");
    if (n_cams > kNoAllocMaxViews)
        return fail(FNR_ERR_INVALID_ARG,
                    "fnr_render_noalloc renders at most %d views per call (its static scratch holds one counter "
                    "per view); got %d",
                    kNoAllocMaxViews, n_cams);
    fnr_context *ctx = cache->ctx;
    if (!ctx || !cache_belongs(ctx, cache)) return fail(FNR_ERR_INVALID_ARG, "unknown cache");
    const int device = ctx->device;
    if (device < 0 || device >= kMaxDevices) return fail(FNR_ERR_UNSUPPORTED, "device index %d", device);
    RenderConst rc;
    fnr_status st = make_render_const(params, &rc);
    if (st != FNR_OK) return st;
    if (cache->view.layout == FNR_LAYOUT_BRICKS)
        return fail(FNR_ERR_UNSUPPORTED, "fnr_render_noalloc reads dense caches (FNR_LAYOUT_DENSE)");
    if (rc.flags & (FNR_RENDER_SKIP_EMPTY | FNR_RENDER_VOXELS))
        return fail(FNR_ERR_UNSUPPORTED,
                    "fnr_render_noalloc renders the plain path only (no FNR_RENDER_SKIP_EMPTY or FNR_RENDER_VOXELS)");
    for (int i = 0; i < n_cams; ++i)
        if ((st = check_camera(&cams[i])) != FNR_OK) return st;
    const int prec = cache->desc.pos_precision, D = cache->desc.D;
    NoAllocFn fn = noalloc_fn(prec, D);
    if (!fn) return fail(FNR_ERR_UNSUPPORTED, "fnr_render_noalloc supports D in {1,2,3,4,6,8,12,16}, got %d", D);
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    // The device address of the static scratch, asked for on every call with the
    // device current (host code cannot use the array's name as a device
    // address). Asking again each time costs no allocation, and it stays right
    // if the caller has reset the device's primary context since the last call.
    unsigned int *scratch = nullptr;
    if ((e = cudaGetSymbolAddress(reinterpret_cast<void **>(&scratch), g_noalloc_scratch)) != cudaSuccess)
        return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    int grid = 0;
    {
        // One-time set-up per device and kernel instance, done by the first call
        // that needs it: the persistent grid size (an occupancy query).
        std::lock_guard<std::mutex> g(g_setup_mu);
        if (!g_grid[device][prec][D]) {
            int per_sm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(fn),
                                                                   FNR_BLOCK, 0)) != cudaSuccess)
                return cuda_fail(e, "occupancy query");
            g_grid[device][prec][D] = (per_sm > 0 ? per_sm : 1) * (ctx->num_sms > 0 ? ctx->num_sms : 1);
        }
        grid = g_grid[device][prec][D];
    }
    MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.c = cache->view;
    a.r = rc;
    int tiles = 0;
    int64_t pix_off = 0;
    for (int j = 0; j < n_cams; ++j) {
        fill_frame(&a.f[j], &cams[j], rgba_dev + pix_off * 4, stats_dev ? stats_dev + pix_off : nullptr, nullptr,
                   tiles);
        tiles += frame_tiles(&cams[j]);
        pix_off += int64_t(cams[j].width) * cams[j].height;
    }
    a.n_frames = n_cams;
    a.total_tiles = tiles;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the counters this call uses start at zero; the rest of the array is left as the last call left it
    if ((e = cudaMemsetAsync(scratch, 0, sizeof(unsigned int) * (1 + n_cams), s)) != cudaSuccess)
        return cuda_fail(e, "scratch clear");
    fn<<<grid, FNR_BLOCK, 0, s>>>(a, scratch, done_words);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "noalloc launch");
    return FNR_OK;
}
