// fnr_internal.h -- structures shared by libfnr's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <set>
#include <string>

#include "fnr.h"

namespace fnr {

// Read-only view of one cache's device data, passed to kernels by value.
struct CacheView {
    const void *sigma;    // [k^3] stored density
    const char *uvw;      // [k^3] records, rec_stride bytes apart
    const void *beta;     // [l*l][D] stored weights
    const float *ct;      // [l] cos(theta_j) boundaries
    const float *qp;      // [l] azimuth-key boundaries
    const float *scales;  // FP8: [1 + 3D]
    const uint16_t *offs; // FP8: binary16 (u, v, w) offsets, [offs_dim^3][offs_stride]
    const uint32_t *occ;  // brick occupancy bits, brick (bz * occ_dim + by) * occ_dim + bx
    const int32_t *page;  // FNR_LAYOUT_BRICKS: brick -> pool slot (-1 empty); sigma / uvw are the pools
    const uint32_t *rank; // FNR_LAYOUT_BRICKS: set occupancy bits in the words before each word
    const uint8_t *dist;  // per jump brick: Chebyshev distance (jump bricks) to the nearest occupied one,
                          // capped at kDistCap + 1
    int32_t occ_shift;    // log2 of the brick side in cells
    int32_t occ_dim;      // bricks per axis, ceil(k / 2^occ_shift)
    int32_t offs_shift;   // FP8: log2 of the offset-brick side in cells
    int32_t offs_dim;     // FP8: offset bricks per axis
    int32_t offs_stride;  // FP8: binary16 elements per offset brick (3D rounded up to 8)
    int32_t dist_shift;   // log2 of the jump-brick side in cells (>= occ_shift)
    int32_t dist_dim;     // jump bricks per axis, ceil(k / 2^dist_shift) <= kDistMaxDim
    int32_t layout;       // FNR_LAYOUT_*
    float bmin[3];
    float scale[3];       // binary32(k / (bmax - bmin)) per axis
    float kf;             // (float)k
    int32_t k, D, l;
    int32_t rec_stride;   // bytes
    int32_t pos_prec, dir_prec;
};

// Per-launch constants of one render request.
struct RenderConst {
    int32_t N;
    float t_near;
    float dt;             // Delta, binary32
    int32_t act;
    long long s_thr;      // termination threshold on the fixed-point optical depth
    float bg[3];
    uint32_t flags;       // FNR_RENDER_* bits
};

// One view inside a launch. Tiles are kTileW x kTileH pixels (8 x 4), one warp each.
struct FrameDesc {
    float c2w[12];
    float fx, fy, cx, cy;
    int32_t W, H;
    int32_t tiles_x;
    int32_t tile_begin;   // first launch-global tile of this frame
    float *rgba;          // [H*W][4]
    fnr_ray_stats *stats; // [H*W] or null
    int32_t *cells;       // [H*W][N] or null
};

#ifndef FNR_TILE_W
#define FNR_TILE_W 8
#endif
constexpr int kTileW = FNR_TILE_W, kTileH = 32 / FNR_TILE_W;  // one warp per tile, one lane per pixel
static_assert(kTileW * kTileH == 32 && (kTileW & (kTileW - 1)) == 0, "a tile is one warp");
// FNR_TILE_2X2: tiles numbered in 2 x 2 groups (the four warps of a block
// render a compact 2 x 2 patch of tiles) instead of row-major over the frame
#ifndef FNR_TILE_2X2
#define FNR_TILE_2X2 1
#endif
constexpr int kMaxFramesPerLaunch = 32;

// Top-left pixel of frame tile t (tiles_x: tiles per row, or 2 x 2 groups per row).
__host__ __device__ inline void tile_origin(const FrameDesc &F, int t, int &x0, int &y0) {
#if FNR_TILE_2X2
    const int g = t >> 2, w = t & 3;
    const int gy = g / F.tiles_x, gx = g - gy * F.tiles_x;
    x0 = (2 * gx + (w & 1)) * kTileW;
    y0 = (2 * gy + (w >> 1)) * kTileH;
#else
    const int ty = t / F.tiles_x, tx = t - ty * F.tiles_x;
    x0 = tx * kTileW;
    y0 = ty * kTileH;
#endif
}

struct MarchArgs {
    CacheView c;
    RenderConst r;
    int32_t n_frames;
    int32_t total_tiles;
    FrameDesc f[kMaxFramesPerLaunch];
};

// Host-side helpers shared by the API and the kernels' launchers.
// Every device allocation of the library goes through dev_malloc (testing.cu),
// so the failure-injection hook of fnr_testing.h reaches all of them.
cudaError_t dev_malloc(void **p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T **p, size_t bytes) {
    return dev_malloc(reinterpret_cast<void **>(p), bytes);
}
// The armed cache-build fault (fnr_testing_mlp_fault), taken once: leaves the
// arguments unchanged when none is armed.
void take_mlp_fault(long long *wait_limit, long long *withhold);
// Whether cache builds use the CTA-pair form of the tensor-core kernel
// (fnr_testing_mlp_cta_pair); the single-CTA form otherwise.
bool mlp_cta_pair();
int rec_stride_bytes(int prec, int D);
size_t elem_bytes(int prec);

// Launchers (march.cu / quant.cu). Return cudaError_t of the launch.
cudaError_t launch_march(const MarchArgs &a, cudaStream_t s);
// Dense cache -> brick pools: pool slot s holds brick slot_brick[s] (k^3 grid, bricks of 2^shift cells).
cudaError_t launch_gather_bricks(const void *sigma, const char *uvw, void *sigma_pool, char *uvw_pool,
                                 const int32_t *slot_brick, int64_t n_bricks, int k, int shift, int dim,
                                 int s_sigma, int rec_stride, cudaStream_t s);
cudaError_t launch_convert_sigma(const float *in, void *out, int64_t n, int prec, const float *scale,
                                 cudaStream_t s);
cudaError_t launch_convert_uvw(const float *in, char *out, int64_t n_cells, int D, int prec, int rec_stride,
                               const float *scales, cudaStream_t s, const uint16_t *offs = nullptr,
                               int64_t c0 = 0, int k = 0, int oshift = 0, int odim = 0, int ostride = 0);
// E4M3 (u, v, w) offsets: the smallest power of two >= 4 with ceil(k / Bo) <= 64, as a shift.
int offset_shift(int k);
// Per offset brick and channel: running min / max of a slab of cells c0 .. c0 + n (order-preserving
// uint keys; initialise with 0xffffffff / 0), then the binary16 midranges.
cudaError_t launch_brick_minmax(const float *uvw, int64_t c0, int64_t n, int k, int nch, int oshift, int odim,
                                unsigned *kmin, unsigned *kmax, cudaStream_t s);
cudaError_t launch_brick_offsets(const unsigned *kmin, const unsigned *kmax, int64_t n_bricks, int nch,
                                 uint16_t *offs, int ostride, cudaStream_t s);
// Per-channel absmax of the residuals from the offsets (atomicMax on the bits of |r|, amax_bits[1 + c]).
cudaError_t launch_residual_absmax(const float *uvw, int64_t c0, int64_t n, int k, int nch, const uint16_t *offs,
                                   int oshift, int odim, int ostride, unsigned *amax_bits, cudaStream_t s);
cudaError_t launch_convert_beta(const float *in, void *out, int64_t n, int prec, cudaStream_t s);
cudaError_t launch_absmax(const float *sigma, const float *uvw, int64_t n_cells, int nch, unsigned *amax_bits,
                          cudaStream_t s);
// Brick occupancy bits from a stored density plane (words must be zeroed first).
cudaError_t launch_occupancy(const CacheView &v, uint32_t *words, cudaStream_t s);
int occupancy_shift(const fnr_cache_desc *d);
uint64_t occupancy_words(const fnr_cache_desc *d);
// Distance field for passing over empty space: the Chebyshev distance transform of the occupancy
// at jump-brick resolution (2^dist_shift cells, at most kDistMaxDim jump bricks per axis, so the
// field is at most 32 KB and stays in L1); distances above kDistCap read kDistCap + 1.
constexpr int kDistCap = 15;
constexpr int kDistMaxDim = 32;
int distance_shift(const fnr_cache_desc *d);
cudaError_t launch_brick_distance(const uint32_t *words, int nb, int occ_shift, uint8_t *dist, int nj,
                                  int dist_shift, cudaStream_t s);
cudaError_t launch_scales_from_absmax(const unsigned *amax_bits, float *scales, int n, cudaStream_t s);

struct Server;
void server_stop(fnr_context *ctx);

// mlp.cu: tensor-core evaluation of F_pos (mode 0) / F_dir (mode 1) into a cache.
fnr_status check_mlp(const fnr_mlp *m, int n_out_min, const char *name);
fnr_status run_mlp_points(const fnr_mlp *m, const float *points, long long n, float *out, int out_stride,
                          bool relu0, int num_sms, cudaStream_t s);
fnr_status run_mlp(const fnr_mlp *m, int mode, const fnr_cache_desc &d, const CacheView &v, int num_sms,
                   cudaStream_t s);

}  // namespace fnr

struct fnr_cache {
    fnr_cache_desc desc;
    void *base = nullptr;
    bool owned = true;
    uint64_t footprint = 0;
    uint64_t n_bricks = 0;  // FNR_LAYOUT_BRICKS: bricks in the pools
    fnr::CacheView view;
    std::atomic<int> inflight{0};
    fnr_context *ctx = nullptr;
};

struct fnr_context {
    int device = 0;
    int num_sms = 0;
    uint64_t budget = 0;
    std::atomic<uint64_t> used{0};
    std::mutex mu;
    std::set<fnr_cache *> caches;
    std::mutex serve_mu;
    fnr::Server *server = nullptr;
};
