// api.cu -- libfnr's C ABI: contexts, cache build/free, plain rendering.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "fnr_internal.h"
#include "nvtx_range.h"

namespace fnr {

// The voxel walk's launcher (march_voxels.cu); r.dt carries t_far in that mode.
cudaError_t launch_march_voxels(const MarchArgs &a, cudaStream_t s);

static thread_local std::string g_last_error;

fnr_status fail(fnr_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

fnr_status cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(FNR_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(FNR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void clear_error() { g_last_error.clear(); }

size_t elem_bytes(int prec) { return prec == FNR_PREC_FP32 ? 4 : prec == FNR_PREC_FP16 ? 2 : 1; }

int rec_stride_bytes(int prec, int D) {
    const int raw = 3 * D * static_cast<int>(elem_bytes(prec));
    const int align = prec == FNR_PREC_FP8_E4M3 ? 8 : 16;
    return (raw + align - 1) / align * align;
}

static uint64_t align256(uint64_t v) { return (v + 255u) & ~uint64_t(255u); }

struct Layout {
    uint64_t off_sigma, off_uvw, off_beta, off_ct, off_qp, off_scales, off_offs, off_occ, off_dist, off_page, off_rank,
        total;
    int rec_stride;
};

// Brick side of the occupancy bits: the descriptor's, or the smallest power of
// two >= 2 with ceil(k / B) <= 64 (the bits then fit in 32 KB, which stays in L1).
int occupancy_shift(const fnr_cache_desc *d) {
    if (d->occupancy_brick > 0) {
        int sh = 0;
        while ((1 << sh) < d->occupancy_brick) ++sh;
        return sh;
    }
    int sh = 1;
    while ((d->k + (1 << sh) - 1) >> sh > 64) ++sh;
    return sh;
}

int offset_shift(int k) {
    int sh = 2;
    while ((k + (1 << sh) - 1) >> sh > 64) ++sh;
    return sh;
}

// binary16 elements per E4M3 offset brick: 3D rounded up to 8 (16-byte records)
static int offset_stride(int D) { return (3 * D + 7) / 8 * 8; }

static uint64_t offset_bytes(const fnr_cache_desc *d) {
    if (d->pos_precision != FNR_PREC_FP8_E4M3) return 0;
    const uint64_t nbo = uint64_t((d->k + (1 << offset_shift(d->k)) - 1) >> offset_shift(d->k));
    return nbo * nbo * nbo * uint64_t(offset_stride(d->D)) * 2u;
}

// Jump-brick side of the distance field: the smallest power-of-two multiple of
// the occupancy brick with ceil(k / J) <= kDistMaxDim.
int distance_shift(const fnr_cache_desc *d) {
    int sh = occupancy_shift(d);
    while ((d->k + (1 << sh) - 1) >> sh > kDistMaxDim) ++sh;
    return sh;
}

uint64_t occupancy_words(const fnr_cache_desc *d) {
    const uint64_t nb = uint64_t((d->k + (1 << occupancy_shift(d)) - 1) >> occupancy_shift(d));
    return (nb * nb * nb + 31u) / 32u;
}

static bool desc_valid(const fnr_cache_desc *d) {
    if (!d) return false;
    if (d->k < 1 || d->k > FNR_MAX_K || d->D < 1 || d->D > FNR_MAX_D || d->l < 2 || d->l > FNR_MAX_L) return false;
    if (d->pos_precision < FNR_PREC_FP32 || d->pos_precision > FNR_PREC_FP8_E4M3) return false;
    if (d->dir_precision != FNR_PREC_FP32 && d->dir_precision != FNR_PREC_FP16) return false;
    for (int a = 0; a < 3; ++a)
        if (!(isfinite(d->bmin[a]) && isfinite(d->bmax[a]) && d->bmax[a] > d->bmin[a])) return false;
    const int B = d->occupancy_brick;
    if (B < 0 || B > 256 || (B & (B - 1)) != 0) return false;
    if ((d->layout != FNR_LAYOUT_DENSE && d->layout != FNR_LAYOUT_BRICKS) || d->reserved != 0) return false;
    return true;
}

// Sections of one cache allocation. Dense: k^3 densities and records. Bricks
// (n_bricks >= 0): pools of n_bricks * B^3 densities and records, then the
// page table after the occupancy bits.
static Layout layout_of(const fnr_cache_desc *d, int64_t n_bricks = -1) {
    Layout L;
    const bool bricks = d->layout == FNR_LAYOUT_BRICKS && n_bricks >= 0;
    const int sh = occupancy_shift(d);
    const uint64_t nb = uint64_t((d->k + (1 << sh) - 1) >> sh);
    const uint64_t k3 = bricks ? uint64_t(n_bricks) << (3 * sh) : uint64_t(d->k) * d->k * d->k;
    L.rec_stride = rec_stride_bytes(d->pos_precision, d->D);
    uint64_t off = 0;
    L.off_sigma = off;
    off = align256(off + k3 * elem_bytes(d->pos_precision));
    L.off_uvw = off;
    off = align256(off + k3 * uint64_t(L.rec_stride));
    L.off_beta = off;
    off = align256(off + uint64_t(d->l) * d->l * d->D * elem_bytes(d->dir_precision));
    L.off_ct = off;
    off = align256(off + uint64_t(d->l) * 4);
    L.off_qp = off;
    off = align256(off + uint64_t(d->l) * 4);
    L.off_scales = off;
    off = align256(off + uint64_t(1 + 3 * d->D) * 4);
    L.off_offs = off;
    off = align256(off + offset_bytes(d));
    L.off_occ = off;
    off = align256(off + occupancy_words(d) * 4);
    L.off_dist = off;
    const uint64_t nj = uint64_t((d->k + (1 << distance_shift(d)) - 1) >> distance_shift(d));
    off = align256(off + nj * nj * nj);
    L.off_page = off;
    if (bricks) off = align256(off + nb * nb * nb * 4);
    L.off_rank = off;
    if (bricks) off = align256(off + occupancy_words(d) * 4);
    L.total = off;
    return L;
}

// Direction-bin boundary tables (see fnr.h): cos(j pi / l) and the azimuth key
// of the unit vector at phi_j = 2 pi j / l, both in FP64 rounded to binary32.
static double azimuth_key64(double x, double y) {
    if (x == 0.0 && y == 0.0) return 0.0;
    if (y >= 0.0) {
        if (x >= 0.0) return y / (x + y);
        return 1.0 + (-x) / (y - x);
    }
    if (x < 0.0) return 2.0 + (-y) / (-x - y);
    return 3.0 + x / (x - y);
}

static void bin_tables(int l, std::vector<float> &ct, std::vector<float> &qp) {
    const double pi = 3.14159265358979323846264338327950288;
    ct.assign(l, 1.0f);
    qp.assign(l, 0.0f);
    for (int j = 1; j < l; ++j) {
        ct[j] = static_cast<float>(cos(static_cast<double>(j) * pi / static_cast<double>(l)));
        const double ph = 2.0 * pi * static_cast<double>(j) / static_cast<double>(l);
        qp[j] = static_cast<float>(azimuth_key64(cos(ph), sin(ph)));
    }
}

bool budget_charge(fnr_context *ctx, uint64_t bytes) {
    uint64_t cur = ctx->used.load();
    for (;;) {
        if (ctx->budget && cur + bytes > ctx->budget) return false;
        if (ctx->used.compare_exchange_weak(cur, cur + bytes)) return true;
    }
}

void budget_uncharge(fnr_context *ctx, uint64_t bytes) { ctx->used.fetch_sub(bytes); }

// RAII device buffer for build-time temporaries.
struct DevBuf {
    void *p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

static fnr_status build_from_arrays(fnr_cache *c, const fnr_cache_source *src, const Layout &L, cudaStream_t s) {
    const fnr_cache_desc &d = c->desc;
    const int64_t k3 = int64_t(d.k) * d.k * d.k;
    const int nch = 3 * d.D;
    const int prec = d.pos_precision;
    char *base = static_cast<char *>(c->base);
    float *scales = reinterpret_cast<float *>(base + L.off_scales);
    cudaError_t e;
    const bool dev = src->location == FNR_LOC_DEVICE;
    // Slab size for staging host arrays (cells per slab).
    const int64_t slab = dev ? k3 : std::max<int64_t>(1, std::min<int64_t>(k3, (int64_t(256) << 20) / (4 * (nch + 1))));
    DevBuf stage;
    if (!dev) {
        if ((e = dev_malloc(&stage.p, size_t(slab) * 4 * (nch + 1))) != cudaSuccess) return cuda_fail(e, "staging");
    }
    auto slab_ptrs = [&](int64_t c0, int64_t n, const float **sp, const float **up) -> cudaError_t {
        if (dev) {
            *sp = src->sigma + c0;
            *up = src->uvw + c0 * nch;
            return cudaSuccess;
        }
        float *ss = static_cast<float *>(stage.p);
        float *uu = ss + slab;
        cudaError_t ee = cudaMemcpyAsync(ss, src->sigma + c0, size_t(n) * 4, cudaMemcpyHostToDevice, s);
        if (ee == cudaSuccess)
            ee = cudaMemcpyAsync(uu, src->uvw + c0 * nch, size_t(n) * 4 * nch, cudaMemcpyHostToDevice, s);
        *sp = ss;
        *up = uu;
        return ee;
    };
    const int osh = offset_shift(d.k), odim = (d.k + (1 << osh) - 1) >> osh, ostride = offset_stride(d.D);
    uint16_t *offs = reinterpret_cast<uint16_t *>(base + L.off_offs);
    if (prec == FNR_PREC_FP8_E4M3) {
        // (1) per offset brick and channel the min and max, then the binary16 midranges; (2) the
        // per-channel absmax of the density and of the residuals; (3) the scales
        const int64_t nbo3 = int64_t(odim) * odim * odim;
        DevBuf amax, kmm;
        if ((e = dev_malloc(&amax.p, sizeof(unsigned) * (1 + nch))) != cudaSuccess) return cuda_fail(e, "absmax");
        if ((e = dev_malloc(&kmm.p, sizeof(unsigned) * 2 * size_t(nbo3) * nch)) != cudaSuccess)
            return cuda_fail(e, "offset min / max");
        unsigned *kmin = static_cast<unsigned *>(kmm.p), *kmax = kmin + size_t(nbo3) * nch;
        if ((e = cudaMemsetAsync(amax.p, 0, sizeof(unsigned) * (1 + nch), s)) != cudaSuccess ||
            (e = cudaMemsetAsync(kmin, 0xff, sizeof(unsigned) * size_t(nbo3) * nch, s)) != cudaSuccess ||
            (e = cudaMemsetAsync(kmax, 0, sizeof(unsigned) * size_t(nbo3) * nch, s)) != cudaSuccess)
            return cuda_fail(e, "memset");
        for (int64_t c0 = 0; c0 < k3; c0 += slab) {
            const int64_t n = std::min(slab, k3 - c0);
            const float *sp, *up;
            if ((e = slab_ptrs(c0, n, &sp, &up)) != cudaSuccess) return cuda_fail(e, "upload");
            if ((e = launch_brick_minmax(up, c0, n, d.k, nch, osh, odim, kmin, kmax, s)) != cudaSuccess)
                return cuda_fail(e, "offset min / max kernel");
            if (!dev && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "min / max sync");
        }
        if ((e = launch_brick_offsets(kmin, kmax, nbo3, nch, offs, ostride, s)) != cudaSuccess)
            return cuda_fail(e, "offsets kernel");
        for (int64_t c0 = 0; c0 < k3; c0 += slab) {
            const int64_t n = std::min(slab, k3 - c0);
            const float *sp, *up;
            if ((e = slab_ptrs(c0, n, &sp, &up)) != cudaSuccess) return cuda_fail(e, "upload");
            // the density channel (and the raw absmax of the others, overwritten below)
            if ((e = launch_absmax(sp, up, n, nch, static_cast<unsigned *>(amax.p), s)) != cudaSuccess)
                return cuda_fail(e, "absmax kernel");
            if (!dev && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "absmax sync");
        }
        if ((e = cudaMemsetAsync(static_cast<unsigned *>(amax.p) + 1, 0, sizeof(unsigned) * nch, s)) != cudaSuccess)
            return cuda_fail(e, "memset");
        for (int64_t c0 = 0; c0 < k3; c0 += slab) {
            const int64_t n = std::min(slab, k3 - c0);
            const float *sp, *up;
            if ((e = slab_ptrs(c0, n, &sp, &up)) != cudaSuccess) return cuda_fail(e, "upload");
            if ((e = launch_residual_absmax(up, c0, n, d.k, nch, offs, osh, odim, ostride,
                                            static_cast<unsigned *>(amax.p), s)) != cudaSuccess)
                return cuda_fail(e, "residual absmax kernel");
            if (!dev && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "residual sync");
        }
        if ((e = launch_scales_from_absmax(static_cast<unsigned *>(amax.p), scales, 1 + nch, s)) != cudaSuccess)
            return cuda_fail(e, "scales kernel");
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "scales sync");
    }
    for (int64_t c0 = 0; c0 < k3; c0 += slab) {
        const int64_t n = std::min(slab, k3 - c0);
        const float *sp, *up;
        if ((e = slab_ptrs(c0, n, &sp, &up)) != cudaSuccess) return cuda_fail(e, "upload");
        if ((e = launch_convert_sigma(sp, base + L.off_sigma + c0 * elem_bytes(prec), n, prec, scales, s)) !=
            cudaSuccess)
            return cuda_fail(e, "density conversion");
        if ((e = launch_convert_uvw(up, base + L.off_uvw + c0 * L.rec_stride, n, d.D, prec, L.rec_stride, scales,
                                    s, offs, c0, d.k, osh, odim, ostride)) != cudaSuccess)
            return cuda_fail(e, "uvw conversion");
        if (!dev && (e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "conversion sync");
    }
    // direction cache
    const int64_t nb = int64_t(d.l) * d.l * d.D;
    const float *bp = src->beta;
    DevBuf bstage;
    if (!dev) {
        if ((e = dev_malloc(&bstage.p, size_t(nb) * 4)) != cudaSuccess) return cuda_fail(e, "beta staging");
        if ((e = cudaMemcpyAsync(bstage.p, src->beta, size_t(nb) * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
            return cuda_fail(e, "beta upload");
        bp = static_cast<const float *>(bstage.p);
    }
    if ((e = launch_convert_beta(bp, base + L.off_beta, nb, d.dir_precision, s)) != cudaSuccess)
        return cuda_fail(e, "beta conversion");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "build sync");
    return FNR_OK;
}

static void fill_view(fnr_cache *c, const Layout &L) {
    const fnr_cache_desc &d = c->desc;
    char *base = static_cast<char *>(c->base);
    CacheView &v = c->view;
    v.sigma = base + L.off_sigma;
    v.uvw = base + L.off_uvw;
    v.beta = base + L.off_beta;
    v.ct = reinterpret_cast<const float *>(base + L.off_ct);
    v.qp = reinterpret_cast<const float *>(base + L.off_qp);
    v.scales = reinterpret_cast<const float *>(base + L.off_scales);
    v.occ = reinterpret_cast<const uint32_t *>(base + L.off_occ);
    v.dist = reinterpret_cast<const uint8_t *>(base + L.off_dist);
    const bool fp8 = d.pos_precision == FNR_PREC_FP8_E4M3;
    v.offs = fp8 ? reinterpret_cast<const uint16_t *>(base + L.off_offs) : nullptr;
    v.offs_shift = fp8 ? offset_shift(d.k) : 0;
    v.offs_dim = fp8 ? (d.k + (1 << v.offs_shift) - 1) >> v.offs_shift : 0;
    v.offs_stride = fp8 ? offset_stride(d.D) : 0;
    v.layout = c->n_bricks > 0 || d.layout == FNR_LAYOUT_BRICKS ? FNR_LAYOUT_BRICKS : FNR_LAYOUT_DENSE;
    v.page = v.layout == FNR_LAYOUT_BRICKS ? reinterpret_cast<const int32_t *>(base + L.off_page) : nullptr;
    v.rank = v.layout == FNR_LAYOUT_BRICKS ? reinterpret_cast<const uint32_t *>(base + L.off_rank) : nullptr;
    v.occ_shift = occupancy_shift(&d);
    v.occ_dim = (d.k + (1 << v.occ_shift) - 1) >> v.occ_shift;
    v.dist_shift = distance_shift(&d);
    v.dist_dim = (d.k + (1 << v.dist_shift) - 1) >> v.dist_shift;
    for (int a = 0; a < 3; ++a) {
        v.bmin[a] = d.bmin[a];
        v.scale[a] = static_cast<float>(static_cast<double>(d.k) /
                                        (static_cast<double>(d.bmax[a]) - static_cast<double>(d.bmin[a])));
    }
    v.kf = static_cast<float>(d.k);
    v.k = d.k;
    v.D = d.D;
    v.l = d.l;
    v.rec_stride = L.rec_stride;
    v.pos_prec = d.pos_precision;
    v.dir_prec = d.dir_precision;
}

// Fill the render constants shared by the plain and served paths.
fnr_status make_render_const(const fnr_render_params *p, RenderConst *rc) {
    if (!p) return fail(FNR_ERR_INVALID_ARG, "params is NULL");
    if (p->n_samples < 1 || p->n_samples > FNR_MAX_SAMPLES)
        return fail(FNR_ERR_INVALID_ARG, "n_samples %d outside [1, %d]", p->n_samples, FNR_MAX_SAMPLES);
    if (!(isfinite(p->t_near) && isfinite(p->t_far) && p->t_far > p->t_near))
        return fail(FNR_ERR_INVALID_ARG, "need finite t_near < t_far");
    if (isnan(p->t_thr)) return fail(FNR_ERR_INVALID_ARG, "t_thr is NaN");
    if (p->activation != FNR_ACT_SIGMOID && p->activation != FNR_ACT_IDENTITY)
        return fail(FNR_ERR_INVALID_ARG, "unknown activation %d", p->activation);
    if ((p->flags & ~(FNR_RENDER_SKIP_EMPTY | FNR_RENDER_DIR_BILINEAR | FNR_RENDER_VOXELS)) != 0u)
        return fail(FNR_ERR_INVALID_ARG, "unknown render flags 0x%x", p->flags);
    if (p->reserved != 0) return fail(FNR_ERR_INVALID_ARG, "reserved field must be 0");
    const bool voxels = (p->flags & FNR_RENDER_VOXELS) != 0u;
    rc->N = p->n_samples;
    rc->t_near = p->t_near;
    // uniform samples: Delta; the voxel walk has no spacing and reads t_far from this field instead
    rc->dt = voxels ? p->t_far : (p->t_far - p->t_near) / static_cast<float>(p->n_samples);
    if (!voxels && !(rc->dt > 0.0f)) return fail(FNR_ERR_INVALID_ARG, "sample spacing underflows");
    rc->act = p->activation;
    if (!(p->t_thr > 0.0f)) {
        rc->s_thr = 0x7fffffffffffffffLL;
    } else {
        // optical depth: Delta sum sigma (threshold divided by Delta) or, for the walk, sum sigma delta
        const double per = voxels ? 1.0 : static_cast<double>(rc->dt);
        const double v = ceil(log(1.0 / static_cast<double>(p->t_thr)) / per * 4294967296.0);
        rc->s_thr = v >= 9223372036854775807.0 ? 0x7fffffffffffffffLL : (v < 0.0 ? 0 : static_cast<long long>(v));
    }
    for (int c = 0; c < 3; ++c) rc->bg[c] = p->bg[c];
    rc->flags = p->flags;
    return FNR_OK;
}

fnr_status check_camera(const fnr_camera *c) {
    if (c->width < 1 || c->height < 1 || c->width > FNR_MAX_IMAGE_SIDE || c->height > FNR_MAX_IMAGE_SIDE)
        return fail(FNR_ERR_INVALID_ARG, "image size %dx%d outside [1, %d]", c->width, c->height, FNR_MAX_IMAGE_SIDE);
    for (int i = 0; i < 12; ++i)
        if (!isfinite(c->c2w[i])) return fail(FNR_ERR_INVALID_ARG, "non-finite c2w");
    if (!(isfinite(c->fx) && isfinite(c->fy) && c->fx != 0.0f && c->fy != 0.0f && isfinite(c->cx) && isfinite(c->cy)))
        return fail(FNR_ERR_INVALID_ARG, "bad intrinsics");
    return FNR_OK;
}

void fill_frame(FrameDesc *f, const fnr_camera *cam, float *rgba, fnr_ray_stats *stats, int32_t *cells,
                int tile_begin) {
    memcpy(f->c2w, cam->c2w, sizeof(f->c2w));
    f->fx = cam->fx;
    f->fy = cam->fy;
    f->cx = cam->cx;
    f->cy = cam->cy;
    f->W = cam->width;
    f->H = cam->height;
    f->tiles_x = (cam->width + kTileW - 1) / kTileW;
    if (FNR_TILE_2X2) f->tiles_x = (f->tiles_x + 1) / 2;  // groups of 2 x 2 tiles per row
    f->tile_begin = tile_begin;
    f->rgba = rgba;
    f->stats = stats;
    f->cells = cells;
}

int frame_tiles(const fnr_camera *cam) {
    const int tx = (cam->width + kTileW - 1) / kTileW, ty = (cam->height + kTileH - 1) / kTileH;
    if (FNR_TILE_2X2) return 4 * ((tx + 1) / 2) * ((ty + 1) / 2);
    return tx * ty;
}

bool cache_belongs(fnr_context *ctx, const fnr_cache *c) {
    std::lock_guard<std::mutex> g(ctx->mu);
    return ctx->caches.count(const_cast<fnr_cache *>(c)) != 0;
}

}  // namespace fnr

using namespace fnr;

extern "C" {

const char *fnr_last_error(void) { return g_last_error.c_str(); }

fnr_status fnr_context_create(int32_t device, uint64_t hbm_budget_bytes, fnr_context **out) {
    clear_error();
    if (!out) return fail(FNR_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(FNR_ERR_INVALID_ARG, "device %d not in [0, %d)", device, n);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    fnr_context *ctx = new fnr_context();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    *out = ctx;
    return FNR_OK;
}

fnr_status fnr_context_destroy(fnr_context *ctx) {
    clear_error();
    if (!ctx) return FNR_OK;
    {
        std::lock_guard<std::mutex> g(ctx->serve_mu);
        server_stop(ctx);  // drains queued and in-flight requests
    }
    cudaSetDevice(ctx->device);
    std::set<fnr_cache *> cs;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        cs.swap(ctx->caches);
    }
    for (fnr_cache *c : cs) {
        if (c->owned && c->base) cudaFree(c->base);
        delete c;
    }
    delete ctx;
    return FNR_OK;
}

uint64_t fnr_context_used_bytes(const fnr_context *ctx) { return ctx ? ctx->used.load() : 0; }

uint64_t fnr_cache_bytes(const fnr_cache_desc *d) {
    if (!desc_valid(d)) return 0;
    const uint64_t k3 = uint64_t(d->k) * d->k * d->k;
    const uint64_t s_sigma = elem_bytes(d->pos_precision) * 8u;
    const uint64_t s_uvw = 3u * elem_bytes(d->pos_precision) * 8u;
    const uint64_t s_beta = elem_bytes(d->dir_precision) * 8u;
    uint64_t bits = (uint64_t(d->D) * s_uvw + s_sigma) * k3 + uint64_t(d->D) * s_beta * d->l * d->l;
    uint64_t bytes = bits / 8u;
    if (d->pos_precision == FNR_PREC_FP8_E4M3) {
        const uint64_t nbo = uint64_t((d->k + (1 << offset_shift(d->k)) - 1) >> offset_shift(d->k));
        bytes += uint64_t(1 + 3 * d->D) * 4u + nbo * nbo * nbo * uint64_t(3 * d->D) * 2u;
    }
    return bytes;
}

uint64_t fnr_cache_footprint(const fnr_cache_desc *d) {
    if (!desc_valid(d)) return 0;
    return layout_of(d).total;
}

// Dense cache -> FNR_LAYOUT_BRICKS cache: pool slots in brick-index order of
// the occupied bricks, densities and records gathered brick by brick on the
// GPU; the direction cache, tables, scales and occupancy bits are copied.
static fnr_status make_bricks(fnr_context *ctx, const fnr_cache *dense, const fnr_cache_desc *desc,
                              cudaStream_t s, fnr_cache **out) {
    const CacheView &dv = dense->view;
    const int64_t nb = dv.occ_dim, nb3 = nb * nb * nb;
    std::vector<uint32_t> words(occupancy_words(desc));
    cudaError_t e;
    if ((e = cudaMemcpyAsync(words.data(), dv.occ, words.size() * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "occupancy read-back");
    std::vector<int32_t> page(size_t(nb3), -1), slot_brick;
    std::vector<uint32_t> rank(words.size());
    for (int64_t b = 0; b < nb3; ++b) {
        if ((b & 31) == 0) rank[size_t(b >> 5)] = uint32_t(slot_brick.size());
        if ((words[size_t(b >> 5)] >> (b & 31)) & 1u) {
            page[size_t(b)] = int32_t(slot_brick.size());
            slot_brick.push_back(int32_t(b));
        }
    }
    const int64_t n_bricks = int64_t(slot_brick.size());
    const Layout L = layout_of(desc, n_bricks);
    const Layout LD = layout_of(&dense->desc);
    if (!budget_charge(ctx, L.total))
        return fail(FNR_ERR_BUDGET, "brick cache needs %llu bytes, budget %llu, in use %llu",
                    (unsigned long long)L.total, (unsigned long long)ctx->budget,
                    (unsigned long long)ctx->used.load());
    fnr_cache *c = new fnr_cache();
    c->desc = *desc;
    c->footprint = L.total;
    c->n_bricks = uint64_t(n_bricks);
    c->ctx = ctx;
    if ((e = dev_malloc(&c->base, L.total)) != cudaSuccess) {
        budget_uncharge(ctx, L.total);
        delete c;
        return cuda_fail(e, "brick cache allocation");
    }
    char *base = static_cast<char *>(c->base);
    const char *dbase = static_cast<const char *>(dense->base);
    DevBuf slots;
    fnr_status st = FNR_OK;
    if (n_bricks > 0 && (e = dev_malloc(&slots.p, size_t(n_bricks) * 4)) != cudaSuccess) st = cuda_fail(e, "slots");
    if (st == FNR_OK &&
        ((n_bricks > 0 && (e = cudaMemcpyAsync(slots.p, slot_brick.data(), size_t(n_bricks) * 4,
                                               cudaMemcpyHostToDevice, s)) != cudaSuccess) ||
         (e = cudaMemcpyAsync(base + L.off_page, page.data(), size_t(nb3) * 4, cudaMemcpyHostToDevice, s)) !=
             cudaSuccess ||
         (e = cudaMemcpyAsync(base + L.off_rank, rank.data(), rank.size() * 4, cudaMemcpyHostToDevice, s)) !=
             cudaSuccess ||
         (e = cudaMemcpyAsync(base + L.off_beta, dbase + LD.off_beta, L.off_page - L.off_beta,
                              cudaMemcpyDeviceToDevice, s)) != cudaSuccess))
        st = cuda_fail(e, "brick cache tables");
    // (beta, the bin tables, the scales, the occupancy bits and the brick distances keep their
    // relative offsets)
    if (st == FNR_OK && n_bricks > 0 &&
        (e = launch_gather_bricks(dv.sigma, dv.uvw, base + L.off_sigma, base + L.off_uvw,
                                  static_cast<const int32_t *>(slots.p), n_bricks, desc->k, dv.occ_shift,
                                  dv.occ_dim, int(elem_bytes(desc->pos_precision)), L.rec_stride, s)) != cudaSuccess)
        st = cuda_fail(e, "brick gather");
    if (st == FNR_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "brick cache sync");
    if (st != FNR_OK) {
        cudaFree(c->base);
        budget_uncharge(ctx, L.total);
        delete c;
        return st;
    }
    fill_view(c, L);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->caches.insert(c);
    }
    *out = c;
    return FNR_OK;
}

fnr_status fnr_build_cache(fnr_context *ctx, const fnr_cache_desc *desc, const fnr_cache_source *src,
                           fnr_stream_t stream, fnr_cache **out) {
    clear_error();
    NvtxRange range("fnr_build_cache");
    if (!ctx || !desc || !src || !out) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (!desc_valid(desc)) return fail(FNR_ERR_INVALID_ARG, "invalid cache descriptor");
    if (desc->layout == FNR_LAYOUT_BRICKS) {  // through a dense cache, freed afterwards
        fnr_cache_desc dd = *desc;
        dd.layout = FNR_LAYOUT_DENSE;
        fnr_cache *dense = nullptr;
        fnr_status st = fnr_build_cache(ctx, &dd, src, stream, &dense);
        if (st != FNR_OK) return st;
        st = make_bricks(ctx, dense, desc, reinterpret_cast<cudaStream_t>(stream), out);
        std::string msg = st != FNR_OK ? std::string(fnr_last_error()) : std::string();
        fnr_cache_free(ctx, dense);
        if (st != FNR_OK) return fail(st, "%s", msg.c_str());
        return FNR_OK;
    }
    fnr_status st0;
    if (src->kind == FNR_SRC_MLP) {
        if ((st0 = check_mlp(src->pos_mlp, 1 + 3 * desc->D, "pos_mlp")) != FNR_OK) return st0;
        if ((st0 = check_mlp(src->dir_mlp, desc->D, "dir_mlp")) != FNR_OK) return st0;
        if (desc->pos_precision == FNR_PREC_FP8_E4M3)
            return fail(FNR_ERR_UNSUPPORTED, "MLP builds write FP32 or FP16 caches (build FP8 from arrays)");
    } else if (src->kind == FNR_SRC_ARRAYS) {
        if (!src->sigma || !src->uvw || !src->beta) return fail(FNR_ERR_INVALID_ARG, "NULL source array");
        if (src->location != FNR_LOC_HOST && src->location != FNR_LOC_DEVICE)
            return fail(FNR_ERR_INVALID_ARG, "unknown source location");
    } else {
        return fail(FNR_ERR_INVALID_ARG, "unknown source kind %d", src->kind);
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    const Layout L = layout_of(desc);
    if (!budget_charge(ctx, L.total))
        return fail(FNR_ERR_BUDGET, "cache needs %llu bytes, budget %llu, in use %llu", (unsigned long long)L.total,
                    (unsigned long long)ctx->budget, (unsigned long long)ctx->used.load());
    fnr_cache *c = new fnr_cache();
    c->desc = *desc;
    c->footprint = L.total;
    c->ctx = ctx;
    if ((e = dev_malloc(&c->base, L.total)) != cudaSuccess) {
        budget_uncharge(ctx, L.total);
        delete c;
        return cuda_fail(e, "cache allocation");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<float> ct, qp;
    bin_tables(desc->l, ct, qp);
    char *base = static_cast<char *>(c->base);
    fnr_status st = FNR_OK;
    if ((e = cudaMemcpyAsync(base + L.off_ct, ct.data(), ct.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(base + L.off_qp, qp.data(), qp.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) {
        st = cuda_fail(e, "table upload");
    }
    if (st == FNR_OK && desc->pos_precision != FNR_PREC_FP8_E4M3) {
        // scales unused: keep them defined (1.0)
        std::vector<float> ones(1 + 3 * desc->D, 1.0f);
        if ((e = cudaMemcpyAsync(base + L.off_scales, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
            st = cuda_fail(e, "scale upload");
        if (st == FNR_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "sync");
    }
    if (st == FNR_OK) {
        if (src->kind == FNR_SRC_ARRAYS) {
            st = build_from_arrays(c, src, L, s);
        } else {
            fill_view(c, L);
            st = run_mlp(src->pos_mlp, 0, c->desc, c->view, ctx->num_sms, s);
            if (st == FNR_OK) st = run_mlp(src->dir_mlp, 1, c->desc, c->view, ctx->num_sms, s);
        }
    }
    if (st == FNR_OK) {
        // brick occupancy bits from the stored densities
        fill_view(c, L);
        if ((e = cudaMemsetAsync(base + L.off_occ, 0, occupancy_words(desc) * 4, s)) != cudaSuccess ||
            (e = launch_occupancy(c->view, reinterpret_cast<uint32_t *>(base + L.off_occ), s)) != cudaSuccess ||
            (e = launch_brick_distance(reinterpret_cast<const uint32_t *>(base + L.off_occ), c->view.occ_dim,
                                       c->view.occ_shift, reinterpret_cast<uint8_t *>(base + L.off_dist),
                                       c->view.dist_dim, c->view.dist_shift, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            st = cuda_fail(e, "occupancy bits");
    }
    if (st != FNR_OK) {
        cudaFree(c->base);
        budget_uncharge(ctx, L.total);
        delete c;
        return st;
    }
    fill_view(c, L);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->caches.insert(c);
    }
    *out = c;
    return FNR_OK;
}

fnr_status fnr_cache_free(fnr_context *ctx, fnr_cache *c) {
    clear_error();
    if (!ctx || !c) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!ctx->caches.count(c)) return fail(FNR_ERR_INVALID_ARG, "cache does not belong to this context");
        if (c->inflight.load() != 0) return fail(FNR_ERR_INVALID_ARG, "cache is referenced by in-flight requests");
        ctx->caches.erase(c);
    }
    cudaSetDevice(ctx->device);
    if (c->owned && c->base) cudaFree(c->base);
    budget_uncharge(ctx, c->footprint);
    delete c;
    return FNR_OK;
}

// ---------------------------------------------------------------- save / load
namespace {
constexpr char kFileMagic[8] = {'F', 'N', 'R', 'C', 'A', 'C', 'H', 'E'};
constexpr uint32_t kFileVersion = 2;  // 2: the brick distance field follows the occupancy bits
struct FileHeader {
    char magic[8];
    uint32_t version;
    uint32_t header_bytes;
    fnr_cache_desc desc;
    uint64_t footprint;
    uint64_t n_bricks;  // FNR_LAYOUT_BRICKS: bricks in the pools
};
constexpr size_t kStageBytes = size_t(64) << 20;  // pinned staging buffer

struct PinnedBuf {
    void *p = nullptr;
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
};
struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};
}  // namespace

fnr_status fnr_cache_save(const fnr_cache *c, const char *path) {
    clear_error();
    NvtxRange range("fnr_cache_save");
    if (!c || !path) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = cudaSetDevice(c->ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "synchronise before save");
    FileHeader h;
    memset(&h, 0, sizeof(h));
    memcpy(h.magic, kFileMagic, 8);
    h.version = kFileVersion;
    h.header_bytes = sizeof(FileHeader);
    h.desc = c->desc;
    h.footprint = c->footprint;
    h.n_bricks = c->n_bricks;
    File F;
    if (!(F.f = fopen(path, "wb"))) return fail(FNR_ERR_IO, "cannot open %s for writing", path);
    if (fwrite(&h, sizeof(h), 1, F.f) != 1) return fail(FNR_ERR_IO, "write failed: %s", path);
    PinnedBuf buf;
    if ((e = cudaMallocHost(&buf.p, kStageBytes)) != cudaSuccess) return cuda_fail(e, "staging buffer");
    const char *src = static_cast<const char *>(c->base);
    for (uint64_t off = 0; off < c->footprint; off += kStageBytes) {
        const size_t n = size_t(std::min<uint64_t>(kStageBytes, c->footprint - off));
        if ((e = cudaMemcpy(buf.p, src + off, n, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return cuda_fail(e, "cache read-back");
        if (fwrite(buf.p, 1, n, F.f) != n) return fail(FNR_ERR_IO, "write failed: %s", path);
    }
    if (fflush(F.f) != 0) return fail(FNR_ERR_IO, "write failed: %s", path);
    return FNR_OK;
}

fnr_status fnr_cache_load(fnr_context *ctx, const char *path, fnr_stream_t stream, fnr_cache **out) {
    clear_error();
    NvtxRange range("fnr_cache_load");
    if (!ctx || !path || !out) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    File F;
    if (!(F.f = fopen(path, "rb"))) return fail(FNR_ERR_IO, "cannot open %s", path);
    FileHeader h;
    if (fread(&h, sizeof(h), 1, F.f) != 1) return fail(FNR_ERR_IO, "%s: truncated header", path);
    if (memcmp(h.magic, kFileMagic, 8) != 0) return fail(FNR_ERR_IO, "%s is not a cache file", path);
    if (h.version != kFileVersion || h.header_bytes != sizeof(FileHeader))
        return fail(FNR_ERR_IO, "%s: format version %u is not supported", path, h.version);
    if (!desc_valid(&h.desc)) return fail(FNR_ERR_IO, "%s: invalid cache descriptor", path);
    const bool bricks = h.desc.layout == FNR_LAYOUT_BRICKS;
    if (bricks && h.n_bricks > (uint64_t(h.desc.k) * h.desc.k * h.desc.k))
        return fail(FNR_ERR_IO, "%s: brick count out of range", path);
    const Layout L = layout_of(&h.desc, bricks ? int64_t(h.n_bricks) : -1);
    if (h.footprint != L.total)
        return fail(FNR_ERR_IO, "%s: footprint %llu does not match the descriptor's %llu", path,
                    (unsigned long long)h.footprint, (unsigned long long)L.total);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    if (!budget_charge(ctx, L.total))
        return fail(FNR_ERR_BUDGET, "cache needs %llu bytes, budget %llu, in use %llu", (unsigned long long)L.total,
                    (unsigned long long)ctx->budget, (unsigned long long)ctx->used.load());
    fnr_cache *c = new fnr_cache();
    c->desc = h.desc;
    c->footprint = L.total;
    c->n_bricks = bricks ? h.n_bricks : 0;
    c->ctx = ctx;
    fnr_status st = FNR_OK;
    if ((e = dev_malloc(&c->base, L.total)) != cudaSuccess) {
        budget_uncharge(ctx, L.total);
        delete c;
        return cuda_fail(e, "cache allocation");
    }
    {
        cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
        PinnedBuf buf;
        if ((e = cudaMallocHost(&buf.p, kStageBytes)) != cudaSuccess) st = cuda_fail(e, "staging buffer");
        char *dst = static_cast<char *>(c->base);
        for (uint64_t off = 0; st == FNR_OK && off < L.total; off += kStageBytes) {
            const size_t n = size_t(std::min<uint64_t>(kStageBytes, L.total - off));
            if (fread(buf.p, 1, n, F.f) != n) {
                st = fail(FNR_ERR_IO, "%s: truncated payload", path);
                break;
            }
            if ((e = cudaMemcpyAsync(dst + off, buf.p, n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                (e = cudaStreamSynchronize(s)) != cudaSuccess)  // the staging buffer is reused
                st = cuda_fail(e, "cache upload");
        }
    }
    if (st != FNR_OK) {
        cudaFree(c->base);
        budget_uncharge(ctx, L.total);
        delete c;
        return st;
    }
    fill_view(c, L);
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        ctx->caches.insert(c);
    }
    *out = c;
    return FNR_OK;
}

fnr_status fnr_cache_get_layout(const fnr_cache *c, fnr_cache_layout *out) {
    clear_error();
    if (!c || !out) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    const CacheView &v = c->view;
    out->sigma_dev = v.sigma;
    out->uvw_dev = v.uvw;
    out->beta_dev = v.beta;
    out->scales_dev = c->desc.pos_precision == FNR_PREC_FP8_E4M3 ? v.scales : nullptr;
    out->cos_theta_dev = v.ct;
    out->phi_key_dev = v.qp;
    out->occupancy_dev = v.occ;
    out->record_stride = v.rec_stride;
    out->occupancy_brick = 1 << v.occ_shift;
    out->layout = v.layout;
    out->reserved1 = 0;
    out->page_table_dev = v.page;
    out->brick_distance_dev = v.dist;
    out->distance_brick = 1 << v.dist_shift;
    out->reserved2 = 0;
    out->offsets_dev = v.offs;
    out->offset_brick = v.offs ? 1 << v.offs_shift : 0;
    out->offset_stride = v.offs ? v.offs_stride : 0;
    out->n_bricks = c->n_bricks;
    out->footprint = c->footprint;
    return FNR_OK;
}

fnr_status fnr_render(fnr_context *ctx, const fnr_cache *cache, const fnr_camera *cams, int32_t n_cams,
                      const fnr_render_params *params, float *rgba_dev, fnr_ray_stats *stats_dev,
                      int32_t *debug_cells_dev, fnr_stream_t stream) {
    clear_error();
    NvtxRange range("fnr_render");
    if (!ctx || !cache || !cams || !rgba_dev) return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    if (n_cams < 1) return fail(FNR_ERR_INVALID_ARG, "n_cams must be >= 1");
    if (!cache_belongs(ctx, cache)) return fail(FNR_ERR_INVALID_ARG, "cache does not belong to this context");
    RenderConst rc;
    fnr_status st = make_render_const(params, &rc);
    if (st != FNR_OK) return st;
    if ((rc.flags & FNR_RENDER_VOXELS) && cache->view.layout != FNR_LAYOUT_DENSE)
        return fail(FNR_ERR_UNSUPPORTED, "the voxel walk reads dense caches only");
    for (int i = 0; i < n_cams; ++i)
        if ((st = check_camera(&cams[i])) != FNR_OK) return st;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    MarchArgs a;
    memset(&a, 0, sizeof(a));
    a.c = cache->view;
    a.r = rc;
    int64_t pix_off = 0;
    for (int f0 = 0; f0 < n_cams; f0 += kMaxFramesPerLaunch) {
        const int nf = std::min(kMaxFramesPerLaunch, n_cams - f0);
        int tiles = 0;
        for (int j = 0; j < nf; ++j) {
            const fnr_camera *cam = &cams[f0 + j];
            fill_frame(&a.f[j], cam, rgba_dev + pix_off * 4, stats_dev ? stats_dev + pix_off : nullptr,
                       debug_cells_dev ? debug_cells_dev + pix_off * rc.N : nullptr, tiles);
            tiles += frame_tiles(cam);
            pix_off += int64_t(cam->width) * cam->height;
        }
        a.n_frames = nf;
        a.total_tiles = tiles;
        if ((e = (rc.flags & FNR_RENDER_VOXELS) ? launch_march_voxels(a, s) : launch_march(a, s)) != cudaSuccess)
            return cuda_fail(e, "march launch");
    }
    return FNR_OK;
}

}  // extern "C"
