// uncached.cu -- the uncached FastNeRF render: F_pos at every sample inside the
// box and F_dir per ray, evaluated by the tensor-core MLP kernel (mlp.cu), then
// composited with Eq. 5 and Eq. 1 exactly as the cached march does.
//
//   samples_kernel: per ray, the inside samples' positions into one compact
//     list (a warp-aggregated atomic hands each ray its range) and the ray's
//     unit direction;
//   F_pos over the list, F_dir over the directions (run_mlp_points);
//   composite_kernel: per ray, beta from F_dir, then the samples in order:
//     sigma and (u, v, w) from F_pos, Eq. 5 + activation, Eq. 1 and the exact
//     integer termination; RGBA and counters.
#include "march_device.cuh"
#include "nvtx_range.h"

namespace fnr {

fnr_status fail(fnr_status st, const char *fmt, ...);
fnr_status cuda_fail(cudaError_t e, const char *what);
void clear_error();
fnr_status make_render_const(const fnr_render_params *p, RenderConst *rc);
fnr_status check_camera(const fnr_camera *c);
void fill_frame(FrameDesc *f, const fnr_camera *cam, float *rgba, fnr_ray_stats *stats, int32_t *cells,
                int tile_begin);
bool budget_charge(fnr_context *ctx, uint64_t bytes);
void budget_uncharge(fnr_context *ctx, uint64_t bytes);

namespace {

struct Ray {
    float d[3], o[3];
};

// a1 with the same binary32 sequence as the cached march
__device__ __forceinline__ Ray make_ray(const FrameDesc &F, int px, int py) {
    Ray r;
    const float dcx = __fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(px), 0.5f), F.cx), F.fx);
    const float dcy = -__fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(py), 0.5f), F.cy), F.fy);
    const float wx = __fmaf_rn(F.c2w[0], dcx, __fmaf_rn(F.c2w[1], dcy, -F.c2w[2]));
    const float wy = __fmaf_rn(F.c2w[4], dcx, __fmaf_rn(F.c2w[5], dcy, -F.c2w[6]));
    const float wz = __fmaf_rn(F.c2w[8], dcx, __fmaf_rn(F.c2w[9], dcy, -F.c2w[10]));
    const float n2 = __fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz)));
    const float len = __fsqrt_rn(n2);
    r.d[0] = __fdiv_rn(wx, len);
    r.d[1] = __fdiv_rn(wy, len);
    r.d[2] = __fdiv_rn(wz, len);
    r.o[0] = F.c2w[3];
    r.o[1] = F.c2w[7];
    r.o[2] = F.c2w[11];
    return r;
}

struct Box {
    float lo[3], hi[3];
};

// sample i of the ray: position and whether it is inside the box
__device__ __forceinline__ bool sample_at(const Ray &r, const RenderConst &rc, const Box &b, int i, float p[3]) {
    const float t = __fmaf_rn(__fadd_rn(static_cast<float>(i), 0.5f), rc.dt, rc.t_near);
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = __fmaf_rn(t, r.d[a], r.o[a]);
        in = in && p[a] >= b.lo[a] && p[a] < b.hi[a];
    }
    return in;
}

__global__ void samples_kernel(const FrameDesc F, const RenderConst rc, const Box b, float *points,
                               unsigned long long *total, long long *offset, int *count, float *dirs) {
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    const int n_rays = F.W * F.H;
    const bool active = ray < n_rays;
    Ray r;
    int n = 0;
    if (active) {
        r = make_ray(F, ray % F.W, ray / F.W);
        float p[3];
        for (int i = 0; i < rc.N; ++i) n += sample_at(r, rc, b, i, p) ? 1 : 0;
    }
    // one atomic per warp for the warp's rays
    const unsigned full = __activemask();
    int incl = n;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        const int v = __shfl_up_sync(full, incl, dd);
        if (lane >= dd) incl += v;
    }
    const int last = 31 - __clz(full);
    unsigned long long base = 0;
    if (lane == last) base = atomicAdd(total, static_cast<unsigned long long>(incl));
    base = __shfl_sync(full, base, last);
    if (!active) return;
    const long long off = static_cast<long long>(base) + incl - n;
    offset[ray] = off;
    count[ray] = n;
    dirs[3 * ray] = r.d[0];
    dirs[3 * ray + 1] = r.d[1];
    dirs[3 * ray + 2] = r.d[2];
    long long j = off;
    float p[3];
    for (int i = 0; i < rc.N; ++i)
        if (sample_at(r, rc, b, i, p)) {
            points[3 * j] = p[0];
            points[3 * j + 1] = p[1];
            points[3 * j + 2] = p[2];
            ++j;
        }
}

template <int D>
__global__ void composite_kernel(const FrameDesc F, const RenderConst rc, const Box b, const float *pos_out,
                                 const float *dir_out, const long long *offset) {
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= F.W * F.H) return;
    const Ray r = make_ray(F, ray % F.W, ray / F.W);
    float beta[D];
#pragma unroll
    for (int i = 0; i < D; ++i) beta[i] = dir_out[static_cast<long long>(ray) * D + i];
    float T = 1.0f, C[3] = {0.0f, 0.0f, 0.0f};
    long long S = 0;
    int n_look = 0, n_occ = 0, n_steps = rc.N;
    long long j = offset[ray];
    float p[3];
    for (int i = 0; i < rc.N; ++i) {
        if (!sample_at(r, rc, b, i, p)) continue;
        const float *o = pos_out + j * (1 + 3 * D);
        ++j;
        ++n_look;
        const float sg = o[0];
        if (!(sg > 0.0f)) continue;
        ++n_occ;
        float col[3];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {  // Eq. 5, each channel's sum in order j = 0 .. D-1
            float x = 0.0f;
#pragma unroll
            for (int k = 0; k < D; ++k) x = __fmaf_rn(beta[k], o[1 + ch * D + k], x);
            col[ch] = rc.act == FNR_ACT_IDENTITY ? x : __fdividef(1.0f, 1.0f + __expf(-x));
        }
        float ext, alpha;
        dev::extinction(__fmul_rn(sg, rc.dt), ext, alpha);
        const float w = T * alpha;
        C[0] = __fmaf_rn(w, col[0], C[0]);
        C[1] = __fmaf_rn(w, col[1], C[1]);
        C[2] = __fmaf_rn(w, col[2], C[2]);
        T = T * ext;
        const long long qd = dev::fixed_depth(sg);
        S = (S > 0x7fffffffffffffffLL - qd) ? 0x7fffffffffffffffLL : S + qd;
        if (S >= rc.s_thr) {
            n_steps = i + 1;
            break;
        }
    }
    float4 out;
    out.x = __fmaf_rn(T, rc.bg[0], C[0]);
    out.y = __fmaf_rn(T, rc.bg[1], C[1]);
    out.z = __fmaf_rn(T, rc.bg[2], C[2]);
    out.w = 1.0f - T;
    reinterpret_cast<float4 *>(F.rgba)[ray] = out;
    if (F.stats) reinterpret_cast<int4 *>(F.stats)[ray] = make_int4(n_steps, n_look, n_occ, -1);
}

template <int D>
cudaError_t launch_composite(const FrameDesc &F, const RenderConst &rc, const Box &b, const float *pos_out,
                             const float *dir_out, const long long *offset, cudaStream_t s) {
    const int n = F.W * F.H;
    composite_kernel<D><<<(n + 127) / 128, 128, 0, s>>>(F, rc, b, pos_out, dir_out, offset);
    return cudaGetLastError();
}

cudaError_t composite(int D, const FrameDesc &F, const RenderConst &rc, const Box &b, const float *pos_out,
                      const float *dir_out, const long long *offset, cudaStream_t s) {
    switch (D) {
        case 1: return launch_composite<1>(F, rc, b, pos_out, dir_out, offset, s);
        case 2: return launch_composite<2>(F, rc, b, pos_out, dir_out, offset, s);
        case 4: return launch_composite<4>(F, rc, b, pos_out, dir_out, offset, s);
        case 6: return launch_composite<6>(F, rc, b, pos_out, dir_out, offset, s);
        case 8: return launch_composite<8>(F, rc, b, pos_out, dir_out, offset, s);
        case 16: return launch_composite<16>(F, rc, b, pos_out, dir_out, offset, s);
        default: return cudaErrorInvalidValue;
    }
}

struct DevMem {
    void *p = nullptr;
    ~DevMem() {
        if (p) cudaFree(p);
    }
};

}  // namespace

}  // namespace fnr

using namespace fnr;

extern "C" fnr_status fnr_render_mlp(fnr_context *ctx, const fnr_mlp *pos_mlp, const fnr_mlp *dir_mlp, int32_t D,
                                     const float *bmin, const float *bmax, const fnr_camera *cam,
                                     const fnr_render_params *params, float *rgba_dev, fnr_ray_stats *stats_dev,
                                     fnr_stream_t stream) {
    clear_error();
    NvtxRange range("fnr_render_mlp");
    if (!ctx || !pos_mlp || !dir_mlp || !bmin || !bmax || !cam || !rgba_dev)
        return fail(FNR_ERR_INVALID_ARG, "NULL argument");
    if (D != 1 && D != 2 && D != 4 && D != 6 && D != 8 && D != 16)
        return fail(FNR_ERR_UNSUPPORTED, "the uncached render supports D in {1,2,4,6,8,16}, got %d", D);
    fnr_status st;
    if ((st = check_mlp(pos_mlp, 1 + 3 * D, "pos_mlp")) != FNR_OK) return st;
    if ((st = check_mlp(dir_mlp, D, "dir_mlp")) != FNR_OK) return st;
    Box b;
    for (int a = 0; a < 3; ++a) {
        if (!(isfinite(bmin[a]) && isfinite(bmax[a]) && bmax[a] > bmin[a]))
            return fail(FNR_ERR_INVALID_ARG, "invalid box");
        b.lo[a] = bmin[a];
        b.hi[a] = bmax[a];
    }
    RenderConst rc;
    if ((st = make_render_const(params, &rc)) != FNR_OK) return st;
    if (rc.flags != 0u) return fail(FNR_ERR_UNSUPPORTED, "the uncached render takes no render flags");
    if ((st = check_camera(cam)) != FNR_OK) return st;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    FrameDesc F;
    fill_frame(&F, cam, rgba_dev, stats_dev, nullptr, 0);
    const long long n_rays = static_cast<long long>(cam->width) * cam->height;
    // temporaries: the sample list is sized for every sample (the worst case), the rest per ray
    const long long max_pts = n_rays * rc.N;
    const uint64_t bytes = uint64_t(max_pts) * (3 + 1 + 3 * D) * 4 + uint64_t(n_rays) * (8 + 4 + 12 + 4 * D) + 8;
    if (!budget_charge(ctx, bytes))
        return fail(FNR_ERR_BUDGET, "the uncached render needs %llu bytes of temporaries",
                    (unsigned long long)bytes);
    DevMem points, pos_out, dirs, dir_out, offset, count, total;
    st = FNR_OK;
    if ((e = dev_malloc(&points.p, size_t(max_pts) * 12)) != cudaSuccess ||
        (e = dev_malloc(&pos_out.p, size_t(max_pts) * (1 + 3 * D) * 4)) != cudaSuccess ||
        (e = dev_malloc(&dirs.p, size_t(n_rays) * 12)) != cudaSuccess ||
        (e = dev_malloc(&dir_out.p, size_t(n_rays) * D * 4)) != cudaSuccess ||
        (e = dev_malloc(&offset.p, size_t(n_rays) * 8)) != cudaSuccess ||
        (e = dev_malloc(&count.p, size_t(n_rays) * 4)) != cudaSuccess ||
        (e = dev_malloc(&total.p, 8)) != cudaSuccess)
        st = cuda_fail(e, "uncached render temporaries");
    unsigned long long n_pts = 0;
    if (st == FNR_OK) {
        if ((e = cudaMemsetAsync(total.p, 0, 8, s)) != cudaSuccess) st = cuda_fail(e, "memset");
    }
    if (st == FNR_OK) {
        samples_kernel<<<unsigned((n_rays + 127) / 128), 128, 0, s>>>(
            F, rc, b, static_cast<float *>(points.p), static_cast<unsigned long long *>(total.p),
            static_cast<long long *>(offset.p), static_cast<int *>(count.p), static_cast<float *>(dirs.p));
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(&n_pts, total.p, 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            st = cuda_fail(e, "sample positions");
    }
    if (st == FNR_OK)
        st = run_mlp_points(pos_mlp, static_cast<const float *>(points.p), (long long)n_pts,
                            static_cast<float *>(pos_out.p), 1 + 3 * D, true, ctx->num_sms, s);
    if (st == FNR_OK)
        st = run_mlp_points(dir_mlp, static_cast<const float *>(dirs.p), n_rays, static_cast<float *>(dir_out.p), D,
                            false, ctx->num_sms, s);
    if (st == FNR_OK) {
        if ((e = composite(D, F, rc, b, static_cast<const float *>(pos_out.p), static_cast<const float *>(dir_out.p),
                           static_cast<const long long *>(offset.p), s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            st = cuda_fail(e, "uncached composite");
    }
    budget_uncharge(ctx, bytes);
    return st;
}
