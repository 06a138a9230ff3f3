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
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "fnr_internal.h"

namespace fnr {

namespace {

constexpr int kUnroll = 4;  // density loads in flight per lane

__device__ __forceinline__ float e4m3_to_float(unsigned int byte) {
    __half_raw h = __nv_cvt_fp8_to_halfraw(static_cast<__nv_fp8_storage_t>(byte), __NV_E4M3);
    return __half2float(__half(h));
}

template <int PREC, int D>
struct Record;

template <int D>
struct Record<FNR_PREC_FP32, D> {
    static constexpr int NV = (3 * D + 3) / 4;
    float4 v[NV];
    __device__ __forceinline__ void load(const char *p) {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = __ldg(reinterpret_cast<const float4 *>(p) + j);
    }
    __device__ __forceinline__ float get(int i) const {
        const float4 &q = v[i >> 2];
        return (i & 3) == 0 ? q.x : (i & 3) == 1 ? q.y : (i & 3) == 2 ? q.z : q.w;
    }
};

template <int D>
struct Record<FNR_PREC_FP16, D> {
    static constexpr int NV = (6 * D + 15) / 16;
    uint4 v[NV];
    __device__ __forceinline__ void load(const char *p) {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = __ldg(reinterpret_cast<const uint4 *>(p) + j);
    }
    __device__ __forceinline__ float get(int i) const {
        const uint4 &q = v[i >> 3];
        const int w = (i >> 1) & 3;
        unsigned int word = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
        unsigned short bits = static_cast<unsigned short>((i & 1) ? (word >> 16) : (word & 0xffffu));
        return __half2float(__ushort_as_half(bits));
    }
};

template <int D>
struct Record<FNR_PREC_FP8_E4M3, D> {
    static constexpr int NV = (3 * D + 7) / 8;
    uint2 v[NV];
    __device__ __forceinline__ void load(const char *p) {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = __ldg(reinterpret_cast<const uint2 *>(p) + j);
    }
    __device__ __forceinline__ float get(int i) const {
        const uint2 &q = v[i >> 3];
        unsigned int word = ((i >> 2) & 1) ? q.y : q.x;
        return e4m3_to_float((word >> (8 * (i & 3))) & 0xffu);
    }
};

template <int PREC>
__device__ __forceinline__ float load_sigma(const CacheView &c, long long cell, float sigma_scale) {
    if constexpr (PREC == FNR_PREC_FP32) {
        return __ldg(static_cast<const float *>(c.sigma) + cell);
    } else if constexpr (PREC == FNR_PREC_FP16) {
        return __half2float(__ldg(static_cast<const __half *>(c.sigma) + cell));
    } else {
        unsigned int q = __ldg(static_cast<const unsigned char *>(c.sigma) + cell);
        return __fmul_rn(e4m3_to_float(q), sigma_scale);  // binary32 dequantisation
    }
}

__device__ __forceinline__ long long fixed_depth(float s) {
    if (!(s > 0.0f)) return 0;
    if (s >= 2147483648.0f) return 0x7fffffffffffffffLL;
    return static_cast<long long>(floorf(__fmul_rn(s, 4294967296.0f)));
}

// Azimuth key in [0, 4], monotone in atan2(y, x) wrapped to [0, 2 pi).
__device__ __forceinline__ float phi_key(float x, float y) {
    if (x == 0.0f && y == 0.0f) return 0.0f;
    if (y >= 0.0f) {
        if (x >= 0.0f) return __fdiv_rn(y, __fadd_rn(x, y));
        return __fadd_rn(1.0f, __fdiv_rn(-x, __fadd_rn(y, -x)));
    }
    if (x < 0.0f) return __fadd_rn(2.0f, __fdiv_rn(-y, __fadd_rn(-x, -y)));
    return __fadd_rn(3.0f, __fdiv_rn(x, __fadd_rn(x, -y)));
}

// Direction cell: counts of boundaries passed; the libm estimate only picks
// where the exact walk over the (monotone) tables starts.
__device__ __forceinline__ int dir_cell(const CacheView &c, float dx, float dy, float dz) {
    const int l = c.l;
    const float inv_pi = 0.318309886183790671538f;
    int it = static_cast<int>(acosf(fminf(fmaxf(dz, -1.0f), 1.0f)) * inv_pi * static_cast<float>(l));
    it = min(max(it, 0), l - 1);
    while (it < l - 1 && dz <= __ldg(c.ct + it + 1)) ++it;
    while (it > 0 && dz > __ldg(c.ct + it)) --it;
    float ph = atan2f(dy, dx);
    if (ph < 0.0f) ph += 6.28318530717958647692f;
    int ip = static_cast<int>(ph * (0.5f * inv_pi) * static_cast<float>(l));
    ip = min(max(ip, 0), l - 1);
    const float q = phi_key(dx, dy);
    while (ip < l - 1 && q >= __ldg(c.qp + ip + 1)) ++ip;
    while (ip > 0 && q < __ldg(c.qp + ip)) --ip;
    return it * l + ip;
}

template <int PREC, int D>
__device__ __forceinline__ void march_ray(const CacheView &c, const RenderConst &r, const FrameDesc &F, int px,
                                          int py) {
    constexpr int NB = (PREC == FNR_PREC_FP8_E4M3) ? 3 * D : D;
    // a1: ray (binary32, fixed sequence)
    const float dcx = __fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(px), 0.5f), F.cx), F.fx);
    const float dcy = -__fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(py), 0.5f), F.cy), F.fy);
    const float wx = __fmaf_rn(F.c2w[0], dcx, __fmaf_rn(F.c2w[1], dcy, -F.c2w[2]));
    const float wy = __fmaf_rn(F.c2w[4], dcx, __fmaf_rn(F.c2w[5], dcy, -F.c2w[6]));
    const float wz = __fmaf_rn(F.c2w[8], dcx, __fmaf_rn(F.c2w[9], dcy, -F.c2w[10]));
    const float n2 = __fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz)));
    const float len = __fsqrt_rn(n2);
    const float dx = __fdiv_rn(wx, len), dy = __fdiv_rn(wy, len), dz = __fdiv_rn(wz, len);
    const float ox = F.c2w[3], oy = F.c2w[7], oz = F.c2w[11];

    // a2: direction cell and beta
    const int dcell = dir_cell(c, dx, dy, dz);
    float bw[NB];
    if constexpr (PREC == FNR_PREC_FP8_E4M3) {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            float b = c.dir_prec == FNR_PREC_FP16
                          ? __half2float(__ldg(static_cast<const __half *>(c.beta) + (long long)dcell * D + i))
                          : __ldg(static_cast<const float *>(c.beta) + (long long)dcell * D + i);
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) bw[ch * D + i] = b * __ldg(c.scales + 1 + ch * D + i);
        }
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i)
            bw[i] = c.dir_prec == FNR_PREC_FP16
                        ? __half2float(__ldg(static_cast<const __half *>(c.beta) + (long long)dcell * D + i))
                        : __ldg(static_cast<const float *>(c.beta) + (long long)dcell * D + i);
    }
    const float sigma_scale = (PREC == FNR_PREC_FP8_E4M3) ? __ldg(c.scales) : 1.0f;

    float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    long long S = 0;
    int n_look = 0, n_occ = 0, n_steps = r.N;
    const long long k = c.k;
    const long long pix = static_cast<long long>(py) * F.W + px;
    int32_t *cells_out = F.cells ? F.cells + pix * r.N : nullptr;
    bool done = false;

    for (int i0 = 0; i0 < r.N && !done; i0 += kUnroll) {
        long long cell[kUnroll];
        float sg[kUnroll];
        // a3, a4: sample positions and cells
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u;
            const float t = __fmaf_rn(__fadd_rn(static_cast<float>(i), 0.5f), r.dt, r.t_near);
            const float gx = __fmul_rn(__fsub_rn(__fmaf_rn(t, dx, ox), c.bmin[0]), c.scale[0]);
            const float gy = __fmul_rn(__fsub_rn(__fmaf_rn(t, dy, oy), c.bmin[1]), c.scale[1]);
            const float gz = __fmul_rn(__fsub_rn(__fmaf_rn(t, dz, oz), c.bmin[2]), c.scale[2]);
            const bool in = i < r.N && gx >= 0.0f && gx < c.kf && gy >= 0.0f && gy < c.kf && gz >= 0.0f &&
                            gz < c.kf;
            cell[u] = in ? (static_cast<long long>(floorf(gz)) * k + static_cast<long long>(floorf(gy))) * k +
                               static_cast<long long>(floorf(gx))
                         : -1;
        }
        // a5: all density loads of the group issued before any is consumed
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) sg[u] = cell[u] >= 0 ? load_sigma<PREC>(c, cell[u], sigma_scale) : 0.0f;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            const int i = i0 + u;
            if (i >= r.N) break;
            if (cells_out) cells_out[i] = cell[u] >= 0 ? static_cast<int32_t>(cell[u]) : -1;
            if (cell[u] < 0) continue;
            ++n_look;
            const float s = sg[u];
            if (!(s > 0.0f)) continue;
            ++n_occ;
            // a6: (u, v, w) record
            Record<PREC, D> rec;
            rec.load(c.uvw + cell[u] * c.rec_stride);
            // a7: Eq. 5 and the activation
            float col[3];
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                float x = 0.0f;
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    const float b = (PREC == FNR_PREC_FP8_E4M3) ? bw[ch * D + j] : bw[j];
                    x = __fmaf_rn(b, rec.get(ch * D + j), x);
                }
                col[ch] = r.act == FNR_ACT_IDENTITY ? x : 1.0f / (1.0f + expf(-x));
            }
            // a8: Eq. 1 and exact termination
            const float od = __fmul_rn(s, r.dt);
            const float alpha = -expm1f(-od);
            const float w = T * alpha;
            Cr = __fmaf_rn(w, col[0], Cr);
            Cg = __fmaf_rn(w, col[1], Cg);
            Cb = __fmaf_rn(w, col[2], Cb);
            T = T * expf(-od);
            const long long f = fixed_depth(s);
            S = (S > 0x7fffffffffffffffLL - f) ? 0x7fffffffffffffffLL : S + f;
            if (S >= r.s_thr) {
                n_steps = i + 1;
                done = true;
                break;
            }
        }
    }
    if (cells_out)
        for (int i = n_steps; i < r.N; ++i) cells_out[i] = -2;
    // a9: output
    float4 o;
    o.x = __fmaf_rn(T, r.bg[0], Cr);
    o.y = __fmaf_rn(T, r.bg[1], Cg);
    o.z = __fmaf_rn(T, r.bg[2], Cb);
    o.w = 1.0f - T;
    reinterpret_cast<float4 *>(F.rgba)[pix] = o;
    if (F.stats) {
        int4 st = make_int4(n_steps, n_look, n_occ, dcell);
        reinterpret_cast<int4 *>(F.stats)[pix] = st;
    }
}

template <int PREC, int D>
__global__ void __launch_bounds__(256) march_kernel(const __grid_constant__ MarchArgs A) {
    const int tile = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (tile >= A.total_tiles) return;
    int f = 0;
    while (f + 1 < A.n_frames && tile >= A.f[f + 1].tile_begin) ++f;
    const FrameDesc &F = A.f[f];
    const int t = tile - F.tile_begin;
    const int ty = t / F.tiles_x, tx = t - ty * F.tiles_x;
    const int lane = threadIdx.x & 31;
    const int px = tx * kTileW + (lane & (kTileW - 1)), py = ty * kTileH + lane / kTileW;
    if (px >= F.W || py >= F.H) return;
    march_ray<PREC, D>(A.c, A.r, F, px, py);
}

template <int PREC, int D>
cudaError_t launch_t(const MarchArgs &a, cudaStream_t s) {
    const int threads = 256;
    const int warps_per_block = threads / 32;
    const unsigned blocks = static_cast<unsigned>((a.total_tiles + warps_per_block - 1) / warps_per_block);
    march_kernel<PREC, D><<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_p(const MarchArgs &a, cudaStream_t s) {
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
