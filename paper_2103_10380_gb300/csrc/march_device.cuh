// march_device.cuh -- device code of the cached ray march, shared by the
// plain render kernel (march.cu), the serving kernel (serve.cu), the
// allocation-free kernel (noalloc.cu) and the occupancy build (quant.cu).
#pragma once

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "fnr_internal.h"

namespace fnr {
namespace dev {


// Tuning knobs (defaults are the best measured on GB300):
//   FNR_UNROLL    density loads issued together per lane
//   FNR_BLOCK / FNR_MINB  threads per block / minimum resident blocks per SM
//   FNR_MINB_FP16 / FNR_MINB_FP8  the same for the quantised caches
//   FNR_FAST_EXP  1: exponentials of the occupied-sample path via ex2.approx
#ifndef FNR_UNROLL
#define FNR_UNROLL 8
#endif
#ifndef FNR_BLOCK
#define FNR_BLOCK 128
#endif
#ifndef FNR_MINB
#define FNR_MINB 7
#endif
#ifndef FNR_MINB_FP16
#define FNR_MINB_FP16 8
#endif
#ifndef FNR_MINB_FP8
#define FNR_MINB_FP8 7
#endif
#ifndef FNR_FAST_EXP
#define FNR_FAST_EXP 1
#endif
// FNR_REC_PREFETCH: when an occupied sample is queued, prefetch its record
// (1: into L2, 2: into L1, 0: no); E4M3 records (24 bytes) measured better without
#ifndef FNR_REC_PREFETCH
#define FNR_REC_PREFETCH 1
#endif
constexpr int kUnroll = FNR_UNROLL;

// prefetch [p, p + n) (n <= 128) into L2 (level 1) or L1 (level 2)
template <int LEVEL>
__device__ __forceinline__ void prefetch_span(const char *p, int n) {
    if constexpr (LEVEL == 1) {
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p + n - 1));
    } else if constexpr (LEVEL == 2) {
        asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(p + n - 1));
    }
}
// minimum resident blocks per SM of the march kernels for a cache precision
__host__ __device__ constexpr int min_blocks(int prec) {
    return prec == FNR_PREC_FP8_E4M3 ? FNR_MINB_FP8 : (prec == FNR_PREC_FP16 ? FNR_MINB_FP16 : FNR_MINB);
}

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
    // codes 2p and 2p + 1 with one paired conversion
    __device__ __forceinline__ float2 get2(int p) const {
        const uint2 &q = v[p >> 2];
        const unsigned int word = ((p >> 1) & 1) ? q.y : q.x;
        const __nv_fp8x2_storage_t two = static_cast<__nv_fp8x2_storage_t>((word >> (16 * (p & 1))) & 0xffffu);
        return __half22float2(__half2(__nv_cvt_fp8x2_to_halfraw2(two, __NV_E4M3)));
    }
};

// The binary16 (u, v, w) offsets of one E4M3 offset brick (3D values, 16-byte aligned).
template <int D>
struct OffsetRecord {
    static constexpr int NV = (3 * D + 7) / 8;
    uint4 v[NV];
    __device__ __forceinline__ void load(const uint16_t *p) {
#pragma unroll
        for (int j = 0; j < NV; ++j) v[j] = __ldg(reinterpret_cast<const uint4 *>(p) + j);
    }
    __device__ __forceinline__ float get(int i) const {
        const uint4 &q = v[i >> 3];
        const int w = (i >> 1) & 3;
        const unsigned int word = w == 0 ? q.x : w == 1 ? q.y : w == 2 ? q.z : q.w;
        return __half2float(__ushort_as_half(static_cast<unsigned short>((i & 1) ? (word >> 16) : (word & 0xffffu))));
    }
};

// E4M3 colour (Eq. 5 on the stored values): component i = ch D + j is
// u_i = fma(s_i, e4m3(q_i), m_i) (its channel scale s_i and offset m_i), and
// x_ch = sum_j beta_j u_{ch D + j} in the order j = 0 .. D-1; scale_of(i) and
// beta_of(j) supply s_i and beta_j.
template <int D, class ScaleOf, class BetaOf>
__device__ __forceinline__ void shade_e4m3(const Record<FNR_PREC_FP8_E4M3, D> &rec, const OffsetRecord<D> &off,
                                           int act, ScaleOf scale_of, BetaOf beta_of, float col[3]) {
    float x[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int p = 0; p < (3 * D + 1) / 2; ++p) {
        const float2 q = rec.get2(p);
        const int i = 2 * p;
        x[i / D] = __fmaf_rn(beta_of(i % D), __fmaf_rn(scale_of(i), q.x, off.get(i)), x[i / D]);
        if (i + 1 < 3 * D)
            x[(i + 1) / D] =
                __fmaf_rn(beta_of((i + 1) % D), __fmaf_rn(scale_of(i + 1), q.y, off.get(i + 1)), x[(i + 1) / D]);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
#if FNR_FAST_EXP
        col[ch] = act == FNR_ACT_IDENTITY ? x[ch] : __fdividef(1.0f, 1.0f + __expf(-x[ch]));
#else
        col[ch] = act == FNR_ACT_IDENTITY ? x[ch] : 1.0f / (1.0f + expf(-x[ch]));
#endif
    }
}

template <int PREC>
__device__ __forceinline__ float load_sigma(const CacheView &c, int cell, float sigma_scale) {
    if constexpr (PREC == FNR_PREC_FP32) {
        return __ldg(static_cast<const float *>(c.sigma) + cell);
    } else if constexpr (PREC == FNR_PREC_FP16) {
        return __half2float(__ldg(static_cast<const __half *>(c.sigma) + cell));
    } else {
        unsigned int q = __ldg(static_cast<const unsigned char *>(c.sigma) + cell);
        return __fmul_rn(e4m3_to_float(q), sigma_scale);  // binary32 dequantisation
    }
}

// Programmatic dependent launch: a render launch may start while the previous
// one in its stream finishes (it reads only the cache, which no launch
// writes); it waits for that launch to complete before its first global write,
// so outputs keep stream order. Without a programmatic dependency (another
// kind of launch, a graph node, the first launch) the wait returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void allow_next_grid() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Occupancy bit of an in-grid brick (the bits are small and stay in L1).
__device__ __forceinline__ unsigned brick_occupied(const CacheView &c, int brick) {
    return (__ldg(c.occ + (brick >> 5)) >> (brick & 31)) & 1u;
}

// floor(s * 2^32) for binary32 s, by integer shifts of the significand (no
// float -> int64 conversion: on this GPU those run on the FP64 pipe).
// s <= 0 or NaN -> 0; s >= 2^31 -> 2^63 - 1 (saturated).
__device__ __forceinline__ long long fixed_depth(float s) {
    if (!(s > 0.0f)) return 0;
    if (s >= 2147483648.0f) return 0x7fffffffffffffffLL;
    const unsigned int bits = __float_as_uint(s);
    const int ex = static_cast<int>((bits >> 23) & 0xffu);
    const unsigned long long mant = (bits & 0x7fffffu) | (ex ? 0x800000u : 0u);
    const int shift = (ex ? ex - 127 : -126) - 23 + 32;  // s * 2^32 = mant * 2^shift
    if (shift >= 0) return static_cast<long long>(mant << shift);
    return -shift >= 64 ? 0 : static_cast<long long>(mant >> (-shift));
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

// Starting estimates for the direction cell; the exact walk over the boundary
// tables corrects any error, so short polynomial approximations suffice.
// Polar angle: acos(x) ~ sqrt(1 - x) (a0 + a1 x + a2 x^2 + a3 x^3) for
// 0 <= x <= 1 (Abramowitz & Stegun, Handbook of Mathematical Functions,
// 4.4.45; |error| <= 7e-5 rad), acos(-x) = pi - acos(x).
__device__ __forceinline__ float acos_estimate(float x) {
    const float ax = fminf(fabsf(x), 1.0f);
    const float p = fmaf(fmaf(fmaf(-0.0187293f, ax, 0.0742610f), ax, -0.2121144f), ax, 1.5707288f);
    const float a = sqrtf(1.0f - ax) * p;
    return x < 0.0f ? 3.14159265f - a : a;
}
// Azimuth from the diamond key q in [0, 4]: quadrant floor(q), and inside it
// the angle pi/4 + atan(2 t - 1) for t = q - floor(q) (tan of the angle is
// t / (1 - t)); atan(z) ~ (pi/4) z - z (|z| - 1)(0.2447 + 0.0663 |z|) on
// [-1, 1] (Rajan, Wang, Inkol and Joyal, "Efficient approximations for the
// arctangent function", IEEE Signal Processing Magazine 23(3), 2006;
// |error| <= 1.5e-3 rad).
__device__ __forceinline__ float azimuth_estimate(float q) {
    const float k = floorf(fminf(q, 3.999999f));
    const float z = 2.0f * (q - k) - 1.0f;
    const float az = fabsf(z);
    const float at = fmaf(0.78539816f, z, -z * (az - 1.0f) * fmaf(0.0663f, az, 0.2447f));
    return fmaf(1.57079633f, k, 0.78539816f + at);
}

// Direction cell: counts of boundaries passed; the estimates only pick where
// the exact walk over the (monotone) tables starts.
__device__ __forceinline__ int dir_cell(const CacheView &c, float dx, float dy, float dz) {
    const int l = c.l;
    const float inv_pi = 0.318309886183790671538f;
    int it = static_cast<int>(acos_estimate(dz) * inv_pi * static_cast<float>(l));
    it = min(max(it, 0), l - 1);
    while (it < l - 1 && dz <= __ldg(c.ct + it + 1)) ++it;
    while (it > 0 && dz > __ldg(c.ct + it)) --it;
    const float q = phi_key(dx, dy);
    int ip = static_cast<int>(azimuth_estimate(q) * (0.5f * inv_pi) * static_cast<float>(l));
    ip = min(max(ip, 0), l - 1);
    while (ip < l - 1 && q >= __ldg(c.qp + ip + 1)) ++ip;
    while (ip > 0 && q < __ldg(c.qp + ip)) --ip;
    return it * l + ip;
}

// Bilinear direction weights (FNR_RENDER_DIR_BILINEAR): beta interpolated in
// (theta, phi) between the bin centres theta_i = (i + 1/2) pi / l and
// phi_j = (j + 1/2) 2 pi / l, theta neighbours clamped at the poles, phi
// neighbours wrapping around 2 pi. Kept out of line: once per ray, and its
// libm calls would otherwise raise the march's register pressure.
template <int D>
__device__ __noinline__ void stage_beta_bilinear(const CacheView &c, float dx, float dy, float dz,
                                                 float (*qbeta)[32], int lane) {
    auto beta_at = [&](long long cell, int i) {
        return c.dir_prec == FNR_PREC_FP16 ? __half2float(__ldg(static_cast<const __half *>(c.beta) + cell * D + i))
                                           : __ldg(static_cast<const float *>(c.beta) + cell * D + i);
    };
    const float pi = 3.14159265358979f;
    const float th = atan2f(sqrtf(dx * dx + dy * dy), dz);
    float ph = atan2f(dy, dx);
    if (ph < 0.0f) ph += 2.0f * pi;
    const float u = th * (static_cast<float>(c.l) / pi) - 0.5f;
    const float v = ph * (static_cast<float>(c.l) / (2.0f * pi)) - 0.5f;
    const float fu = floorf(u), fv = floorf(v);
    const float a = u - fu, b = v - fv;
    const int i0 = min(max(static_cast<int>(fu), 0), c.l - 1);
    const int i1 = min(max(static_cast<int>(fu) + 1, 0), c.l - 1);
    int j0 = static_cast<int>(fv) % c.l;
    if (j0 < 0) j0 += c.l;
    const int j1 = j0 + 1 == c.l ? 0 : j0 + 1;
    const long long c00 = (long long)i0 * c.l + j0, c01 = (long long)i0 * c.l + j1;
    const long long c10 = (long long)i1 * c.l + j0, c11 = (long long)i1 * c.l + j1;
    const float w00 = (1.0f - a) * (1.0f - b), w01 = (1.0f - a) * b, w10 = a * (1.0f - b), w11 = a * b;
#pragma unroll
    for (int i = 0; i < D; ++i)
        qbeta[i][lane] = w00 * beta_at(c00, i) + w01 * beta_at(c01, i) + w10 * beta_at(c10, i) + w11 * beta_at(c11, i);
}

// Per-ray setup: a1 (ray), a2 (direction cell), and the per-ray affine
// coefficients of the sample cells with the sample range that can reach the box.
template <int PREC, int D>
struct RaySetup {
    float e[3], f[3];
    float inv_emax;    // approximate 1 / max_a |e_a| (skipping only)
    int i_lo, i_hi;
    int in_lo, in_hi;  // samples certainly inside the box (the exact test is then redundant)
    int dcell;
    float sigma_scale;

    // qbeta / lane: where this ray's D direction weights (unscaled) are staged
    __device__ __forceinline__ void init(const CacheView &c, const RenderConst &r, const FrameDesc &F, int px,
                                         int py, float (*qbeta)[32], int lane) {
        // a1: ray (binary32, fixed sequence)
        const float dcx = __fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(px), 0.5f), F.cx), F.fx);
        const float dcy = -__fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(py), 0.5f), F.cy), F.fy);
        const float wx = __fmaf_rn(F.c2w[0], dcx, __fmaf_rn(F.c2w[1], dcy, -F.c2w[2]));
        const float wy = __fmaf_rn(F.c2w[4], dcx, __fmaf_rn(F.c2w[5], dcy, -F.c2w[6]));
        const float wz = __fmaf_rn(F.c2w[8], dcx, __fmaf_rn(F.c2w[9], dcy, -F.c2w[10]));
        const float n2 = __fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz)));
        const float len = __fsqrt_rn(n2);
        const float dd[3] = {__fdiv_rn(wx, len), __fdiv_rn(wy, len), __fdiv_rn(wz, len)};
        const float oo[3] = {F.c2w[3], F.c2w[7], F.c2w[11]};

        // a2: direction cell and beta
        dcell = dir_cell(c, dd[0], dd[1], dd[2]);
        stage_beta(c, r, dd, qbeta, lane);
        sigma_scale = (PREC == FNR_PREC_FP8_E4M3) ? __ldg(c.scales) : 1.0f;

        // a3/a4 per ray: cell coordinates of sample i are g_a = fma(i + 1/2, e_a, f_a)
        // with e_a = (d_a s_a) Delta and f_a = fma(near, d_a s_a, (o_a - bmin_a) s_a)
        // (binary32, the order fixed in fnr.h).
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float ua = __fmul_rn(dd[a], c.scale[a]);
            e[a] = __fmul_rn(ua, r.dt);
            f[a] = __fmaf_rn(r.t_near, ua, __fmul_rn(__fsub_rn(oo[a], c.bmin[a]), c.scale[a]));
        }
        // Samples that can reach the box: a range widened by one cell on every face
        // and two samples at each end, so every sample the exact test puts inside
        // lies in [i_lo, i_hi); samples outside it are outside the box.
        i_lo = 0;
        i_hi = r.N;
        const bool finite_dir = (dd[0] == dd[0]) && (dd[1] == dd[1]) && (dd[2] == dd[2]);
        if (!finite_dir) i_hi = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (e[a] == 0.0f) {
                if (!(f[a] >= -1.0f && f[a] <= c.kf + 1.0f)) i_hi = 0;
            } else {
                // approximate reciprocal (a few ulp; an e_a so small that 1/e_a overflows gives
                // infinity either way): these bounds carry two samples of margin and only narrow the
                // range the exact per-sample test runs over
                const float re = __fdividef(1.0f, e[a]);
                const float ta = (-1.0f - f[a]) * re - 0.5f;
                const float tb = (c.kf + 1.0f - f[a]) * re - 0.5f;
                const float lo = fmaxf(fminf(ta, tb) - 2.0f, -1.0f);
                const float hi = fminf(fmaxf(ta, tb) + 2.0f, static_cast<float>(r.N) + 1.0f);
                i_lo = max(i_lo, __float2int_rd(lo));
                i_hi = min(i_hi, __float2int_ru(hi) + 1);
            }
        }
        i_lo = min(i_lo, r.N);
        inv_emax = __fdividef(1.0f, fmaxf(fabsf(e[0]), fmaxf(fabsf(e[1]), fabsf(e[2]))));
        // The same bound narrowed by one cell on every face and two samples at
        // each end: samples in [in_lo, in_hi) have 1 <= g_a <= k - 1 on every axis
        // with room to spare for the rounding of g and of these bounds, so the
        // exact per-sample test would pass there.
        in_lo = 0;
        in_hi = finite_dir ? r.N : 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (e[a] == 0.0f) {
                if (!(f[a] >= 1.0f && f[a] <= c.kf - 1.0f)) in_hi = 0;
            } else {
                const float re = __fdividef(1.0f, e[a]);
                const float ta = (1.0f - f[a]) * re - 0.5f;
                const float tb = (c.kf - 1.0f - f[a]) * re - 0.5f;
                const float lo = fminf(fmaxf(fminf(ta, tb) + 2.0f, -1.0f), static_cast<float>(r.N) + 1.0f);
                const float hi = fmaxf(fminf(fmaxf(ta, tb) - 2.0f, static_cast<float>(r.N) + 1.0f), -1.0f);
                in_lo = max(in_lo, __float2int_ru(lo));
                in_hi = min(in_hi, __float2int_rd(hi));
            }
        }
        in_lo = max(in_lo, i_lo);
        in_hi = min(in_hi, i_hi);
    }

    // The ray's D direction weights (unscaled; FP8 folds the channel scales at
    // shading) into qbeta[i][lane]: the nearest bin's, or bilinear in
    // (theta, phi) between bin centres (FNR_RENDER_DIR_BILINEAR).
    __device__ __forceinline__ void stage_beta(const CacheView &c, const RenderConst &r, const float dd[3],
                                               float (*qbeta)[32], int lane) const {
        auto beta_at = [&](long long cell, int i) {
            return c.dir_prec == FNR_PREC_FP16
                       ? __half2float(__ldg(static_cast<const __half *>(c.beta) + cell * D + i))
                       : __ldg(static_cast<const float *>(c.beta) + cell * D + i);
        };
        if (r.flags & FNR_RENDER_DIR_BILINEAR) {
            stage_beta_bilinear<D>(c, dd[0], dd[1], dd[2], qbeta, lane);
        } else {
#pragma unroll
            for (int i = 0; i < D; ++i) qbeta[i][lane] = beta_at(dcell, i);
        }
    }

    // Cell of sample i (fi = i + 0.5) or -1 outside the box. For finite g,
    // 0 <= g < k iff 0 <= floor(g) < k; floor goes straight to int32.
    __device__ __forceinline__ int cell_of(const CacheView &c, float fi) const {
        const float gx = __fmaf_rn(fi, e[0], f[0]);
        const float gy = __fmaf_rn(fi, e[1], f[1]);
        const float gz = __fmaf_rn(fi, e[2], f[2]);
        const int ix = __float2int_rd(gx), iy = __float2int_rd(gy), iz = __float2int_rd(gz);
        const unsigned int ku = static_cast<unsigned int>(c.k);
        const bool in = static_cast<unsigned int>(ix) < ku && static_cast<unsigned int>(iy) < ku &&
                        static_cast<unsigned int>(iz) < ku;
        return in ? (iz * c.k + iy) * c.k + ix : -1;  // k^3 < 2^31
    }

    // Cell of a sample known to be inside the box.
    __device__ __forceinline__ int cell_inside(const CacheView &c, float fi) const {
        const int ix = __float2int_rd(__fmaf_rn(fi, e[0], f[0]));
        const int iy = __float2int_rd(__fmaf_rn(fi, e[1], f[1]));
        const int iz = __float2int_rd(__fmaf_rn(fi, e[2], f[2]));
        return (iz * c.k + iy) * c.k + ix;
    }

    // Brick and brick-local index ((z mod B) B + (y mod B)) B + (x mod B) of
    // sample fi; false if the sample is outside the box (checked when `check`).
    __device__ __forceinline__ bool cell_bl(const CacheView &c, float fi, int &brick, int &local, bool check) const {
        const int ix = __float2int_rd(__fmaf_rn(fi, e[0], f[0]));
        const int iy = __float2int_rd(__fmaf_rn(fi, e[1], f[1]));
        const int iz = __float2int_rd(__fmaf_rn(fi, e[2], f[2]));
        if (check) {
            const unsigned int ku = static_cast<unsigned int>(c.k);
            if (!(static_cast<unsigned int>(ix) < ku && static_cast<unsigned int>(iy) < ku &&
                  static_cast<unsigned int>(iz) < ku))
                return false;
        }
        const int sh = c.occ_shift, m = (1 << sh) - 1;
        brick = ((iz >> sh) * c.occ_dim + (iy >> sh)) * c.occ_dim + (ix >> sh);
        local = ((((iz & m) << sh) | (iy & m)) << sh) | (ix & m);
        return true;
    }

    // The same two with the sample's occupancy brick (meaningful when inside).
    __device__ __forceinline__ int cell_of_b(const CacheView &c, float fi, int &brick) const {
        const int ix = __float2int_rd(__fmaf_rn(fi, e[0], f[0]));
        const int iy = __float2int_rd(__fmaf_rn(fi, e[1], f[1]));
        const int iz = __float2int_rd(__fmaf_rn(fi, e[2], f[2]));
        const unsigned int ku = static_cast<unsigned int>(c.k);
        const bool in = static_cast<unsigned int>(ix) < ku && static_cast<unsigned int>(iy) < ku &&
                        static_cast<unsigned int>(iz) < ku;
        brick = ((iz >> c.occ_shift) * c.occ_dim + (iy >> c.occ_shift)) * c.occ_dim + (ix >> c.occ_shift);
        return in ? (iz * c.k + iy) * c.k + ix : -1;
    }
    __device__ __forceinline__ int cell_inside_b(const CacheView &c, float fi, int &brick) const {
        const int ix = __float2int_rd(__fmaf_rn(fi, e[0], f[0]));
        const int iy = __float2int_rd(__fmaf_rn(fi, e[1], f[1]));
        const int iz = __float2int_rd(__fmaf_rn(fi, e[2], f[2]));
        brick = ((iz >> c.occ_shift) * c.occ_dim + (iy >> c.occ_shift)) * c.occ_dim + (ix >> c.occ_shift);
        return (iz * c.k + iy) * c.k + ix;
    }

    // Empty-space skipping over runs of samples (FNR_RENDER_SKIP_EMPTY), one
    // step: the first sample >= s that this lane must still test -- s itself
    // unless s lies in an empty jump brick, INT_MAX when no sample is left in
    // [s, i_hi). A sample in jump brick b (J cells a side) at distance d >= 1
    // from every occupied one lies in the cube of jump bricks b - (d - 1) ..
    // b + (d - 1), which holds no density. Along axis a the sample's binary32
    // coordinate g_a is r_a = ((b_a + 1) J - g_a or g_a - b_a J, by the sign
    // of e_a) from the face of its brick ahead of it, so (d - 1) J + r_a from the
    // cube's face (an axis with e_a = 0 never reaches it), and no sample moves
    // more than emax = max_a |e_a| cells along any axis: after n samples with n emax <= (d - 1) J + min_a r_a - 1/100 the
    // ray is still inside the cube (1/100 cell covers the roundings, each below
    // 2^-12 cell for k < 2048), and by monotonicity of the per-axis binary32
    // coordinate in the sample index so is every sample in between. Those
    // samples lie in empty bricks: the per-sample test would not look them up.
    __device__ __forceinline__ int skip_empty_step(const CacheView &c, int s) const {
        if (s >= i_hi) return 0x7fffffff;
        const float fs = __fadd_rn(static_cast<float>(s), 0.5f);
        float g[3];
        int ci[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g[a] = __fmaf_rn(fs, e[a], f[a]);
            ci[a] = __float2int_rd(g[a]);
        }
        const unsigned int ku = static_cast<unsigned int>(c.k);
        if (!(static_cast<unsigned int>(ci[0]) < ku && static_cast<unsigned int>(ci[1]) < ku &&
              static_cast<unsigned int>(ci[2]) < ku))
            return s;
        const int sh = c.dist_shift;
        const int d = __ldg(c.dist + ((ci[2] >> sh) * c.dist_dim + (ci[1] >> sh)) * c.dist_dim + (ci[0] >> sh));
        if (d == 0) return s;
        float reach = 3.0e38f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int face = ((ci[a] >> sh) + (e[a] > 0.0f ? 1 : 0)) << sh;
            const float ra = e[a] > 0.0f ? static_cast<float>(face) - g[a] : g[a] - static_cast<float>(face);
            if (e[a] != 0.0f) reach = fminf(reach, ra);  // no motion along a: no limit
        }
        reach += static_cast<float>((d - 1) << sh) - 0.01f;
        const int n = __float2int_rd(fminf(reach * inv_emax, 1.0e9f));
        if (n <= 0) return s;
        return n < i_hi - s ? s + n + 1 : 0x7fffffff;
    }

    // a7: Eq. 5 and the activation for one record.
    __device__ __forceinline__ void shade(const Record<PREC, D> &rec, int act, const float *b, float col[3]) const {
        shade_with(rec, act, [&](int ch, int j) { return b[(PREC == FNR_PREC_FP8_E4M3) ? ch * D + j : j]; }, col);
    }
    // the same with beta_j (times the FP8 scale of channel (ch, j)) supplied by beta_of(ch, j); the
    // loops run component-major, but each channel's sum keeps the order j = 0 .. D-1
    template <class BetaOf>
    __device__ __forceinline__ static void shade_with(const Record<PREC, D> &rec, int act, BetaOf beta_of,
                                                      float col[3]) {
        float x[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int j = 0; j < D; ++j) {
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) x[ch] = __fmaf_rn(beta_of(ch, j), rec.get(ch * D + j), x[ch]);
        }
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
#if FNR_FAST_EXP
            col[ch] = act == FNR_ACT_IDENTITY ? x[ch] : __fdividef(1.0f, 1.0f + __expf(-x[ch]));
#else
            col[ch] = act == FNR_ACT_IDENTITY ? x[ch] : 1.0f / (1.0f + expf(-x[ch]));
#endif
        }
    }
};

// exp(-od) and 1 - exp(-od) for the Eq. 1 update.
__device__ __forceinline__ void extinction(float od, float &ext, float &alpha) {
#if FNR_FAST_EXP
    ext = __expf(-od);
    alpha = 1.0f - ext;
#else
    ext = expf(-od);
    alpha = -expm1f(-od);
#endif
}

// ---------------------------------------------------------------------------
// Queued variant. The transmittance, the weights w_i = T_i alpha_i and the
// termination step depend on the densities only, so each lane marches its ray
// with density loads alone and appends (cell, w_i) of every occupied sample to
// a per-warp queue in shared memory. Whenever 32 entries are queued the warp
// shades them together -- 32 independent record loads in one round trip --
// and every owner lane adds w_i * c_i to its colour in sample order, so the
// binary32 result equals the sequential form bit for bit.
constexpr int kQCap = 32 * (kUnroll + 1);  // entries left after a flush (< 32) plus one group's appends

// OFFS (E4M3 caches): each entry also carries its offset brick, and the warp
// keeps the 3D channel scales.
template <int D, bool OFFS = false>
struct WarpQueue {
    int cell[kQCap];
    float w[kQCap];
    unsigned char owner[kQCap];
    float col[3][32];
    float beta[D][32];     // beta of each lane's ray (unscaled)
    unsigned int own_mask[32];
    int obr[OFFS ? kQCap : 1];  // offset brick of each entry
    float sc[OFFS ? 3 * D : 1]; // scale of (u, v, w) channel ch D + j
};
template <int PREC, int D>
using QueueFor = WarpQueue<D, PREC == FNR_PREC_FP8_E4M3>;

// SKIP (FNR_RENDER_SKIP_EMPTY): a sample in a brick without stored density is
// known to be empty, so only samples in occupied bricks load their density; the
// lookup counter counts those loads. Everything else is unchanged.
// BRICKS (FNR_LAYOUT_BRICKS, implies SKIP): densities and records live in brick
// pools in brick-index order; an occupied sample's pool slot is the brick's rank
// among the occupied bricks, and the queue carries pool indices instead of cells.
template <int PREC, int D, bool SKIP, bool BRICKS = false>
__device__ __forceinline__ void march_tile_queued(const CacheView &c, const RenderConst &r, const FrameDesc &F,
                                                  int px, int py, bool active, QueueFor<PREC, D> &q) {
    constexpr bool kOffs = PREC == FNR_PREC_FP8_E4M3;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    RaySetup<PREC, D> R;
    if (active) {
        R.init(c, r, F, px, py, q.beta, lane);
    } else {
        R.i_lo = R.i_hi = 0;
        R.dcell = 0;
        R.sigma_scale = 1.0f;
    }
    if (!active)
        for (int i = 0; i < D; ++i) q.beta[i][lane] = 0.0f;
    if constexpr (kOffs) {
        for (int i = lane; i < 3 * D; i += 32) q.sc[i] = __ldg(c.scales + 1 + i);
        __syncwarp();
    }
    float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    long long S = 0;
    int n_look = 0, n_occ = 0, n_steps = r.N;
    const long long pix = active ? static_cast<long long>(py) * F.W + px : 0;
    int32_t *cells_out = (active && F.cells) ? F.cells + pix * r.N : nullptr;
    if (F.cells) wait_prior_grid();  // per-sample cells are written while marching
    bool done = !active;
    if (cells_out)
        for (int i = 0; i < R.i_lo; ++i) cells_out[i] = -1;
    const bool has_range = active && R.i_lo < R.i_hi;
    const int lo_w = __reduce_min_sync(FULL, has_range ? R.i_lo : 0x7fffffff);
    const int hi_w = __reduce_max_sync(FULL, has_range ? R.i_hi : 0);

    // Shade queue entries [base, base + n) and add them to their owners.
    auto flush = [&](int base, int n) {
        float col[3] = {0.0f, 0.0f, 0.0f};
        int own = 32 + lane;  // distinct dummy for lanes without an entry
        if (lane < n) {
            const int e = base + lane;
            own = q.owner[e];
            Record<PREC, D> rec;
            rec.load(c.uvw + static_cast<long long>(q.cell[e]) * c.rec_stride);
            if constexpr (kOffs) {
                OffsetRecord<D> off;
                off.load(c.offs + static_cast<long long>(q.obr[e]) * c.offs_stride);
                shade_e4m3<D>(
                    rec, off, r.act, [&](int i) { return q.sc[i]; }, [&](int j) { return q.beta[j][own]; }, col);
            } else {
                float b[D];
#pragma unroll
                for (int i = 0; i < D; ++i) b[i] = q.beta[i][own];
                R.shade(rec, r.act, b, col);
            }
        }
        q.col[0][lane] = col[0];
        q.col[1][lane] = col[1];
        q.col[2][lane] = col[2];
        q.own_mask[lane] = 0u;
        __syncwarp();
        const unsigned m = __match_any_sync(FULL, own);
        if (lane < n && lane == __ffs(m) - 1) q.own_mask[own] = m;
        __syncwarp();
        unsigned mine = q.own_mask[lane];
        while (mine) {  // this lane's entries, in queue (= sample) order
            const int j = __ffs(mine) - 1;
            mine &= mine - 1;
            const float w = q.w[base + j];
            Cr = __fmaf_rn(w, q.col[0][j], Cr);
            Cg = __fmaf_rn(w, q.col[1][j], Cg);
            Cb = __fmaf_rn(w, q.col[2][j], Cb);
        }
        __syncwarp();
    };

    // empty-group test by the maximum density (measured faster for binary32 densities only)
    constexpr bool kMaxTest = PREC == FNR_PREC_FP32;
    // skipping passes over runs of samples in empty space (not when every sample's cell is written)
    const bool jump = SKIP && F.cells == nullptr;
    int qn = 0;
    for (int i0 = lo_w; i0 < hi_w; i0 += kUnroll) {
        if (!__any_sync(FULL, !done)) break;
        if (SKIP && jump) {
            // The warp moves on, a step at a time, to the first sample some marching lane must
            // still test; each step is one cube of empty jump bricks for every lane, and the
            // steps stop as soon as one lane cannot advance.
#pragma unroll 1
            for (int st = 0; st < 4; ++st) {
                const int t = done ? 0x7fffffff : R.skip_empty_step(c, max(i0, R.i_lo));
                const int m = __reduce_min_sync(FULL, t);
                if (m <= i0) break;
                i0 = m;
                if (i0 >= hi_w) break;
            }
            if (i0 >= hi_w) break;
        }
        // samples of this group the lane visits: [i_lo, i_hi) before termination
        const int vlo = min(max(R.i_lo - i0, 0), kUnroll), vhi = min(max(R.i_hi - i0, 0), kUnroll);
        const unsigned vis = done ? 0u : (((1u << vhi) - 1u) & ~((1u << vlo) - 1u));
        int cell[kUnroll];
        float sg[kUnroll];
        float fi = __fadd_rn(static_cast<float>(i0), 0.5f);
        unsigned in_m = 0u, occ_m = 0u;
        // Groups certainly inside the box for every lane still marching take the
        // path without per-sample range tests (warp-uniform choice).
        const bool inside = done || (i0 >= R.in_lo && i0 + kUnroll <= R.in_hi);
        if constexpr (BRICKS) {
            // First the occupancy bits, exactly as the dense skip path; then, only if some lane
            // of the warp has a sample in an occupied brick, those samples' pool indices: the
            // brick's slot is its rank among the occupied bricks (a per-word prefix count plus a
            // popcount, both from L1-resident arrays) and the cell's brick-local index.
            const float fi0 = fi;
            if (__all_sync(FULL, inside)) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    int br;
                    R.cell_inside_b(c, fi, br);
                    in_m |= (!done ? brick_occupied(c, br) : 0u) << u;
                    fi = __fadd_rn(fi, 1.0f);
                }
            } else {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    int br = 0;
                    const bool in = ((vis >> u) & 1u) && R.cell_of_b(c, fi, br) >= 0;
                    in_m |= (in ? brick_occupied(c, br) : 0u) << u;
                    fi = __fadd_rn(fi, 1.0f);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) cell[u] = -1;
            if (__any_sync(FULL, in_m != 0u)) {
                float fu = fi0;
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    if ((in_m >> u) & 1u) {
                        int br, loc;
                        R.cell_bl(c, fu, br, loc, false);
                        const uint32_t wb = __ldg(c.occ + (br >> 5));
                        const uint32_t slot = __ldg(c.rank + (br >> 5)) + __popc(wb & ((1u << (br & 31)) - 1u));
                        cell[u] = static_cast<int>((slot << (3 * c.occ_shift)) | static_cast<uint32_t>(loc));
                    }
                    fu = __fadd_rn(fu, 1.0f);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                sg[u] = ((in_m >> u) & 1u) ? load_sigma<PREC>(c, cell[u], R.sigma_scale) : 0.0f;
            if constexpr (!kMaxTest) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) occ_m |= (sg[u] > 0.0f ? 1u : 0u) << u;
            }
        } else if constexpr (SKIP) {
            // density lookups only in occupied bricks: in_m = the lookups made
            if (__all_sync(FULL, inside)) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    int br;
                    cell[u] = R.cell_inside_b(c, fi, br);
                    in_m |= (!done ? brick_occupied(c, br) : 0u) << u;
                    fi = __fadd_rn(fi, 1.0f);
                }
            } else {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) {
                    int br = 0;
                    cell[u] = ((vis >> u) & 1u) ? R.cell_of_b(c, fi, br) : -1;
                    in_m |= (cell[u] >= 0 ? brick_occupied(c, br) : 0u) << u;
                    fi = __fadd_rn(fi, 1.0f);
                }
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                sg[u] = ((in_m >> u) & 1u) ? load_sigma<PREC>(c, cell[u], R.sigma_scale) : 0.0f;
            if constexpr (!kMaxTest) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) occ_m |= (sg[u] > 0.0f ? 1u : 0u) << u;
            }
        } else if (__all_sync(FULL, inside)) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                cell[u] = R.cell_inside(c, fi);
                fi = __fadd_rn(fi, 1.0f);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) sg[u] = !done ? load_sigma<PREC>(c, cell[u], R.sigma_scale) : 0.0f;
            in_m = vis;  // every visited sample of the group is in the box
            if constexpr (!kMaxTest) {
#pragma unroll
                for (int u = 0; u < kUnroll; ++u) occ_m |= (sg[u] > 0.0f ? 1u : 0u) << u;
            }
        } else {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                cell[u] = ((vis >> u) & 1u) ? R.cell_of(c, fi) : -1;
                fi = __fadd_rn(fi, 1.0f);
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                sg[u] = cell[u] >= 0 ? load_sigma<PREC>(c, cell[u], R.sigma_scale) : 0.0f;
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                in_m |= (cell[u] >= 0 ? 1u : 0u) << u;
                if constexpr (!kMaxTest) occ_m |= (sg[u] > 0.0f ? 1u : 0u) << u;
            }
        }
        if (cells_out) {
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                if ((vis >> u) & 1u)  // past termination: overwritten by -2 below
                    cells_out[i0 + u] =
                        BRICKS ? R.cell_of(c, __fadd_rn(static_cast<float>(i0 + u), 0.5f)) : cell[u];
        }
        if constexpr (kMaxTest) {
            // Any occupied sample in the warp? Densities are finite and >= 0 (negative
            // and NaN values are stored as 0), so the group's maximum decides.
            float smax = sg[0];
#pragma unroll
            for (int u = 1; u < kUnroll; ++u) smax = fmaxf(smax, sg[u]);
            if (!__any_sync(FULL, smax > 0.0f)) {  // empty space for the whole warp
                n_look += __popc(in_m);
                continue;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) occ_m |= (sg[u] > 0.0f ? 1u : 0u) << u;
        } else if (!__any_sync(FULL, occ_m != 0u)) {  // empty space for the whole warp
            n_look += __popc(in_m);
            continue;
        }
        // Occupied samples of this lane, in order: weights, transmittance, termination.
        unsigned app = 0u, counted = in_m;
        float aw[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            aw[u] = 0.0f;
            if (((occ_m >> u) & 1u) && !done) {
                float ext, alpha;
                extinction(__fmul_rn(sg[u], r.dt), ext, alpha);
                aw[u] = T * alpha;
                T = T * ext;
                app |= 1u << u;
                const long long qd = fixed_depth(sg[u]);
                S = (S > 0x7fffffffffffffffLL - qd) ? 0x7fffffffffffffffLL : S + qd;
                if (S >= r.s_thr) {
                    n_steps = i0 + u + 1;
                    done = true;
                    counted = in_m & ((2u << u) - 1u);
                }
            }
        }
        n_look += __popc(counted);
        const int cnt = __popc(app);
        n_occ += cnt;
        // append lane by lane (per owner: sample order)
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += v;
        }
        int pos = qn + incl - cnt;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
            if ((app >> u) & 1u) {
                if constexpr (FNR_REC_PREFETCH != 0 && PREC != FNR_PREC_FP8_E4M3)
                    prefetch_span<FNR_REC_PREFETCH>(c.uvw + static_cast<long long>(cell[u]) * c.rec_stride,
                                                    c.rec_stride);
                q.cell[pos] = cell[u];
                q.w[pos] = aw[u];
                q.owner[pos] = static_cast<unsigned char>(lane);
                if constexpr (kOffs) {
                    // the sample's offset brick, from its cell coordinates
                    const float fu = __fadd_rn(static_cast<float>(i0 + u), 0.5f);
                    const int sh = c.offs_shift;
                    const int ox = __float2int_rd(__fmaf_rn(fu, R.e[0], R.f[0])) >> sh;
                    const int oy = __float2int_rd(__fmaf_rn(fu, R.e[1], R.f[1])) >> sh;
                    const int oz = __float2int_rd(__fmaf_rn(fu, R.e[2], R.f[2])) >> sh;
                    q.obr[pos] = (oz * c.offs_dim + oy) * c.offs_dim + ox;
                }
                ++pos;
            }
        }
        qn += __shfl_sync(FULL, incl, 31);
        if (qn >= 32) {
            __syncwarp();
            int base = 0;
            for (; base + 32 <= qn; base += 32) flush(base, 32);
            const int rem = qn - base;  // < 32, moved to the front (source >= 32 > target)
            if (lane < rem) {
                q.cell[lane] = q.cell[base + lane];
                q.w[lane] = q.w[base + lane];
                q.owner[lane] = q.owner[base + lane];
                if constexpr (kOffs) q.obr[lane] = q.obr[base + lane];
            }
            __syncwarp();
            qn = rem;
        }
    }
    if (qn > 0) {
        __syncwarp();
        flush(0, qn);
    }
    wait_prior_grid();
    if (!active) return;
    if (cells_out) {
        if (done)
            for (int i = n_steps; i < r.N; ++i) cells_out[i] = -2;
        else
            for (int i = max(R.i_hi, R.i_lo); i < r.N; ++i) cells_out[i] = -1;
    }
    float4 o;
    o.x = __fmaf_rn(T, r.bg[0], Cr);
    o.y = __fmaf_rn(T, r.bg[1], Cg);
    o.z = __fmaf_rn(T, r.bg[2], Cb);
    o.w = 1.0f - T;
    reinterpret_cast<float4 *>(F.rgba)[pix] = o;
    if (F.stats) reinterpret_cast<int4 *>(F.stats)[pix] = make_int4(n_steps, n_look, n_occ, R.dcell);
}

}  // namespace dev
}  // namespace fnr
