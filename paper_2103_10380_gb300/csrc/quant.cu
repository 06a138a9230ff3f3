// quant.cu -- cache storage conversion: binary32 source arrays -> FP32 / FP16 /
// FP8-E4M3 cache records, with per-channel FP8 scales from a device absmax.
//
// Densities are clamped to >= 0 (NaN -> 0) before storage. FP16 rounds to
// nearest even; FP8 stores E4M3(x / scale_c) rounded to nearest even and
// saturated to +-448, scale_c = absmax_c / 448 (binary32 division; 1 for an
// all-zero channel). For the (u, v, w) channels x is the residual from the
// cell's offset brick: the binary16 midrange of the channel over the brick. The (u, v, w) records are padded to rec_stride bytes with
// zeros so every record starts on a 16-byte (FP8: 8-byte) boundary.
// The brick occupancy bits are derived from the stored densities with the
// march's own dequantisation, so "brick empty" means exactly that every
// density the march could load there is 0.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "fnr_internal.h"
#include "march_device.cuh"

namespace fnr {

namespace {

__device__ __forceinline__ float clamp_density(float v) { return v > 0.0f ? v : 0.0f; }

__device__ __forceinline__ unsigned char to_e4m3(float v) {
    return static_cast<unsigned char>(__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3));
}

unsigned grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 64) b = 152 * 64;
    return static_cast<unsigned>(b < 1 ? 1 : b);
}

// Order-preserving uint key of a binary32 value (NaN excluded by the callers).
__device__ __forceinline__ unsigned order_key(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_order_key(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Offset brick of cell index `cell` (x fastest): (z >> sh, y >> sh, x >> sh).
__device__ __forceinline__ int64_t offset_brick_of(int64_t cell, int k, int sh, int dim) {
    const int64_t x = cell % k, y = (cell / k) % k, z = cell / (static_cast<int64_t>(k) * k);
    return ((z >> sh) * dim + (y >> sh)) * dim + (x >> sh);
}

// One thread per cell of the slab, all channels; lanes of a warp whose cells
// share an offset brick combine their keys first, so each (warp, brick,
// channel) makes one atomic min and one atomic max.
__global__ void brick_minmax_kernel(const float *__restrict__ uvw, int64_t c0, int64_t n, int k, int nch, int sh,
                                    int dim, unsigned *__restrict__ kmin, unsigned *__restrict__ kmax) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t n_iter = (n + stride - 1) / stride;  // the same trip count for every lane (warp-wide sync)
    const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    for (int64_t it = 0; it < n_iter; ++it) {
        const int64_t i = first + it * stride;
        const bool in = i < n;
        const long long b = in ? offset_brick_of(c0 + i, k, sh, dim) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, b);
        const bool leader = in && (threadIdx.x & 31) == __ffs(same) - 1;
        for (int c = 0; c < nch; ++c) {
            const float v = in ? uvw[i * nch + c] : 0.0f;
            const bool ok = in && v == v;
            const unsigned lo = __reduce_min_sync(same, ok ? order_key(v) : 0xffffffffu);
            const unsigned hi = __reduce_max_sync(same, ok ? order_key(v) : 0u);
            if (leader) {
                if (lo != 0xffffffffu) atomicMin(kmin + b * nch + c, lo);
                if (hi != 0u) atomicMax(kmax + b * nch + c, hi);
            }
        }
    }
}

// Offsets: the binary16 (nearest even) value of (min + max) * 0.5 in binary32, 0 for a brick
// whose values were all NaN; the padding of each offset record is 0.
__global__ void brick_offsets_kernel(const unsigned *__restrict__ kmin, const unsigned *__restrict__ kmax,
                                     int64_t n_bricks, int nch, uint16_t *__restrict__ offs, int ostride) {
    const int64_t total = n_bricks * ostride;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / ostride;
        const int c = static_cast<int>(e - b * ostride);
        float m = 0.0f;
        if (c < nch && kmin[b * nch + c] != 0xffffffffu)
            m = (from_order_key(kmin[b * nch + c]) + from_order_key(kmax[b * nch + c])) * 0.5f;
        offs[e] = __half_as_ushort(__float2half_rn(m));
    }
}

__device__ __forceinline__ float offset_of(const uint16_t *__restrict__ offs, int64_t cell, int c, int k, int sh,
                                           int dim, int ostride) {
    return __half2float(__ushort_as_half(offs[offset_brick_of(cell, k, sh, dim) * ostride + c]));
}

// Per-channel absmax of |binary32(u - offset)| (NaN skipped) into amax_bits[1 + c].
__global__ void residual_absmax_kernel(const float *__restrict__ uvw, int64_t c0, int64_t n, int k, int nch,
                                       const uint16_t *__restrict__ offs, int sh, int dim, int ostride,
                                       unsigned *__restrict__ amax_bits) {
    __shared__ unsigned smax[3 * FNR_MAX_D];
    for (int c = threadIdx.x; c < nch; c += blockDim.x) smax[c] = 0u;
    __syncthreads();
    const int64_t total = n * nch;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nch;
        const int c = static_cast<int>(e - i * nch);
        const float r = fabsf(uvw[e] - offset_of(offs, c0 + i, c, k, sh, dim, ostride));
        if (r == r) atomicMax(&smax[c], __float_as_uint(r));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < nch; c += blockDim.x) atomicMax(&amax_bits[1 + c], smax[c]);
}

__global__ void convert_sigma_kernel(const float *__restrict__ in, void *__restrict__ out, int64_t n, int prec,
                                     const float *__restrict__ scale) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = clamp_density(in[i]);
        if (prec == FNR_PREC_FP32) static_cast<float *>(out)[i] = v;
        else if (prec == FNR_PREC_FP16) static_cast<__half *>(out)[i] = __float2half_rn(v);
        else static_cast<unsigned char *>(out)[i] = to_e4m3(__fdiv_rn(v, scale[0]));
    }
}

// One thread per output byte-group would waste bandwidth on the padding; one
// thread per (cell, channel) element, padding written by channel-0 threads.
__global__ void convert_uvw_kernel(const float *__restrict__ in, char *__restrict__ out, int64_t n_cells, int nch,
                                   int prec, int rec_stride, const float *__restrict__ scales,
                                   const uint16_t *__restrict__ offs, int64_t c0, int k, int sh, int dim,
                                   int ostride) {
    const int64_t total = n_cells * nch;
    const int es = prec == FNR_PREC_FP32 ? 4 : prec == FNR_PREC_FP16 ? 2 : 1;
    const int pad_bytes = rec_stride - nch * es;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t cell = e / nch;
        const int ch = static_cast<int>(e - cell * nch);
        char *rec = out + cell * rec_stride;
        const float v = in[e];
        if (prec == FNR_PREC_FP32) reinterpret_cast<float *>(rec)[ch] = v;
        else if (prec == FNR_PREC_FP16) reinterpret_cast<__half *>(rec)[ch] = __float2half_rn(v);
        else
            reinterpret_cast<unsigned char *>(rec)[ch] =
                to_e4m3(__fdiv_rn(__fsub_rn(v, offset_of(offs, c0 + cell, ch, k, sh, dim, ostride)), scales[1 + ch]));
        if (ch == 0)
            for (int b = 0; b < pad_bytes; ++b) rec[nch * es + b] = 0;
    }
}

__global__ void convert_beta_kernel(const float *__restrict__ in, void *__restrict__ out, int64_t n, int prec) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (prec == FNR_PREC_FP16) static_cast<__half *>(out)[i] = __float2half_rn(in[i]);
        else static_cast<float *>(out)[i] = in[i];
    }
}

// Channel absmax: channel 0 = clamped density, 1..nch = (u, v, w) channels.
// Non-negative binary32 values order like their bit patterns, so an unsigned
// atomicMax on the bits is an exact max. NaNs are skipped.
__global__ void absmax_kernel(const float *__restrict__ sigma, const float *__restrict__ uvw, int64_t n_cells, int nch,
                              unsigned *__restrict__ amax_bits) {
    __shared__ unsigned smax[1 + 3 * FNR_MAX_D];
    for (int c = threadIdx.x; c <= nch; c += blockDim.x) smax[c] = 0u;
    __syncthreads();
    unsigned local_s = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_cells; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = fabsf(clamp_density(sigma[i]));
        local_s = max(local_s, __float_as_uint(v));
    }
    atomicMax(&smax[0], local_s);
    const int64_t total = n_cells * nch;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const float v = fabsf(uvw[e]);
        if (v == v) atomicMax(&smax[1 + static_cast<int>(e % nch)], __float_as_uint(v));
    }
    __syncthreads();
    for (int c = threadIdx.x; c <= nch; c += blockDim.x) atomicMax(&amax_bits[c], smax[c]);
}

__global__ void scales_kernel(const unsigned *__restrict__ amax_bits, float *__restrict__ scales, int n) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n) {
        const float a = __uint_as_float(amax_bits[c]);
        scales[c] = a > 0.0f ? __fdiv_rn(a, 448.0f) : 1.0f;
    }
}

template <int PREC>
__global__ void occupancy_kernel(const CacheView v, uint32_t *__restrict__ words) {
    const int64_t k = v.k, n = k * k * k;
    const float sscale = PREC == FNR_PREC_FP8_E4M3 ? v.scales[0] : 1.0f;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        int brick = -1;
        if (dev::load_sigma<PREC>(v, static_cast<int>(i), sscale) > 0.0f) {
            const int x = static_cast<int>(i % k), y = static_cast<int>((i / k) % k), z = static_cast<int>(i / (k * k));
            brick = ((z >> v.occ_shift) * v.occ_dim + (y >> v.occ_shift)) * v.occ_dim + (x >> v.occ_shift);
        }
        // one atomic per distinct brick among the warp's active lanes
        const unsigned act = __activemask();
        const unsigned same = __match_any_sync(act, brick);
        if (brick >= 0 && (threadIdx.x & 31) == __ffs(same) - 1)
            atomicOr(words + (brick >> 5), 1u << (brick & 31));
    }
}

// Distance field for passing over empty space: the Chebyshev (L-infinity)
// distance, in jump bricks (2^m occupancy bricks a side), from each jump brick
// to the nearest occupied one. Initial pass: 0 for jump bricks holding an
// occupied brick, unset (255) for the others; pass r = 1 .. kDistCap gives r
// to every unset jump brick with a neighbour (3 x 3 x 3) at r - 1 -- one at
// distance r always has one, and one still unset after pass r - 1 is at
// distance >= r; updating in place is safe since a pass reads only r - 1 and
// writes r; the last pass gives kDistCap + 1 to those still unset.
__global__ void dist_init_kernel(const uint32_t *__restrict__ words, int nb, int m, uint8_t *__restrict__ dist,
                                 int nj) {
    const int64_t nj3 = static_cast<int64_t>(nj) * nj * nj;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < nj3; j += stride) {
        const int jx = static_cast<int>(j % nj), jy = static_cast<int>((j / nj) % nj), jz = static_cast<int>(j / nj / nj);
        bool occ = false;
        for (int z = jz << m; z < min((jz + 1) << m, nb) && !occ; ++z)
            for (int y = jy << m; y < min((jy + 1) << m, nb) && !occ; ++y)
                for (int x = jx << m; x < min((jx + 1) << m, nb) && !occ; ++x) {
                    const int64_t b = (static_cast<int64_t>(z) * nb + y) * nb + x;
                    occ = (words[b >> 5] >> (b & 31)) & 1u;
                }
        dist[j] = occ ? uint8_t(0) : uint8_t(255);
    }
}

__global__ void dist_pass_kernel(uint8_t *__restrict__ dist, int nb, int r) {
    const int64_t nb3 = static_cast<int64_t>(nb) * nb * nb;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < nb3; b += stride) {
        if (dist[b] != 255) continue;
        const int x = static_cast<int>(b % nb), y = static_cast<int>((b / nb) % nb), z = static_cast<int>(b / nb / nb);
        bool near = false;
        for (int dz = -1; dz <= 1 && !near; ++dz)
            for (int dy = -1; dy <= 1 && !near; ++dy)
                for (int dx = -1; dx <= 1 && !near; ++dx) {
                    const int xx = x + dx, yy = y + dy, zz = z + dz;
                    if (xx < 0 || yy < 0 || zz < 0 || xx >= nb || yy >= nb || zz >= nb) continue;
                    near = dist[(static_cast<int64_t>(zz) * nb + yy) * nb + xx] == r - 1;
                }
        if (near) dist[b] = static_cast<uint8_t>(r);
    }
}

__global__ void dist_cap_kernel(uint8_t *__restrict__ dist, int64_t nb3) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t b = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < nb3; b += stride)
        if (dist[b] == 255) dist[b] = static_cast<uint8_t>(kDistCap + 1);
}

// One pool element per thread: cell (x, y, z) of brick slot_brick[slot] at
// pool index slot B^3 + (lz B + ly) B + lx; cells past the grid edge are 0.
__global__ void gather_bricks_kernel(const char *__restrict__ sigma, const char *__restrict__ uvw,
                                     char *__restrict__ sigma_pool, char *__restrict__ uvw_pool,
                                     const int32_t *__restrict__ slot_brick, int64_t n_elems, int k, int shift,
                                     int dim, int s_sigma, int rec_stride) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int mask = (1 << shift) - 1;
    for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n_elems; e += stride) {
        const int64_t slot = e >> (3 * shift);
        const int local = static_cast<int>(e & ((int64_t(1) << (3 * shift)) - 1));
        const int brick = slot_brick[slot];
        const int bx = brick % dim, by = (brick / dim) % dim, bz = brick / (dim * dim);
        const int x = (bx << shift) + (local & mask), y = (by << shift) + ((local >> shift) & mask),
                  z = (bz << shift) + (local >> (2 * shift));
        const bool in = x < k && y < k && z < k;
        const int64_t cell = in ? (static_cast<int64_t>(z) * k + y) * k + x : 0;
        for (int b = 0; b < s_sigma; ++b) sigma_pool[e * s_sigma + b] = in ? sigma[cell * s_sigma + b] : char(0);
        const uint64_t *src = reinterpret_cast<const uint64_t *>(uvw + cell * rec_stride);
        uint64_t *dst = reinterpret_cast<uint64_t *>(uvw_pool + e * rec_stride);
        for (int w = 0; w < rec_stride / 8; ++w) dst[w] = in ? src[w] : 0ull;
    }
}

}  // namespace

cudaError_t launch_gather_bricks(const void *sigma, const char *uvw, void *sigma_pool, char *uvw_pool,
                                 const int32_t *slot_brick, int64_t n_bricks, int k, int shift, int dim,
                                 int s_sigma, int rec_stride, cudaStream_t s) {
    const int64_t n = n_bricks << (3 * shift);
    gather_bricks_kernel<<<grid_for(n, 256), 256, 0, s>>>(static_cast<const char *>(sigma), uvw,
                                                          static_cast<char *>(sigma_pool), uvw_pool, slot_brick, n, k,
                                                          shift, dim, s_sigma, rec_stride);
    return cudaGetLastError();
}

cudaError_t launch_occupancy(const CacheView &v, uint32_t *words, cudaStream_t s) {
    const int64_t n = static_cast<int64_t>(v.k) * v.k * v.k;
    const unsigned blocks = grid_for(n, 256);
    if (v.pos_prec == FNR_PREC_FP16) occupancy_kernel<FNR_PREC_FP16><<<blocks, 256, 0, s>>>(v, words);
    else if (v.pos_prec == FNR_PREC_FP8_E4M3) occupancy_kernel<FNR_PREC_FP8_E4M3><<<blocks, 256, 0, s>>>(v, words);
    else occupancy_kernel<FNR_PREC_FP32><<<blocks, 256, 0, s>>>(v, words);
    return cudaGetLastError();
}

cudaError_t launch_brick_distance(const uint32_t *words, int nb, int occ_shift, uint8_t *dist, int nj,
                                  int dist_shift, cudaStream_t s) {
    const int64_t nj3 = static_cast<int64_t>(nj) * nj * nj;
    if (nj3 <= 0) return cudaSuccess;
    const unsigned blocks = grid_for(nj3, 256);
    dist_init_kernel<<<blocks, 256, 0, s>>>(words, nb, dist_shift - occ_shift, dist, nj);
    for (int r = 1; r <= kDistCap; ++r) dist_pass_kernel<<<blocks, 256, 0, s>>>(dist, nj, r);
    dist_cap_kernel<<<blocks, 256, 0, s>>>(dist, nj3);
    return cudaGetLastError();
}

cudaError_t launch_convert_sigma(const float *in, void *out, int64_t n, int prec, const float *scale, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    convert_sigma_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n, prec, scale);
    return cudaGetLastError();
}

cudaError_t launch_convert_uvw(const float *in, char *out, int64_t n_cells, int D, int prec, int rec_stride,
                               const float *scales, cudaStream_t s, const uint16_t *offs, int64_t c0, int k,
                               int oshift, int odim, int ostride) {
    if (n_cells <= 0) return cudaSuccess;
    if (prec == FNR_PREC_FP8_E4M3 && !offs) return cudaErrorInvalidValue;
    convert_uvw_kernel<<<grid_for(n_cells * 3 * D, 256), 256, 0, s>>>(in, out, n_cells, 3 * D, prec, rec_stride,
                                                                        scales, offs, c0, k, oshift, odim, ostride);
    return cudaGetLastError();
}

cudaError_t launch_brick_minmax(const float *uvw, int64_t c0, int64_t n, int k, int nch, int oshift, int odim,
                                unsigned *kmin, unsigned *kmax, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    brick_minmax_kernel<<<grid_for(n, 256), 256, 0, s>>>(uvw, c0, n, k, nch, oshift, odim, kmin, kmax);
    return cudaGetLastError();
}

cudaError_t launch_brick_offsets(const unsigned *kmin, const unsigned *kmax, int64_t n_bricks, int nch,
                                 uint16_t *offs, int ostride, cudaStream_t s) {
    if (n_bricks <= 0) return cudaSuccess;
    brick_offsets_kernel<<<grid_for(n_bricks * ostride, 256), 256, 0, s>>>(kmin, kmax, n_bricks, nch, offs, ostride);
    return cudaGetLastError();
}

cudaError_t launch_residual_absmax(const float *uvw, int64_t c0, int64_t n, int k, int nch, const uint16_t *offs,
                                   int oshift, int odim, int ostride, unsigned *amax_bits, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    residual_absmax_kernel<<<grid_for(n * nch, 256), 256, 0, s>>>(uvw, c0, n, k, nch, offs, oshift, odim, ostride,
                                                                   amax_bits);
    return cudaGetLastError();
}

cudaError_t launch_convert_beta(const float *in, void *out, int64_t n, int prec, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    convert_beta_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n, prec);
    return cudaGetLastError();
}

cudaError_t launch_absmax(const float *sigma, const float *uvw, int64_t n_cells, int nch, unsigned *amax_bits,
                          cudaStream_t s) {
    if (n_cells <= 0) return cudaSuccess;
    absmax_kernel<<<grid_for(n_cells * nch, 256), 256, 0, s>>>(sigma, uvw, n_cells, nch, amax_bits);
    return cudaGetLastError();
}

cudaError_t launch_scales_from_absmax(const unsigned *amax_bits, float *scales, int n, cudaStream_t s) {
    scales_kernel<<<1, 64, 0, s>>>(amax_bits, scales, n);
    return cudaGetLastError();
}

}  // namespace fnr
