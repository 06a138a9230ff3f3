// mlp.cu -- cache build from the F_pos / F_dir MLPs on the 5th-generation
// tensor cores (Section 3.3: the caches hold F evaluated at every grid sample;
// Section 3.2 Eqs. 3-4 and Section 4: F_pos and F_dir are ReLU MLPs on
// positionally encoded inputs).
//
// One CTA per SM walks tiles of 128 grid points. Per tile:
//   1. every thread encodes one point (gamma(x) = sin / cos(2^j pi x), binary32,
//      rounded to bf16) into shared memory, in the UMMA K-major no-swizzle
//      layout (8 x 8 core matrices, 16 bytes per core-matrix row);
//   2. per layer: the layer's bf16 weights -- pre-arranged once in the same
//      core-matrix layout -- arrive in shared memory by bulk async copy
//      (cp.async.bulk, completion on an mbarrier); one elected thread issues
//      K/16 tcgen05.mma (M=128, N=layer width, bf16 x bf16 -> fp32) into a
//      tensor-memory accumulator and commits them to an mbarrier; four warps
//      read the accumulator back (tcgen05.ld, one 32-lane quarter each), add
//      the bias, apply ReLU, round to bf16 and write the next layer's input;
//   3. the last layer's outputs go straight to the cache: sigma = ReLU(out_0),
//      (u, v, w) = out_1..3D for F_pos; beta = out_0..D-1 for F_dir.
// Every mbarrier wait is bounded; a wait that runs out sets the error word and
// the CTA stops issuing work, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <vector>

#include "fnr_internal.h"

namespace fnr {

fnr_status fail(fnr_status st, const char *fmt, ...);
fnr_status cuda_fail(cudaError_t e, const char *what);

namespace {

constexpr int kTileM = 128;
constexpr int kMaxK = 256;
constexpr int kMaxN = 256;
constexpr int kThreads = 128;
constexpr int kMaxLayers = 16;
constexpr uint32_t kTmemCols = 256;
constexpr size_t kSmemA = size_t(kTileM) * kMaxK * 2;   // 64 KB activations
constexpr size_t kSmemB = size_t(kMaxN) * kMaxK * 2;    // 128 KB one layer of weights
constexpr size_t kSmemBytes = kSmemA + kSmemB + 64;
constexpr long long kWaitLimit = 1LL << 22;             // try_wait polls before giving up

struct MlpLayerDev {
    const __nv_bfloat16 *w;  // core-matrix layout, Np x Kp
    const float *b;          // Np (zero padded)
    int K, N;                // padded to multiples of 16
};

struct MlpArgs {
    MlpLayerDev L[kMaxLayers];
    int n_layers;
    int mode;        // 0: F_pos over the k^3 cell centres, 1: F_dir over the l x l bin centres
    int pe_freqs;
    int k, l;
    float bmin[3], h[3];
    long long n_points;
    // outputs
    void *sigma_out;   // mode 0
    char *uvw_out;     // mode 0
    int rec_stride, prec, D;
    void *beta_out;    // mode 1
    int dprec;
    int *err;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait: false (and the error word set) when the limit runs out.
// Only thread 0 waits; the CTA learns the outcome through a barrier.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err) {
    for (long long it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    atomicExch(err, 1);
    return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, no swizzle, 8x8 core matrices;
// lbo = byte distance between core matrices along K, sbo = along M / N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
    d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
    d |= uint64_t(1) << 46;  // descriptor version for this architecture
    return d;                // base offset 0, swizzle none
}

// Instruction descriptor, kind::f16: bf16 A and B (both K-major), fp32 D.
__device__ __forceinline__ uint32_t instr_desc(int M, int N) {
    uint32_t d = 0;
    d |= 1u << 4;                            // D format fp32
    d |= 1u << 7;                            // A format bf16
    d |= 1u << 10;                           // B format bf16
    d |= uint32_t(N >> 3) << 17;
    d |= uint32_t(M >> 4) << 24;
    return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, k) in a K-major core-matrix tile with Kp columns.
__device__ __forceinline__ uint32_t cm_offset(int row, int k, int Kp) {
    return uint32_t((row >> 3) * (Kp >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return uint32_t(__bfloat16_as_ushort(x)) | (uint32_t(__bfloat16_as_ushort(y)) << 16);
}

// Positional encoding of this thread's point into row `row` of the A tile.
__device__ __forceinline__ void encode_point(const MlpArgs &A, long long p, int row, char *sa) {
    const int K0 = A.L[0].K;
    float x[3] = {0.0f, 0.0f, 0.0f};
    const bool valid = p < A.n_points;
    if (valid) {
        if (A.mode == 0) {
            const long long kk = A.k;
            const int ix = int(p % kk), iy = int((p / kk) % kk), iz = int(p / (kk * kk));
            x[0] = fmaf(float(ix) + 0.5f, A.h[0], A.bmin[0]);
            x[1] = fmaf(float(iy) + 0.5f, A.h[1], A.bmin[1]);
            x[2] = fmaf(float(iz) + 0.5f, A.h[2], A.bmin[2]);
        } else {
            const int it = int(p / A.l), ip = int(p % A.l);
            float st, ct, sp, cp;
            sincospif((float(it) + 0.5f) / float(A.l), &st, &ct);          // theta / pi
            sincospif(2.0f * (float(ip) + 0.5f) / float(A.l), &sp, &cp);   // phi / pi
            x[0] = st * cp;
            x[1] = st * sp;
            x[2] = ct;
        }
    }
    const int Lf = A.pe_freqs;
    for (int g = 0; g < K0; g += 8) {  // 8 encoded values per 16-byte store
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int col = g + q;
            float val = 0.0f;
            if (valid && col < 6 * Lf) {
                const int a = col / (2 * Lf), r = col % (2 * Lf), j = r >> 1;
                const float arg = ldexpf(x[a], j);  // 2^j x, exact
                val = (r & 1) ? cospif(arg) : sinpif(arg);
            }
            v[q] = val;
        }
        uint4 pk;
        pk.x = pack_bf16(v[0], v[1]);
        pk.y = pack_bf16(v[2], v[3]);
        pk.z = pack_bf16(v[4], v[5]);
        pk.w = pack_bf16(v[6], v[7]);
        *reinterpret_cast<uint4 *>(sa + cm_offset(row, g, K0)) = pk;
    }
}

__global__ void __launch_bounds__(kThreads, 1) mlp_kernel(const __grid_constant__ MlpArgs A) {
    extern __shared__ __align__(1024) char smem[];
    char *sa = smem;
    char *sb = smem + kSmemA;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kSmemA + kSmemB);  // [0] weights, [1] mma
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2);
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar_w = smem_u32(&bars[0]), bar_m = smem_u32(&bars[1]);

    if (tid == 0) {
        mbar_init(bar_w, 1);
        mbar_init(bar_m, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    uint32_t ph_w = 0, ph_m = 0;

    const long long n_tiles = (A.n_points + kTileM - 1) / kTileM;
    bool aborted = false;  // uniform across the CTA: read only after a barrier
    for (long long tile = blockIdx.x; tile < n_tiles && !aborted; tile += gridDim.x) {
        const long long p = tile * kTileM + tid;
        encode_point(A, p, tid, sa);
        fence_proxy_async();
        __syncthreads();
        for (int li = 0; li < A.n_layers; ++li) {
            const MlpLayerDev &Ly = A.L[li];
            const int K = Ly.K, N = Ly.N;
            const bool last = li + 1 == A.n_layers;
            // Thread 0 stages the layer's weights, issues its MMAs and waits for
            // them; the other threads learn the outcome at the barrier.
            if (tid == 0) {
                const uint32_t bytes = uint32_t(N) * uint32_t(K) * 2u;
                mbar_expect_tx(bar_w, bytes);
                const char *src = reinterpret_cast<const char *>(Ly.w);
                for (uint32_t off = 0; off < bytes; off += 32768u) {
                    const uint32_t chunk = bytes - off < 32768u ? bytes - off : 32768u;
                    bulk_g2s(smem_u32(sb) + off, src + off, chunk, bar_w);
                }
                bool ok = mbar_wait(bar_w, ph_w, A.err);
                if (ok) {
                    tc_fence_after();
                    const uint32_t idesc = instr_desc(kTileM, N);
                    const uint32_t sbo = uint32_t(K >> 3) * 128u;
                    for (int s = 0; s < K / 16; ++s) {
                        const uint64_t ad = smem_desc(smem_u32(sa) + uint32_t(s) * 256u, 128u, sbo);
                        const uint64_t bd = smem_desc(smem_u32(sb) + uint32_t(s) * 256u, 128u, sbo);
                        umma_bf16(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
                    }
                    umma_commit(bar_m);
                    ok = mbar_wait(bar_m, ph_m, A.err);
                }
                abort_flag = ok ? 0 : 1;
                tc_fence_before();
            }
            ph_w ^= 1u;
            ph_m ^= 1u;
            __syncthreads();
            tc_fence_after();
            if (abort_flag) {
                aborted = true;
                break;
            }
            // epilogue: this warp's 32 rows of the accumulator (warp-collective
            // loads; stores predicated per row)
            const uint32_t trow = tmem + (uint32_t(warp * 32) << 16);
            const int row = tid;
            const bool valid = p < A.n_points;
            for (int c0 = 0; c0 < N; c0 += 16) {
                float v[16];
                tmem_ld16(trow + uint32_t(c0), v);
                if (!last) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = fmaxf(v[q] + __ldg(Ly.b + c0 + q), 0.0f);
#pragma unroll
                    for (int g = 0; g < 16; g += 8) {
                        uint4 pk;
                        pk.x = pack_bf16(v[g + 0], v[g + 1]);
                        pk.y = pack_bf16(v[g + 2], v[g + 3]);
                        pk.z = pack_bf16(v[g + 4], v[g + 5]);
                        pk.w = pack_bf16(v[g + 6], v[g + 7]);
                        *reinterpret_cast<uint4 *>(sa + cm_offset(row, c0 + g, N)) = pk;
                    }
                } else if (valid) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int c = c0 + q;
                        const float o = v[q] + __ldg(Ly.b + c);
                        if (A.mode == 0) {
                            if (c == 0) {
                                const float sg = fmaxf(o, 0.0f);
                                if (A.prec == FNR_PREC_FP16) static_cast<__half *>(A.sigma_out)[p] = __float2half_rn(sg);
                                else static_cast<float *>(A.sigma_out)[p] = sg;
                            } else if (c <= 3 * A.D) {
                                char *rec = A.uvw_out + p * A.rec_stride;
                                if (A.prec == FNR_PREC_FP16)
                                    reinterpret_cast<__half *>(rec)[c - 1] = __float2half_rn(o);
                                else reinterpret_cast<float *>(rec)[c - 1] = o;
                            }
                        } else if (c < A.D) {
                            if (A.dprec == FNR_PREC_FP16)
                                static_cast<__half *>(A.beta_out)[p * A.D + c] = __float2half_rn(o);
                            else static_cast<float *>(A.beta_out)[p * A.D + c] = o;
                        }
                    }
                }
            }
            tc_fence_before();
            fence_proxy_async();
            __syncthreads();
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
    }
}

// W [N][K] row-major bf16 bits -> padded core-matrix layout [Np][Kp].
__global__ void relayout_kernel(const uint16_t *__restrict__ w, int N, int K, uint16_t *__restrict__ out, int Np,
                                int Kp) {
    const int total = Np * Kp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int n = e / Kp, k = e - n * Kp;
        const uint16_t v = (n < N && k < K) ? w[size_t(n) * K + k] : uint16_t(0);
        const size_t off = size_t(n >> 3) * (Kp >> 3) * 64 + size_t(k >> 3) * 64 + size_t(n & 7) * 8 + (k & 7);
        out[off] = v;
    }
}

__global__ void pad_bias_kernel(const float *__restrict__ b, int N, float *__restrict__ out, int Np) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np) out[i] = i < N ? b[i] : 0.0f;
}

int round16(int v) { return (v + 15) / 16 * 16; }

}  // namespace

// Validate one MLP description; n_out_min is the number of outputs needed.
fnr_status check_mlp(const fnr_mlp *m, int n_out_min, const char *name) {
    if (!m) return fail(FNR_ERR_INVALID_ARG, "%s is NULL", name);
    if (m->n_layers < 1 || m->n_layers > kMaxLayers)
        return fail(FNR_ERR_INVALID_ARG, "%s: n_layers %d outside [1, %d]", name, m->n_layers, kMaxLayers);
    if (m->pe_in != 3) return fail(FNR_ERR_UNSUPPORTED, "%s: pe_in must be 3", name);
    if (m->pe_freqs < 1 || 6 * m->pe_freqs > m->dims[0])
        return fail(FNR_ERR_INVALID_ARG, "%s: dims[0]=%d cannot hold 2*3*%d encoded inputs", name, m->dims[0],
                    m->pe_freqs);
    for (int i = 0; i <= m->n_layers; ++i)
        if (m->dims[i] < 1 || round16(m->dims[i]) > kMaxK)
            return fail(FNR_ERR_UNSUPPORTED, "%s: layer width %d outside [1, %d]", name, m->dims[i], kMaxK);
    if (m->dims[m->n_layers] < n_out_min)
        return fail(FNR_ERR_INVALID_ARG, "%s: %d outputs, need %d", name, m->dims[m->n_layers], n_out_min);
    for (int i = 0; i < m->n_layers; ++i)
        if (!m->weights[i] || !m->biases[i]) return fail(FNR_ERR_INVALID_ARG, "%s: NULL layer %d", name, i);
    return FNR_OK;
}

// Evaluate one MLP over its grid into the cache (mode 0: F_pos, 1: F_dir).
fnr_status run_mlp(const fnr_mlp *m, int mode, const fnr_cache_desc &d, const CacheView &v, int num_sms,
                   cudaStream_t s) {
    struct Buf {
        void *p = nullptr;
        ~Buf() {
            if (p) cudaFree(p);
        }
    } wbuf, bbuf, ebuf;
    size_t welems = 0, belems = 0;
    for (int i = 0; i < m->n_layers; ++i) {
        welems += size_t(round16(m->dims[i + 1])) * round16(m->dims[i]);
        belems += size_t(round16(m->dims[i + 1]));
    }
    cudaError_t e;
    if ((e = cudaMalloc(&wbuf.p, welems * 2)) != cudaSuccess) return cuda_fail(e, "MLP weights");
    if ((e = cudaMalloc(&bbuf.p, belems * 4)) != cudaSuccess) return cuda_fail(e, "MLP biases");
    if ((e = cudaMalloc(&ebuf.p, 4)) != cudaSuccess) return cuda_fail(e, "MLP error word");
    if ((e = cudaMemsetAsync(ebuf.p, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "memset");
    MlpArgs A;
    memset(&A, 0, sizeof(A));
    size_t wo = 0, bo = 0;
    for (int i = 0; i < m->n_layers; ++i) {
        const int K = m->dims[i], N = m->dims[i + 1], Kp = round16(K), Np = round16(N);
        uint16_t *wd = static_cast<uint16_t *>(wbuf.p) + wo;
        float *bd = static_cast<float *>(bbuf.p) + bo;
        relayout_kernel<<<(Np * Kp + 255) / 256, 256, 0, s>>>(m->weights[i], N, K, wd, Np, Kp);
        pad_bias_kernel<<<(Np + 255) / 256, 256, 0, s>>>(m->biases[i], N, bd, Np);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "MLP weight layout");
        A.L[i].w = reinterpret_cast<const __nv_bfloat16 *>(wd);
        A.L[i].b = bd;
        A.L[i].K = Kp;
        A.L[i].N = Np;
        wo += size_t(Np) * Kp;
        bo += size_t(Np);
    }
    A.n_layers = m->n_layers;
    A.mode = mode;
    A.pe_freqs = m->pe_freqs;
    A.k = d.k;
    A.l = d.l;
    for (int a = 0; a < 3; ++a) {
        A.bmin[a] = d.bmin[a];
        A.h[a] = static_cast<float>((static_cast<double>(d.bmax[a]) - d.bmin[a]) / d.k);
    }
    A.n_points = mode == 0 ? (long long)d.k * d.k * d.k : (long long)d.l * d.l;
    A.sigma_out = const_cast<void *>(v.sigma);
    A.uvw_out = const_cast<char *>(v.uvw);
    A.rec_stride = v.rec_stride;
    A.prec = d.pos_precision;
    A.D = d.D;
    A.beta_out = const_cast<void *>(v.beta);
    A.dprec = d.dir_precision;
    A.err = static_cast<int *>(ebuf.p);
    if ((e = cudaFuncSetAttribute(mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kSmemBytes))) !=
        cudaSuccess)
        return cuda_fail(e, "MLP smem attribute");
    const long long tiles = (A.n_points + kTileM - 1) / kTileM;
    const int grid = int(tiles < num_sms ? tiles : num_sms);
    mlp_kernel<<<grid, kThreads, kSmemBytes, s>>>(A);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "MLP launch");
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, ebuf.p, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "MLP sync");
    if (herr) return fail(FNR_ERR_DEVICE, "MLP kernel: an mbarrier wait ran out");
    return FNR_OK;
}

}  // namespace fnr
