// mlp.cu -- cache build from the F_pos / F_dir MLPs on the 5th-generation
// tensor cores (Section 3.3: the caches hold F evaluated at every grid sample;
// Section 3.2 Eqs. 3-4 and Section 4: F_pos and F_dir are ReLU MLPs on
// positionally encoded inputs).
//
// The kernel has two forms (template parameter CTAS). The default, CTAS = 1:
// one CTA per SM walks tiles of 128 grid points. CTAS = 2: a cluster of two
// CTAs on an SM pair walks tiles of 256 points, 128 per CTA; rank 0 issues
// M = 256 MMAs for both (tcgen05.mma.cta_group::2), which read each CTA's A
// rows and each CTA's half of the weight chunk from that CTA's own shared
// memory and accumulate into each CTA's own tensor memory, so each SM streams
// half of every chunk. Warp roles, in every CTA:
//   producer (warp 0): streams every layer's bf16 weights (this CTA's half of
//     each chunk in the pair form), pre-arranged in 64-column K chunks of the
//     K-major 128-byte swizzled operand layout, through a shared-memory ring by
//     bulk async copy (cp.async.bulk, completion on the slot's "full"
//     mbarrier), running ahead across layers and tiles. The single-CTA ring has
//     2 slots of 32 KB, loaded once per tile; the pair form's has 4 slots of
//     16 KB -- a whole layer -- loaded once per layer for both tiles in flight;
//   two tiles are in flight: each has its own A tile (same swizzled layout)
//     and its own tensor-memory accumulator, so one tile's epilogue runs while
//     the other's MMAs do;
//   encoders (warps 2-3): encode each tile's points (gamma(x) = sin / cos(2^j
//     pi x), rounded to bf16) into the tile's layer-0 staging buffer one tile
//     pair ahead, as soon as the MMAs that read the buffer's previous contents
//     have completed, so encoding never waits between tiles;
//   MMA issuer (warp 1, one lane; rank 0 in the pair form): waits for the layer
//     input and each chunk, issues tcgen05.mma (K=16 steps, bf16 x bf16 -> fp32
//     in tensor memory; layer 0 reads the staging buffer), releases each slot
//     with tcgen05.commit on its "empty" mbarrier and signals the finished
//     accumulator with one more commit; in rank 1 of a pair the same lane tells
//     rank 0 when each chunk half has landed;
//   epilogue (warps 4-19, four per 32-lane quarter of tensor memory): per
//     hidden layer read the accumulator (tcgen05.ld), add the bias, apply
//     ReLU, round to bf16 and write the next layer's A tile; after the head,
//     stage the outputs in the (now free) A tile as fp32 rows and write the
//     tile's sigma = ReLU(out_0), (u, v, w) = out_1..3D (F_pos) or beta =
//     out_0..D-1 (F_dir) -- contiguous ranges of the cache -- with coalesced
//     stores by all sixteen warps.
// In the pair form rank 0 issues each tcgen05.commit twice, on its own copy of
// the barrier and, through the barrier's cluster address, on rank 1's; rank 1's
// threads arrive on rank 0's barriers with remote mbarrier arrives. The next
// layer's weights load while the epilogue runs. Every mbarrier wait is bounded;
// a wait that runs out sets the error word and the abort flags of the CTA (and
// of its pair), every role leaves its loop, each producer waits (bounded) for
// the copies it has in flight, the MMA issuer for its tensor-core operations
// (rank 1 for the same commit), and the tensor memory is freed. Both forms
// compute every product in the same order; the pair form measured slower (its
// hand-offs between the two SMs lengthen the refill and epilogue chains), so
// the single-CTA form is the default and the pair form is chosen only through
// the test hook fnr_testing_mlp_cta_pair.
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
constexpr int kChunkK = 64;                          // K columns per weight chunk: one 128-byte swizzle row
#ifndef FNR_MLP_PAIR
#define FNR_MLP_PAIR 2
#endif
#ifndef FNR_MLP_BIAS_SMEM
#define FNR_MLP_BIAS_SMEM 0
#endif
constexpr int kPair = FNR_MLP_PAIR;                  // tiles in flight per CTA
#ifndef FNR_MLP_FIRST_EPI
#define FNR_MLP_FIRST_EPI 4
#endif
#ifndef FNR_MLP_KATTR
#define FNR_MLP_KATTR __launch_bounds__(kThreads, 1)
#endif
// epilogue warp w reads tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31
constexpr int kProducerWarp = 0, kMmaWarp = 1, kEncWarp0 = 2, kEncWarps = 2;
constexpr int kFirstEpiWarp = FNR_MLP_FIRST_EPI, kEpiWarps = 16;
static_assert(kFirstEpiWarp >= kEncWarp0 + kEncWarps && kFirstEpiWarp % 4 == 0, "warp roles");
constexpr int kThreads = (kFirstEpiWarp + kEpiWarps) * 32;
constexpr int kMaxK0 = kChunkK;     // the encoded input (layer 0's K) fits one staging chunk
constexpr int kMaxHeadOut = 64;     // outputs per point staged after the head
constexpr int kMaxLayers = 16;
constexpr int kMaxBias = kMaxLayers * kMaxN;
constexpr uint32_t kTmemCols = 256 * kPair;                                // one accumulator per tile
constexpr size_t kSmemA = size_t(kPair) * kTileM * kMaxK * 2;               // 64 KB activations per tile
constexpr size_t kStageBytes = size_t(kTileM) * kMaxK0 * 2;                 // 16 KB layer-0 input per tile
constexpr size_t kSmemStage = size_t(kPair) * kStageBytes;
constexpr size_t kSmemBias = FNR_MLP_BIAS_SMEM ? size_t(kMaxBias) * 4 : 0;  // 16 KB biases (else read via L1)
static_assert(size_t(kTileM) * (kMaxHeadOut + 4) * 4 <= size_t(kTileM) * kMaxK * 2, "head staging fits an A tile");

// The two forms of the kernel. CTAS = 1: one CTA per SM issues M = 128 MMAs
// and streams whole 64-column weight chunks through a 2-slot ring. CTAS = 2:
// a cluster of two CTAs on an SM pair; rank 0 issues M = 256 MMAs for both
// (tcgen05 cta_group::2), each CTA holds 128 rows of A and half of every weight
// chunk, and the 4-slot ring holds a whole layer's chunk halves, which both
// tiles in flight read from one load.
template <int CTAS>
struct Form {
    static_assert(CTAS == 1 || CTAS == 2, "CTAs per MMA");
    static constexpr bool kShare = CTAS == 2;                       // a layer's chunks serve both tiles
    static constexpr int kSuperM = kTileM * CTAS;                   // points per MMA tile
    static constexpr int kSlots = 2 * CTAS;                         // ring slots
    static constexpr int kSlotBytes = kMaxN / CTAS * kChunkK * 2;   // this CTA's rows of one weight chunk
    static constexpr size_t kSmemRing = size_t(kSlots) * kSlotBytes;
    // full, empty, pair_full; per tile slot acc_full, a_ready, enc_ready, enc_free, head_ready; drain
    static constexpr int kBars = 3 * kSlots + 5 * kPair + 1;
    static constexpr size_t kSmemBars = (size_t(kBars) * 8 + 16 + 127) / 128 * 128;
    static constexpr size_t kSmemBytes = kSmemA + kSmemStage + kSmemRing + kSmemBias + kSmemBars + 1024;  // + slack
    static_assert(kSmemBytes <= 232448, "shared memory per CTA");
    static_assert(!kShare || kMaxK / kChunkK <= kSlots, "a layer's chunks fit the ring");
};
constexpr long long kWaitLimit = 1LL << 22;                                 // try_wait polls before giving up
constexpr long long kDrainLimit = 1LL << 22;                                // polls for in-flight work at exit

struct MlpLayerDev {
    const __nv_bfloat16 *w;  // chunk-major: chunk c = [Np][64] in the 128-byte swizzled K-major layout
    int K, N;                // padded to multiples of 16
    int bias_off;            // offset of this layer's Np biases in the bias table
};

struct MlpArgs {
    MlpLayerDev L[kMaxLayers];
    const float *bias;       // all layers' padded biases
    int n_bias;
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
    // mode 2: F evaluated at listed points (positions, or unit directions for F_dir); the head's
    // first out_stride outputs go to out[p * out_stride + c] in FP32 (channel 0 through ReLU if relu0)
    const float *points;  // [n_points][3]
    float *out;
    int out_stride, relu0;
    int n_out;        // outputs stored per point: 1 + 3D (mode 0), D (mode 1), out_stride (mode 2)
    int head_stride;  // floats per staged head row: round16(n_out) + 4
    int *err;
    long long wait_limit;  // polls before a wait gives up (kWaitLimit unless a test armed a fault)
    long long withhold;    // test fault: the producer withholds its chunk of this index (-1: none)
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

// kCluster: acquire at cluster scope, for a barrier that the other CTA of the
// pair arrives on with data of its own to order (epilogue and encoder
// hand-offs); else the default CTA scope (weight chunks, slot releases,
// accumulators: completions of the pair's own copies and tensor-core work).
template <bool kCluster>
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    if (kCluster)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
    return ok != 0;
}

// The same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cluster_addr(uint32_t local, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

// Arrive on an mbarrier of the other CTA of the pair (address from cluster_addr).
__device__ __forceinline__ void mbar_arrive_remote(uint32_t addr) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release;\n barrier.cluster.wait.acquire;" ::: "memory");
}

// Bounded wait: false when `limit` polls run out (the error word and the
// CTA's abort flag -- and the peer CTA's, at cluster address peer_abort if
// non-zero -- are then set) or when another role has aborted.
template <bool kCluster>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, volatile int *abort_flag,
                                          long long limit, uint32_t peer_abort) {
    for (long long it = 0; it < limit; ++it) {
        if (mbar_try_wait<kCluster>(bar, parity)) return true;
        if ((it & 1023) == 1023 && *abort_flag) return false;
    }
    atomicExch(err, 1);
    *abort_flag = 1;
    if (peer_abort) asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(peer_abort), "r"(1) : "memory");
    return false;
}

// Bounded wait at exit for work this CTA has in flight, abort or not; false
// (and the error word set) if it does not complete within kDrainLimit polls.
template <bool kCluster>
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity, int *err) {
    for (long long it = 0; it < kDrainLimit; ++it)
        if (mbar_try_wait<kCluster>(bar, parity)) return true;
    atomicExch(err, 2);
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major with the 128-byte swizzle: rows of
// 64 bf16 (128 bytes), 8-row atoms of 1024 bytes stacked along M / N
// (stride 1024), the 16-byte pieces of row r stored at piece index ^ (r & 7).
// Atoms start on 1024-byte boundaries; a K step of 16 inside the atom row
// advances the start address by 32 bytes. The leading-dimension offset is
// unused by this layout (encoded as 1).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= uint64_t((addr >> 4) & 0x3FFFu);
    d |= uint64_t(1) << 16;                 // leading byte offset (unused), 16 bytes
    d |= uint64_t(1024 >> 4) << 32;         // stride byte offset: 8 rows x 128 bytes
    d |= uint64_t(1) << 46;                 // descriptor version for this architecture
    d |= uint64_t(2) << 61;                 // swizzle mode: 128 bytes
    return d;                               // base offset 0
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

template <int CTAS>
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    if constexpr (CTAS == 2)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::
                "r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
}

// Arrive on the mbarrier at shared::cluster address `bar` when every tcgen05
// operation this thread has issued so far has completed.
template <int CTAS>
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    if constexpr (CTAS == 2)
        asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
    else
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// Tensor-memory allocation of `cols` columns by one whole warp (in both CTAs of a pair,
// together), its address written to shared memory at `slot`; and its release.
template <int CTAS>
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t cols) {
    if constexpr (CTAS == 2) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
}

template <int CTAS>
__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t cols) {
    if constexpr (CTAS == 2)
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
    else
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(cols) : "memory");
}

// 16 columns of this warp's TMEM lane quarter, without waiting (see tmem_wait).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Byte offset of element (row, k) of the A tile (kTileM rows) in the 128-byte
// swizzled K-major layout: 64-column K blocks of kTileM / 8 atoms each.
__device__ __forceinline__ uint32_t a_offset(int row, int k) {
    return uint32_t((k >> 6) * (kTileM / 8) * 1024 + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((k >> 3) & 7) ^ (row & 7)) << 4) + (k & 7) * 2);
}

// ReLU(a), ReLU(b) rounded to bf16 (nearest even) and packed, a in the low
// half, in one conversion; a negative value rounds to a negative bf16, so
// clamping after rounding equals rounding after clamping.
__device__ __forceinline__ uint32_t pack_relu_bf16(float a, float b) {
    uint32_t d;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(b), "f"(a));
    return d;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat16 x = __float2bfloat16_rn(a), y = __float2bfloat16_rn(b);
    return uint32_t(__bfloat16_as_ushort(x)) | (uint32_t(__bfloat16_as_ushort(y)) << 16);
}

// Positional encoding of point p into row `row` of a layer-0 A tile (K0 <= 64
// columns, one 128-byte swizzled row): column 2 P + 0 / 1 holds sin / cos(2^j
// pi x_a) with P = a L + j, rounded to bf16; columns from 6 L on, and every
// column of a point past the end, are 0.
__device__ __forceinline__ void encode_point(const MlpArgs &A, long long p, int row, char *sa) {
    const int K0 = A.L[0].K;
    float x0 = 0.0f, x1 = 0.0f, x2 = 0.0f;
    const bool valid = p < A.n_points;
    if (valid) {
        if (A.mode == 2) {
            x0 = A.points[3 * p];
            x1 = A.points[3 * p + 1];
            x2 = A.points[3 * p + 2];
        } else if (A.mode == 0) {
            int ix, iy, iz;
            if (A.n_points <= 0x7fffffffLL) {  // 32-bit index arithmetic
                const unsigned k = unsigned(A.k), q = unsigned(p);
                const unsigned yz = q / k;
                ix = int(q - yz * k);
                iz = int(yz / k);
                iy = int(yz - unsigned(iz) * k);
            } else {
                const long long kk = A.k;
                ix = int(p % kk);
                iy = int((p / kk) % kk);
                iz = int(p / (kk * kk));
            }
            x0 = fmaf(float(ix) + 0.5f, A.h[0], A.bmin[0]);
            x1 = fmaf(float(iy) + 0.5f, A.h[1], A.bmin[1]);
            x2 = fmaf(float(iz) + 0.5f, A.h[2], A.bmin[2]);
        } else {
            const unsigned q = unsigned(p), l = unsigned(A.l);
            const int it = int(q / l), ip = int(q - unsigned(it) * l);
            float st, ct, sp, cp;
            sincospif((float(it) + 0.5f) / float(A.l), &st, &ct);         // theta / pi
            sincospif(2.0f * (float(ip) + 0.5f) / float(A.l), &sp, &cp);  // phi / pi
            x0 = st * cp;
            x1 = st * sp;
            x2 = ct;
        }
    }
    const int nP = valid ? 3 * A.pe_freqs : 0;
    int a = 0, j = 0;  // (a, j) of P, advanced with P
    for (int g = 0; g < K0; g += 8) {  // 8 encoded values per 16-byte store
        float v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int P = (g >> 1) + q;
            float sv = 0.0f, cv = 0.0f;
            if (P < nP) {
                const float xa = a == 0 ? x0 : (a == 1 ? x1 : x2);
                sincospif(xa * __int_as_float((127 + j) << 23), &sv, &cv);  // 2^j x_a, exact
                if (++j == A.pe_freqs) {
                    j = 0;
                    ++a;
                }
            }
            v[2 * q] = sv;
            v[2 * q + 1] = cv;
        }
        uint4 pk;
        pk.x = pack_bf16(v[0], v[1]);
        pk.y = pack_bf16(v[2], v[3]);
        pk.z = pack_bf16(v[4], v[5]);
        pk.w = pack_bf16(v[6], v[7]);
        *reinterpret_cast<uint4 *>(sa + a_offset(row, g)) = pk;
    }
}

__device__ __forceinline__ int n_chunks(int K) { return K / kChunkK; }  // K is padded to a multiple of 64

template <int CTAS>
__global__ void FNR_MLP_KATTR mlp_kernel(const __grid_constant__ MlpArgs A) {
    using F = Form<CTAS>;
    constexpr int kCtas = CTAS, kSlots = F::kSlots, kSlotBytes = F::kSlotBytes, kBars = F::kBars;
    constexpr long long kSuperM = F::kSuperM;
    constexpr bool kShare = F::kShare;
    constexpr size_t kSmemRing = F::kSmemRing;
    extern __shared__ __align__(1024) char smem_raw[];
    // the swizzled operand tiles start on 1024-byte boundaries
    char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    char *sa = smem;                 // A tile of slot t at sa + t * kTileM * kMaxK * 2
    char *stage = smem + kSmemA;     // layer-0 input of slot t at stage + t * kStageBytes
    char *ring = stage + kSmemStage;
    float *sbias = reinterpret_cast<float *>(ring + kSmemRing);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ring + kSmemRing + kSmemBias);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + kBars);
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // Rank in the CTA pair: rank 0 issues the MMAs for both; every shared-memory
    // layout below is the same in both CTAs, so an address names the same
    // object in either.
    uint32_t rank = 0;
    if (kCtas == 2) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const bool leader = rank == 0;
    // bars: [0, kSlots) full, [kSlots, 2 kSlots) empty, [2 kSlots, 3 kSlots) pair_full, then per tile slot:
    // acc_full, a_ready, enc_ready, enc_free, head_ready
    const uint32_t bar0 = smem_u32(bars);
    auto full_bar = [&](int s) { return bar0 + 8u * uint32_t(s); };
    auto empty_bar = [&](int s) { return bar0 + 8u * uint32_t(kSlots + s); };
    // pair_full(s) (rank 0): the other CTA's part of the chunk in slot s has landed
    auto pair_full = [&](int s) { return bar0 + 8u * uint32_t(2 * kSlots + s); };
    auto tile_bar = [&](int which, int t) { return bar0 + 8u * uint32_t(3 * kSlots + which * kPair + t); };
    // acc_full(t): the tile's accumulator holds a finished layer (one tcgen05.commit; rank 1: one relayed arrive)
    auto acc_full = [&](int t) { return tile_bar(0, t); };
    // a_ready(t) (rank 0): the accumulators have been read and the next layer's A tiles written (every epilogue
    // warp of both CTAs)
    auto a_ready = [&](int t) { return tile_bar(1, t); };
    // enc_ready(t) (rank 0): the staging buffers hold the encoded points of the tile's next pair (the encoder
    // warps of both CTAs)
    auto enc_ready = [&](int t) { return tile_bar(2, t); };
    // enc_free(t): the layer-0 MMAs that read the staging buffers have completed (commit; rank 1: relayed)
    auto enc_free = [&](int t) { return tile_bar(3, t); };
    // head_ready(t): every epilogue warp of this CTA has staged its head outputs
    auto head_ready = [&](int t) { return tile_bar(4, t); };
    // drain: every tensor-core operation of the pair has completed (commit; rank 1: relayed)
    const uint32_t drain_bar = bar0 + 8u * uint32_t(3 * kSlots + 5 * kPair);
    constexpr uint32_t kATileBytes = uint32_t(kTileM) * kMaxK * 2;
    // the same barrier in the other CTA of the pair, and arrivals that go to rank 0's copy
    auto other = [&](uint32_t bar) { return cluster_addr(bar, rank ^ 1u); };
    auto arrive_at_leader = [&](uint32_t bar) {
        if (leader) mbar_arrive(bar);
        else mbar_arrive_remote(other(bar));
    };
    const uint32_t peer_abort =
        kCtas == 2 ? cluster_addr(smem_u32(const_cast<int *>(&abort_flag)), rank ^ 1u) : 0u;

    if (FNR_MLP_BIAS_SMEM)
        for (int i = tid; i < A.n_bias; i += kThreads) sbias[i] = A.bias[i];
    if (tid == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
            mbar_init(pair_full(s), 1);
        }
        for (int t = 0; t < kPair; ++t) {
            mbar_init(acc_full(t), 1);
            mbar_init(a_ready(t), kEpiWarps * kCtas);
            mbar_init(enc_ready(t), kEncWarps * kCtas);
            mbar_init(enc_free(t), 1);
            mbar_init(head_ready(t), kEpiWarps);
        }
        mbar_init(drain_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kMmaWarp) tmem_alloc<CTAS>(smem_u32(tmem_slot), kTmemCols);  // both CTAs of a pair together
    tc_fence_before();
    __syncthreads();
    if (kCtas == 2) cluster_sync();  // both CTAs' barriers are initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    // MMA tiles of kSuperM points go to CTAs (pairs) in groups of kPair: group r holds tiles
    // (kPair r + t) * grid + bid, t < kPair; a tile past the end is carried as an empty one (no outputs).
    // CTA `rank` of a pair holds rows [rank kTileM, rank kTileM + kTileM) of each tile.
    const long long n_tiles = (A.n_points + kSuperM - 1) / kSuperM;
    const long long G = gridDim.x / kCtas;
    const long long bid = blockIdx.x / kCtas;
    auto pair_tile = [&](long long r, int t) { return (kPair * r + t) * G + bid; };
    const long long n_pairs = n_tiles > bid ? (n_tiles - bid + kPair * G - 1) / (kPair * G) : 0;
    // bounded waits: hand-offs between the CTAs of a pair (cluster scope), and completions
    // of copies and tensor-core work (CTA scope)
    auto wait = [&](uint32_t bar, uint32_t parity) {
        return mbar_wait<kCtas == 2>(bar, parity, A.err, &abort_flag, A.wait_limit, peer_abort);
    };
    auto wait_done = [&](uint32_t bar, uint32_t parity) {
        return mbar_wait<false>(bar, parity, A.err, &abort_flag, A.wait_limit, peer_abort);
    };
    // a warp-wide bounded wait on a completion or a hand-off within the CTA (lane 0 polls); false
    // when it ran out or another role aborted
    auto warp_wait = [&](uint32_t bar, uint32_t parity) {
        int ok = 1;
        if (lane == 0) ok = wait_done(bar, parity) ? 1 : 0;
        return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };

    if (warp == kProducerWarp) {
        if (lane == 0) {
            long long it = 0, last = -1;  // last: index of the last chunk copied
            for (long long r = 0; r < n_pairs && !abort_flag; ++r)
                for (int li = 0; li < A.n_layers && !abort_flag; ++li)
                    for (int t = 0; t < (kShare ? 1 : kPair) && !abort_flag; ++t) {  // once per tile, or once
                        const MlpLayerDev &Ly = A.L[li];
                        const int nc = n_chunks(Ly.K);
                        // this CTA's rows of each chunk: [rank N / kCtas, (rank + 1) N / kCtas), whole 8-row atoms
                        const uint32_t bytes = uint32_t(Ly.N / kCtas) * uint32_t(kChunkK) * 2u;
                        for (int c = 0; c < nc; ++c, ++it) {
                            const int slot = int(it % kSlots);
                            const long long round = it / kSlots;
                            if (round > 0 && !wait_done(empty_bar(slot), uint32_t((round - 1) & 1))) break;
                            if (it == A.withhold) continue;  // test fault: this chunk never arrives
                            mbar_expect_tx(full_bar(slot), bytes);
                            const char *src = reinterpret_cast<const char *>(Ly.w) + size_t(c) * Ly.N * kChunkK * 2 +
                                              size_t(rank) * bytes;
                            bulk_g2s(smem_u32(ring) + uint32_t(slot) * kSlotBytes, src, bytes, full_bar(slot));
                            last = it;
                        }
                    }
            // Every copy issued has landed before the CTA's shared memory goes away
            // (after an abort some may not have been waited for): the last kSlots
            // copies, one per slot; earlier ones were consumed before their slot was reused.
            for (long long j = last >= kSlots ? last - kSlots + 1 : 0; j <= last; ++j)
                if (j != A.withhold) mbar_drain<kCtas == 2>(full_bar(int(j % kSlots)), uint32_t((j / kSlots) & 1), A.err);
        }
    } else if (warp == kMmaWarp) {
        if (lane == 0 && leader) {
            long long it = 0, uses = 0;  // uses: (layer, tile) steps per slot t, same count for both
            for (long long r = 0; r < n_pairs && !abort_flag; ++r)
                for (int li = 0; li < A.n_layers && !abort_flag; ++li, ++uses)
                    for (int t = 0; t < kPair && !abort_flag; ++t) {
                        const MlpLayerDev &Ly = A.L[li];
                        if (kShare && t > 0) it -= n_chunks(Ly.K);  // the layer's chunks again, still in the ring
                        if (li == 0 && !wait(enc_ready(t), uint32_t(r & 1))) break;
                        if (!wait(a_ready(t), uint32_t(uses & 1))) break;
                        tc_fence_after();
                        const uint32_t idesc = instr_desc(kSuperM, Ly.N);
                        const uint32_t a_base =
                            li == 0 ? smem_u32(stage) + uint32_t(t) * uint32_t(kStageBytes)
                                    : smem_u32(sa) + uint32_t(t) * kATileBytes;
                        const uint32_t d_tmem = tmem + uint32_t(t * 256);
                        const int nc = n_chunks(Ly.K);
                        for (int c = 0; c < nc; ++c, ++it) {
                            const int slot = int(it % kSlots);
                            const uint32_t par = uint32_t((it / kSlots) & 1);
                            const bool first = !kShare || t == 0;  // the chunk's first use: wait for it to land
                            if (first && !wait_done(full_bar(slot), par)) break;
                            if (kCtas == 2 && first && !wait_done(pair_full(slot), par)) break;
                            tc_fence_after();
#pragma unroll
                            for (int s = 0; s < kChunkK / 16; ++s) {
                                const uint64_t ad = smem_desc_sw128(a_base + uint32_t(c) * (kTileM / 8) * 1024u +
                                                                    uint32_t(s) * 32u);
                                const uint64_t bd =
                                    smem_desc_sw128(smem_u32(ring) + uint32_t(slot) * kSlotBytes + uint32_t(s) * 32u);
                                umma_bf16<CTAS>(d_tmem, ad, bd, idesc, (c > 0 || s > 0) ? 1u : 0u);
                            }
                            if (!kShare || t == kPair - 1) {  // its last use: the slot may be refilled
                                umma_commit<CTAS>(empty_bar(slot));
                                if (kCtas == 2) umma_commit<CTAS>(other(empty_bar(slot)));
                            }
                        }
                        if (abort_flag) break;
                        if (li == 0) {  // the staging buffers may be refilled
                            umma_commit<CTAS>(enc_free(t));
                            if (kCtas == 2) umma_commit<CTAS>(other(enc_free(t)));
                        }
                        umma_commit<CTAS>(acc_full(t));
                        if (kCtas == 2) umma_commit<CTAS>(other(acc_full(t)));
                    }
            // every tensor-core operation issued (and every commit before this one) has
            // completed before the tensor memory is freed and the CTAs leave
            umma_commit<CTAS>(drain_bar);
            if (kCtas == 2) umma_commit<CTAS>(other(drain_bar));
            mbar_drain<kCtas == 2>(drain_bar, 0u, A.err);
        } else if (lane == 0) {
            // rank 1: tell rank 0 when each of this CTA's chunk parts has landed, in chunk order
            long long it = 0;
            for (long long r = 0; r < n_pairs && !abort_flag; ++r)
                for (int li = 0; li < A.n_layers && !abort_flag; ++li)
                    for (int t = 0; t < (kShare ? 1 : kPair) && !abort_flag; ++t) {
                        const int nc = n_chunks(A.L[li].K);
                        for (int c = 0; c < nc; ++c, ++it) {
                            const int slot = int(it % kSlots);
                            if (!wait_done(full_bar(slot), uint32_t((it / kSlots) & 1))) break;
                            mbar_arrive_remote(other(pair_full(slot)));
                        }
                    }
            // rank 0's MMAs read this CTA's shared memory and write its tensor memory:
            // they have completed before either is released
            mbar_drain<kCtas == 2>(drain_bar, 0u, A.err);
        }
    } else if (warp >= kEncWarp0 && warp < kEncWarp0 + kEncWarps) {
        // encoders: rows (warp - kEncWarp0) * 32 + lane + 32 kEncWarps i of this CTA's part of each tile
        const int e = warp - kEncWarp0;
        for (long long r = 0; r < n_pairs && !abort_flag; ++r) {
            bool ok = true;
            for (int t = 0; t < kPair && ok; ++t) {
                // pair r - 1's layer-0 MMAs of this slot have read the buffers
                if (r > 0 && !(ok = warp_wait(enc_free(t), uint32_t((r - 1) & 1)))) break;
                const long long tile = pair_tile(r, t);
                char *st = stage + size_t(t) * kStageBytes;
                for (int row = e * 32 + lane; row < kTileM; row += 32 * kEncWarps) {
                    const long long p =
                        tile < n_tiles ? tile * kSuperM + rank * kTileM + row : A.n_points;  // past the end: zeros
                    encode_point(A, p, row, st);
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) arrive_at_leader(enc_ready(t));
            }
            if (!ok) break;
        }
    } else if (warp >= kFirstEpiWarp) {
        const int q = warp & 3, g = (warp - kFirstEpiWarp) >> 2;  // lane quarter, column group
        const int row = q * 32 + lane;
        const int te = (warp - kFirstEpiWarp) * 32 + lane;       // 0 .. 32 kEpiWarps - 1
        long long uses = 0;
        bool stop = false;
        // the accumulators are free for the first pair's layer 0
        if (n_pairs > 0)
            for (int t = 0; t < kPair; ++t) {
                __syncwarp();
                if (lane == 0) arrive_at_leader(a_ready(t));
            }
        for (long long r = 0; r < n_pairs && !stop; ++r) {
            for (int li = 0; li < A.n_layers && !stop; ++li, ++uses) {
                const MlpLayerDev &Ly = A.L[li];
                const int N = Ly.N;
                const bool last = li + 1 == A.n_layers;
                const float *bias = (FNR_MLP_BIAS_SMEM ? sbias : A.bias) + Ly.bias_off;
                for (int t = 0; t < kPair; ++t) {
                    if (!warp_wait(acc_full(t), uint32_t(uses & 1))) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    char *sa_t = sa + size_t(t) * kATileBytes;
                    const uint32_t trow = tmem + uint32_t(t * 256) + (uint32_t(q * 32) << 16);
                    if (!last) {
                        // this warp's 16-column chunks j = g, g+4, g+8, g+12, two loads in flight per wait
                        const int nj = N / 16;
                        auto process = [&](const uint32_t (&rr)[16], int j) {
                            const int c0 = j * 16;
#pragma unroll
                            for (int u = 0; u < 16; u += 8) {
                                const float4 b0 = FNR_MLP_BIAS_SMEM
                                                      ? *reinterpret_cast<const float4 *>(bias + c0 + u)
                                                      : __ldg(reinterpret_cast<const float4 *>(bias + c0 + u));
                                const float4 b1 = FNR_MLP_BIAS_SMEM
                                                      ? *reinterpret_cast<const float4 *>(bias + c0 + u + 4)
                                                      : __ldg(reinterpret_cast<const float4 *>(bias + c0 + u + 4));
                                uint4 pk;
                                pk.x = pack_relu_bf16(__uint_as_float(rr[u + 0]) + b0.x, __uint_as_float(rr[u + 1]) + b0.y);
                                pk.y = pack_relu_bf16(__uint_as_float(rr[u + 2]) + b0.z, __uint_as_float(rr[u + 3]) + b0.w);
                                pk.z = pack_relu_bf16(__uint_as_float(rr[u + 4]) + b1.x, __uint_as_float(rr[u + 5]) + b1.y);
                                pk.w = pack_relu_bf16(__uint_as_float(rr[u + 6]) + b1.z, __uint_as_float(rr[u + 7]) + b1.w);
                                *reinterpret_cast<uint4 *>(sa_t + a_offset(row, c0 + u)) = pk;
                            }
                        };
                        for (int j0 = g; j0 < nj; j0 += 8) {  // warp-uniform
                            uint32_t r0[16], r1[16];
                            const bool two = j0 + 4 < nj;
                            tmem_ld16_nowait(trow + uint32_t(j0 * 16), r0);
                            if (two) tmem_ld16_nowait(trow + uint32_t((j0 + 4) * 16), r1);
                            tmem_wait();
                            process(r0, j0);
                            if (two) process(r1, j0 + 4);
                        }
                        // K padding of the next layer: columns [N, roundup(N, 64)) are 0
                        const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                        for (int c8 = N + 8 * g; c8 < ((N + 63) & ~63); c8 += 32)
                            *reinterpret_cast<uint4 *>(sa_t + a_offset(row, c8)) = z;
                        tc_fence_before();
                        fence_proxy_async();
                        __syncwarp();
                        if (lane == 0) arrive_at_leader(a_ready(t));
                        continue;
                    }
                    // head: stage out_c + bias (c < n_out) as fp32 rows of head_stride floats in the A tile,
                    // which the head's MMAs no longer read
                    float *hst = reinterpret_cast<float *>(sa_t);
                    const int hs = A.head_stride;
                    for (int j = g; j * 16 < A.n_out; j += 4) {  // warp-uniform
                        uint32_t rr[16];
                        tmem_ld16_nowait(trow + uint32_t(j * 16), rr);
                        tmem_wait();
#pragma unroll
                        for (int u = 0; u < 16; u += 4) {
                            const float4 b4 = FNR_MLP_BIAS_SMEM
                                                  ? *reinterpret_cast<const float4 *>(bias + j * 16 + u)
                                                  : __ldg(reinterpret_cast<const float4 *>(bias + j * 16 + u));
                            *reinterpret_cast<float4 *>(hst + row * hs + j * 16 + u) =
                                make_float4(__uint_as_float(rr[u + 0]) + b4.x, __uint_as_float(rr[u + 1]) + b4.y,
                                            __uint_as_float(rr[u + 2]) + b4.z, __uint_as_float(rr[u + 3]) + b4.w);
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(head_ready(t));
                    if (!warp_wait(head_ready(t), uint32_t(r & 1))) {
                        stop = true;
                        break;
                    }
                    // this CTA's outputs of the tile are contiguous ranges of the cache (or of out):
                    // element e of the range belongs to row e / n and output e % n
                    const long long tile = pair_tile(r, t);
                    const long long p0 = tile * kSuperM + rank * kTileM;
                    const int nv = tile < n_tiles && p0 < A.n_points
                                       ? int(A.n_points - p0 < kTileM ? A.n_points - p0 : kTileM)
                                       : 0;
                    constexpr int kEpiThreads = 32 * kEpiWarps;
                    if (A.mode == 0) {
                        for (int i = te; i < nv; i += kEpiThreads) {
                            const float sg = fmaxf(hst[i * hs], 0.0f);
                            if (A.prec == FNR_PREC_FP16) static_cast<__half *>(A.sigma_out)[p0 + i] = __float2half_rn(sg);
                            else static_cast<float *>(A.sigma_out)[p0 + i] = sg;
                        }
                        const int n = 3 * A.D;
                        char *rec0 = A.uvw_out + p0 * A.rec_stride;
                        for (int e = te; e < nv * n; e += kEpiThreads) {
                            const int i = e / n, c = e - i * n;
                            const float o = hst[i * hs + 1 + c];
                            char *rec = rec0 + size_t(i) * A.rec_stride;
                            if (A.prec == FNR_PREC_FP16) reinterpret_cast<__half *>(rec)[c] = __float2half_rn(o);
                            else reinterpret_cast<float *>(rec)[c] = o;
                        }
                    } else if (A.mode == 1) {
                        const int n = A.D;
                        for (int e = te; e < nv * n; e += kEpiThreads) {
                            const int i = e / n, c = e - i * n;
                            const float o = hst[i * hs + c];
                            if (A.dprec == FNR_PREC_FP16)
                                static_cast<__half *>(A.beta_out)[p0 * n + e] = __float2half_rn(o);
                            else static_cast<float *>(A.beta_out)[p0 * n + e] = o;
                        }
                    } else {
                        const int n = A.out_stride;
                        for (int e = te; e < nv * n; e += kEpiThreads) {
                            const int i = e / n, c = e - i * n;
                            const float o = hst[i * hs + c];
                            A.out[p0 * n + e] = (c == 0 && A.relu0) ? fmaxf(o, 0.0f) : o;
                        }
                    }
                    // the staged rows have been read: the next pair's layer 0 may use the accumulator
                    // and its epilogue may overwrite the A tile
                    __syncwarp();
                    if (r + 1 < n_pairs && lane == 0) arrive_at_leader(a_ready(t));
                }
            }
        }
    }
    __syncthreads();
    // no arrive or MMA of one CTA of the pair targets the other after this point
    if (kCtas == 2) cluster_sync();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_free<CTAS>(tmem, kTmemCols);
    }
}

// W [N][K] row-major bf16 bits -> padded, chunk-major 128-byte swizzled layout:
// chunk c holds columns [64 c, 64 c + 64) as [Np][64] K-major rows of 128
// bytes, 8-row atoms of 1024 bytes, piece (k / 8) of row n at (k / 8) ^ (n & 7).
__global__ void relayout_kernel(const uint16_t *__restrict__ w, int N, int K, uint16_t *__restrict__ out, int Np,
                                int Kp) {
    const int total = Np * Kp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int n = e / Kp, k = e - n * Kp;
        const uint16_t v = (n < N && k < K) ? w[size_t(n) * K + k] : uint16_t(0);
        const int c = k / kChunkK, kk = k - c * kChunkK;
        const size_t off = size_t(c) * Np * kChunkK + size_t(n >> 3) * 512 + size_t(n & 7) * 64 +
                           size_t(((kk >> 3) ^ (n & 7)) & 7) * 8 + (kk & 7);
        out[off] = v;
    }
}

__global__ void pad_bias_kernel(const float *__restrict__ b, int N, float *__restrict__ out, int Np) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Np) out[i] = i < N ? b[i] : 0.0f;
}

int round16(int v) { return (v + 15) / 16 * 16; }
int round64(int v) { return (v + 63) / 64 * 64; }

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
    if (m->dims[0] > kMaxK0)
        return fail(FNR_ERR_UNSUPPORTED, "%s: encoded width dims[0]=%d above %d", name, m->dims[0], kMaxK0);
    for (int i = 0; i <= m->n_layers; ++i)
        if (m->dims[i] < 1 || round64(m->dims[i]) > kMaxK)
            return fail(FNR_ERR_UNSUPPORTED, "%s: layer width %d outside [1, %d]", name, m->dims[i], kMaxK);
    if (m->dims[m->n_layers] < n_out_min)
        return fail(FNR_ERR_INVALID_ARG, "%s: %d outputs, need %d", name, m->dims[m->n_layers], n_out_min);
    for (int i = 0; i < m->n_layers; ++i)
        if (!m->weights[i] || !m->biases[i]) return fail(FNR_ERR_INVALID_ARG, "%s: NULL layer %d", name, i);
    return FNR_OK;
}

namespace {

// Launch one form of the kernel: one CTA (pair) per SM (pair) that can be
// resident at once, at most one per MMA tile.
template <int CTAS>
fnr_status launch_form(const MlpArgs &A, int num_sms, cudaStream_t s) {
    using F = Form<CTAS>;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(mlp_kernel<CTAS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(F::kSmemBytes))) != cudaSuccess)
        return cuda_fail(e, "MLP smem attribute");
    const long long tiles = (A.n_points + F::kSuperM - 1) / F::kSuperM;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = unsigned(CTAS);
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = F::kSmemBytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = CTAS > 1 ? 1 : 0;
    int units = num_sms;
    if (CTAS > 1) {
        cfg.gridDim = dim3(unsigned(num_sms / CTAS * CTAS));
        int clusters = 0;
        if ((e = cudaOccupancyMaxActiveClusters(&clusters, mlp_kernel<CTAS>, &cfg)) != cudaSuccess)
            return cuda_fail(e, "MLP cluster occupancy");
        if (clusters < 1) return fail(FNR_ERR_UNSUPPORTED, "MLP kernel: no SM pair can hold a CTA pair");
        units = clusters;
    }
    const int grid = int(tiles < units ? tiles : units) * CTAS;
    cfg.gridDim = dim3(unsigned(grid));
    if ((e = cudaLaunchKernelEx(&cfg, mlp_kernel<CTAS>, A)) != cudaSuccess) return cuda_fail(e, "MLP launch");
    return FNR_OK;
}

// Lay out the weights and biases of m, fill the layer table of A, launch the
// kernel on the mode-specific arguments already in A, and wait for it.
fnr_status mlp_launch(const fnr_mlp *m, MlpArgs &A, int num_sms, cudaStream_t s) {
    struct Buf {
        void *p = nullptr;
        ~Buf() {
            if (p) cudaFree(p);
        }
    } wbuf, bbuf, ebuf;
    size_t welems = 0, belems = 0;
    for (int i = 0; i < m->n_layers; ++i) {
        welems += size_t(round16(m->dims[i + 1])) * round64(m->dims[i]);
        belems += size_t(round16(m->dims[i + 1]));
    }
    cudaError_t e;
    if ((e = dev_malloc(&wbuf.p, welems * 2)) != cudaSuccess) return cuda_fail(e, "MLP weights");
    if ((e = dev_malloc(&bbuf.p, belems * 4)) != cudaSuccess) return cuda_fail(e, "MLP biases");
    if ((e = dev_malloc(&ebuf.p, 4)) != cudaSuccess) return cuda_fail(e, "MLP error word");
    if ((e = cudaMemsetAsync(ebuf.p, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "memset");
    size_t wo = 0, bo = 0;
    for (int i = 0; i < m->n_layers; ++i) {
        const int K = m->dims[i], N = m->dims[i + 1], Kp = round64(K), Np = round16(N);
        uint16_t *wd = static_cast<uint16_t *>(wbuf.p) + wo;
        float *bd = static_cast<float *>(bbuf.p) + bo;
        relayout_kernel<<<(Np * Kp + 255) / 256, 256, 0, s>>>(m->weights[i], N, K, wd, Np, Kp);
        pad_bias_kernel<<<(Np + 255) / 256, 256, 0, s>>>(m->biases[i], N, bd, Np);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "MLP weight layout");
        A.L[i].w = reinterpret_cast<const __nv_bfloat16 *>(wd);
        A.L[i].bias_off = int(bo);
        A.L[i].K = Kp;
        A.L[i].N = Np;
        wo += size_t(Np) * Kp;
        bo += size_t(Np);
    }
    A.bias = static_cast<const float *>(bbuf.p);
    A.n_bias = int(bo);
    A.n_layers = m->n_layers;
    A.pe_freqs = m->pe_freqs;
    A.err = static_cast<int *>(ebuf.p);
    A.wait_limit = kWaitLimit;
    A.withhold = -1;
    take_mlp_fault(&A.wait_limit, &A.withhold);
    A.n_out = A.mode == 0 ? 1 + 3 * A.D : (A.mode == 1 ? A.D : A.out_stride);
    A.head_stride = round16(A.n_out) + 4;
    if (A.n_out < 1 || A.n_out > kMaxHeadOut || A.n_out > A.L[m->n_layers - 1].N)
        return fail(FNR_ERR_UNSUPPORTED, "MLP kernel: %d outputs per point (at most %d)", A.n_out, kMaxHeadOut);
    if (A.n_points <= 0) return FNR_OK;
    const fnr_status st = mlp_cta_pair() ? launch_form<2>(A, num_sms, s) : launch_form<1>(A, num_sms, s);
    if (st != FNR_OK) return st;
    int herr = 0;
    if ((e = cudaMemcpyAsync(&herr, ebuf.p, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "MLP sync");
    if (herr == 1) return fail(FNR_ERR_DEVICE, "MLP kernel: an mbarrier wait ran out");
    if (herr) return fail(FNR_ERR_DEVICE, "MLP kernel: work in flight did not drain at exit");
    return FNR_OK;
}

}  // namespace

// Evaluate one MLP over its grid into the cache (mode 0: F_pos, 1: F_dir).
fnr_status run_mlp(const fnr_mlp *m, int mode, const fnr_cache_desc &d, const CacheView &v, int num_sms,
                   cudaStream_t s) {
    MlpArgs A;
    memset(&A, 0, sizeof(A));
    A.mode = mode;
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
    return mlp_launch(m, A, num_sms, s);
}

// Evaluate one MLP at n listed points ([n][3] on the device): the first
// out_stride head outputs of point p go to out[p * out_stride + c] in FP32.
fnr_status run_mlp_points(const fnr_mlp *m, const float *points, long long n, float *out, int out_stride,
                          bool relu0, int num_sms, cudaStream_t s) {
    MlpArgs A;
    memset(&A, 0, sizeof(A));
    A.mode = 2;
    A.n_points = n;
    A.points = points;
    A.out = out;
    A.out_stride = out_stride;
    A.relu0 = relu0 ? 1 : 0;
    return mlp_launch(m, A, num_sms, s);
}

}  // namespace fnr
