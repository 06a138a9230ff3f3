// march_voxels.cuh -- the voxel walk (FNR_RENDER_VOXELS): every cell a ray
// passes through is one sample whose delta is the ray's length inside the cell
// (Section 4 integrates every voxel a ray passes through once it has reached
// the density).
//
// One lane per ray, one warp per 8 x 4 pixel tile as in the uniform march. The
// walk itself (a 3-D digital differential analyser in binary32, the sequence
// fixed in fnr.h) is arithmetic only, so each lane generates kVU cells ahead,
// issues their density loads together, composites them in walk order
// (weights, transmittance, exact fixed-point termination) and only then loads
// the records of the cells it composited. In this mode the launcher passes
// t_far in r.dt (the walk has no sample spacing) and r.s_thr is the threshold
// on sum floor(fp32(sigma delta) 2^32).
//
// The kernel is instantiated three times per (precision, D), one form per
// translation unit: the plain walk (march_voxels.cu), the walk that skips the
// density loads of empty bricks (march_voxels_skip.cu), and the same with the
// one-step passes over empty cubes, used when no per-cell output is asked for
// (march_voxels_jump.cu). Each form carries only its own code: the brick
// arithmetic alone cost the plain walk 10%.
#pragma once
#include "march_device.cuh"

namespace fnr {

enum VoxelForm { kVoxPlain = 0, kVoxSkip = 1, kVoxJump = 2 };

namespace {

using namespace dev;

constexpr int kVU = 8;  // cells generated ahead of their density loads

// The cells of one ray in walk order (fnr.h, FNR_RENDER_VOXELS).
struct VoxelWalk {
    float u0, u1, u2, w0, w1, w2;  // g_a(t) = t u_a + w_a in grid units
    float tn0, tn1, tn2;           // next crossing per axis
    int c0, c1, c2;                // current cell
    float t, t1;
    int k;
    bool live;

    __device__ __forceinline__ static float crossing(int c, float u, float w) {
        if (u > 0.0f) return __fdiv_rn(__fsub_rn(static_cast<float>(c + 1), w), u);
        if (u < 0.0f) return __fdiv_rn(__fsub_rn(static_cast<float>(c), w), u);
        return __int_as_float(0x7f800000);  // +infinity
    }

    // Box clipping, start cell and first crossings; live = false if the ray
    // has no cells in [t_near, t_far].
    __device__ __forceinline__ void init(const CacheView &cv, const float o[3], const float d[3], float t_near,
                                         float t_far) {
        k = cv.k;
        const float kf = cv.kf;
        float uu[3], ww[3];
        float t0 = t_near, te = t_far;
        live = true;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            uu[a] = __fmul_rn(d[a], cv.scale[a]);
            ww[a] = __fmul_rn(__fsub_rn(o[a], cv.bmin[a]), cv.scale[a]);
            if (uu[a] != uu[a] || ww[a] != ww[a]) live = false;
            if (uu[a] == 0.0f) {
                if (!(ww[a] >= 0.0f && ww[a] < kf)) live = false;
            } else {
                const float ta = __fdiv_rn(-ww[a], uu[a]);
                const float tb = __fdiv_rn(__fsub_rn(kf, ww[a]), uu[a]);
                const float lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
                if (lo > t0) t0 = lo;
                if (hi < te) te = hi;
            }
        }
        if (!(t0 < te)) live = false;
        u0 = uu[0], u1 = uu[1], u2 = uu[2];
        w0 = ww[0], w1 = ww[1], w2 = ww[2];
        t = t0;
        t1 = te;
        auto start = [&](float u, float w) {
            const int ci = __float2int_rd(__fmaf_rn(t0, u, w));
            return ci < 0 ? 0 : (ci > k - 1 ? k - 1 : ci);
        };
        c0 = live ? start(u0, w0) : 0;
        c1 = live ? start(u1, w1) : 0;
        c2 = live ? start(u2, w2) : 0;
        tn0 = crossing(c0, u0, w0);
        tn1 = crossing(c1, u1, w1);
        tn2 = crossing(c2, u2, w2);
    }

    // The current cell, its occupancy brick (bricks of 2^sh cells, od per axis),
    // its E4M3 offset brick (2^osh cells, odim per axis) and its length;
    // advances to the next cell, or clears live after the last one. The step is
    // branch-free: lanes of a warp step different axes.
    __device__ __forceinline__ int next(float &delta, int &brick, int sh, int od, int &obrick, int osh, int odim) {
        int a = 0;
        float tnext = tn0;
        if (tn1 < tnext) {
            a = 1;
            tnext = tn1;
        }
        if (tn2 < tnext) {
            a = 2;
            tnext = tn2;
        }
        const float end = tnext < t1 ? tnext : t1;
        const int cell = (c2 * k + c1) * k + c0;  // k^3 < 2^31
        brick = ((c2 >> sh) * od + (c1 >> sh)) * od + (c0 >> sh);
        obrick = ((c2 >> osh) * odim + (c1 >> osh)) * odim + (c0 >> osh);
        delta = __fsub_rn(end, t);
        if (!(tnext < t1)) {
            live = false;
            return cell;
        }
        if (tnext > t) t = tnext;
        // the stepped axis has u != 0 (a +infinity crossing is never below t1)
        const bool x = a == 0, y = a == 1;
        const float ua = x ? u0 : (y ? u1 : u2);
        const float wa = x ? w0 : (y ? w1 : w2);
        const int ca = (x ? c0 : (y ? c1 : c2)) + (ua > 0.0f ? 1 : -1);
        const float tna = __fdiv_rn(__fsub_rn(static_cast<float>(ua > 0.0f ? ca + 1 : ca), wa), ua);
        c0 = x ? ca : c0;
        c1 = y ? ca : c1;
        c2 = (x || y) ? c2 : ca;
        tn0 = x ? tna : tn0;
        tn1 = y ? tna : tn1;
        tn2 = (x || y) ? tn2 : tna;
        if (ca < 0 || ca >= k) live = false;
        return cell;
    }

    // Crossings the walk makes along one axis from cell c on (n = 0: the one out
    // of c) at times before X, and at X too when `at`: counted with the crossing
    // formula itself, which is monotone in the cell index, from an estimate out
    // of the grid coordinate at X. -1 if the estimate is off by more than a few.
    // `next` receives the first crossing not counted: the one out of the cell
    // the axis has reached.
    __device__ __forceinline__ static int crossings_until(int c, float u, float w, float X, bool at, float &next) {
        next = __int_as_float(0x7f800000);
        if (u == 0.0f) return 0;
        const int s = u > 0.0f ? 1 : -1;
        auto before = [&](int n) {
            const float tc = crossing(c + s * n, u, w);
            const bool b = tc < X || (at && tc == X);
            if (!b) next = tc;
            return b;
        };
        const float g = floorf(__fmaf_rn(X, u, w));
        const float est = s > 0 ? g - static_cast<float>(c) : static_cast<float>(c) - g;
        int n = static_cast<int>(fminf(fmaxf(est, 0.0f), 16777216.0f));
        int fixes = 0;
        while (n > 0 && !before(n - 1))
            if (--n, ++fixes > 4) return -1;
        while (before(n))
            if (++n, ++fixes > 4) return -1;
        return n;
    }

    // One step over the cells of an empty cube [lo_a, hi_a] of cells that holds
    // the current cell: the number of cells the walk would return, one by one,
    // until it leaves the cube (or ends inside it), and its state after that,
    // both exactly as next() would leave them -- every crossing time comes from
    // a cell index alone, crossings at one time go in axis order, and each
    // crossing moves one axis by one cell. Returns the cells passed; at most
    // `cap`, which spends the walk; 0 if it took no step.
    __device__ __forceinline__ int pass_cube(const int lo[3], const int hi[3], int cap) {
        const float uu[3] = {u0, u1, u2}, ww[3] = {w0, w1, w2};
        const int cc[3] = {c0, c1, c2};
        float X = __int_as_float(0x7f800000);
        int ax = 3;  // the axis whose crossing leaves the cube first (the lowest on a tie)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (uu[a] != 0.0f) {
                const float xa = crossing(uu[a] > 0.0f ? hi[a] : lo[a], uu[a], ww[a]);
                if (xa < X) {
                    X = xa;
                    ax = a;
                }
            }
        const bool ends = !(X < t1);  // the walk ends inside the cube
        int n[3], total = ends ? 1 : 0;
        float nx[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            n[a] = crossings_until(cc[a], uu[a], ww[a], ends ? t1 : X, !ends && a <= ax, nx[a]);
            if (n[a] < 0) return 0;
            total += n[a];
        }
        if (total <= 1) return 0;
        if (total >= cap) return cap;
        if (ends) {
            live = false;
            return total;
        }
        c0 = cc[0] + (uu[0] > 0.0f ? n[0] : -n[0]);
        c1 = cc[1] + (uu[1] > 0.0f ? n[1] : -n[1]);
        c2 = cc[2] + (uu[2] > 0.0f ? n[2] : -n[2]);
        if (X > t) t = X;
        tn0 = nx[0];  // = crossing(c0, u0, w0), computed by the count
        tn1 = nx[1];
        tn2 = nx[2];
        const int ca = ax == 0 ? c0 : (ax == 1 ? c1 : c2);
        if (ca < 0 || ca >= k) live = false;
        return total;
    }
};

template <int PREC, int D, int FORM>
__global__ void __launch_bounds__(FNR_BLOCK) march_voxels_kernel(const __grid_constant__ MarchArgs A) {
    allow_next_grid();
    constexpr unsigned FULL = 0xffffffffu;
    const int tile = static_cast<int>((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (tile >= A.total_tiles) return;  // whole warp
    int f = 0;
    while (f + 1 < A.n_frames && tile >= A.f[f + 1].tile_begin) ++f;
    const FrameDesc &F = A.f[f];
    const CacheView &c = A.c;
    const RenderConst &r = A.r;
    int x0, y0;
    tile_origin(F, tile - F.tile_begin, x0, y0);
    const int lane = threadIdx.x & 31;
    const int px = x0 + (lane & (kTileW - 1)), py = y0 + lane / kTileW;
    const bool active = px < F.W && py < F.H;
    constexpr bool kOffs = PREC == FNR_PREC_FP8_E4M3;
    __shared__ float sbeta[FNR_BLOCK / 32][D][32];
    __shared__ float wsc[FNR_BLOCK / 32][kOffs ? 3 * D : 1];  // E4M3: the (u, v, w) channel scales, per warp
    float (*qbeta)[32] = sbeta[threadIdx.x >> 5];
    float *ssc = wsc[threadIdx.x >> 5];
    if constexpr (kOffs) {
        for (int i = lane; i < 3 * D; i += 32) ssc[i] = __ldg(c.scales + 1 + i);
        __syncwarp();
    }

    RaySetup<PREC, D> R;  // a1/a2: direction cell and beta (the uniform-sample fields go unused)
    VoxelWalk Wk;
    Wk.live = false;
    R.dcell = 0;
    R.sigma_scale = 1.0f;
    if (active) {
        R.init(c, r, F, px, py, qbeta, lane);
        // the ray again (the fixed a1 sequence) for the walk
        const float dcx = __fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(px), 0.5f), F.cx), F.fx);
        const float dcy = -__fdiv_rn(__fsub_rn(__fadd_rn(static_cast<float>(py), 0.5f), F.cy), F.fy);
        const float wx = __fmaf_rn(F.c2w[0], dcx, __fmaf_rn(F.c2w[1], dcy, -F.c2w[2]));
        const float wy = __fmaf_rn(F.c2w[4], dcx, __fmaf_rn(F.c2w[5], dcy, -F.c2w[6]));
        const float wz = __fmaf_rn(F.c2w[8], dcx, __fmaf_rn(F.c2w[9], dcy, -F.c2w[10]));
        const float n2 = __fmaf_rn(wx, wx, __fmaf_rn(wy, wy, __fmul_rn(wz, wz)));
        const float len = __fsqrt_rn(n2);
        const float dd[3] = {__fdiv_rn(wx, len), __fdiv_rn(wy, len), __fdiv_rn(wz, len)};
        const float oo[3] = {F.c2w[3], F.c2w[7], F.c2w[11]};
        Wk.init(c, oo, dd, r.t_near, r.dt);  // r.dt holds t_far in this mode
    }
    const bool skip = FORM != kVoxPlain && (r.flags & FNR_RENDER_SKIP_EMPTY) != 0u;
    // Skipping without per-cell output also passes over whole empty cubes of jump
    // bricks in one step (VoxelWalk::pass_cube), from the cache's distance field.
    const bool jumps = FORM == kVoxJump && skip && F.cells == nullptr && c.dist != nullptr;
    float T = 1.0f, Cr = 0.0f, Cg = 0.0f, Cb = 0.0f;
    long long S = 0;
    int n_gen = 0, n_steps = 0, n_look = 0, n_occ = 0;
    bool term = false;
    const long long pix = active ? static_cast<long long>(py) * F.W + px : 0;
    int32_t *cells_out = (active && F.cells) ? F.cells + pix * r.N : nullptr;
    if (F.cells) wait_prior_grid();  // cells are written while walking

    while (__any_sync(FULL, Wk.live && !term && n_gen < r.N)) {
        // kVU cells ahead, their densities loaded together
        int cell[kVU], brick[kVU], obr[kVU];
        float dl[kVU], sg[kVU];
        unsigned gen = 0u, looked = 0u;
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            cell[u] = 0;
            brick[u] = 0;
            obr[u] = 0;
            dl[u] = 0.0f;
            if (jumps && u == 0 && Wk.live && !term && n_gen < r.N) {
                // One pass per group (more per group measured slower: each costs a dozen exact divisions
                // and the lanes of a warp take different ones). d > 0: the jump bricks within Chebyshev
                // distance d - 1 of the current one are empty.
                const int sh = c.dist_shift;
                const int d = __ldg(c.dist + ((Wk.c2 >> sh) * c.dist_dim + (Wk.c1 >> sh)) * c.dist_dim + (Wk.c0 >> sh));
                if (d > 0) {
                    const int cw[3] = {Wk.c0, Wk.c1, Wk.c2};
                    int lo[3], hi[3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        lo[a] = max(((cw[a] >> sh) - (d - 1)) << sh, 0);
                        hi[a] = min((((cw[a] >> sh) + d) << sh) - 1, Wk.k - 1);
                    }
                    const int m = Wk.pass_cube(lo, hi, r.N - n_gen);
                    n_gen += m;
                    n_steps += m;
                }
            }
            if (Wk.live && !term && n_gen < r.N) {
                cell[u] = Wk.next(dl[u], brick[u], c.occ_shift, c.occ_dim, obr[u], c.offs_shift, c.offs_dim);
                gen |= 1u << u;
                ++n_gen;
            }
        }
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            sg[u] = 0.0f;
            if (((gen >> u) & 1u) && dl[u] > 0.0f) {
                const bool load = !skip || brick_occupied(c, brick[u]) != 0u;
                if (load) {
                    sg[u] = load_sigma<PREC>(c, cell[u], R.sigma_scale);
                    looked |= 1u << u;
                }
            }
        }
        // walk order: weights, transmittance and termination from the densities alone
        float wgt[kVU];
        unsigned occ = 0u;
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            wgt[u] = 0.0f;
            if (!((gen >> u) & 1u) || term) continue;
            ++n_steps;
            if (cells_out) cells_out[n_steps - 1] = cell[u];
            if ((looked >> u) & 1u) ++n_look;
            if (sg[u] > 0.0f) {
                ++n_occ;
                const float od = __fmul_rn(sg[u], dl[u]);
                float ext, alpha;
                extinction(od, ext, alpha);
                wgt[u] = T * alpha;
                T = T * ext;
                occ |= 1u << u;
                const long long qd = fixed_depth(od);
                S = (S > 0x7fffffffffffffffLL - qd) ? 0x7fffffffffffffffLL : S + qd;
                if (S >= r.s_thr) term = true;
            }
        }
        // records of the composited cells, colour added in walk order
#pragma unroll
        for (int u = 0; u < kVU; ++u) {
            if (!((occ >> u) & 1u)) continue;
            Record<PREC, D> rec;
            rec.load(c.uvw + static_cast<long long>(cell[u]) * c.rec_stride);
            float col[3];
            if constexpr (kOffs) {
                OffsetRecord<D> off;
                off.load(c.offs + static_cast<long long>(obr[u]) * c.offs_stride);
                shade_e4m3<D>(
                    rec, off, r.act, [&](int i) { return ssc[i]; }, [&](int j) { return qbeta[j][lane]; }, col);
            } else {
                RaySetup<PREC, D>::shade_with(rec, r.act, [&](int ch, int j) { return qbeta[j][lane]; }, col);
            }
            Cr = __fmaf_rn(wgt[u], col[0], Cr);
            Cg = __fmaf_rn(wgt[u], col[1], Cg);
            Cb = __fmaf_rn(wgt[u], col[2], Cb);
        }
    }
    wait_prior_grid();
    if (!active) return;
    if (cells_out)
        for (int j = n_steps; j < r.N; ++j) cells_out[j] = term ? -2 : -1;
    float4 o;
    o.x = __fmaf_rn(T, r.bg[0], Cr);
    o.y = __fmaf_rn(T, r.bg[1], Cg);
    o.z = __fmaf_rn(T, r.bg[2], Cb);
    o.w = 1.0f - T;
    reinterpret_cast<float4 *>(F.rgba)[pix] = o;
    if (F.stats) reinterpret_cast<int4 *>(F.stats)[pix] = make_int4(n_steps, n_look, n_occ, R.dcell);
}

template <int PREC, int D, int FORM>
cudaError_t launch_v(const MarchArgs &a, cudaStream_t s) {
    const int warps_per_block = FNR_BLOCK / 32;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>((a.total_tiles + warps_per_block - 1) / warps_per_block));
    cfg.blockDim = dim3(FNR_BLOCK);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, march_voxels_kernel<PREC, D, FORM>, a);
}

template <int PREC, int FORM>
cudaError_t launch_vp(const MarchArgs &a, cudaStream_t s) {
    switch (a.c.D) {
        case 1: return launch_v<PREC, 1, FORM>(a, s);
        case 2: return launch_v<PREC, 2, FORM>(a, s);
        case 3: return launch_v<PREC, 3, FORM>(a, s);
        case 4: return launch_v<PREC, 4, FORM>(a, s);
        case 5: return launch_v<PREC, 5, FORM>(a, s);
        case 6: return launch_v<PREC, 6, FORM>(a, s);
        case 7: return launch_v<PREC, 7, FORM>(a, s);
        case 8: return launch_v<PREC, 8, FORM>(a, s);
        case 9: return launch_v<PREC, 9, FORM>(a, s);
        case 10: return launch_v<PREC, 10, FORM>(a, s);
        case 11: return launch_v<PREC, 11, FORM>(a, s);
        case 12: return launch_v<PREC, 12, FORM>(a, s);
        case 13: return launch_v<PREC, 13, FORM>(a, s);
        case 14: return launch_v<PREC, 14, FORM>(a, s);
        case 15: return launch_v<PREC, 15, FORM>(a, s);
        case 16: return launch_v<PREC, 16, FORM>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

// Every form dispatches on the position-cache precision the same way.
template <int FORM>
cudaError_t launch_voxels_prec(const MarchArgs &a, cudaStream_t s) {
    switch (a.c.pos_prec) {
        case FNR_PREC_FP32: return launch_vp<FNR_PREC_FP32, FORM>(a, s);
        case FNR_PREC_FP16: return launch_vp<FNR_PREC_FP16, FORM>(a, s);
        case FNR_PREC_FP8_E4M3: return launch_vp<FNR_PREC_FP8_E4M3, FORM>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// The skipping forms of the walk (march_voxels_skip.cu, march_voxels_jump.cu).
cudaError_t launch_march_voxels_skip(const MarchArgs &a, cudaStream_t s);
cudaError_t launch_march_voxels_jump(const MarchArgs &a, cudaStream_t s);

}  // namespace fnr
