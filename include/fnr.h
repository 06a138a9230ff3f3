/*
 * fnr.h -- C ABI of libfnr, a GB300 (sm_103a) renderer for FastNeRF's cached
 * representation (Garbin et al., "FastNeRF: High-Fidelity Neural Rendering at
 * 200FPS", 2021).
 *
 * Problem statement (Sections 3.3 and 4): given a position cache (density
 * sigma and a D-component deep radiance map (u, v, w) sampled on a k^3 grid
 * over a bounding box) and a direction cache (D weights beta on an l x l grid
 * of (theta, phi)), and a set of camera parameters, generate one ray per
 * pixel, sample it, look both caches up by nearest neighbour, form the colour
 * c = act(sum_i beta_i (u_i, v_i, w_i)) (Eq. 5) and alpha-composite the
 * samples front to back (Eq. 1) until the transmittance is saturated
 * (supplementary "Meshing & Rendering"), filling an RGBA buffer.
 *
 * Conventions
 *  - Every call returns fnr_status; FNR_OK is 0. No C++ exception crosses the
 *    ABI. fnr_last_error() returns a message for the calling thread's last
 *    failed call; the library owns that string until the thread's next call.
 *  - Pointers named *_dev are CUDA device pointers; they stay owned by the
 *    caller, who must keep them alive until the work that uses them has
 *    completed on its stream. Other pointers are host pointers, read during
 *    the call only.
 *  - fnr_stream_t is a cudaStream_t (NULL = legacy default stream).
 *  - Work is stream-ordered: argument errors are returned at once; a CUDA
 *    launch failure is returned as FNR_ERR_CUDA by the call that saw it.
 *
 * Geometry (exact definitions; the integer results -- cells, direction cell,
 * termination step -- are bit-reproducible):
 *  - Pixel (px, py), py = 0 the top row; camera looks down its -z axis.
 *    binary32, correctly rounded, no contraction:
 *      dcx = ((px + 0.5) - cx) / fx,  dcy = -(((py + 0.5) - cy) / fy)
 *      w_r = fma(R_r0, dcx, fma(R_r1, dcy, -R_r2)), r = 0, 1, 2 (c2w rotation)
 *      n2 = fma(wx, wx, fma(wy, wy, wz * wz)), d = w / sqrt(n2), o = c2w eye.
 *  - Samples (Section 3.1, N midpoints t_i = t_near + (i + 0.5) Delta on
 *    [t_near, t_far], delta_i = Delta = (t_far - t_near) / N). The grid
 *    coordinates g_a = (o_a + t_i d_a - bmin_a) s_a, s_a = binary32(k / (bmax_a -
 *    bmin_a)) evaluated in FP64, are computed as the affine map in i:
 *      u_a = d_a * s_a, e_a = u_a * Delta, f_a = fma(t_near, u_a, (o_a - bmin_a) * s_a),
 *      g_a(i) = fma(i + 0.5, e_a, f_a).
 *    The sample is inside the cache iff 0 <= g_a < k on all axes; its cell is
 *    floor(g) and its linear index (z * k + y) * k + x (Section 3.3, cell-
 *    centred grid, nearest neighbour as in Section 4).
 *  - Direction cell (Section 3.3, theta in [0, pi] from +z, phi = atan2(y, x)
 *    in [0, 2 pi), l bins each):
 *      i_theta = #{ j in 1..l-1 : d_z <= binary32(cos(j pi / l)) }
 *      i_phi   = #{ j in 1..l-1 : key(d_x, d_y) >= binary32(key64(cos phi_j, sin phi_j)) },
 *    phi_j = 2 pi j / l, key the monotone "diamond" azimuth key in [0, 4]:
 *      y >= 0, x >= 0: y / (x + y);         y >= 0, x < 0: 1 + (-x) / (y + (-x));
 *      y <  0, x <  0: 2 + (-y) / ((-x) + (-y)); y < 0, x >= 0: 3 + x / (x + (-y));
 *      (0, 0) -> 0; key in binary32, key64 the same formula in FP64.
 *  - Per occupied sample (sigma > 0): colour (Eq. 5) then Eq. 1 with
 *    alpha = 1 - exp(-sigma Delta), T <- T exp(-sigma Delta). Termination:
 *    S += floor(sigma * 2^32) (int64, saturating; 2^63-1 when sigma >= 2^31);
 *    the ray stops after the first sample with S >= S_thr,
 *    S_thr = ceil(ln(1 / t_thr) / Delta * 2^32) in FP64 (t_thr <= 0: never).
 *    The background is added with the final transmittance:
 *    RGB += T * bg, alpha = 1 - T.
 */
#ifndef FNR_H
#define FNR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FNR_API __attribute__((visibility("default")))
#else
#define FNR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fnr_status;
#define FNR_OK 0
#define FNR_ERR_INVALID_ARG 1 /* malformed argument; nothing was launched */
#define FNR_ERR_UNSUPPORTED 2 /* valid but not supported by this build (e.g. D > 16) */
#define FNR_ERR_OOM 3         /* a device allocation failed */
#define FNR_ERR_BUDGET 4      /* the context's HBM budget would be exceeded */
#define FNR_ERR_QUEUE_FULL 5  /* the request queue is full; retry later */
#define FNR_ERR_NOT_READY 6   /* the request is still queued or in flight */
#define FNR_ERR_TIMEOUT 7     /* a host wait ran out */
#define FNR_ERR_CUDA 8        /* a CUDA runtime call failed */
#define FNR_ERR_DEVICE 9      /* a kernel reported an error through its status word */
#define FNR_ERR_IO 10         /* a file could not be read or written, or is not a cache file */

#define FNR_PREC_FP32 0
#define FNR_PREC_FP16 1
#define FNR_PREC_FP8_E4M3 2 /* OCP E4M3 with one binary32 scale per channel */

#define FNR_ACT_SIGMOID 0  /* c = 1 / (1 + exp(-x)) per channel */
#define FNR_ACT_IDENTITY 1 /* c = x */

#define FNR_SRC_ARRAYS 1
#define FNR_SRC_MLP 2

#define FNR_LOC_HOST 0
#define FNR_LOC_DEVICE 1

#define FNR_MAX_D 16
#define FNR_MAX_K 1290 /* k^3 < 2^31: cell indices are int32 */
#define FNR_MAX_L 4096
#define FNR_MAX_SAMPLES 4096
#define FNR_MAX_IMAGE_SIDE 16384

typedef struct CUstream_st *fnr_stream_t;
typedef struct fnr_context fnr_context;
typedef struct fnr_cache fnr_cache;

/* ------------------------------------------------------------------ context */
/* Create a context on CUDA device `device`. hbm_budget_bytes caps the device
 * memory the context allocates for caches plus the outputs of admitted
 * serving requests (0 = no cap). Errors: INVALID_ARG (bad device), CUDA. */
FNR_API fnr_status fnr_context_create(int32_t device, uint64_t hbm_budget_bytes, fnr_context **out);
/* Stops the request loop (outstanding requests finish first), frees every
 * cache the context still owns and the context. NULL is a no-op. */
FNR_API fnr_status fnr_context_destroy(fnr_context *ctx);
/* Bytes currently charged against the budget. */
FNR_API uint64_t fnr_context_used_bytes(const fnr_context *ctx);

/* Thread-local message of the last failed call ("" if none). */
FNR_API const char *fnr_last_error(void);

/* ------------------------------------------------------------------ caches */
typedef struct {
    int32_t k;             /* grid samples per axis of the position cache, 1..FNR_MAX_K */
    int32_t D;             /* components of the deep radiance map, 1..FNR_MAX_D */
    int32_t l;             /* direction bins per angle, 2..FNR_MAX_L */
    int32_t pos_precision; /* storage of sigma and (u, v, w): FNR_PREC_* */
    int32_t dir_precision; /* storage of beta: FNR_PREC_FP32 or FNR_PREC_FP16 */
    int32_t occupancy_brick; /* cells per side of an occupancy brick (FNR_RENDER_SKIP_EMPTY):
                                a power of two 1..256, or 0 = the smallest power of two >= 2
                                with ceil(k / B) <= 64 (8 at k = 512, 16 at k = 1024) */
    int32_t layout;        /* FNR_LAYOUT_DENSE or FNR_LAYOUT_BRICKS */
    int32_t reserved;      /* must be 0 */
    float bmin[3], bmax[3]; /* bounding box V, bmax > bmin on every axis */
} fnr_cache_desc;

/* Storage of the position cache. DENSE: the k^3 sigma plane and k^3 records.
 * BRICKS (sparse; the paper stores its caches sparsely, Section 3.3 and the
 * supplementary cache sizes): only the occupancy bricks (B^3 cells, B =
 * occupancy_brick) holding a stored density > 0 keep their sigma and records,
 * in a pool of bricks reached through a page table of ceil(k / B)^3 entries.
 * Renders from a BRICKS cache (fnr_render, fnr_submit) have
 * FNR_RENDER_SKIP_EMPTY semantics whether or not the flag is set (an empty
 * brick has no storage); fnr_render_noalloc reads dense caches only. */
#define FNR_LAYOUT_DENSE 0
#define FNR_LAYOUT_BRICKS 1

/* One MLP for the tensor-core cache build (Section 3.2, Eqs. 3 and 4; Section 4):
 * input = positional encoding gamma(x) = [sin(2^j pi x_a), cos(2^j pi x_a)],
 * a = 0..pe_in-1 (coordinate-major), j = 0..pe_freqs-1 (sin before cos),
 * zero padded to dims[0]; hidden layers ReLU; last layer linear.
 * weights[i]: device bf16 bits, [dims[i+1]][dims[i]] row-major;
 * biases[i]: device float[dims[i+1]]. */
typedef struct {
    int32_t n_layers;  /* 1..16 */
    int32_t pe_in;     /* raw inputs: 3 (position) */
    int32_t pe_freqs;  /* L */
    int32_t dims[17];  /* dims[0] = padded encoded width (6 pe_freqs .. 64), other widths 1..256,
                          dims[n_layers] = outputs; wider inputs: FNR_ERR_UNSUPPORTED */
    const uint16_t *weights[16];
    const float *biases[16];
} fnr_mlp;

typedef struct {
    int32_t kind;     /* FNR_SRC_ARRAYS or FNR_SRC_MLP */
    int32_t location; /* FNR_SRC_ARRAYS: FNR_LOC_HOST or FNR_LOC_DEVICE */
    /* FNR_SRC_ARRAYS, binary32:
     *   sigma [k^3] at (z*k + y)*k + x; negative and NaN densities are stored as 0
     *   uvw   [k^3][3D], channels u_1..u_D, v_1..v_D, w_1..w_D
     *   beta  [l][l][D] at (i_theta*l + i_phi)*D + i, sampled at bin centres
     * FP16: round to nearest even. FP8 (E4M3, round to nearest even, saturating
     * to +-448): the density as one channel, scale_0 = absmax / 448 in binary32
     * (1 if all zero), q = E4M3(sigma / scale_0). Each (u, v, w) channel c is
     * stored as the residual from a per-brick offset: the grid is cut into
     * offset bricks of Bo cells a side (the smallest power of two >= 4 with
     * ceil(k / Bo) <= 64), and per brick the offset m is the binary16 (nearest
     * even) value of the binary32 midrange (min + max) * 0.5 of the channel
     * over the brick's cells (NaN ignored; 0 if all NaN); r = binary32(x - m),
     * scale_c = absmax over the grid of |r| / 448 (1 if 0), q = E4M3(r /
     * scale_c). The stored value is m + scale_c * e4m3(q). */
    const float *sigma;
    const float *uvw;
    const float *beta;
    /* FNR_SRC_MLP (device bf16 MLPs, built on the tensor cores):
     * F_pos: 3 -> dims_out = 1 + 3D; sigma = ReLU(out[0]), (u, v, w) = out[1..3D]
     * evaluated at the cell centres bmin + (j + 1/2)(bmax - bmin)/k.
     * F_dir: unit direction (3 inputs) -> D outputs = beta, evaluated at the bin
     * centres theta = (i + 1/2) pi / l, phi = (j + 1/2) 2 pi / l. */
    const fnr_mlp *pos_mlp;
    const fnr_mlp *dir_mlp;
} fnr_cache_source;

/* Bytes of the dense caches by the supplementary "Cache size calculation"
 * (second version, alpha = 1): k^3 (s_sigma + D s_uvw) + D s_beta l^2, where
 * s_uvw is one (u_i, v_i, w_i) triple; FP8 adds its (1 + 3D) binary32 scales
 * and its 3D binary16 offsets per offset brick. Returns 0 for an invalid
 * descriptor. */
FNR_API uint64_t fnr_cache_bytes(const fnr_cache_desc *desc);
/* Device bytes one dense cache occupies: the above plus record padding to 16
 * bytes (8 for FP8), 256-byte section alignment, the two direction-bin tables
 * and the occupancy bits. For FNR_LAYOUT_BRICKS it is the bound with every
 * brick stored; a built cache reports its own footprint (fnr_cache_get_layout).
 * A BRICKS build passes through a dense cache, which is charged to the budget
 * while it exists. */
FNR_API uint64_t fnr_cache_footprint(const fnr_cache_desc *desc);

/* Build a cache on `stream`. Returns when the cache is complete (the call
 * synchronises `stream`). The library owns the cache until fnr_cache_free.
 * Errors: INVALID_ARG, UNSUPPORTED, BUDGET, OOM, CUDA. */
FNR_API fnr_status fnr_build_cache(fnr_context *ctx, const fnr_cache_desc *desc, const fnr_cache_source *src,
                           fnr_stream_t stream, fnr_cache **out);
/* Free a cache. INVALID_ARG if serving requests still reference it. */
FNR_API fnr_status fnr_cache_free(fnr_context *ctx, fnr_cache *cache);

/* Device layout of a built cache (read-only views, owned by the cache). */
typedef struct {
    const void *sigma_dev;     /* [k^3] stored density (float / half / e4m3) */
    const void *uvw_dev;       /* [k^3] records of 3D stored values, record_stride bytes apart */
    const void *beta_dev;      /* [l][l][D] stored weights */
    const float *scales_dev;   /* FP8: [1 + 3D] (sigma first), else NULL */
    const float *cos_theta_dev;/* [l] binary32(cos(j pi / l)); entry 0 = 1 */
    const float *phi_key_dev;  /* [l] azimuth-key boundaries; entry 0 = 0 */
    const uint32_t *occupancy_dev; /* brick occupancy bits: with B = occupancy_brick and
                                      nb = ceil(k / B), brick (bx, by, bz) holds the cells
                                      [bx B, bx B + B) x ... clipped to the grid; its index is
                                      b = (bz nb + by) nb + bx and bit (b & 31) of word b >> 5 is
                                      set iff one of its stored densities is > 0 */
    int32_t record_stride;     /* bytes between (u, v, w) records */
    int32_t occupancy_brick;   /* B */
    uint64_t footprint;        /* device bytes */
    int32_t layout;            /* FNR_LAYOUT_*; for BRICKS, sigma_dev and uvw_dev hold n_bricks
                                  bricks of B^3 cells each, cell (x, y, z) of brick slot s at index
                                  s B^3 + ((z mod B) B + (y mod B)) B + (x mod B) */
    int32_t reserved1;
    const int32_t *page_table_dev; /* BRICKS: [nb^3] brick slot, -1 for an empty brick (same brick
                                      index as the occupancy bits); NULL for DENSE */
    uint64_t n_bricks;         /* BRICKS: bricks stored */
    const uint8_t *brick_distance_dev; /* distance field for passing over empty space: the grid is
                                      cut into jump bricks of J = distance_brick cells a side (J =
                                      B 2^m, the smallest with nj = ceil(k / J) <= 32); a jump brick
                                      is occupied iff one of its occupancy bricks is; entry
                                      (jz nj + jy) nj + jx holds the Chebyshev distance, in jump
                                      bricks, to the nearest occupied jump brick, capped at 16 (0 when
                                      occupied); every jump brick within distance - 1 of it is empty.
                                      Used by FNR_RENDER_SKIP_EMPTY renders. [nj^3] bytes */
    int32_t distance_brick;    /* J */
    int32_t reserved2;
    const uint16_t *offsets_dev; /* FP8: binary16 (u, v, w) offsets, offset brick (bz nbo + by) nbo + bx
                                    at element offset_stride * brick + c, c < 3D; NULL otherwise */
    int32_t offset_brick;      /* FP8: Bo (cells per side of an offset brick), else 0 */
    int32_t offset_stride;     /* FP8: binary16 elements between bricks (3D rounded up to 8), else 0 */
} fnr_cache_layout;
FNR_API fnr_status fnr_cache_get_layout(const fnr_cache *cache, fnr_cache_layout *out);

/* Persist a built cache (no counterpart in the paper, which keeps its caches
 * in memory): the file holds a header -- the 8 bytes "FNRCACHE", a uint32
 * format version (2), the uint32 header size, the fnr_cache_desc, the uint64
 * device footprint and the uint64 brick count (FNR_LAYOUT_BRICKS; else 0) --
 * followed by the cache's device allocation byte
 * for byte (every section of fnr_cache_layout, whose offsets follow from the
 * descriptor). Saving reads the device through a pinned staging buffer after
 * synchronising the context's device. Errors: INVALID_ARG, IO, CUDA. */
FNR_API fnr_status fnr_cache_save(const fnr_cache *cache, const char *path);
/* Load a saved cache into ctx (charged against its budget like a build) and
 * upload it on `stream`; the call returns after the upload. Errors:
 * INVALID_ARG, IO (unreadable, truncated, wrong magic / version / size),
 * BUDGET, CUDA. */
FNR_API fnr_status fnr_cache_load(fnr_context *ctx, const char *path, fnr_stream_t stream, fnr_cache **out);

/* ------------------------------------------------------------------ rendering */
typedef struct {
    float c2w[12]; /* row-major 3x4 [R | eye], camera-to-world */
    float fx, fy, cx, cy;
    int32_t width, height; /* 1..FNR_MAX_IMAGE_SIDE */
} fnr_camera;

typedef struct {
    int32_t n_samples;     /* N, 1..FNR_MAX_SAMPLES */
    float t_near, t_far;   /* finite, t_far > t_near */
    float t_thr;           /* termination transmittance; <= 0 disables */
    float bg[3];           /* background colour */
    int32_t activation;    /* FNR_ACT_* */
    uint32_t flags;        /* FNR_RENDER_* bits */
    int32_t reserved;      /* must be 0 */
} fnr_render_params;

/* Empty-space skipping (the paper renders with its collision mesh so that
 * empty space costs no queries, Section 4 and supplementary "Meshing &
 * Rendering"; here with the cache's brick occupancy bits instead of a mesh):
 * a sample whose brick has no stored density > 0 is known to have sigma = 0,
 * so its density is not looked up. The samples stay the N uniform ones, so
 * RGBA, n_steps, n_occupied and dir_cell equal the plain render's bit for bit;
 * n_lookups counts only the density lookups made (in-box samples in occupied
 * bricks, up to termination). */
#define FNR_RENDER_SKIP_EMPTY 1u
/* Interpolated direction lookup (the paper samples F_view with interpolation,
 * Section 4): beta bilinear in (theta, phi) between the bin centres
 * theta_i = (i + 1/2) pi / l, phi_j = (j + 1/2) 2 pi / l, theta neighbours
 * clamped at the poles, phi neighbours wrapping around 2 pi. The angles are
 * binary32 atan2f values, so colours differ from an FP64 evaluation by up to
 * ~1e-4 rather than 1e-5; dir_cell still reports the nearest bin. */
#define FNR_RENDER_DIR_BILINEAR 2u
/* Voxel walk (the paper integrates every voxel a ray passes through once the
 * ray has reached the density, Section 4): instead of N uniform samples, each
 * cell the ray passes through is one sample whose delta is the ray's length
 * inside the cell. The cells of the segment [t0, t1] = [max(t_near, t_enter),
 * min(t_far, t_exit)] inside the box are walked in order, in binary32 with
 * this sequence, in grid units g_a(t) = t u_a + w_a:
 *   u_a = d_a s_a, w_a = (o_a - bmin_a) s_a (s_a = k / (bmax_a - bmin_a) in
 *     binary32, the cache's scale; o, d from the fixed ray sequence);
 *   box: for u_a != 0 the entry / exit times are -w_a / u_a and (k - w_a) / u_a
 *     (the smaller enters); u_a == 0 needs 0 <= w_a < k; t0 = the largest
 *     entry and t_near, t1 = the smallest exit and t_far; no cells unless
 *     t0 < t1;
 *   start cell c_a = floor(fma(t0, u_a, w_a)) clamped to [0, k - 1];
 *   next crossing along a: ((c_a + 1) - w_a) / u_a (u_a > 0), (c_a - w_a) / u_a
 *     (u_a < 0), +infinity (u_a == 0);
 *   per cell: a* = the axis with the smallest crossing (x, then y, then z on
 *     ties), t_next its crossing, delta = min(t_next, t1) - t (t = t0 at the
 *     start); the walk ends after this cell unless t_next < t1; t = max(t,
 *     t_next); c_a* moves one cell and the walk ends if it leaves [0, k);
 *     otherwise a*'s crossing is recomputed.
 * A cell with delta <= 0 (rounding at a corner) is visited without a lookup.
 * n_samples caps the walk (n_samples >= 3k never cuts a ray short). Eq. 1 per
 * cell with delta_i = delta; termination when sum floor(fp32(sigma delta) 2^32)
 * >= ceil(ln(1/T_thr) 2^32). Stats: n_steps = cells walked, n_lookups =
 * density lookups (cells with delta > 0; with FNR_RENDER_SKIP_EMPTY those in
 * occupied bricks), n_occupied = composited cells. debug cells: the walked
 * cells in order, then -1 (walk ended) or -2 (terminated). With
 * FNR_RENDER_SKIP_EMPTY and no debug cells the walk may pass over a cube of
 * empty cells in one step; every output (RGBA, the three counters) is the
 * cell-by-cell walk's, bit for bit. Combines with
 * FNR_RENDER_SKIP_EMPTY and FNR_RENDER_DIR_BILINEAR; dense caches only, and
 * not for served requests, fnr_render_noalloc or fnr_render_mlp
 * (FNR_ERR_UNSUPPORTED). */
#define FNR_RENDER_VOXELS 4u

typedef struct {
    int32_t n_steps;    /* samples visited (i + 1 of the terminating sample, else N) */
    int32_t n_lookups;  /* visited samples inside the cache box (with FNR_RENDER_SKIP_EMPTY:
                           those in occupied bricks) */
    int32_t n_occupied; /* visited samples with sigma > 0 */
    int32_t dir_cell;   /* i_theta * l + i_phi */
} fnr_ray_stats;

/* Render n_cams views of one cache (the plain path: one launch per call; up
 * to 32 views share a launch). Frame f's pixels start at pixel offset
 * P_f = sum_{g<f} W_g H_g:
 *   rgba_dev        float[P][4], (R, G, B, alpha) at P_f + py * W_f + px
 *   stats_dev       fnr_ray_stats[P] or NULL
 *   debug_cells_dev int32[P][n_samples] or NULL: per sample its cell index,
 *                   -1 outside the box, -2 after termination.
 * Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
FNR_API fnr_status fnr_render(fnr_context *ctx, const fnr_cache *cache, const fnr_camera *cams, int32_t n_cams,
                      const fnr_render_params *params, float *rgba_dev, fnr_ray_stats *stats_dev,
                      int32_t *debug_cells_dev, fnr_stream_t stream);


/* The uncached render ("no cache" in the paper's timings, Section 5): F_pos
 * evaluated at every sample inside the box and F_dir at the ray direction on
 * the tensor cores, then Eq. 5 and Eq. 1 exactly as fnr_render composites
 * them. Samples: t_i = fma(i + 1/2, Delta, near) and p_a = fma(t_i, d_a, o_a)
 * in binary32 (d, o from the fixed ray sequence); p is inside iff
 * bmin_a <= p_a < bmax_a on every axis. F_pos reads the raw position (its
 * positional encoding as for the cache build); sigma = ReLU(output 0), u_i,
 * v_i, w_i = outputs 1..3D; F_dir reads the unit direction; beta = outputs
 * 0..D-1. One view per call; device temporaries are allocated per call and
 * charged to the budget. Stats: n_lookups = inside samples up to termination,
 * n_occupied = those with sigma > 0, dir_cell = -1. Errors: INVALID_ARG,
 * UNSUPPORTED, BUDGET, CUDA, DEVICE. */
FNR_API fnr_status fnr_render_mlp(fnr_context *ctx, const fnr_mlp *pos_mlp, const fnr_mlp *dir_mlp, int32_t D,
                                  const float *bmin, const float *bmax, const fnr_camera *cam,
                                  const fnr_render_params *params, float *rgba_dev, fnr_ray_stats *stats_dev,
                                  fnr_stream_t stream);

/* ------------------------------------------------------------------ serving */
/* A request for one view (Section 4's per-view render, served). The request
 * is copied at submit; rgba_dev / stats_dev stay caller-owned and must stay
 * valid until the request has completed. The cache cannot be freed while one
 * of its requests is queued or in flight.
 * Ordering: the launch that renders the request first waits for all work that
 * was queued on `stream` when fnr_submit was called (NULL: the legacy default
 * stream), so outputs prepared on that stream are not overwritten. After
 * fnr_poll / fnr_wait report completion the outputs may be read on any stream. */
typedef struct {
    const fnr_cache *cache;
    fnr_camera camera;
    fnr_render_params params;
    float *rgba_dev;          /* float[H*W][4] */
    fnr_ray_stats *stats_dev; /* [H*W] or NULL */
    fnr_stream_t stream;      /* the producer stream of the outputs (see above) */
    int32_t priority;         /* reserved, must be 0 */
    int32_t reserved;
} fnr_request;

typedef struct {
    fnr_status status;        /* FNR_OK, or the error that ended the request */
    int32_t reserved;
    uint64_t t_submit_ns;     /* steady-clock nanoseconds */
    uint64_t t_admit_ns;      /* 0 while queued */
    uint64_t t_done_ns;       /* when the host saw the completion word */
    uint64_t n_rays;
    int64_t batch;            /* launch the request ran in (-1 while queued) */
    uint64_t ticket;
} fnr_result;

typedef struct {
    int32_t queue_capacity;     /* queued requests before FNR_ERR_QUEUE_FULL (0: 4096) */
    int32_t max_batch_requests; /* requests per persistent launch, <= 64 (0: 64) */
    int64_t max_batch_rays;     /* rays per launch (0: 16 Mi) */
    int32_t n_slots;            /* launches in flight at once, <= 8 (0: 3) */
    int32_t use_graphs;         /* 1: each slot replays a captured CUDA graph */
    int32_t idle_spin_us;       /* the scheduler thread keeps polling for submits and completions this
                                   long after its last event, then sleeps until a submit (0: 5000;
                                   -1: it never sleeps while the loop runs, for the lowest latency at
                                   the cost of one busy host thread); < -1: INVALID_ARG */
    int32_t reserved;           /* 0 */
} fnr_serve_config;

/* Start the request loop (a host scheduler thread plus n_slots streams).
 * fnr_submit starts it with the defaults if it is not running.
 * Errors: INVALID_ARG (already running, bad config), CUDA. */
FNR_API fnr_status fnr_serve_start(fnr_context *ctx, const fnr_serve_config *cfg);
/* Drain queued and in-flight requests, then stop the loop. */
FNR_API fnr_status fnr_serve_stop(fnr_context *ctx);
/* Queue one request; returns at once with a ticket. Requests are admitted in
 * arrival order into persistent launches as slots free up and as the HBM
 * budget allows (each admitted request charges its output bytes until it
 * completes). Errors: INVALID_ARG, UNSUPPORTED (D not served), BUDGET (the
 * output alone exceeds the budget), QUEUE_FULL. */
FNR_API fnr_status fnr_submit(fnr_context *ctx, const fnr_request *req, uint64_t *ticket);
/* FNR_ERR_NOT_READY while queued or in flight (out is filled with the times so
 * far); otherwise fills out, forgets the ticket and returns FNR_OK (the
 * request's own outcome is out->status). INVALID_ARG for an unknown ticket. */
FNR_API fnr_status fnr_poll(fnr_context *ctx, uint64_t ticket, fnr_result *out);
/* As fnr_poll, blocking up to timeout_ms; FNR_ERR_TIMEOUT if still not done. */
FNR_API fnr_status fnr_wait(fnr_context *ctx, uint64_t ticket, uint32_t timeout_ms, fnr_result *out);

/* ------------------------------------------------------------------ rendering without allocation */
/* The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory: a process whose HBM is owned by another allocator
 * that has already reserved nearly all of it, a render loop that must never
 * stall on cudaMalloc / cudaFree (cudaFree synchronises the device), or a host
 * that plans every byte of device memory up front.
 *
 * Renders up to 32 views of one cache, like fnr_render, with the persistent
 * tile-popping kernel of the request loop, and allocates nothing: the kernel's
 * scratch (a tile counter and one finished-tile counter per view) is a 256-byte
 * static __device__ array that every GPU loading the library holds until the
 * process exits. Views, caches and outputs are the caller's, laid out as for
 * fnr_render; done_words (nullable; device-visible, e.g. host-mapped) gets 1
 * in word f when view f is finished. Stream-ordered on `stream`.
 * Every call looks up the array's device address with the device current (a
 * context reset between calls therefore does no harm); the first call for a
 * device and cache format also queries the kernel's occupancy, so make that
 * first call before any stream capture. Every
 * call shares the array and clears the counters it uses before its launch:
 * calls whose launches overlap on the GPU race, so keep them on one stream or
 * order them. Errors: INVALID_ARG (more than 32 views: the scratch holds one
 * counter per view; NULL arguments; bad params), UNSUPPORTED (D not in
 * {1,2,3,4,6,8,12,16}; FNR_RENDER_SKIP_EMPTY, which this entry point does not
 * render), CUDA. */
FNR_API fnr_status fnr_render_noalloc(const fnr_cache *cache, const fnr_camera *cams, int32_t n_cams,
                                      const fnr_render_params *params, float *rgba_dev, fnr_ray_stats *stats_dev,
                                      uint32_t *done_words, fnr_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* FNR_H */
