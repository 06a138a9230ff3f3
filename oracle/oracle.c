/*
 * oracle.c -- plain FP64 CPU oracle for FastNeRF's cached rendering path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. The renderer never calls it
 * and shares no code, header, table or constant generator with it.
 *
 * What it computes (paper: FastNeRF, Garbin et al. 2021):
 *   - Section 3.1, Eq. 1: c_hat = sum_i T_i (1 - exp(-sigma_i delta_i)) c_i,
 *     T_i = exp(-sum_{j<i} sigma_j delta_j) (the garbled lower index of the sum
 *     is read as j = 1 .. i-1), delta_i = Delta for every sample (midpoint
 *     samples on [near, far], unit-length ray direction).
 *   - Section 3.2, Eq. 5: c = sum_{i=1..D} beta_i (u_i, v_i, w_i), followed by
 *     the output activation (sigmoid by default, identity selectable; the text
 *     does not state one).
 *   - Section 3.3: position cache = k samples per axis of the bounding box,
 *     cell-centred, looked up by nearest neighbour (Section 4); direction
 *     cache = l x l samples of (theta in [0, pi], phi in [0, 2 pi)), polar
 *     angle from +z, phi = atan2(y, x) wrapped to [0, 2 pi).
 *   - Supplementary "Meshing & Rendering": Beer-Lambert extinction with early
 *     ray termination; here: stop after the first sample whose transmittance
 *     falls to T_thr, decided by an exact integer optical-depth sum.
 *   - Section 4 (integration over every voxel on the ray): the voxel walk, one sample per cell
 *     the ray passes through with delta = the ray's length inside the cell
 *     (orc_voxel_walk).
 *   - Supplementary "Cache size calculation" (second version): dense cache
 *     sizes for NeRF and FastNeRF.
 *
 * Integer decisions (which cell a sample or a direction falls in, and when a
 * ray stops) are taken on binary32 values computed with a fixed sequence of
 * correctly rounded operations; this file must be compiled with
 * -ffp-contract=off so that C's float arithmetic is exactly that sequence.
 * Everything else (weights, colour, transmittance) is FP64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FP32 0
#define ORC_FP16 1
#define ORC_FP8 2

#define FNR_ORC_MAX_N 4096 /* longest voxel walk */

#define ORC_ACT_SIGMOID 0
#define ORC_ACT_IDENTITY 1

typedef void (*orc_field_fn)(int64_t cell, int want_uvw, double *sigma, double *uvw, void *user);

typedef struct {
    int32_t k, D, l;
    float bmin[3], bmax[3];
    int32_t pos_prec, dir_prec;
    const void *sigma;    /* [k^3] stored values */
    const void *uvw;      /* [k^3][3D] stored values, u_1..u_D v_1..v_D w_1..w_D */
    const void *beta;     /* [l][l][D] stored values */
    const float *scales;  /* FP8 only: [1 + 3D] per-channel scales (sigma first) */
    orc_field_fn field;   /* optional: FP64 cell accessor that replaces sigma/uvw */
    void *field_user;
    const uint8_t *occ;   /* optional: [nb^3] brick occupancy (nb = ceil(k / occ_brick)), brick
                             (bz nb + by) nb + bx nonzero iff one of its cells has sigma > 0 */
    int32_t occ_brick;    /* cells per brick side */
    int32_t off_brick;    /* FP8 only: cells per side of an offset brick */
    const uint16_t *offsets; /* FP8 only: [nbo^3][3D] binary16 offsets of the (u, v, w) channels */
} orc_cache;

typedef struct {
    float c2w[12]; /* row-major 3x4 camera-to-world [R | eye] */
    float fx, fy, cx, cy;
    int32_t W, H;
} orc_camera;

typedef struct {
    int32_t N;
    float t_near, t_far, t_thr;
    float bg[3];
    int32_t act;
    int32_t skip_empty; /* nonzero: samples in bricks without density are not looked up */
    int32_t dir_bilinear; /* nonzero: beta interpolated bilinearly in (theta, phi) between bin centres */
    int32_t voxels;       /* nonzero: visit every cell the ray passes through (orc_voxel_walk), at most N */
} orc_params;

/* ------------------------------------------------------------ number formats */
/* IEEE binary16 decode (1 sign, 5 exponent, 10 fraction bits, bias 15). */
double orc_f16_decode(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp(1024.0 + m, e - 25);
    return s ? -v : v;
}

/* binary32 -> binary16, round to nearest even, overflow to infinity. */
uint16_t orc_f16_encode(float f) {
    uint16_t sign = signbit(f) ? 0x8000 : 0;
    if (isnan(f)) return sign | 0x7e00;
    double a = fabs((double)f);
    if (isinf(f) || a >= 65520.0) return sign | 0x7c00;
    if (a < ldexp(1.0, -14)) {
        double r = rint(a * ldexp(1.0, 24)); /* quantum 2^-24, exact scaling */
        return sign | (uint16_t)r;           /* r == 1024 is the smallest normal */
    }
    int e;
    frexp(a, &e); /* a in [2^(e-1), 2^e) */
    int E = e - 1;
    double r = rint(ldexp(a, 10 - E)); /* in [1024, 2048] */
    if (r == 2048.0) { r = 1024.0; E += 1; }
    if (E + 15 >= 31) return sign | 0x7c00;
    return sign | (uint16_t)(((E + 15) << 10) | ((int)r - 1024));
}

/* OCP FP8 E4M3 ("fn": no infinities, NaN = S.1111.111, max 448) decode. */
double orc_e4m3_decode(uint8_t q) {
    int s = (q >> 7) & 1, e = (q >> 3) & 15, m = q & 7;
    double v;
    if (e == 15 && m == 7) v = NAN;
    else if (e == 0) v = ldexp((double)m, -9);
    else v = ldexp(8.0 + m, e - 10);
    return s ? -v : v;
}

/* binary32 -> E4M3, round to nearest even, saturating to +-448 (also for
 * infinities); NaN -> 0x7f. */
uint8_t orc_e4m3_encode(float f) {
    if (isnan(f)) return 0x7f;
    uint8_t sign = signbit(f) ? 0x80 : 0;
    double a = fabs((double)f);
    if (a >= 448.0) return sign | 0x7e;
    if (a < ldexp(1.0, -6)) {
        double r = rint(a * 512.0); /* quantum 2^-9 */
        return sign | (uint8_t)r;   /* r == 8 is the smallest normal */
    }
    int e;
    frexp(a, &e);
    int E = e - 1;
    double r = rint(ldexp(a, 3 - E)); /* in [8, 16] */
    if (r == 16.0) { r = 8.0; E += 1; }
    return sign | (uint8_t)(((E + 7) << 3) | ((int)r - 8));
}

/* Cache quantisation as the precision forms define it: density is clamped
 * to >= 0 (NaN -> 0) first; FP8 uses one scale per channel,
 * scale = absmax / 448 in binary32 (1 when the channel is all zero), and
 * q = e4m3(x / scale) with a binary32 division. For the (u, v, w) channels
 * the quantised quantity is the residual from a per-brick offset
 * (orc_fp8_offsets / orc_fp8_uvw_quantize below); the density has none. */
float orc_fp8_scale(int64_t n, int64_t stride, const float *x, int clamp_nonneg) {
    float amax = 0.0f;
    for (int64_t i = 0; i < n; ++i) {
        float v = x[i * stride];
        if (clamp_nonneg) v = (v > 0.0f) ? v : 0.0f;
        float a = fabsf(v);
        if (a > amax) amax = a;
    }
    return amax > 0.0f ? amax / 448.0f : 1.0f;
}

void orc_quantize(int prec, int64_t n, int64_t stride, const float *x, int clamp_nonneg, float scale, void *out) {
    for (int64_t i = 0; i < n; ++i) {
        float v = x[i * stride];
        if (clamp_nonneg) v = (v > 0.0f) ? v : 0.0f;
        if (prec == ORC_FP16) ((uint16_t *)out)[i * stride] = orc_f16_encode(v);
        else if (prec == ORC_FP8) ((uint8_t *)out)[i * stride] = orc_e4m3_encode(v / scale);
        else ((float *)out)[i * stride] = v;
    }
}

/* E4M3 (u, v, w) offsets. The grid is cut into offset bricks of Bo cells a
 * side (clipped to the grid; nbo = ceil(k / Bo) per axis, brick index
 * (bz nbo + by) nbo + bx). Per brick and channel the offset is the binary16
 * (nearest even) value of the binary32 midrange (min + max) * 0.5 of the
 * channel's values over the brick's cells; NaN values are ignored, and a
 * brick whose values are all NaN gets 0. out: [nbo^3][nch] binary16 bits. */
void orc_fp8_offsets(int32_t k, int32_t nch, int32_t Bo, const float *uvw, uint16_t *out) {
    const int64_t nbo = (k + Bo - 1) / Bo;
    for (int64_t bz = 0; bz < nbo; ++bz)
        for (int64_t by = 0; by < nbo; ++by)
            for (int64_t bx = 0; bx < nbo; ++bx)
                for (int c = 0; c < nch; ++c) {
                    int any = 0;
                    float mn = 0.0f, mx = 0.0f;
                    for (int64_t z = bz * Bo; z < (bz + 1) * Bo && z < k; ++z)
                        for (int64_t y = by * Bo; y < (by + 1) * Bo && y < k; ++y)
                            for (int64_t x = bx * Bo; x < (bx + 1) * Bo && x < k; ++x) {
                                const float v = uvw[((z * k + y) * k + x) * nch + c];
                                if (v != v) continue;
                                if (!any || v < mn) mn = v;
                                if (!any || v > mx) mx = v;
                                any = 1;
                            }
                    const float mid = any ? (mn + mx) * 0.5f : 0.0f;
                    out[((bz * nbo + by) * nbo + bx) * nch + c] = orc_f16_encode(mid);
                }
}

/* The offset of cell (x, y, z) in channel c, as binary32. */
static float fp8_offset(int32_t k, int32_t nch, int32_t Bo, const uint16_t *offsets, int64_t cell, int c) {
    const int64_t nbo = (k + Bo - 1) / Bo;
    const int64_t x = cell % k, y = (cell / k) % k, z = cell / ((int64_t)k * k);
    return (float)orc_f16_decode(offsets[(((z / Bo) * nbo + y / Bo) * nbo + x / Bo) * nch + c]);
}

/* Per-channel scale of the (u, v, w) residuals r = binary32(u - offset):
 * absmax_c |r| / 448 in binary32 (NaN skipped; 1 when all are zero). */
float orc_fp8_uvw_scale(int32_t k, int32_t nch, int32_t Bo, const float *uvw, const uint16_t *offsets, int c) {
    const int64_t k3 = (int64_t)k * k * k;
    float amax = 0.0f;
    for (int64_t cell = 0; cell < k3; ++cell) {
        const float r = uvw[cell * nch + c] - fp8_offset(k, nch, Bo, offsets, cell, c);
        const float a = fabsf(r);
        if (a > amax) amax = a;
    }
    return amax > 0.0f ? amax / 448.0f : 1.0f;
}

/* codes[cell][c] = E4M3(binary32(r / scale_c)), r = binary32(u - offset). The
 * stored value is offset + scale_c * e4m3(q). */
void orc_fp8_uvw_quantize(int32_t k, int32_t nch, int32_t Bo, const float *uvw, const uint16_t *offsets,
                          const float *scales, uint8_t *codes) {
    const int64_t k3 = (int64_t)k * k * k;
    for (int64_t cell = 0; cell < k3; ++cell)
        for (int c = 0; c < nch; ++c) {
            const float r = uvw[cell * nch + c] - fp8_offset(k, nch, Bo, offsets, cell, c);
            codes[cell * nch + c] = orc_e4m3_encode(r / scales[c]);
        }
}

/* ------------------------------------------------------------ cache sizes */
/* Supplementary "Cache size calculation": M_NeRF = a (s_sigma + s_rgb) k^3 l^2 and
 * M_FastNeRF = a (D s_uvw + s_sigma) k^3 + D s_beta l^2, sizes in bits, dense
 * (a = 1); returned in bytes. s_uvw is the size of one (u_i, v_i, w_i) triple. */
uint64_t orc_bytes_nerf(uint64_t k, uint64_t l, uint64_t s_sigma_bits, uint64_t s_rgb_bits) {
    return (s_sigma_bits + s_rgb_bits) * k * k * k * l * l / 8u;
}
uint64_t orc_bytes_fastnerf_pos(uint64_t k, uint64_t D, uint64_t s_sigma_bits, uint64_t s_uvw_bits) {
    return (D * s_uvw_bits + s_sigma_bits) * k * k * k / 8u;
}
uint64_t orc_bytes_fastnerf_dir(uint64_t l, uint64_t D, uint64_t s_beta_bits) {
    return D * s_beta_bits * l * l / 8u;
}

/* ------------------------------------------------------------ geometry */
/* Pixel (px, py) -> unit direction d and origin o. Camera looks down its -z,
 * pixel centres at +0.5, py = 0 is the top row. binary32 op sequence:
 *   dcx = ((px + 0.5) - cx) / fx,  dcy = -(((py + 0.5) - cy) / fy),  dcz = -1
 *   w_r = fma(R_r0, dcx, fma(R_r1, dcy, -R_r2))
 *   n2 = fma(wx, wx, fma(wy, wy, wz * wz)),  d = w / sqrt(n2). */
void orc_ray(const orc_camera *c, int32_t px, int32_t py, float d[3], float o[3]) {
    const float *M = c->c2w;
    float dcx = (((float)px + 0.5f) - c->cx) / c->fx;
    float dcy = -((((float)py + 0.5f) - c->cy) / c->fy);
    float w[3];
    for (int r = 0; r < 3; ++r) w[r] = fmaf(M[4 * r + 0], dcx, fmaf(M[4 * r + 1], dcy, -M[4 * r + 2]));
    float n2 = fmaf(w[0], w[0], fmaf(w[1], w[1], w[2] * w[2]));
    float len = sqrtf(n2);
    for (int r = 0; r < 3; ++r) d[r] = w[r] / len;
    o[0] = M[3]; o[1] = M[7]; o[2] = M[11];
}

/* Monotone binary32 key of the azimuth phi = atan2(y, x) in [0, 2 pi):
 * q in [0, 4], one unit per quadrant ("diamond angle"). (0, 0) -> 0. */
float orc_phi_key(float x, float y) {
    if (x == 0.0f && y == 0.0f) return 0.0f;
    if (y >= 0.0f) {
        if (x >= 0.0f) return y / (x + y);
        return 1.0f + (-x) / (y + (-x));
    }
    if (x < 0.0f) return 2.0f + (-y) / ((-x) + (-y));
    return 3.0f + x / (x + (-y));
}

static double phi_key_fp64(double x, double y) {
    if (x == 0.0 && y == 0.0) return 0.0;
    if (y >= 0.0) {
        if (x >= 0.0) return y / (x + y);
        return 1.0 + (-x) / (y - x);
    }
    if (x < 0.0) return 2.0 + (-y) / (-x - y);
    return 3.0 + x / (x - y);
}

/* Direction-cell boundaries: theta_j = j pi / l (key d_z, boundary cos theta_j,
 * rounded to binary32) and phi_j = 2 pi j / l (boundary key of the unit
 * vector at phi_j, FP64 then rounded), j = 1 .. l-1; entry 0 unused. */
static void dir_tables(int l, float *ct, float *qp) {
    const double pi = 3.14159265358979323846264338327950288;
    ct[0] = 1.0f; qp[0] = 0.0f;
    for (int j = 1; j < l; ++j) {
        ct[j] = (float)cos((double)j * pi / (double)l);
        double ph = 2.0 * pi * (double)j / (double)l;
        qp[j] = (float)phi_key_fp64(cos(ph), sin(ph));
    }
}

/* Direction cell: i_theta = #{j in 1..l-1 : d_z <= cos(theta_j)},
 * i_phi = #{j in 1..l-1 : key(d) >= key(phi_j)}. Plain counts over the table. */
static void dir_cell_tab(int l, const float *ct, const float *qp, const float d[3], int32_t *it, int32_t *ip) {
    int a = 0, b = 0;
    float q = orc_phi_key(d[0], d[1]);
    for (int j = 1; j < l; ++j) {
        if (d[2] <= ct[j]) ++a;
        if (q >= qp[j]) ++b;
    }
    *it = a;
    *ip = b;
}

void orc_dir_cell(int l, const float d[3], int32_t *it, int32_t *ip) {
    float *ct = (float *)malloc(sizeof(float) * (size_t)l * 2);
    dir_tables(l, ct, ct + l);
    dir_cell_tab(l, ct, ct + l, d, it, ip);
    free(ct);
}

/* Sample spacing Delta = (far - near) / N in binary32. */
float orc_dt(float t_near, float t_far, int32_t N) { return (t_far - t_near) / (float)N; }

/* Termination threshold on the fixed-point optical depth S = sum floor(sigma 2^32):
 * S_thr = ceil(ln(1/T_thr) / Delta * 2^32) in FP64; T_thr <= 0 disables it. */
int64_t orc_s_thr(float t_thr, float dt) {
    if (!(t_thr > 0.0f)) return INT64_MAX;
    double v = ceil(log(1.0 / (double)t_thr) / (double)dt * 4294967296.0);
    if (v >= 9223372036854775807.0) return INT64_MAX;
    if (v < 0.0) return 0;
    return (int64_t)v;
}

int64_t orc_fix(double sigma) {
    if (!(sigma > 0.0)) return 0;
    if (sigma >= 2147483648.0) return INT64_MAX;
    return (int64_t)floor(sigma * 4294967296.0);
}

/* ------------------------------------------------------------ cache access */
static double stored_scalar(int prec, const void *base, int64_t idx, float scale) {
    if (prec == ORC_FP16) return orc_f16_decode(((const uint16_t *)base)[idx]);
    if (prec == ORC_FP8) {
        float v = (float)orc_e4m3_decode(((const uint8_t *)base)[idx]);
        return (double)(v * scale); /* binary32 product */
    }
    return (double)((const float *)base)[idx];
}

static double cache_sigma(const orc_cache *c, int64_t cell) {
    if (c->field) {
        double s;
        c->field(cell, 0, &s, NULL, c->field_user);
        return s;
    }
    return stored_scalar(c->pos_prec, c->sigma, cell, c->pos_prec == ORC_FP8 ? c->scales[0] : 1.0f);
}

static void cache_uvw(const orc_cache *c, int64_t cell, double *out) {
    if (c->field) {
        double s;
        c->field(cell, 1, &s, out, c->field_user);
        return;
    }
    int n = 3 * c->D;
    if (c->pos_prec == ORC_FP8) {
        /* the exact value of the stored (code, scale, offset): offset + scale e4m3(code), FP64 */
        for (int j = 0; j < n; ++j)
            out[j] = orc_e4m3_decode(((const uint8_t *)c->uvw)[cell * n + j]) * (double)c->scales[1 + j] +
                     (double)fp8_offset(c->k, n, c->off_brick, c->offsets, cell, j);
        return;
    }
    for (int j = 0; j < n; ++j) out[j] = stored_scalar(c->pos_prec, c->uvw, cell * n + j, 1.0f);
}

/* ------------------------------------------------------------ cell table
 * A field accessor for grids too large to hold densely on the host: a dense
 * binary32 sigma plane plus binary32 uvw records for a listed set of cells
 * (ascending cell index). The cells a ray shades and its termination depend on
 * sigma alone, so a first pass with an empty table lists them (its colours are
 * discarded) and a second pass reads their records. A cell missing from the
 * table reads as uvw = 0 and is counted. Storage only: the values returned are
 * exactly those a dense FP32 cache would give. */
typedef struct {
    const float *sigma;   /* [k^3] */
    int64_t n;            /* cells in the table */
    const int64_t *cells; /* [n], ascending */
    const float *rec;     /* [n][nch] */
    int32_t nch;
    int64_t missing;      /* uvw reads of cells not in the table */
} orc_table;

void orc_table_field(int64_t cell, int want_uvw, double *sigma, double *uvw, void *user) {
    orc_table *t = (orc_table *)user;
    *sigma = (double)t->sigma[cell];
    if (!want_uvw) return;
    int64_t lo = 0, hi = t->n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (t->cells[mid] < cell) lo = mid + 1; else hi = mid;
    }
    if (lo < t->n && t->cells[lo] == cell) {
        for (int j = 0; j < t->nch; ++j) uvw[j] = (double)t->rec[lo * t->nch + j];
    } else {
        for (int j = 0; j < t->nch; ++j) uvw[j] = 0.0;
        __atomic_fetch_add(&t->missing, 1, __ATOMIC_RELAXED);
    }
}

static double stored_beta(const orc_cache *c, int64_t cell, int i) {
    return c->dir_prec == ORC_FP16 ? orc_f16_decode(((const uint16_t *)c->beta)[cell * c->D + i])
                                   : (double)((const float *)c->beta)[cell * c->D + i];
}

/* Interpolated direction lookup (Section 4 samples F_view with interpolation
 * rather than nearest neighbour): beta bilinear in (theta, phi) between the
 * bin centres theta_i = (i + 1/2) pi / l, phi_j = (j + 1/2) 2 pi / l, with
 * theta from +z and phi = atan2(y, x) in [0, 2 pi). Continuous indices
 * u = theta l / pi - 1/2, v = phi l / (2 pi) - 1/2; the theta neighbours are
 * clamped to [0, l - 1] (no data beyond the poles), the phi neighbours wrap. */
void orc_beta_bilinear(const orc_cache *c, const float d[3], double *beta) {
    const double pi = 3.14159265358979323846264338327950288;
    const int l = c->l;
    const double x = d[0], y = d[1], z = d[2];
    const double theta = atan2(sqrt(x * x + y * y), z);
    double phi = atan2(y, x);
    if (phi < 0.0) phi += 2.0 * pi;
    const double u = theta * l / pi - 0.5, v = phi * l / (2.0 * pi) - 0.5;
    const double fu = floor(u), fv = floor(v);
    const double a = u - fu, b = v - fv;
    int i0 = (int)fu, i1 = i0 + 1;
    i0 = i0 < 0 ? 0 : (i0 > l - 1 ? l - 1 : i0);
    i1 = i1 < 0 ? 0 : (i1 > l - 1 ? l - 1 : i1);
    const int j0 = (((int)fv % l) + l) % l, j1 = (j0 + 1) % l;
    for (int i = 0; i < c->D; ++i)
        beta[i] = (1.0 - a) * (1.0 - b) * stored_beta(c, (int64_t)i0 * l + j0, i) +
                  (1.0 - a) * b * stored_beta(c, (int64_t)i0 * l + j1, i) +
                  a * (1.0 - b) * stored_beta(c, (int64_t)i1 * l + j0, i) + a * b * stored_beta(c, (int64_t)i1 * l + j1, i);
}

/* ------------------------------------------------------------ voxel walk */
/* Section 4 integrates every voxel a ray passes through. The walk below visits
 * the cells of the segment [t0, t1] = [max(t_near, t_enter), min(t_far, t_exit)]
 * of the ray inside the box in order (a 3-D digital differential analyser),
 * in binary32 with this fixed sequence, in grid units g_a(t) = t u_a + w_a:
 *   u_a = d_a s_a, w_a = (o_a - bmin_a) s_a   (s_a = k / (bmax_a - bmin_a))
 *   box: for u_a != 0 the axis' entry and exit times are -w_a / u_a and
 *     (k - w_a) / u_a (the smaller one enters); u_a == 0 needs 0 <= w_a < k;
 *     t0 = the largest entry (and t_near), t1 = the smallest exit (and t_far);
 *     no cells unless t0 < t1
 *   start cell c_a = floor(fma(t0, u_a, w_a)) clamped to [0, k - 1]
 *   next crossing along a: ((c_a + 1) - w_a) / u_a for u_a > 0, (c_a - w_a) / u_a
 *     for u_a < 0, +infinity for u_a == 0
 *   per step: a* = the axis with the smallest crossing (x before y before z on
 *     ties), t_next its crossing; the cell's length delta = min(t_next, t1) - t
 *     (t = t0 at the start); the walk ends after this cell unless t_next < t1;
 *     t = max(t, t_next); c_a* moves one cell along the ray and the walk ends
 *     if it leaves [0, k); otherwise a*'s next crossing is recomputed.
 * delta <= 0 (rounding at a corner) is a zero-length visit. cells[j] is the
 * linear index (z k + y) k + x of the j-th cell, delta[j] its length; returns
 * the number of cells, at most max_steps. */
static float next_crossing(int32_t c, float u, float w) {
    if (u > 0.0f) return ((float)(c + 1) - w) / u;
    if (u < 0.0f) return ((float)c - w) / u;
    return INFINITY;
}

int orc_voxel_walk(int32_t k, const float bmin[3], const float sc[3], const float o[3], const float d[3],
                   float t_near, float t_far, int32_t max_steps, int32_t *cells, float *delta) {
    const float kf = (float)k;
    float u[3], w[3], t0 = t_near, t1 = t_far;
    for (int a = 0; a < 3; ++a) {
        u[a] = d[a] * sc[a];
        w[a] = (o[a] - bmin[a]) * sc[a];
        if (u[a] != u[a] || w[a] != w[a]) return 0;
        if (u[a] == 0.0f) {
            if (!(w[a] >= 0.0f && w[a] < kf)) return 0;
        } else {
            const float ta = -w[a] / u[a], tb = (kf - w[a]) / u[a];
            const float lo = ta < tb ? ta : tb, hi = ta < tb ? tb : ta;
            if (lo > t0) t0 = lo;
            if (hi < t1) t1 = hi;
        }
    }
    if (!(t0 < t1)) return 0;
    int32_t c[3], step[3];
    float tn[3];
    for (int a = 0; a < 3; ++a) {
        int32_t ci = (int32_t)floorf(fmaf(t0, u[a], w[a]));
        c[a] = ci < 0 ? 0 : (ci > k - 1 ? k - 1 : ci);
        step[a] = u[a] > 0.0f ? 1 : (u[a] < 0.0f ? -1 : 0);
        tn[a] = next_crossing(c[a], u[a], w[a]);
    }
    float t = t0;
    int32_t n = 0;
    while (n < max_steps) {
        int a = 0;
        if (tn[1] < tn[a]) a = 1;
        if (tn[2] < tn[a]) a = 2;
        const float tnext = tn[a];
        const float end = tnext < t1 ? tnext : t1;
        cells[n] = (int32_t)(((int64_t)c[2] * k + c[1]) * k + c[0]);
        delta[n] = end - t;
        ++n;
        if (!(tnext < t1)) break;
        if (tnext > t) t = tnext;
        c[a] += step[a];
        if (c[a] < 0 || c[a] >= k) break;
        tn[a] = next_crossing(c[a], u[a], w[a]);
    }
    return n;
}

/* ------------------------------------------------------------ one ray */
typedef struct {
    const orc_cache *c;
    const orc_camera *cam;
    const orc_params *p;
    const float *ct, *qp;
    float dt;
    int64_t s_thr;
    float scale[3];
} ray_ctx;

static void render_ray(const ray_ctx *X, int32_t px, int32_t py, double *rgba, int32_t *stats, int32_t *cells) {
    const orc_cache *c = X->c;
    const orc_params *p = X->p;
    const int D = c->D, k = c->k, N = p->N;
    float d[3], o[3];
    orc_ray(X->cam, px, py, d, o);
    int32_t it, ip;
    dir_cell_tab(c->l, X->ct, X->qp, d, &it, &ip);
    int64_t dcell = (int64_t)it * c->l + ip;
    double beta[16];
    if (p->dir_bilinear) {
        orc_beta_bilinear(c, d, beta);
    } else {
        for (int i = 0; i < D; ++i) beta[i] = stored_beta(c, dcell, i);
    }
    double T = 1.0, C[3] = {0.0, 0.0, 0.0};
    int64_t S = 0;
    int32_t n_steps = N, n_look = 0, n_occ = 0;
    double uvw[48];
    const float kf = (float)k;
    if (p->voxels) {
        /* Section 4: every cell the ray passes through is one sample whose
         * delta is the ray's length inside it (Eq. 1 with delta_i = that length);
         * termination sums floor(fp32(sigma delta) 2^32) against
         * ceil(ln(1 / T_thr) 2^32). */
        int32_t wc[FNR_ORC_MAX_N];
        float wd[FNR_ORC_MAX_N];
        const int32_t nw = orc_voxel_walk(k, c->bmin, X->scale, o, d, p->t_near, p->t_far, N, wc, wd);
        n_steps = nw;
        int terminated = 0;
        for (int j = 0; j < nw; ++j) {
            if (cells) cells[j] = wc[j];
            if (!(wd[j] > 0.0f)) continue;
            if (p->skip_empty) {
                const int64_t B = c->occ_brick, nb = (k + B - 1) / B, cell = wc[j];
                const int64_t ix = cell % k, iy = (cell / k) % k, iz = cell / ((int64_t)k * k);
                if (!c->occ[((iz / B) * nb + iy / B) * nb + ix / B]) continue;
            }
            n_look += 1;
            const double sig = cache_sigma(c, wc[j]);
            if (!(sig > 0.0)) continue;
            n_occ += 1;
            cache_uvw(c, wc[j], uvw);
            double col[3];
            for (int ch = 0; ch < 3; ++ch) {
                double x = 0.0;
                for (int q = 0; q < D; ++q) x += beta[q] * uvw[ch * D + q]; /* Eq. 5 */
                col[ch] = p->act == ORC_ACT_IDENTITY ? x : 1.0 / (1.0 + exp(-x));
            }
            const double od = sig * (double)wd[j];
            const double alpha = -expm1(-od); /* Eq. 1 */
            for (int ch = 0; ch < 3; ++ch) C[ch] += T * alpha * col[ch];
            T *= exp(-od);
            const int64_t f = orc_fix((double)((float)sig * wd[j]));
            S = (S > INT64_MAX - f) ? INT64_MAX : S + f;
            if (S >= X->s_thr) {
                n_steps = j + 1;
                terminated = 1;
                break;
            }
        }
        if (cells)
            for (int j = n_steps; j < N; ++j) cells[j] = terminated ? -2 : -1;
        for (int ch = 0; ch < 3; ++ch) rgba[ch] = C[ch] + T * (double)p->bg[ch];
        rgba[3] = 1.0 - T;
        if (stats) {
            stats[0] = n_steps;
            stats[1] = n_look;
            stats[2] = n_occ;
            stats[3] = (int32_t)dcell;
        }
        return;
    }
    /* Cell coordinates of sample i: g_a = (o_a + t_i d_a - bmin_a) s_a with
     * t_i = near + (i + 1/2) Delta, evaluated in binary32 as
     * g_a = fma(i + 1/2, e_a, f_a), e_a = (d_a s_a) Delta,
     * f_a = fma(near, d_a s_a, (o_a - bmin_a) s_a). */
    float e[3], f[3];
    for (int a = 0; a < 3; ++a) {
        float ua = d[a] * X->scale[a];
        e[a] = ua * X->dt;
        f[a] = fmaf(p->t_near, ua, (o[a] - c->bmin[a]) * X->scale[a]);
    }
    for (int i = 0; i < N; ++i) {
        float fi = (float)i + 0.5f;
        float g[3];
        int inside = 1;
        for (int a = 0; a < 3; ++a) {
            g[a] = fmaf(fi, e[a], f[a]);
            if (!(g[a] >= 0.0f && g[a] < kf)) inside = 0;
        }
        if (!inside) {
            if (cells) cells[i] = -1;
            continue;
        }
        const int64_t ix = (int64_t)floorf(g[0]), iy = (int64_t)floorf(g[1]), iz = (int64_t)floorf(g[2]);
        int64_t cell = (iz * k + iy) * k + ix;
        if (cells) cells[i] = (int32_t)cell;
        if (p->skip_empty) {
            /* Empty-space skipping (Section 4, supplementary "Meshing & Rendering"):
             * a brick with no density holds only sigma = 0, so its samples are
             * known to be empty without a lookup. */
            const int64_t B = c->occ_brick, nb = (k + B - 1) / B;
            if (!c->occ[((iz / B) * nb + iy / B) * nb + ix / B]) continue;
        }
        n_look += 1;
        double sig = cache_sigma(c, cell);
        if (!(sig > 0.0)) continue;
        n_occ += 1;
        cache_uvw(c, cell, uvw);
        double col[3];
        for (int ch = 0; ch < 3; ++ch) {
            double x = 0.0;
            for (int j = 0; j < D; ++j) x += beta[j] * uvw[ch * D + j]; /* Eq. 5 */
            col[ch] = p->act == ORC_ACT_IDENTITY ? x : 1.0 / (1.0 + exp(-x));
        }
        double od = sig * (double)X->dt;
        double alpha = -expm1(-od); /* Eq. 1 */
        for (int ch = 0; ch < 3; ++ch) C[ch] += T * alpha * col[ch];
        T *= exp(-od);
        int64_t f = orc_fix(sig);
        S = (S > INT64_MAX - f) ? INT64_MAX : S + f;
        if (S >= X->s_thr) {
            n_steps = i + 1;
            if (cells)
                for (int j = i + 1; j < N; ++j) cells[j] = -2;
            break;
        }
    }
    for (int ch = 0; ch < 3; ++ch) rgba[ch] = C[ch] + T * (double)p->bg[ch];
    rgba[3] = 1.0 - T;
    if (stats) {
        stats[0] = n_steps;
        stats[1] = n_look;
        stats[2] = n_occ;
        stats[3] = (int32_t)dcell;
    }
}

typedef struct {
    const ray_ctx *X;
    int64_t n;
    const int32_t *px, *py;
    double *rgba;
    int32_t *stats, *cells;
    int tid, nth;
} job_t;

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    int N = J->X->p->N;
    for (int64_t i = J->tid; i < J->n; i += J->nth)
        render_ray(J->X, J->px[i], J->py[i], J->rgba + 4 * i, J->stats ? J->stats + 4 * i : NULL,
                   J->cells ? J->cells + (int64_t)N * i : NULL);
    return NULL;
}

/* Render the listed pixels. rgba: [n][4] FP64 (R, G, B, alpha = 1 - T);
 * stats (nullable): [n][4] int32 (n_steps, n_lookups, n_occupied, dir cell
 * i_theta*l + i_phi); cells (nullable): [n][N] int32 cell index per sample,
 * -1 outside the box, -2 after termination. Returns 0, or -1 on bad input. */
int orc_render_pixels(const orc_cache *c, const orc_camera *cam, const orc_params *p, int64_t n,
                      const int32_t *px, const int32_t *py, double *rgba, int32_t *stats, int32_t *cells,
                      int nthreads) {
    if (c->k <= 0 || c->D < 1 || c->D > 16 || c->l < 1 || p->N < 1 || nthreads < 1) return -1;
    if (p->voxels && p->N > FNR_ORC_MAX_N) return -1;
    if (p->skip_empty && (!c->occ || c->occ_brick < 1)) return -1;
    float *tab = (float *)malloc(sizeof(float) * (size_t)c->l * 2);
    if (!tab) return -1;
    dir_tables(c->l, tab, tab + c->l);
    ray_ctx X;
    X.c = c; X.cam = cam; X.p = p; X.ct = tab; X.qp = tab + c->l;
    X.dt = orc_dt(p->t_near, p->t_far, p->N);
    X.s_thr = orc_s_thr(p->t_thr, p->voxels ? 1.0f : X.dt); /* voxels: the optical depth is sum sigma delta */
    for (int a = 0; a < 3; ++a) X.scale[a] = (float)((double)c->k / ((double)c->bmax[a] - (double)c->bmin[a]));
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * (size_t)nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        job_t J = {&X, n, px, py, rgba, stats, cells, t, nthreads};
        jobs[t] = J;
        pthread_create(&th[t], NULL, worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th); free(tab);
    return 0;
}

/* ------------------------------------------------------------ uncached samples */
/* Sample positions of the uncached render (F_pos evaluated at the samples
 * themselves rather than at cell centres): t_i = fma(i + 1/2, Delta, near) and
 * p_a = fma(t_i, d_a, o_a) in binary32, inside iff bmin_a <= p_a < bmax_a on
 * every axis. Per pixel: points [N][3], inside [N] (0 / 1), the unit direction. */
void orc_mlp_samples(const orc_camera *cam, const orc_params *p, const float *bmin, const float *bmax, int64_t n,
                     const int32_t *px, const int32_t *py, float *points, uint8_t *inside, float *dirs) {
    const float dt = orc_dt(p->t_near, p->t_far, p->N);
    for (int64_t r = 0; r < n; ++r) {
        float d[3], o[3];
        orc_ray(cam, px[r], py[r], d, o);
        for (int a = 0; a < 3; ++a) dirs[3 * r + a] = d[a];
        for (int i = 0; i < p->N; ++i) {
            const float t = fmaf((float)i + 0.5f, dt, p->t_near);
            int in = 1;
            for (int a = 0; a < 3; ++a) {
                const float v = fmaf(t, d[a], o[a]);
                points[(r * p->N + i) * 3 + a] = v;
                if (!(v >= bmin[a] && v < bmax[a])) in = 0;
            }
            inside[r * p->N + i] = (uint8_t)in;
        }
    }
}

/* ------------------------------------------------------------ FP64 geometry */
/* The same sample positions with every step in FP64 and libm acos/atan2 for the
 * direction, to cross-check the binary32 index decisions: for each sample,
 * the FP64 cell (or -1) and the distance, in cells, from the FP64 position to
 * the nearest cell face or box face; for the ray, the FP64 direction cell and
 * the angular distance (radians) to its nearest bin edge. */
void orc_trace_fp64(const orc_cache *c, const orc_camera *cam, const orc_params *p, int32_t px, int32_t py,
                    int32_t *cells, double *margin, int32_t *dcell, double *dmargin) {
    const double pi = 3.14159265358979323846264338327950288;
    const float *M = cam->c2w;
    double dcx = ((double)px + 0.5 - cam->cx) / cam->fx;
    double dcy = -(((double)py + 0.5 - cam->cy) / cam->fy);
    double w[3];
    for (int r = 0; r < 3; ++r) w[r] = M[4 * r] * dcx + M[4 * r + 1] * dcy - M[4 * r + 2];
    double len = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    double d[3] = {w[0] / len, w[1] / len, w[2] / len};
    double th = acos(d[2] > 1.0 ? 1.0 : (d[2] < -1.0 ? -1.0 : d[2]));
    double ph = atan2(d[1], d[0]);
    if (ph < 0.0) ph += 2.0 * pi;
    int l = c->l;
    double ut = th * l / pi, up = ph * l / (2.0 * pi);
    int it = (int)floor(ut), ip = (int)floor(up);
    if (it > l - 1) it = l - 1;
    ip %= l;
    *dcell = it * l + ip;
    double mt = fabs(ut - floor(ut + 0.5)) * pi / l, mp = fabs(up - floor(up + 0.5)) * 2.0 * pi / l;
    *dmargin = mt < mp ? mt : mp;
    double dt = (double)orc_dt(p->t_near, p->t_far, p->N);
    for (int i = 0; i < p->N; ++i) {
        double t = p->t_near + (i + 0.5) * dt;
        int inside = 1;
        int64_t ix[3];
        double mg = 1e30;
        for (int a = 0; a < 3; ++a) {
            double pa = M[4 * a + 3] + t * d[a];
            double g = (pa - c->bmin[a]) * ((double)c->k / ((double)c->bmax[a] - (double)c->bmin[a]));
            if (!(g >= 0.0 && g < c->k)) inside = 0;
            double fr = fabs(g - floor(g + 0.5));
            if (fr < mg) mg = fr;
            ix[a] = (int64_t)floor(g);
        }
        cells[i] = inside ? (int32_t)((ix[2] * c->k + ix[1]) * c->k + ix[0]) : -1;
        margin[i] = mg;
    }
}

/* ------------------------------------------------------------ F_pos / F_dir MLPs */
/* Positional encoding gamma(x) = [sin(2^j pi x), cos(2^j pi x)]_{j=0..L-1} per
 * input coordinate, coordinate-major, sin before cos (no raw input), zero
 * padded to n_out columns. */
void orc_posenc(int64_t n, int n_in, int L, const double *x, int n_out, double *out) {
    const double pi = 3.14159265358979323846264338327950288;
    for (int64_t r = 0; r < n; ++r) {
        double *o = out + r * n_out;
        int col = 0;
        for (int a = 0; a < n_in; ++a)
            for (int j = 0; j < L; ++j) {
                double v = ldexp(pi, j) * x[r * n_in + a];
                o[col++] = sin(v);
                o[col++] = cos(v);
            }
        for (; col < n_out; ++col) o[col] = 0.0;
    }
}

/* Rounding of an activation as a bf16 tensor-core chain stores it: to binary32
 * first (round to nearest even), then to bfloat16 (8 exponent bits, 7 fraction
 * bits; round to nearest even on the 16 dropped bits). Infinities and NaN pass
 * through unchanged. */
double orc_round_bf16(double v) {
    float f = (float)v;
    if (isnan(f) || isinf(f)) return f;
    uint32_t u;
    memcpy(&u, &f, 4);
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

/* Dense MLP, one point at a time: h_{i+1} = relu(W_i h_i + b_i) for hidden
 * layers, linear last layer. W_i is [out][in] row-major. round_mode 1 rounds
 * the network input and every hidden activation to bf16 (as a bf16 tensor-core
 * chain stores them between layers); 0 keeps FP64 throughout. */
typedef struct {
    int n_layers;
    const int32_t *dims; /* n_layers + 1 */
    const double *const *W;
    const double *const *b;
    int round_mode;
    int64_t n;
    const double *in;
    double *out;
    int tid, nth;
} mlp_job;

static void *mlp_worker(void *arg) {
    mlp_job *J = (mlp_job *)arg;
    int maxw = 0;
    for (int i = 0; i <= J->n_layers; ++i)
        if (J->dims[i] > maxw) maxw = J->dims[i];
    double *h = (double *)malloc(sizeof(double) * (size_t)maxw * 2);
    double *g = h + maxw;
    for (int64_t r = J->tid; r < J->n; r += J->nth) {
        int din = J->dims[0];
        for (int j = 0; j < din; ++j) h[j] = J->round_mode ? orc_round_bf16(J->in[r * din + j]) : J->in[r * din + j];
        for (int L = 0; L < J->n_layers; ++L) {
            int di = J->dims[L], dout = J->dims[L + 1];
            for (int o = 0; o < dout; ++o) {
                double acc = J->b[L][o];
                const double *w = J->W[L] + (int64_t)o * di;
                for (int i = 0; i < di; ++i) acc += w[i] * h[i];
                if (L + 1 < J->n_layers) {
                    acc = acc > 0.0 ? acc : 0.0;
                    if (J->round_mode) acc = orc_round_bf16(acc);
                }
                g[o] = acc;
            }
            double *tmp = h; h = g; g = tmp;
        }
        int dl = J->dims[J->n_layers];
        for (int o = 0; o < dl; ++o) J->out[r * dl + o] = h[o];
    }
    free(h < g ? h : g);
    return NULL;
}

int orc_mlp_forward(int n_layers, const int32_t *dims, const double *const *W, const double *const *b,
                    int round_mode, int64_t n, const double *in, double *out, int nthreads) {
    if (n_layers < 1 || nthreads < 1) return -1;
    mlp_job *jobs = (mlp_job *)malloc(sizeof(mlp_job) * (size_t)nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        mlp_job J = {n_layers, dims, W, b, round_mode, n, in, out, t, nthreads};
        jobs[t] = J;
        pthread_create(&th[t], NULL, mlp_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th);
    return 0;
}
