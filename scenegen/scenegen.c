/*
 * scenegen.c -- seeded procedural scene fields evaluated on a grid.
 *
 * This is the input generator shared by the renderer's tests/benchmarks and
 * by the oracle. It holds none of the rendering method's arithmetic: it only
 * evaluates a procedural density field (spheres and thin axis-aligned box
 * shells) and a procedural deep-radiance field (sums of sinusoids) at the
 * grid sample points it is given, in FP64, and rounds the result to FP32.
 *
 * Field definitions (all FP64):
 *   sigma(x) = sigma_val if x lies strictly inside any sphere
 *              (|x-c|^2 < r^2) or inside any shell (strictly inside the outer
 *              box |x_a-c_a| < h_a for all axes, and not strictly inside the
 *              inner box |x_a-c_a| < h_a - thick for all axes); else 0.
 *   chan_c(x) = sum_t a_{c,t} * sin(2*pi*(f_{c,t} . x) + phase_{c,t}).
 *
 * The grid fill evaluates sin(2*pi*f.x + phase) through separable complex
 * exponentials: exp(i*phase) * E_x[f_x] * E_y[f_y] * E_z[f_z] with per-axis
 * tables E_a[f][j] = exp(i*2*pi*f*a_j). Build with -ffp-contract=off so that
 * the rounding sequence is the same on every host.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SG_FMAX 2 /* integer frequencies lie in [-SG_FMAX, SG_FMAX] */
#define SG_NF (2 * SG_FMAX + 1)

typedef struct {
    int k;
    int64_t z0, nz;
    const double *xs, *ys, *zs; /* per-axis sample coordinates, length k */
    int n_sph;
    const double *sph; /* [n_sph][4] cx,cy,cz,r */
    int n_shell;
    const double *shell; /* [n_shell][6] cx,cy,cz,hx,hy,hz */
    double thick, sigma_val;
    int n_ch, n_terms;
    const double *amp;   /* [n_ch*n_terms] */
    const int32_t *freq; /* [n_ch*n_terms][3] */
    const double *phase; /* [n_ch*n_terms] */
    float *sigma_out;    /* [nz*k*k] */
    float *chan_out;     /* [nz*k*k][n_ch] (may be NULL) */
    /* per-axis complex tables: [SG_NF][k] re/im */
    double *ex_re, *ex_im, *ey_re, *ey_im, *ez_re, *ez_im;
    int nthreads, tid;
} sg_job;

static int inside_density(const sg_job *J, double x, double y, double z) {
    for (int s = 0; s < J->n_sph; ++s) {
        const double *S = J->sph + 4 * s;
        double dx = x - S[0], dy = y - S[1], dz = z - S[2];
        if (dx * dx + dy * dy + dz * dz < S[3] * S[3]) return 1;
    }
    for (int s = 0; s < J->n_shell; ++s) {
        const double *B = J->shell + 6 * s;
        double ax = fabs(x - B[0]), ay = fabs(y - B[1]), az = fabs(z - B[2]);
        int in_outer = ax < B[3] && ay < B[4] && az < B[5];
        int in_inner = ax < B[3] - J->thick && ay < B[4] - J->thick && az < B[5] - J->thick;
        if (in_outer && !in_inner) return 1;
    }
    return 0;
}

static void *sg_worker(void *arg) {
    const sg_job *J = (const sg_job *)arg;
    const int k = J->k;
    const int nterm_all = J->n_ch * J->n_terms;
    double *pre_re = NULL, *pre_im = NULL;
    if (J->chan_out) {
        pre_re = (double *)malloc(sizeof(double) * (size_t)nterm_all);
        pre_im = (double *)malloc(sizeof(double) * (size_t)nterm_all);
    }
    const int64_t rows = J->nz * (int64_t)k;
    for (int64_t row = J->tid; row < rows; row += J->nthreads) {
        int64_t zl = row / k;
        int y = (int)(row % k);
        int64_t zg = J->z0 + zl;
        double yv = J->ys[y], zv = J->zs[zg];
        if (J->chan_out) {
            for (int t = 0; t < nterm_all; ++t) {
                const int32_t *f = J->freq + 3 * t;
                double pr = cos(J->phase[t]), pi = sin(J->phase[t]);
                double yr = J->ey_re[(f[1] + SG_FMAX) * k + y], yi = J->ey_im[(f[1] + SG_FMAX) * k + y];
                double zr = J->ez_re[(f[2] + SG_FMAX) * (int64_t)k + zg], zi = J->ez_im[(f[2] + SG_FMAX) * (int64_t)k + zg];
                double ar = pr * yr - pi * yi, ai = pr * yi + pi * yr;
                pre_re[t] = ar * zr - ai * zi;
                pre_im[t] = ar * zi + ai * zr;
            }
        }
        for (int x = 0; x < k; ++x) {
            int64_t cell = row * k + x;
            double xv = J->xs[x];
            J->sigma_out[cell] = inside_density(J, xv, yv, zv) ? (float)J->sigma_val : 0.0f;
            if (J->chan_out) {
                float *out = J->chan_out + cell * J->n_ch;
                for (int c = 0; c < J->n_ch; ++c) {
                    double acc = 0.0;
                    for (int m = 0; m < J->n_terms; ++m) {
                        int t = c * J->n_terms + m;
                        int fx = J->freq[3 * t];
                        double er = J->ex_re[(fx + SG_FMAX) * k + x], ei = J->ex_im[(fx + SG_FMAX) * k + x];
                        /* Im(pre * E_x) */
                        double im = pre_re[t] * ei + pre_im[t] * er;
                        acc += J->amp[t] * im;
                    }
                    out[c] = (float)acc;
                }
            }
        }
    }
    free(pre_re);
    free(pre_im);
    return NULL;
}

static void axis_table(int k, const double *a, double *re, double *im) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int f = -SG_FMAX; f <= SG_FMAX; ++f)
        for (int j = 0; j < k; ++j) {
            double ang = two_pi * (double)f * a[j];
            re[(f + SG_FMAX) * k + j] = cos(ang);
            im[(f + SG_FMAX) * k + j] = sin(ang);
        }
}

/* Fill z-slab [z0, z0+nz) of a k^3 grid. Returns 0 on success, -1 on bad
 * arguments or allocation failure. chan_out may be NULL (density only). */
int sg_fill_grid(int k, const double *xs, const double *ys, const double *zs, int64_t z0, int64_t nz,
                 int n_sph, const double *sph, int n_shell, const double *shell, double thick,
                 double sigma_val, int n_ch, int n_terms, const double *amp, const int32_t *freq,
                 const double *phase, float *sigma_out, float *chan_out, int nthreads) {
    if (k <= 0 || z0 < 0 || nz < 0 || z0 + nz > k || nthreads <= 0) return -1;
    for (int t = 0; t < n_ch * n_terms; ++t)
        for (int a = 0; a < 3; ++a)
            if (freq[3 * t + a] < -SG_FMAX || freq[3 * t + a] > SG_FMAX) return -1;
    size_t tab = (size_t)SG_NF * (size_t)k;
    double *buf = (double *)malloc(sizeof(double) * tab * 6);
    if (!buf) return -1;
    sg_job base;
    memset(&base, 0, sizeof(base));
    base.k = k; base.z0 = z0; base.nz = nz; base.xs = xs; base.ys = ys; base.zs = zs;
    base.n_sph = n_sph; base.sph = sph; base.n_shell = n_shell; base.shell = shell;
    base.thick = thick; base.sigma_val = sigma_val; base.n_ch = n_ch; base.n_terms = n_terms;
    base.amp = amp; base.freq = freq; base.phase = phase;
    base.sigma_out = sigma_out; base.chan_out = chan_out;
    base.ex_re = buf; base.ex_im = buf + tab; base.ey_re = buf + 2 * tab; base.ey_im = buf + 3 * tab;
    base.ez_re = buf + 4 * tab; base.ez_im = buf + 5 * tab;
    axis_table(k, xs, base.ex_re, base.ex_im);
    axis_table(k, ys, base.ey_re, base.ey_im);
    axis_table(k, zs, base.ez_re, base.ez_im);
    base.nthreads = nthreads;
    sg_job *jobs = (sg_job *)malloc(sizeof(sg_job) * (size_t)nthreads);
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    if (!jobs || !th) { free(buf); free(jobs); free(th); return -1; }
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = base;
        jobs[t].tid = t;
        pthread_create(&th[t], NULL, sg_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(jobs); free(th); free(buf);
    return 0;
}

/* FP64 field at arbitrary points (direct sin, no tables): used where the
 * unquantised field is wanted at a few points. out_chan may be NULL. */
int sg_eval_points(int64_t n, const double *xyz, int n_sph, const double *sph, int n_shell,
                   const double *shell, double thick, double sigma_val, int n_ch, int n_terms,
                   const double *amp, const int32_t *freq, const double *phase, double *out_sigma,
                   double *out_chan) {
    const double two_pi = 6.283185307179586476925286766559;
    sg_job J;
    memset(&J, 0, sizeof(J));
    J.n_sph = n_sph; J.sph = sph; J.n_shell = n_shell; J.shell = shell; J.thick = thick;
    for (int64_t i = 0; i < n; ++i) {
        double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        out_sigma[i] = inside_density(&J, x, y, z) ? sigma_val : 0.0;
        if (!out_chan) continue;
        for (int c = 0; c < n_ch; ++c) {
            double acc = 0.0;
            for (int m = 0; m < n_terms; ++m) {
                int t = c * n_terms + m;
                const int32_t *f = freq + 3 * t;
                acc += amp[t] * sin(two_pi * (f[0] * x + f[1] * y + f[2] * z) + phase[t]);
            }
            out_chan[i * n_ch + c] = acc;
        }
    }
    return 0;
}
