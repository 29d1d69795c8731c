/*
 * FP64 CPU oracle for the one-way coupled Eulerian-Lagrangian method of
 * "A coupled Eulerian-Lagrangian approach for fluid and particle dynamics"
 * (arxiv 2607.17836).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  It
 * shares no code, header, table or constant with the CUDA library, and only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  Nothing in the product path calls it.
 *
 * Everything is double precision.  Every array is row-major [j][i]
 * (y slow, x fast) on the periodic square [0, 2*pi)^2 with nodes x_i = i*dx.
 *
 * Contents, in the paper's order:
 *   - a radix-2 complex FFT (its own; no library), Sec. 3.1 ("forward and
 *     inverse fast Fourier transforms are performed at each timestep");
 *   - the pseudospectral vorticity solver, Sec. 3.1, Eqs. 1, 4-10;
 *   - the three spatial interpolants, Sec. 3.4, Eqs. 15-22, plus the
 *     periodic cubic-spline prefilter (physical-space cyclic tridiagonal
 *     solve) used for interpolating B-spline coefficients;
 *   - linear temporal interpolation, Eqs. 23-24;
 *   - RK4 for tracers (Eq. 12) and Stokes-drag inertial particles
 *     (Eqs. 3, 13, 14), in unwrapped FP64 coordinates with periodic
 *     evaluation (Sec. 3.2, Algorithm 1).
 *
 * OpenMP (when compiled with -fopenmp) only splits independent loops over
 * rows, columns and particles; it changes no arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define TWO_PI 6.283185307179586476925286766559

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------
 * Radix-2 complex FFT.
 *   X_k = sum_j x_j exp(sign * 2 pi i j k / n)
 * sign = -1 is the forward transform, sign = +1 the unnormalised inverse.
 * Iterative Cooley-Tukey: bit-reversal permutation, then log2(n) butterfly
 * stages.  tw holds exp(sign * 2 pi i k / n) for k < n/2.
 * --------------------------------------------------------------------- */
static void fft_twiddles(int n, int sign, double *twr, double *twi) {
    for (int k = 0; k < n / 2; k++) {
        double a = sign * TWO_PI * (double)k / (double)n;
        twr[k] = cos(a);
        twi[k] = sin(a);
    }
}

static void fft_core(double *re, double *im, int n, const double *twr,
                     const double *twi) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = re[i]; re[i] = re[j]; re[j] = t;
            t = im[i]; im[i] = im[j]; im[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2, step = n / len;
        for (int s = 0; s < n; s += len) {
            for (int k = 0; k < half; k++) {
                double wr = twr[k * step], wi = twi[k * step];
                int a = s + k, b = s + k + half;
                double br = re[b] * wr - im[b] * wi;
                double bi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - br; im[b] = im[a] - bi;
                re[a] = re[a] + br; im[a] = im[a] + bi;
            }
        }
    }
}

/* One 1-D transform of length n (power of two). */
void orc_fft1(double *re, double *im, int n, int sign) {
    double *twr = malloc(sizeof(double) * (n / 2 + 1));
    double *twi = malloc(sizeof(double) * (n / 2 + 1));
    fft_twiddles(n, sign, twr, twi);
    fft_core(re, im, n, twr, twi);
    free(twr);
    free(twi);
}

/* 2-D transform of an n x n row-major array: every row, then every column. */
void orc_fft2(double *re, double *im, int n, int sign) {
    double *twr = malloc(sizeof(double) * (n / 2 + 1));
    double *twi = malloc(sizeof(double) * (n / 2 + 1));
    fft_twiddles(n, sign, twr, twi);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; j++) fft_core(re + (size_t)j * n, im + (size_t)j * n, n, twr, twi);
#pragma omp parallel
    {
        double *cr = malloc(sizeof(double) * n);
        double *ci = malloc(sizeof(double) * n);
#pragma omp for schedule(static)
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < n; j++) { cr[j] = re[(size_t)j * n + i]; ci[j] = im[(size_t)j * n + i]; }
            fft_core(cr, ci, n, twr, twi);
            for (int j = 0; j < n; j++) { re[(size_t)j * n + i] = cr[j]; im[(size_t)j * n + i] = ci[j]; }
        }
        free(cr);
        free(ci);
    }
    free(twr);
    free(twi);
}

/* ------------------------------------------------------------------------
 * Pseudospectral vorticity solver, Sec. 3.1.
 * The oracle keeps the full n x n complex spectrum (no half-spectrum
 * storage), indexed like the physical array: [jy][ix].
 * Wavenumber of index m: m for m < n/2, m - n otherwise (so n/2 -> -n/2).
 * --------------------------------------------------------------------- */
typedef struct {
    int n;
    double nu, dt;
    int ab2_mode;     /* 0: viscous integrating factor, 1: explicit AB2 (Eq. 10) */
    int64_t step;
    double *wr, *wi;  /* omega-hat */
    double *hr, *hi;  /* AB2 history: N-hat^{n-1} (mode 0) or R^{n-1} (mode 1) */
    double *t0r, *t0i, *t1r, *t1i, *t2r, *t2i, *t3r, *t3i; /* scratch */
} orc_flow;

static double wavenum(int m, int n) { return (m < n / 2) ? (double)m : (double)(m - n); }

/* Derivative multiplier: the wavenumber, with the unpaired Nyquist mode
 * (k = -n/2) given a zero derivative. */
static double dwavenum(int m, int n) { return (m == n / 2) ? 0.0 : wavenum(m, n); }

/* 2/3 rule (Sec. 3.1): the highest third of the resolved modes is zeroed.
 * Read as a square mask: keep mode k iff 3|kx| < n and 3|ky| < n. */
static int kept_two_thirds(int ix, int jy, int n) {
    double kx = fabs(wavenum(ix, n)), ky = fabs(wavenum(jy, n));
    return (3.0 * kx < (double)n) && (3.0 * ky < (double)n);
}

orc_flow *orc_flow_new(int n, double nu, double dt, int ab2_mode, const double *omega0) {
    size_t nn = (size_t)n * n;
    orc_flow *f = calloc(1, sizeof(orc_flow));
    f->n = n; f->nu = nu; f->dt = dt; f->ab2_mode = ab2_mode; f->step = 0;
    double **bufs[] = {&f->wr, &f->wi, &f->hr, &f->hi, &f->t0r, &f->t0i, &f->t1r,
                       &f->t1i, &f->t2r, &f->t2i, &f->t3r, &f->t3i};
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); b++) *bufs[b] = calloc(nn, sizeof(double));
    /* Initial condition: transform, remove the mean (psi-hat(0) = 0 makes the
     * k = 0 vorticity mode inert) and apply the 2/3 projection once. */
    memcpy(f->wr, omega0, nn * sizeof(double));
    orc_fft2(f->wr, f->wi, n, -1);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            size_t q = (size_t)j * n + i;
            if ((i == 0 && j == 0) || !kept_two_thirds(i, j, n)) { f->wr[q] = 0.0; f->wi[q] = 0.0; }
        }
    return f;
}

void orc_flow_free(orc_flow *f) {
    if (!f) return;
    double *bufs[] = {f->wr, f->wi, f->hr, f->hi, f->t0r, f->t0i, f->t1r,
                      f->t1i, f->t2r, f->t2i, f->t3r, f->t3i};
    for (size_t b = 0; b < sizeof(bufs) / sizeof(bufs[0]); b++) free(bufs[b]);
    free(f);
}

int64_t orc_flow_step_count(const orc_flow *f) { return f->step; }

void orc_flow_get_spectrum(const orc_flow *f, double *re, double *im) {
    size_t nn = (size_t)f->n * f->n;
    memcpy(re, f->wr, nn * sizeof(double));
    memcpy(im, f->wi, nn * sizeof(double));
}

/* Inverse transform of a spectrum into its (real) physical field, with the
 * 1/(NxNy) normalisation of Sec. 3.1. */
static void to_physical(int n, double *re, double *im, double *out) {
    size_t nn = (size_t)n * n;
    orc_fft2(re, im, n, +1);
    double s = 1.0 / (double)nn;
    for (size_t q = 0; q < nn; q++) out[q] = re[q] * s;
}

/* Physical velocity (Eqs. 5, 6), vorticity and vorticity gradient (Eq. 4)
 * of the current spectrum.  Any output pointer may be NULL. */
void orc_flow_fields(orc_flow *f, double *u, double *v, double *w, double *wx, double *wy) {
    int n = f->n;
    size_t nn = (size_t)n * n;
    double *outs[5] = {u, v, w, wx, wy};
    for (int which = 0; which < 5; which++) {
        if (!outs[which]) continue;
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                size_t q = (size_t)j * n + i;
                double kx = wavenum(i, n), ky = wavenum(j, n);
                double dkx = dwavenum(i, n), dky = dwavenum(j, n);
                double k2 = kx * kx + ky * ky;
                double ar = f->wr[q], ai = f->wi[q];
                /* Eq. 5: psi-hat = omega-hat / |k|^2, psi-hat(0) = 0. */
                double pr = (k2 > 0.0) ? ar / k2 : 0.0, pi = (k2 > 0.0) ? ai / k2 : 0.0;
                double rr, ri;
                switch (which) {
                case 0: rr = -dky * pi; ri = dky * pr; break;  /* u-hat = i ky psi-hat  (Eq. 6) */
                case 1: rr = dkx * pi; ri = -dkx * pr; break;  /* v-hat = -i kx psi-hat (Eq. 6) */
                case 2: rr = ar; ri = ai; break;               /* omega-hat */
                case 3: rr = -dkx * ai; ri = dkx * ar; break;  /* i kx omega-hat (Eq. 4) */
                default: rr = -dky * ai; ri = dky * ar; break; /* i ky omega-hat (Eq. 4) */
                }
                f->t0r[q] = rr;
                f->t0i[q] = ri;
            }
        to_physical(n, f->t0r, f->t0i, outs[which]);
    }
    (void)nn;
}

/* Physical streamfunction psi of the current spectrum (Eq. 5). */
void orc_flow_psi(orc_flow *f, double *psi) {
    int n = f->n;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            size_t q = (size_t)j * n + i;
            double kx = wavenum(i, n), ky = wavenum(j, n), k2 = kx * kx + ky * ky;
            f->t0r[q] = k2 > 0.0 ? f->wr[q] / k2 : 0.0;
            f->t0i[q] = k2 > 0.0 ? f->wi[q] / k2 : 0.0;
        }
    to_physical(n, f->t0r, f->t0i, psi);
}

/* Dealiased spectral nonlinear term N-hat = FFT(u d(omega)/dx + v d(omega)/dy)
 * (Eqs. 7, 8), with the 2/3 rule applied, into (nr, ni). */
static void nonlinear_hat(orc_flow *f, double *nr, double *ni) {
    int n = f->n;
    size_t nn = (size_t)n * n;
    double *u = f->t1r, *v = f->t1i, *wx = f->t2r, *wy = f->t2i;
    orc_flow_fields(f, u, v, NULL, wx, wy);
    for (size_t q = 0; q < nn; q++) {
        nr[q] = u[q] * wx[q] + v[q] * wy[q];
        ni[q] = 0.0;
    }
    orc_fft2(nr, ni, n, -1);
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++)
            if (!kept_two_thirds(i, j, n)) { nr[(size_t)j * n + i] = 0.0; ni[(size_t)j * n + i] = 0.0; }
}

/* Physical-space nonlinear term u d(omega)/dx + v d(omega)/dy (Eq. 7) of
 * the current state, for tests. */
void orc_flow_nonlinear(orc_flow *f, double *out) {
    int n = f->n;
    size_t nn = (size_t)n * n;
    double *u = malloc(nn * sizeof(double)), *v = malloc(nn * sizeof(double));
    double *wx = malloc(nn * sizeof(double)), *wy = malloc(nn * sizeof(double));
    orc_flow_fields(f, u, v, NULL, wx, wy);
    for (size_t q = 0; q < nn; q++) out[q] = u[q] * wx[q] + v[q] * wy[q];
    free(u); free(v); free(wx); free(wy);
}

/* Advance omega-hat by nsteps AB2 steps of size dt (Sec. 3.1).
 * Eq. 9: d omega-hat/dt = -N-hat - nu |k|^2 omega-hat.
 * ab2_mode 1 is Eq. 10 as printed, with R = right-hand side of Eq. 9.
 * ab2_mode 0 treats the viscous term with the integrating factor
 * E = exp(-nu |k|^2 dt) and AB2 on the rest:
 *   omega^{n+1} = E omega^n - dt (3/2 E N^n - 1/2 E^2 N^{n-1}).
 * The first step of either mode is forward Euler (its Eq. 10 needs a
 * history term that does not exist yet). */
void orc_flow_step(orc_flow *f, int nsteps) {
    int n = f->n;
    double *nr = f->t3r, *ni = f->t3i;
    for (int s = 0; s < nsteps; s++) {
        nonlinear_hat(f, nr, ni);
        int first = (f->step == 0);
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                size_t q = (size_t)j * n + i;
                double kx = wavenum(i, n), ky = wavenum(j, n);
                double k2 = kx * kx + ky * ky;
                if (f->ab2_mode == 0) {
                    double E = exp(-f->nu * k2 * f->dt);
                    double ar, ai;
                    if (first) {
                        ar = E * (f->wr[q] - f->dt * nr[q]);
                        ai = E * (f->wi[q] - f->dt * ni[q]);
                    } else {
                        ar = E * f->wr[q] - f->dt * (1.5 * E * nr[q] - 0.5 * E * E * f->hr[q]);
                        ai = E * f->wi[q] - f->dt * (1.5 * E * ni[q] - 0.5 * E * E * f->hi[q]);
                    }
                    f->wr[q] = ar; f->wi[q] = ai;
                    f->hr[q] = nr[q]; f->hi[q] = ni[q];
                } else {
                    double rr = -nr[q] - f->nu * k2 * f->wr[q];
                    double ri = -ni[q] - f->nu * k2 * f->wi[q];
                    if (first) {
                        f->wr[q] += f->dt * rr;
                        f->wi[q] += f->dt * ri;
                    } else {
                        f->wr[q] += f->dt * (1.5 * rr - 0.5 * f->hr[q]);
                        f->wi[q] += f->dt * (1.5 * ri - 0.5 * f->hi[q]);
                    }
                    f->hr[q] = rr; f->hi[q] = ri;
                }
            }
        f->step++;
    }
}

/* Energy, enstrophy and palinstrophy of the current state as plain means of
 * the physical fields: E = 1/2 <u^2+v^2>, Z = 1/2 <omega^2>,
 * P = 1/2 <|grad omega|^2>. */
void orc_flow_diagnostics(orc_flow *f, double *out3) {
    int n = f->n;
    size_t nn = (size_t)n * n;
    double *u = malloc(nn * sizeof(double)), *v = malloc(nn * sizeof(double));
    double *w = malloc(nn * sizeof(double)), *wx = malloc(nn * sizeof(double));
    double *wy = malloc(nn * sizeof(double));
    orc_flow_fields(f, u, v, w, wx, wy);
    double se = 0, sz = 0, sp = 0;
    for (size_t q = 0; q < nn; q++) {
        se += u[q] * u[q] + v[q] * v[q];
        sz += w[q] * w[q];
        sp += wx[q] * wx[q] + wy[q] * wy[q];
    }
    out3[0] = 0.5 * se / (double)nn;
    out3[1] = 0.5 * sz / (double)nn;
    out3[2] = 0.5 * sp / (double)nn;
    free(u); free(v); free(w); free(wx); free(wy);
}

/* ------------------------------------------------------------------------
 * Interpolation, Sec. 3.4.
 * --------------------------------------------------------------------- */
enum { ORC_BILINEAR = 0, ORC_CATMULL_ROM = 1, ORC_BSPLINE = 2 };

static int pmod(int a, int n) { int r = a % n; return r < 0 ? r + n : r; }

/* Cell containing coordinate x (any real) and the normalised offset in it
 * (Eqs. 15, 17, 20).  x is first mapped periodically onto [0, 2 pi); a
 * point on a node belongs to the cell on its right. */
static void locate(double x, int n, int *cell, double *off) {
    double xw = x - TWO_PI * floor(x / TWO_PI);
    double s = xw * (double)n / TWO_PI;
    double c = floor(s);
    *off = s - c;
    *cell = pmod((int)c, n);
}

/* Catmull-Rom weights, Eq. 19: nodes i-1, i, i+1, i+2. */
static void w_catmull_rom(double s, double w[4]) {
    double s2 = s * s, s3 = s2 * s;
    w[0] = -0.5 * s + s2 - 0.5 * s3;
    w[1] = 1.0 - 2.5 * s2 + 1.5 * s3;
    w[2] = 0.5 * s + 2.0 * s2 - 1.5 * s3;
    w[3] = -0.5 * s2 + 0.5 * s3;
}

/* Cubic B-spline weights, Eq. 22: nodes i-1, i, i+1, i+2. */
static void w_bspline(double s, double w[4]) {
    double s2 = s * s, s3 = s2 * s;
    w[0] = (1.0 - s) * (1.0 - s) * (1.0 - s) / 6.0;
    w[1] = (3.0 * s3 - 6.0 * s2 + 4.0) / 6.0;
    w[2] = (-3.0 * s3 + 3.0 * s2 + 3.0 * s + 1.0) / 6.0;
    w[3] = s3 / 6.0;
}

/* Value at (x, y) of the periodic grid function f by the given scheme.
 * Bilinear is Eq. 16.  Catmull-Rom (Eq. 18) and B-spline (Eq. 21) use the
 * 4 x 4 stencil f_{i+m-2, j+n-2}, m, n = 1..4, wrapped periodically.
 * For the B-spline scheme f holds whatever the stencil is to weight: raw
 * samples, or coefficients from orc_bspline_prefilter. */
double orc_interp(int n, const double *f, int scheme, double x, double y) {
    int i, j;
    double xi, eta;
    locate(x, n, &i, &xi);
    locate(y, n, &j, &eta);
    if (scheme == ORC_BILINEAR) {
        int i1 = pmod(i + 1, n), j1 = pmod(j + 1, n);
        return (1.0 - xi) * (1.0 - eta) * f[(size_t)j * n + i] + xi * (1.0 - eta) * f[(size_t)j * n + i1] +
               (1.0 - xi) * eta * f[(size_t)j1 * n + i] + xi * eta * f[(size_t)j1 * n + i1];
    }
    double wx[4], wy[4];
    if (scheme == ORC_CATMULL_ROM) { w_catmull_rom(xi, wx); w_catmull_rom(eta, wy); }
    else { w_bspline(xi, wx); w_bspline(eta, wy); }
    double acc = 0.0;
    for (int b = 0; b < 4; b++) {
        int jj = pmod(j + b - 1, n);
        for (int a = 0; a < 4; a++) {
            int ii = pmod(i + a - 1, n);
            acc += wx[a] * wy[b] * f[(size_t)jj * n + ii];
        }
    }
    return acc;
}

void orc_interp_many(int n, const double *f, int scheme, int64_t np, const double *x,
                     const double *y, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) out[p] = orc_interp(n, f, scheme, x[p], y[p]);
}

/* Periodic tridiagonal solve of (c_{i-1} + 4 c_i + c_{i+1}) / 6 = d_i for
 * one line of length n (in place in d).  Sherman-Morrison: the periodic
 * matrix is a tridiagonal T plus a rank-one corner correction u v^T with
 * u = (g, 0, .., 0, a)^T, v = (1, 0, .., 0, b/g)^T, a = b = 1/6, g = -4/6;
 * solve T y = d and T z = u by elimination, then c = y - (v.y)/(1+v.z) z. */
static void cyclic_tridiag_line(int n, double *d, double *y, double *z, double *cp) {
    const double lo = 1.0 / 6.0, di = 4.0 / 6.0, up = 1.0 / 6.0;
    const double a = lo, b = up, g = -di;
    /* T: diagonal di except T00 = di - g and T(n-1,n-1) = di - a b / g. */
    for (int pass = 0; pass < 2; pass++) {
        double *rhs = pass == 0 ? y : z;
        for (int i = 0; i < n; i++) rhs[i] = pass == 0 ? d[i] : 0.0;
        if (pass == 1) { z[0] = g; z[n - 1] = a; }
        /* forward elimination (Thomas) */
        double diag0 = di - g;
        cp[0] = up / diag0;
        rhs[0] = rhs[0] / diag0;
        for (int i = 1; i < n; i++) {
            double dii = (i == n - 1) ? di - a * b / g : di;
            double m = dii - lo * cp[i - 1];
            cp[i] = (i < n - 1) ? up / m : 0.0;
            rhs[i] = (rhs[i] - lo * rhs[i - 1]) / m;
        }
        for (int i = n - 2; i >= 0; i--) rhs[i] -= cp[i] * rhs[i + 1];
    }
    double vy = y[0] + (b / g) * y[n - 1];
    double vz = z[0] + (b / g) * z[n - 1];
    double fac = vy / (1.0 + vz);
    for (int i = 0; i < n; i++) d[i] = y[i] - fac * z[i];
}

/* In-place cubic-spline prefilter of an n x n periodic grid: the solve along
 * x for every row, then along y for every column.  The result c makes the
 * B-spline stencil of Eq. 21 reproduce the samples at every node. */
void orc_bspline_prefilter(int n, double *f) {
#pragma omp parallel
    {
        double *line = malloc(sizeof(double) * n), *y = malloc(sizeof(double) * n);
        double *z = malloc(sizeof(double) * n), *cp = malloc(sizeof(double) * n);
#pragma omp for schedule(static)
        for (int j = 0; j < n; j++) {
            memcpy(line, f + (size_t)j * n, sizeof(double) * n);
            cyclic_tridiag_line(n, line, y, z, cp);
            memcpy(f + (size_t)j * n, line, sizeof(double) * n);
        }
#pragma omp barrier
#pragma omp for schedule(static)
        for (int i = 0; i < n; i++) {
            for (int j = 0; j < n; j++) line[j] = f[(size_t)j * n + i];
            cyclic_tridiag_line(n, line, y, z, cp);
            for (int j = 0; j < n; j++) f[(size_t)j * n + i] = line[j];
        }
        free(line); free(y); free(z); free(cp);
    }
}

/* ------------------------------------------------------------------------
 * Particles, Secs. 3.2, 3.3 and Algorithm 1.
 * Fluid velocity at a stage: spatial interpolation of both time levels at
 * the periodically mapped stage position, then linear blending in time
 * (Eq. 23) with theta = 0, 1/2, 1/2, 1 for the four stages.
 * --------------------------------------------------------------------- */
typedef struct {
    int n, scheme;
    const double *un, *vn, *un1, *vn1;
} orc_vel;

static void stage_velocity(const orc_vel *c, double x, double y, double theta, double *u, double *v) {
    double a0 = orc_interp(c->n, c->un, c->scheme, x, y);
    double b0 = orc_interp(c->n, c->vn, c->scheme, x, y);
    double a1 = orc_interp(c->n, c->un1, c->scheme, x, y);
    double b1 = orc_interp(c->n, c->vn1, c->scheme, x, y);
    *u = (1.0 - theta) * a0 + theta * a1;
    *v = (1.0 - theta) * b0 + theta * b1;
}

/* Tracer velocity from the streamfunction, Sec. 3.2 and Eq. 11: psi at the
 * four points (x +- dx, y), (x, y +- dy) (mapped periodically inside
 * orc_interp), each interpolated in space by the scheme and blended linearly
 * in time; u = (psi_N - psi_S) / 2dy, v = -(psi_E - psi_W) / 2dx. */
static void psi_velocity(int n, int scheme, const double *pn, const double *pn1, double x,
                         double y, double theta, double *u, double *v) {
    double d = TWO_PI / (double)n;
    double px[4] = {x, x, x + d, x - d}, py[4] = {y + d, y - d, y, y};
    double val[4];
    for (int k = 0; k < 4; k++) {
        double a = orc_interp(n, pn, scheme, px[k], py[k]);
        double b = orc_interp(n, pn1, scheme, px[k], py[k]);
        val[k] = (1.0 - theta) * a + theta * b;
    }
    *u = (val[0] - val[1]) / (2.0 * d);
    *v = -(val[2] - val[3]) / (2.0 * d);
}

void orc_psi_velocity_many(int n, int scheme, const double *psi, int64_t np, const double *x,
                           const double *y, double *u, double *v) {
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) psi_velocity(n, scheme, psi, psi, x[p], y[p], 0.0, &u[p], &v[p]);
}

/* One RK4 step (Eq. 12) of np tracers whose velocity comes from the
 * streamfunction (levels psin, psin1; coefficients for the B-spline scheme). */
void orc_tracers_rk4_psi(int n, int scheme, double dt, const double *psin, const double *psin1,
                         int64_t np, double *x, double *y) {
    const double theta[4] = {0.0, 0.5, 0.5, 1.0};
    const double frac[4] = {0.0, 0.5, 0.5, 1.0};
    const double wgt[4] = {1.0, 2.0, 2.0, 1.0};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) {
        double x0 = x[p], y0 = y[p], kx = 0.0, ky = 0.0, sx = 0.0, sy = 0.0;
        for (int s = 0; s < 4; s++) {
            psi_velocity(n, scheme, psin, psin1, x0 + frac[s] * dt * kx, y0 + frac[s] * dt * ky,
                         theta[s], &kx, &ky);
            sx += wgt[s] * kx;
            sy += wgt[s] * ky;
        }
        x[p] = x0 + dt / 6.0 * sx;
        y[p] = y0 + dt / 6.0 * sy;
    }
}

/* One RK4 step of length dt for np particles, from time level n (fields
 * un, vn) to n+1 (fields un1, vn1).  Positions x, y are unwrapped.
 * st == 0: tracers, Eq. 2 integrated by Eq. 12 (vx, vy untouched, may be
 * NULL).  st > 0: inertial particles, Eq. 3 with the drag of Eq. 13,
 * integrated jointly in (x, v) by Eq. 14.  For the B-spline scheme the
 * field arrays are the (prefiltered or raw) stencil values. */
void orc_particles_rk4(int n, int scheme, double dt, double st, const double *un,
                       const double *vn, const double *un1, const double *vn1, int64_t np,
                       double *x, double *y, double *vx, double *vy) {
    orc_vel c = {n, scheme, un, vn, un1, vn1};
    const double theta[4] = {0.0, 0.5, 0.5, 1.0};
    const double frac[4] = {0.0, 0.5, 0.5, 1.0};  /* stage position = x + frac * dt * k_prev */
    const double wgt[4] = {1.0, 2.0, 2.0, 1.0};
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; p++) {
        double x0 = x[p], y0 = y[p];
        if (st == 0.0) {
            double kx = 0.0, ky = 0.0, sx = 0.0, sy = 0.0;
            for (int s = 0; s < 4; s++) {
                double xs = x0 + frac[s] * dt * kx, ys = y0 + frac[s] * dt * ky;
                stage_velocity(&c, xs, ys, theta[s], &kx, &ky);
                sx += wgt[s] * kx;
                sy += wgt[s] * ky;
            }
            x[p] = x0 + dt / 6.0 * sx;
            y[p] = y0 + dt / 6.0 * sy;
        } else {
            double u0 = vx[p], v0 = vy[p];
            double kxx = 0.0, kxy = 0.0, kvx = 0.0, kvy = 0.0;
            double sxx = 0.0, sxy = 0.0, svx = 0.0, svy = 0.0;
            for (int s = 0; s < 4; s++) {
                double xs = x0 + frac[s] * dt * kxx, ys = y0 + frac[s] * dt * kxy;
                double us = u0 + frac[s] * dt * kvx, vs = v0 + frac[s] * dt * kvy;
                double fu, fv;
                stage_velocity(&c, xs, ys, theta[s], &fu, &fv);
                kxx = us; kxy = vs;             /* dx/dt = v_p          */
                kvx = (fu - us) / st;           /* dv/dt = (u - v_p)/St */
                kvy = (fv - vs) / st;
                sxx += wgt[s] * kxx; sxy += wgt[s] * kxy;
                svx += wgt[s] * kvx; svy += wgt[s] * kvy;
            }
            x[p] = x0 + dt / 6.0 * sxx;
            y[p] = y0 + dt / 6.0 * sxy;
            vx[p] = u0 + dt / 6.0 * svx;
            vy[p] = v0 + dt / 6.0 * svy;
        }
    }
}
