/*
 * eor_oracle.c — plain FP64 CPU oracle of the excursion-set 21-cm likelihood path
 * (Greig & Mesinger 2015, "21CMMC", arXiv:1501.06576).
 *
 * TEST INFRASTRUCTURE ONLY: see eor_oracle.h for who may load it and what pins it.
 * It shares no code with the CUDA library. Written for clarity, not speed.
 */
#include "eor_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
/* Critical density today, 3 H0^2 / (8 pi G) = 2.775e11 h^2 Msun / Mpc^3. */
#define OR_RHO_CRIT_H2 2.775e11

/* ------------------------------------------------------------------ threads */

static int g_threads = 0;

void or_set_threads(int n) {
    g_threads = n;
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- FFT */

/* Textbook iterative radix-2 Cooley-Tukey; every twiddle taken directly from cos/sin. */
static void fft_pow2(double* a, int n, int sign) {
    for (int i = 1, j = 0; i < n; i++) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = a[2 * i], ti = a[2 * i + 1];
            a[2 * i] = a[2 * j]; a[2 * i + 1] = a[2 * j + 1];
            a[2 * j] = tr; a[2 * j + 1] = ti;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int j = 0; j < half; j++) {
            double ang = sign * 2.0 * OR_PI * (double)j / (double)len;
            double wr = cos(ang), wi = sin(ang);
            for (int i = 0; i < n; i += len) {
                double* u = a + 2 * (i + j);
                double* v = a + 2 * (i + j + half);
                double vr = v[0] * wr - v[1] * wi;
                double vi = v[0] * wi + v[1] * wr;
                v[0] = u[0] - vr; v[1] = u[1] - vi;
                u[0] += vr;       u[1] += vi;
            }
        }
    }
}

/* Direct O(n^2) DFT for lengths that are not powers of two. */
static void dft_direct(double* a, int n, int sign) {
    double* t = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    for (int k = 0; k < n; k++) {
        double sr = 0.0, si = 0.0;
        for (int j = 0; j < n; j++) {
            double ang = sign * 2.0 * OR_PI * (double)(((long long)j * k) % n) / (double)n;
            double c = cos(ang), s = sin(ang);
            sr += a[2 * j] * c - a[2 * j + 1] * s;
            si += a[2 * j] * s + a[2 * j + 1] * c;
        }
        t[2 * k] = sr; t[2 * k + 1] = si;
    }
    memcpy(a, t, sizeof(double) * 2 * (size_t)n);
    free(t);
}

void or_fft1d(double* a, int n, int sign) {
    if (n <= 1) return;
    if ((n & (n - 1)) == 0) fft_pow2(a, n, sign);
    else dft_direct(a, n, sign);
}

/* 3D transform as 1D transforms along z, then y, then x. */
void or_fft3d(double* a, int n, int sign) {
    const long long n2 = (long long)n * n;
    /* z lines are contiguous */
#pragma omp parallel for schedule(static)
    for (long long line = 0; line < n2; line++) or_fft1d(a + 2 * line * n, n, sign);
    /* y lines: stride n */
#pragma omp parallel
    {
        double* buf = (double*)malloc(sizeof(double) * 2 * (size_t)n);
#pragma omp for schedule(static)
        for (long long line = 0; line < n2; line++) {
            long long ix = line / n, iz = line % n;
            for (int iy = 0; iy < n; iy++) {
                long long idx = (ix * n + iy) * n + iz;
                buf[2 * iy] = a[2 * idx]; buf[2 * iy + 1] = a[2 * idx + 1];
            }
            or_fft1d(buf, n, sign);
            for (int iy = 0; iy < n; iy++) {
                long long idx = (ix * n + iy) * n + iz;
                a[2 * idx] = buf[2 * iy]; a[2 * idx + 1] = buf[2 * iy + 1];
            }
        }
        free(buf);
    }
    /* x lines: stride n^2 */
#pragma omp parallel
    {
        double* buf = (double*)malloc(sizeof(double) * 2 * (size_t)n);
#pragma omp for schedule(static)
        for (long long line = 0; line < n2; line++) {
            for (int ix = 0; ix < n; ix++) {
                long long idx = ix * n2 + line;
                buf[2 * ix] = a[2 * idx]; buf[2 * ix + 1] = a[2 * idx + 1];
            }
            or_fft1d(buf, n, sign);
            for (int ix = 0; ix < n; ix++) {
                long long idx = ix * n2 + line;
                a[2 * idx] = buf[2 * ix]; a[2 * idx + 1] = buf[2 * ix + 1];
            }
        }
        free(buf);
    }
}

/* Signed frequency index of grid index i: 0..n/2-1, then -n/2..-1 (Nyquist is -n/2). */
static int freq_index(int i, int n) { return i < n / 2 ? i : i - n; }

/* --------------------------------------------------------------- quadrature */

typedef double (*or_fn)(double x, const void* ctx);

static double simpson_adapt(or_fn f, const void* ctx, double a, double b, double fa, double fm,
                            double fb, double whole, double eps, int depth) {
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = f(lm, ctx), frm = f(rm, ctx);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    if (depth <= 0 || fabs(delta) <= 15.0 * eps) return left + right + delta / 15.0;
    return simpson_adapt(f, ctx, a, m, fa, flm, fm, left, 0.5 * eps, depth - 1) +
           simpson_adapt(f, ctx, m, b, fm, frm, fb, right, 0.5 * eps, depth - 1);
}

/* Adaptive Simpson on [a, b], split into `panels` equal panels, absolute tolerance eps. */
static double integrate(or_fn f, const void* ctx, double a, double b, int panels, double eps) {
    double total = 0.0, h = (b - a) / panels;
    for (int p = 0; p < panels; p++) {
        double lo = a + p * h, hi = lo + h, mid = 0.5 * (lo + hi);
        double flo = f(lo, ctx), fmid = f(mid, ctx), fhi = f(hi, ctx);
        double whole = h / 6.0 * (flo + 4.0 * fmid + fhi);
        total += simpson_adapt(f, ctx, lo, hi, flo, fmid, fhi, whole, eps / panels, 48);
    }
    return total;
}

/* Adaptive Simpson on [a, b] that also stops where a panel's estimate changes by less than
 * rel of itself (so that rounding in a narrow peak cannot drive the recursion to its depth). */
static double simpson_rel(or_fn f, const void* ctx, double a, double b, double fa, double fm, double fb,
                          double whole, double eps, double rel, int depth) {
    double m = 0.5 * (a + b);
    double lm = 0.5 * (a + m), rm = 0.5 * (m + b);
    double flm = f(lm, ctx), frm = f(rm, ctx);
    double left = (m - a) / 6.0 * (fa + 4.0 * flm + fm);
    double right = (b - m) / 6.0 * (fm + 4.0 * frm + fb);
    double delta = left + right - whole;
    if (depth <= 0 || fabs(delta) <= 15.0 * eps || fabs(delta) <= rel * fabs(left + right))
        return left + right + delta / 15.0;
    return simpson_rel(f, ctx, a, m, fa, flm, fm, left, 0.5 * eps, rel, depth - 1) +
           simpson_rel(f, ctx, m, b, fm, frm, fb, right, 0.5 * eps, rel, depth - 1);
}

static double integrate_rel(or_fn f, const void* ctx, double a, double b, double eps, double rel) {
    double m = 0.5 * (a + b), fa = f(a, ctx), fm = f(m, ctx), fb = f(b, ctx);
    return simpson_rel(f, ctx, a, b, fa, fm, fb, (b - a) / 6.0 * (fa + 4.0 * fm + fb), eps, rel, 40);
}

/* ---------------------------------------------------------------- cosmology */

/* Bardeen, Bond, Kaiser & Szalay (1986), App. G: adiabatic CDM transfer function. */
double or_bbks_transfer(double q) {
    if (q <= 0.0) return 1.0;
    double poly = 1.0 + 3.89 * q + pow(16.1 * q, 2) + pow(5.46 * q, 3) + pow(6.71 * q, 4);
    return log(1.0 + 2.34 * q) / (2.34 * q) * pow(poly, -0.25);
}

static double pk_shape(const or_cosmo* c, double k) {
    double t = 1.0;
    if (c->use_transfer) t = or_bbks_transfer(k / (c->omega_m * c->h * c->h));  /* q = k / (Omega_m h^2 Mpc^-1) */
    return pow(k, c->n_s) * t * t;
}

double or_pk(const or_cosmo* c, double k) { return c->amp * pk_shape(c, k); }

/* Fourier transform of the real-space top-hat of unit volume. */
double or_tophat_w(double x) {
    if (fabs(x) < 0.05) {   /* Taylor series: the closed form cancels for small x */
        double x2 = x * x;
        return 1.0 - x2 / 10.0 + x2 * x2 / 280.0 - x2 * x2 * x2 / 15120.0;
    }
    return 3.0 * (sin(x) - x * cos(x)) / (x * x * x);
}

typedef struct { const or_cosmo* c; double r; } sig_ctx;

/* d sigma^2 / d ln k = k^3 P(k) W^2(kR) / (2 pi^2), P without amplitude. */
static double sigma2_integrand(double lnk, const void* vctx) {
    const sig_ctx* s = (const sig_ctx*)vctx;
    double k = exp(lnk);
    double w = or_tophat_w(k * s->r);
    return k * k * k * pk_shape(s->c, k) * w * w / (2.0 * OR_PI * OR_PI);
}

static double sigma2_shape(const or_cosmo* c, double r) {
    sig_ctx s = {c, r};
    const double a = log(1e-6), b = log(1e4);
    /* coarse estimate sets the absolute tolerance (relative 1e-11) */
    double coarse = 0.0;
    const int m = 4000;
    for (int i = 0; i <= m; i++) {
        double w = (i == 0 || i == m) ? 1.0 : (i % 2 ? 4.0 : 2.0);
        coarse += w * sigma2_integrand(a + (b - a) * i / m, &s);
    }
    coarse *= (b - a) / m / 3.0;
    return integrate(sigma2_integrand, &s, a, b, 64, 1e-11 * fabs(coarse));
}

void or_cosmo_init(or_cosmo* c) {
    double r8 = 8.0 / c->h;
    c->amp = c->sigma8 * c->sigma8 / sigma2_shape(c, r8);
}

double or_sigma2(const or_cosmo* c, double r) { return c->amp * sigma2_shape(c, r); }

typedef struct { const or_cosmo* c; } gr_ctx;

static double hubble_e(const or_cosmo* c, double a) {
    return sqrt(c->omega_m / (a * a * a) + c->omega_l);
}

static double growth_integrand(double a, const void* vctx) {
    const or_cosmo* c = ((const gr_ctx*)vctx)->c;
    if (a <= 0.0) return 0.0;
    double ae = a * hubble_e(c, a);
    return 1.0 / (ae * ae * ae);
}

/* Linear growth D(a) proportional to H(a) Int_0^a da' / (a' H(a'))^3 (flat LCDM), normalised to D(0) = 1. */
static double growth_unnorm(const or_cosmo* c, double a) {
    gr_ctx g = {c};
    double coarse = 0.0;
    const int m = 2000;
    for (int i = 0; i <= m; i++) {
        double w = (i == 0 || i == m) ? 1.0 : (i % 2 ? 4.0 : 2.0);
        coarse += w * growth_integrand(a * i / m, &g);
    }
    coarse *= a / m / 3.0;
    return hubble_e(c, a) * integrate(growth_integrand, &g, 0.0, a, 16, 1e-13 * fabs(coarse));
}

double or_growth(const or_cosmo* c, double z) {
    return growth_unnorm(c, 1.0 / (1.0 + z)) / growth_unnorm(c, 1.0);
}

/* Growth rate f = d ln D / d ln a of D(a) = E(a) I(a), I(a) = Int_0^a da'/(a' E(a'))^3:
 * a D'/D = d ln E / d ln a + 1 / (a^2 E^3 I), with d ln E / d ln a = -1.5 Omega_m / (a^3 E^2)
 * for flat LCDM. */
double or_growth_rate(const or_cosmo* c, double z) {
    double a = 1.0 / (1.0 + z);
    double e = hubble_e(c, a);
    double i_a = growth_unnorm(c, a) / e;
    return -1.5 * c->omega_m / (a * a * a * e * e) + 1.0 / (a * a * e * e * e * i_a);
}

double or_rho_mean(const or_cosmo* c) { return c->omega_m * OR_RHO_CRIT_H2 * c->h * c->h; }

double or_mass_to_radius(const or_cosmo* c, double m) {
    return cbrt(3.0 * m / (4.0 * OR_PI * or_rho_mean(c)));
}

/* Virial temperature -> halo mass (Sec. 2.1.3, after Barkana & Loeb 2001). */
double or_mmin(const or_cosmo* c, double tvir, double z, double mu) {
    double zp = 1.0 + z;
    double om_z = c->omega_m * zp * zp * zp / (c->omega_m * zp * zp * zp + c->omega_l);
    double d = om_z - 1.0;
    double dc = 18.0 * OR_PI * OR_PI + 82.0 * d - 39.0 * d * d;
    return 1e8 / c->h * pow(mu / 0.6, -1.5) *
           pow(c->omega_m / om_z * dc / (18.0 * OR_PI * OR_PI), -0.5) *
           pow(tvir / 1.98e4, 1.5) * pow(zp / 10.0, -1.5);
}

/* Brightness-temperature prefactor of Sec. 2.2 with T_S >> T_gamma and no velocity term. */
double or_t0_mk(const or_cosmo* c, double z) {
    double h2 = c->h * c->h;
    return 27.0 * sqrt((1.0 + z) / 10.0 * 0.15 / (c->omega_m * h2)) * (c->omega_b * h2 / 0.023);
}

/* ---------------------------------------------------------------- ionization */

double or_r_cell(const or_ion_cfg* cfg, int n, double box_mpc) {
    double dx = box_mpc / n;
    if (cfg->r_cell_rule == 1) return dx;
    return cbrt(3.0 / (4.0 * OR_PI)) * dx;
}

/* Radii from R_mfp downwards by the factor r_factor while above R_cell, then R_cell once (Sec. 2.1). */
int or_radius_ladder(const or_ion_cfg* cfg, int n, double box_mpc, double r_mfp, double* radii, int cap) {
    double r_cell = or_r_cell(cfg, n, box_mpc);
    int count = 0;
    double r = r_mfp;
    while (r > r_cell) {
        if (count < cap) radii[count] = r;
        count++;
        r = r / cfg->r_factor;
    }
    if (count < cap) radii[count] = r_cell;
    return count + 1;
}

/* Extended Press-Schechter conditional collapsed fraction inside a sphere of variance
 * sigma2_r and overdensity delta_r, in haloes above the mass of variance sigma2_min. */
double or_fcoll(double delta_r, double sigma2_min, double sigma2_r, double delta_c) {
    double s2 = sigma2_min - sigma2_r;
    if (s2 <= 0.0) return 0.0;              /* region lighter than M_min: no such haloes */
    if (delta_r >= delta_c) return 1.0;     /* region itself collapsed */
    return erfc((delta_c - delta_r) / sqrt(2.0 * s2));
}

/* ------------------------------------------ mass-dependent efficiency (Sec. 5) */

/* dW/dx of the top-hat transform: 3 (x^2 sin x - 3 sin x + 3 x cos x) / x^4. */
static double tophat_dw(double x) {
    if (fabs(x) < 0.05) {
        double x2 = x * x;
        return x * (-1.0 / 5.0 + x2 / 70.0 - x2 * x2 / 2520.0);
    }
    double s = sin(x), c = cos(x);
    return 3.0 * (x * x * s - 3.0 * s + 3.0 * x * c) / (x * x * x * x);
}

/* d sigma^2 / d ln R integrand: k^3 P(k) 2 W(kR) W'(kR) kR / (2 pi^2), P without amplitude. */
static double dsigma2_integrand(double lnk, const void* vctx) {
    const sig_ctx* s = (const sig_ctx*)vctx;
    double k = exp(lnk), x = k * s->r;
    return k * k * k * pk_shape(s->c, k) * 2.0 * or_tophat_w(x) * tophat_dw(x) * x / (2.0 * OR_PI * OR_PI);
}

double or_dsigma2_dlnr(const or_cosmo* c, double r) {
    sig_ctx s = {c, r};
    const double a = log(1e-6), b = log(1e4);
    double coarse = 0.0;   /* integral of |integrand| sets the absolute tolerance */
    const int m = 4000;
    for (int i = 0; i <= m; i++) {
        double w = (i == 0 || i == m) ? 1.0 : (i % 2 ? 4.0 : 2.0);
        coarse += w * fabs(dsigma2_integrand(a + (b - a) * i / m, &s));
    }
    coarse *= (b - a) / m / 3.0;
    return c->amp * integrate(dsigma2_integrand, &s, a, b, 64, 1e-11 * coarse);
}

/* S(M) = D^2 sigma^2(R(M)) and dS/dln M = D^2 (d sigma^2/d ln R) / 3 on a uniform ln M grid,
 * each node by the two quadratures above; or_var_s interpolates with cubic Hermite
 * polynomials through the values and the derivatives. */
or_var_table* or_var_table_new(const or_cosmo* c, double growth, double m_lo, double m_hi, double dlnm) {
    or_var_table* t = (or_var_table*)calloc(1, sizeof(or_var_table));
    t->lnm0 = log(m_lo);
    t->n = (int)ceil((log(m_hi) - t->lnm0) / dlnm) + 1;
    if (t->n < 2) t->n = 2;
    t->dlnm = (log(m_hi) - t->lnm0) / (t->n - 1);
    t->s = (double*)malloc(sizeof(double) * t->n);
    t->ds = (double*)malloc(sizeof(double) * t->n);
    double g2 = growth * growth;
#pragma omp parallel for schedule(dynamic)
    for (int i = 0; i < t->n; i++) {
        double r = or_mass_to_radius(c, exp(t->lnm0 + i * t->dlnm));
        t->s[i] = g2 * or_sigma2(c, r);
        t->ds[i] = g2 * or_dsigma2_dlnr(c, r) / 3.0;
    }
    return t;
}

void or_var_table_free(or_var_table* t) {
    if (!t) return;
    free(t->s);
    free(t->ds);
    free(t);
}

double or_var_s(const or_var_table* t, double lnm, double* dsdlnm) {
    double u = (lnm - t->lnm0) / t->dlnm;
    int i = (int)floor(u);
    if (i < 0) i = 0;
    if (i > t->n - 2) i = t->n - 2;
    double x = u - i, h = t->dlnm;
    double p0 = t->s[i], p1 = t->s[i + 1], m0 = t->ds[i] * h, m1 = t->ds[i + 1] * h;
    double x2 = x * x, x3 = x2 * x;
    if (dsdlnm)
        *dsdlnm = ((6.0 * x2 - 6.0 * x) * p0 + (3.0 * x2 - 4.0 * x + 1.0) * m0 + (-6.0 * x2 + 6.0 * x) * p1 +
                   (3.0 * x2 - 2.0 * x) * m1) / h;
    return (2.0 * x3 - 3.0 * x2 + 1.0) * p0 + (x3 - 2.0 * x2 + x) * m0 + (-2.0 * x3 + 3.0 * x2) * p1 +
           (x3 - x2) * m1;
}

/* S(lb - gap) - S(lb) for gap >= 0 without cancellation: for gaps below a quarter of the grid
 * step both points use the cubic of lb's cell, whose Hermite basis differences factor as
 * (u - v) = -gap / h times a polynomial; larger gaps subtract directly. */
static double var_diff(const or_var_table* t, double lb, double gap) {
    double h = t->dlnm;
    if (gap >= 0.25 * h) return or_var_s(t, lb - gap, NULL) - or_var_s(t, lb, NULL);
    int i = (int)floor((lb - t->lnm0) / h);
    i = i < 0 ? 0 : (i > t->n - 2 ? t->n - 2 : i);
    double x0 = t->lnm0 + i * h;
    double v = (lb - x0) / h, u = v - gap / h;
    double p0 = t->s[i], p1 = t->s[i + 1], m0 = t->ds[i] * h, m1 = t->ds[i + 1] * h;
    double q = u * u + u * v + v * v, l = u + v;
    return (-gap / h) * (p0 * (2.0 * q - 3.0 * l) + m0 * (q - 2.0 * l + 1.0) + p1 * (-2.0 * q + 3.0 * l) +
                         m1 * (q - l));
}

static double pop_zeta(const or_pop* p, double m) { return p->zeta0 * pow(m / p->m_pivot, p->slope); }

typedef struct {
    const or_var_table* t;
    const or_pop* p;
    double top_lnm;   /* ln of the upper end of the mass range */
    double lnm_r;     /* ln M_R, or 0 without a region (S_R = 0) */
    double nu;        /* delta_c - delta_R > 0 */
} pops_ctx;

/* In x = ln(top / M): zeta(M) f(S(M) | delta_R, S_R) (-dS/d ln M), with the first-crossing
 * distribution f(S) = nu / sqrt(2 pi) (S - S_R)^(-3/2) exp(-nu^2 / (2 (S - S_R))) of the
 * extended Press-Schechter conditional mass function (Lacey & Cole 1993). */
static double pops_integrand(double x, const void* v) {
    const pops_ctx* c = (const pops_ctx*)v;
    double lnm = c->top_lnm - x, ds;
    double s = or_var_s(c->t, lnm, &ds);
    double d = c->lnm_r != 0.0 ? var_diff(c->t, c->lnm_r, (c->lnm_r - c->top_lnm) + x) : s;
    if (d <= 0.0) return 0.0;
    double f = c->nu / sqrt(2.0 * OR_PI) * pow(d, -1.5) * exp(-c->nu * c->nu / (2.0 * d));
    return pop_zeta(c->p, exp(lnm)) * f * (-ds);
}

double or_fcoll_pops(const or_var_table* t, const or_pop* pops, int n_pops, double m_r, double delta_r,
                     double delta_c) {
    double nu = delta_c - delta_r, total = 0.0;
    for (int i = 0; i < n_pops; i++) {
        const or_pop* p = &pops[i];
        double hi = p->m_hi > 0.0 ? p->m_hi : exp(t->lnm0 + (t->n - 1) * t->dlnm);
        if (nu <= 0.0) {   /* region collapsed into one halo of mass M_R */
            if (m_r > 0.0 && m_r >= p->m_lo && (p->m_hi <= 0.0 || m_r < p->m_hi)) total += pop_zeta(p, m_r);
            continue;
        }
        double top = m_r > 0.0 ? fmin(hi, m_r) : hi;
        if (top <= p->m_lo) continue;
        pops_ctx c = {t, p, log(top), m_r > 0.0 ? log(m_r) : 0.0, nu};
        double span = log(top / p->m_lo);
        double eps = 1e-12 * (pop_zeta(p, p->m_lo) + pop_zeta(p, top));
        /* panels halving towards x = 0 (M -> top), where the integrand narrows as nu -> 0 */
        double b = span;
        for (int k = 0; k < 50; k++) {
            double a = 0.5 * b;
            total += integrate_rel(pops_integrand, &c, a, b, eps / 50.0, 1e-11);
            b = a;
        }
    }
    return total;
}

static double* forward_spectrum(int n, const float* delta) {
    size_t n3 = (size_t)n * n * n;
    double* spec = (double*)malloc(sizeof(double) * 2 * n3);
    for (size_t i = 0; i < n3; i++) { spec[2 * i] = delta[i]; spec[2 * i + 1] = 0.0; }
    or_fft3d(spec, n, -1);
    return spec;
}

/* buf = IDFT(W(|k| R) spec) / n^3 (real part), using the signed frequencies of each axis. */
static void filter_from_spectrum(int n, double box_mpc, const double* spec, double r, double* work,
                                 double* out) {
    size_t n3 = (size_t)n * n * n;
    double kf = 2.0 * OR_PI / box_mpc;
#pragma omp parallel for schedule(static)
    for (long long ix = 0; ix < n; ix++) {
        double kx = kf * freq_index((int)ix, n);
        for (int iy = 0; iy < n; iy++) {
            double ky = kf * freq_index(iy, n);
            for (int iz = 0; iz < n; iz++) {
                double kz = kf * freq_index(iz, n);
                double k = sqrt(kx * kx + ky * ky + kz * kz);
                double w = or_tophat_w(k * r);
                size_t idx = ((size_t)ix * n + iy) * n + iz;
                work[2 * idx] = spec[2 * idx] * w;
                work[2 * idx + 1] = spec[2 * idx + 1] * w;
            }
        }
    }
    or_fft3d(work, n, +1);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)n3; i++) out[i] = work[2 * i] / (double)n3;
}

/* Line-of-sight (last axis) second derivative field: out = IDFT(k_z^2 / k^2 DFT(delta)) / n^3,
 * zero at k = 0. In linear theory dv_r/dr = -f H out. */
void or_los_gradient(int n, double box_mpc, const float* delta, double* out) {
    size_t n3 = (size_t)n * n * n;
    double* spec = forward_spectrum(n, delta);
    (void)box_mpc;   /* the ratio k_z^2 / k^2 does not depend on the box size */
#pragma omp parallel for schedule(static)
    for (long long ix = 0; ix < n; ix++) {
        double mx = freq_index((int)ix, n);
        for (int iy = 0; iy < n; iy++) {
            double my = freq_index(iy, n);
            for (int iz = 0; iz < n; iz++) {
                double mz = freq_index(iz, n);
                double m2 = mx * mx + my * my + mz * mz;
                double w = m2 > 0.0 ? mz * mz / m2 : 0.0;
                size_t idx = ((size_t)ix * n + iy) * n + iz;
                spec[2 * idx] *= w;
                spec[2 * idx + 1] *= w;
            }
        }
    }
    or_fft3d(spec, n, +1);
#pragma omp parallel for schedule(static)
    for (long long i = 0; i < (long long)n3; i++) out[i] = spec[2 * i] / (double)n3;
    free(spec);
}

void or_filter_box(int n, double box_mpc, const float* delta, double r, double* out) {
    size_t n3 = (size_t)n * n * n;
    double* spec = forward_spectrum(n, delta);
    double* work = (double*)malloc(sizeof(double) * 2 * n3);
    filter_from_spectrum(n, box_mpc, spec, r, work, out);
    free(work);
    free(spec);
}

int or_ionize(const or_cosmo* c, const or_ion_cfg* cfg, int n, double box_mpc, double z,
              const float* delta, double zeta, double r_mfp, double log10_tvir,
              double* xhi, uint8_t* flag, double* dtb, double* xhi_mean) {
    size_t n3 = (size_t)n * n * n;
    /* radii */
    int nr = or_radius_ladder(cfg, n, box_mpc, r_mfp, NULL, 0);
    double* radii = (double*)malloc(sizeof(double) * nr);
    or_radius_ladder(cfg, n, box_mpc, r_mfp, radii, nr);
    /* variance of the halo-mass threshold and of each sphere, at redshift z */
    double g = or_growth(c, z);
    double m_min = or_mmin(c, pow(10.0, log10_tvir), z, cfg->mu);
    double s2_min = g * g * or_sigma2(c, or_mass_to_radius(c, m_min));

    double* spec = forward_spectrum(n, delta);
    double* work = (double*)malloc(sizeof(double) * 2 * n3);
    double* dr = (double*)malloc(sizeof(double) * n3);
    double* f_cell = (double*)malloc(sizeof(double) * n3);
    uint8_t* ion = (uint8_t*)calloc(n3, 1);

    for (int j = 0; j < nr; j++) {
        double r = radii[j];
        double s2_r = g * g * or_sigma2(c, r);
        filter_from_spectrum(n, box_mpc, spec, r, work, dr);
        int last = (j == nr - 1);
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)n3; i++) {
            double f = or_fcoll(dr[i], s2_min, s2_r, cfg->delta_c);
            if (zeta * f >= 1.0) ion[i] = 1;             /* Eq. 1 */
            if (last) f_cell[i] = f;
        }
    }

    double t0 = or_t0_mk(c, z);
    double sum = 0.0;
    for (size_t i = 0; i < n3; i++) {
        double xhii = ion[i] ? 1.0 : fmin(1.0, zeta * f_cell[i]);   /* partial ionization at R_cell */
        double x = 1.0 - xhii;
        if (xhi) xhi[i] = x;
        if (flag) flag[i] = ion[i];
        if (dtb) dtb[i] = t0 * x * (1.0 + (double)delta[i]);
        sum += x;
    }
    if (xhi_mean) *xhi_mean = sum / (double)n3;

    free(ion); free(f_cell); free(dr); free(work); free(spec); free(radii);
    return nr;
}

/* Overdensities where zeta f_coll crosses 1 for one radius: a scan of nu = delta_c - delta_R
 * from nu_max down (geometric, 400 points, then nu = 0, where F is the collapsed value),
 * each sign change of F - 1 refined by bisection. Returns the count (<= cap), roots as
 * delta values in increasing order of nu, i.e. decreasing delta. */
static int pops_roots(const or_var_table* t, const or_pop* pops, int n_pops, double m_r, double delta_c,
                      double nu_max, double* roots, int cap) {
    const int m = 400;
    int count = 0;
    double nu_prev = nu_max;
    double g_prev = or_fcoll_pops(t, pops, n_pops, m_r, delta_c - nu_prev, delta_c) - 1.0;
    for (int k = 1; k <= m + 1; k++) {
        double nu = k <= m ? nu_max * pow(1e-10, (double)k / m) : 0.0;
        double g = or_fcoll_pops(t, pops, n_pops, m_r, delta_c - nu, delta_c) - 1.0;
        if ((g >= 0.0) != (g_prev >= 0.0)) {
            double lo = nu, hi = nu_prev;   /* g(lo) and g(hi) differ in sign */
            double glo = g;
            for (int it = 0; it < 200 && hi - lo > 1e-15 * (1.0 + hi); it++) {
                double mid = 0.5 * (lo + hi);
                double gm = or_fcoll_pops(t, pops, n_pops, m_r, delta_c - mid, delta_c) - 1.0;
                if ((gm >= 0.0) == (glo >= 0.0)) { lo = mid; glo = gm; } else hi = mid;
            }
            if (count < cap) roots[count] = delta_c - 0.5 * (lo + hi);
            count++;
        }
        nu_prev = nu;
        g_prev = g;
    }
    return count;
}

int or_ionize_pops(const or_cosmo* c, const or_ion_cfg* cfg, int n, double box_mpc, double z,
                   const float* delta, const or_pop* pops, int n_pops, double r_mfp,
                   double* xhi, uint8_t* flag, double* dtb, double* xhi_mean) {
    size_t n3 = (size_t)n * n * n;
    int nr = or_radius_ladder(cfg, n, box_mpc, r_mfp, NULL, 0);
    double* radii = (double*)malloc(sizeof(double) * nr);
    or_radius_ladder(cfg, n, box_mpc, r_mfp, radii, nr);
    double g = or_growth(c, z);
    double rho = or_rho_mean(c);
    double m_lo = INFINITY;
    for (int i = 0; i < n_pops; i++) m_lo = fmin(m_lo, pops[i].m_lo);
    double m_top = 4.0 / 3.0 * OR_PI * radii[0] * radii[0] * radii[0] * rho;
    or_var_table* t = or_var_table_new(c, g, 0.25 * m_lo, 4.0 * m_top, 0.03);

    double* spec = forward_spectrum(n, delta);
    double* work = (double*)malloc(sizeof(double) * 2 * n3);
    double* dr = (double*)malloc(sizeof(double) * n3);
    uint8_t* ion = (uint8_t*)calloc(n3, 1);
    double roots[64];

    for (int j = 0; j < nr; j++) {
        double r = radii[j];
        double m_r = 4.0 / 3.0 * OR_PI * r * r * r * rho;
        filter_from_spectrum(n, box_mpc, spec, r, work, dr);
        double s_r = or_var_s(t, log(m_r), NULL);
        double ds = or_var_s(t, log(m_lo), NULL) - s_r;
        double nu_max = ds > 0.0 ? 12.0 * sqrt(2.0 * ds) : 1.0;
        int nroot = pops_roots(t, pops, n_pops, m_r, cfg->delta_c, nu_max, roots, 64);
        if (nroot > 64) nroot = 64;
        double f_top = or_fcoll_pops(t, pops, n_pops, m_r, cfg->delta_c, cfg->delta_c);
        int last = (j == nr - 1);
        /* Eq. 1 per cell: zeta f_coll >= 1, i.e. an odd number of crossings at or above delta_R */
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < (long long)n3; i++) {
            int on;
            if (dr[i] >= cfg->delta_c) {
                on = f_top >= 1.0;
            } else {
                int above = 0;
                for (int q = 0; q < nroot; q++) above += roots[q] <= dr[i];
                on = above & 1;
            }
            if (on) ion[i] = 1;
            if (last) work[i] = ion[i] ? 1.0 : fmin(1.0, or_fcoll_pops(t, pops, n_pops, m_r, dr[i], cfg->delta_c));
        }
    }

    double t0 = or_t0_mk(c, z);
    double sum = 0.0;
    for (size_t i = 0; i < n3; i++) {
        double x = 1.0 - work[i];   /* partial ionization at R_cell, 1 where flagged */
        if (xhi) xhi[i] = x;
        if (flag) flag[i] = ion[i];
        if (dtb) dtb[i] = t0 * x * (1.0 + (double)delta[i]);
        sum += x;
    }
    if (xhi_mean) *xhi_mean = sum / (double)n3;
    or_var_table_free(t);
    free(ion); free(dr); free(work); free(spec); free(radii);
    return nr;
}

/* ---------------------------------------------------------------- spectrum */

void or_power_spectrum(int n, double box_mpc, const double* box, int nbins, double k_lo, double k_hi,
                       double* d2, double* kmean, int64_t* nmodes) {
    size_t n3 = (size_t)n * n * n;
    double dx = box_mpc / n;
    double vol = box_mpc * box_mpc * box_mpc;
    double kf = 2.0 * OR_PI / box_mpc;
    double* spec = (double*)malloc(sizeof(double) * 2 * n3);
    for (size_t i = 0; i < n3; i++) { spec[2 * i] = box[i]; spec[2 * i + 1] = 0.0; }
    or_fft3d(spec, n, -1);

    double* s = (double*)calloc(nbins, sizeof(double));
    double* ks = (double*)calloc(nbins, sizeof(double));
    int64_t* cnt = (int64_t*)calloc(nbins, sizeof(int64_t));
    double log_ratio = log(k_hi / k_lo);
    double dx3 = dx * dx * dx;
    for (int ix = 0; ix < n; ix++)
        for (int iy = 0; iy < n; iy++)
            for (int iz = 0; iz < n; iz++) {
                int mx = freq_index(ix, n), my = freq_index(iy, n), mz = freq_index(iz, n);
                if (mx == 0 && my == 0 && mz == 0) continue;
                double k = kf * sqrt((double)(mx * mx + my * my + mz * mz));
                if (k < k_lo || k >= k_hi) continue;
                int b = (int)floor(nbins * log(k / k_lo) / log_ratio);
                if (b < 0 || b >= nbins) continue;
                size_t idx = ((size_t)ix * n + iy) * n + iz;
                double xr = spec[2 * idx] * dx3, xi = spec[2 * idx + 1] * dx3;   /* X = dx^3 DFT */
                s[b] += k * k * k * (xr * xr + xi * xi) / (2.0 * OR_PI * OR_PI * vol);
                ks[b] += k;
                cnt[b] += 1;
            }
    for (int b = 0; b < nbins; b++) {
        if (d2) d2[b] = cnt[b] ? s[b] / cnt[b] : NAN;
        if (kmean) kmean[b] = cnt[b] ? ks[b] / cnt[b] : NAN;
        if (nmodes) nmodes[b] = cnt[b];
    }
    free(cnt); free(ks); free(s); free(spec);
}

double or_chi2(int nbins, double k_lo, double k_hi, double chi_lo, double chi_hi,
               const double* d2, const int64_t* nmodes, const double* mock, const double* sigma) {
    double chi2 = 0.0;
    for (int b = 0; b < nbins; b++) {
        double centre = k_lo * pow(k_hi / k_lo, (b + 0.5) / nbins);
        if (centre < chi_lo || centre > chi_hi) continue;
        if (nmodes && nmodes[b] == 0) continue;
        double r = (d2[b] - mock[b]) / sigma[b];
        chi2 += r * r;
    }
    return chi2;
}
