// tables.cu — FP64 cosmology and per-walker tables of the excursion-set path, built on
// the GPU (sm_103a). FP64 is kept to these small tables: the growth factor, the
// top-hat mass variance sigma^2(R), the virial mass threshold, each walker's radius
// ladder and the overdensity at which Eq. 1 switches; the per-cell work stays FP32.
#include <math.h>

#include "eor_internal.cuh"

namespace eor {

namespace {

constexpr int kGL = 8;   // Gauss-Legendre points per panel

// Nodes and weights of the kGL-point Gauss-Legendre rule on [-1, 1], by Newton's method
// on the Legendre recurrence (one thread per node).
__device__ void gauss_legendre(double* x, double* w) {
    int i = threadIdx.x;
    if (i < kGL) {
        double z = cos(kPi * (i + 0.75) / (kGL + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 1; k < kGL; k++) {
                double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
                p0 = p1; p1 = p2;
            }
            dp = kGL * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Bardeen et al. (1986) App. G transfer function, q = k / (Omega_m h^2 Mpc^-1).
__device__ double transfer_bbks(double q) {
    if (q <= 0.0) return 1.0;
    double q2 = q * q;
    double poly = 1.0 + 3.89 * q + 259.21 * q2 + 162.771336 * q2 * q + 2027.16958081 * q2 * q2;
    return log1p(2.34 * q) / (2.34 * q) / sqrt(sqrt(poly));
}

__device__ double window_tophat(double x) {
    if (x < 0.05) {
        double x2 = x * x;
        return 1.0 - x2 * (0.1 - x2 * (1.0 / 280.0 - x2 / 15120.0));
    }
    double s, c;
    sincos(x, &s, &c);
    return 3.0 * (s - x * c) / (x * x * x);
}

// k^3 T(k)^2 k^n_s W(kR)^2 / (2 pi^2): d sigma^2 / d ln k without the amplitude.
__device__ double dsigma2_dlnk(double k, double r, double om_h2, double n_s) {
    double t = transfer_bbks(k / om_h2);
    double w = window_tophat(k * r);
    return k * k * k * pow(k, n_s) * t * t * w * w / (2.0 * kPi * kPi);
}

__device__ double block_sum(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    __syncthreads();
    return s;   // valid in thread 0
}

// One block per radius: sigma^2 shape integral over ln k in [ln 1e-6, ln(1/R)] (panels
// of width <= 0.1) and over x = kR in [1, min(400, 1e4 R)] (panels of pi/8, resolving
// the window's oscillation). Beyond x = 400 the integrand is below 1e-10 of the total.
__global__ void k_sigma2_shape(double lnr_lo, double dlnr, int n_table, double r8, double om_h2,
                               double n_s, double* out) {
    __shared__ double gx[kGL], gw[kGL], red[32];
    gauss_legendre(gx, gw);
    __syncthreads();
    int idx = blockIdx.x;
    double r = idx < n_table ? exp(lnr_lo + dlnr * idx) : r8;
    double acc = 0.0;
    // part A: ln k panels
    double a = log(1e-6), b = log(fmin(1.0 / r, 1e4));
    int na = (int)ceil((b - a) / 0.1);
    double ha = (b - a) / na;
    for (int p = threadIdx.x; p < na; p += blockDim.x) {
        double lo = a + p * ha;
        for (int g = 0; g < kGL; g++) {
            double lnk = lo + 0.5 * ha * (gx[g] + 1.0);
            acc += 0.5 * ha * gw[g] * dsigma2_dlnk(exp(lnk), r, om_h2, n_s);
        }
    }
    // part B: x panels, integrand in k: (1/k) dsigma2_dlnk, dk = dx / r
    double x0 = 1.0, x1 = fmin(400.0, 1e4 * r);
    if (x1 > x0) {
        int nb = (int)ceil((x1 - x0) / (kPi / 8.0));
        double hb = (x1 - x0) / nb;
        for (int p = threadIdx.x; p < nb; p += blockDim.x) {
            double lo = x0 + p * hb;
            for (int g = 0; g < kGL; g++) {
                double x = lo + 0.5 * hb * (gx[g] + 1.0);
                double k = x / r;
                acc += 0.5 * hb * gw[g] * dsigma2_dlnk(k, r, om_h2, n_s) / x;
            }
        }
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) out[idx] = s;
}

// amp = sigma_8^2 / shape(8/h); table -> ln(amp * shape).
__global__ void k_sigma2_normalise(double* shape, int n_table, double sigma8, double* amp_out) {
    double amp = sigma8 * sigma8 / shape[n_table];
    for (int i = threadIdx.x; i < n_table; i += blockDim.x) shape[i] = log(amp * shape[i]);
    if (threadIdx.x == 0) amp_out[0] = amp;
}

// Linear growth D(z) = E(a) Int_0^a da'/(a' E(a'))^3 / (same at a = 1), flat LCDM, and its
// rate f = d ln D / d ln a into out[n_z + j];
// substituting a' = u^2 makes the integrand smooth at 0. One block per redshift.
__global__ void k_growth(const double* zs, int n_z, double om, double ol, double* out) {
    __shared__ double gx[kGL], gw[kGL], red[32];
    gauss_legendre(gx, gw);
    __syncthreads();
    const int panels = 256;
    double res[2], integ0 = 0.0;
    for (int which = 0; which < 2; which++) {
        double a = which == 0 ? 1.0 / (1.0 + zs[blockIdx.x]) : 1.0;
        double umax = sqrt(a), h = umax / panels, acc = 0.0;
        for (int p = threadIdx.x; p < panels; p += blockDim.x) {
            for (int g = 0; g < kGL; g++) {
                double u = p * h + 0.5 * h * (gx[g] + 1.0);
                double ap = u * u;
                double e = sqrt(om / (ap * ap * ap) + ol);
                double d = ap * e;
                acc += 0.5 * h * gw[g] * 2.0 * u / (d * d * d);
            }
        }
        double s = block_sum(acc, red);
        res[which] = sqrt(om / (a * a * a) + ol) * s;
        if (which == 0) integ0 = s;
    }
    if (threadIdx.x == 0) {
        out[blockIdx.x] = res[0] / res[1];
        // f = d ln D / d ln a = d ln E / d ln a + 1 / (a^2 E^3 I), d ln E / d ln a = -1.5 Om / (a^3 E^2)
        const double a = 1.0 / (1.0 + zs[blockIdx.x]);
        const double e = sqrt(om / (a * a * a) + ol);
        out[n_z + blockIdx.x] = -1.5 * om / (a * a * a * e * e) + 1.0 / (a * a * e * e * e * integ0);
    }
}

// Bin of every |m|^2 = mx^2 + my^2 + mz^2 (FP64 decision, -1 outside [k_lo, k_hi) or k = 0).
__global__ void k_bin_table(int n_m2, double kf, double k_lo, double k_hi, int n_bins, signed char* bin) {
    int m2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (m2 >= n_m2) return;
    int b = -1;
    if (m2 > 0) {
        double k = kf * sqrt((double)m2);
        if (k >= k_lo && k < k_hi) {
            b = (int)floor(n_bins * log(k / k_lo) / log(k_hi / k_lo));
            if (b < 0 || b >= n_bins) b = -1;
        }
    }
    bin[m2] = (signed char)b;
}

// Mode count and summed |k| per bin over the full n^3 grid (data independent).
__global__ void k_mode_counts(int n, double kf, const signed char* bin, int n_bins, long long* cnt,
                              double* ksum) {
    __shared__ unsigned long long s_cnt[EOR21_MAX_BINS];
    __shared__ double s_k[EOR21_MAX_BINS];
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) { s_cnt[b] = 0ull; s_k[b] = 0.0; }
    __syncthreads();
    long long n3 = (long long)n * n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n3;
         idx += (long long)gridDim.x * blockDim.x) {
        int ix = (int)(idx / ((long long)n * n)), iy = (int)((idx / n) % n), iz = (int)(idx % n);
        int mx = ix < n / 2 ? ix : ix - n, my = iy < n / 2 ? iy : iy - n, mz = iz < n / 2 ? iz : iz - n;
        int m2 = mx * mx + my * my + mz * mz;
        int b = bin[m2];
        if (b >= 0) {
            atomicAdd(&s_cnt[b], 1ull);
            atomicAdd(&s_k[b], kf * sqrt((double)m2));
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) {
        atomicAdd((unsigned long long*)&cnt[b], s_cnt[b]);
        atomicAdd(&ksum[b], s_k[b]);
    }
}

// Bins that enter chi^2: geometric centre k_lo (k_hi/k_lo)^((b + 1/2)/n_bins) in [lo, hi].
__global__ void k_chi2_bins(int n_bins, double k_lo, double k_hi, double lo, double hi, signed char* use) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins) return;
    double centre = k_lo * pow(k_hi / k_lo, (b + 0.5) / n_bins);
    use[b] = (centre >= lo && centre <= hi) ? 1 : 0;
}

__device__ double interp_lnsig(const double* lnsig, double lnr_lo, double dlnr, double r, int* err) {
    double u = (log(r) - lnr_lo) / dlnr;
    int i = (int)floor(u);
    if (!(i >= 1 && i <= kSigmaTable - 3)) {
        atomicOr(err, kErrSigmaRange);
        i = i < 1 ? 1 : kSigmaTable - 3;
    }
    double t = u - i;
    // 4-point Lagrange through i-1, i, i+1, i+2
    double f0 = lnsig[i - 1], f1 = lnsig[i], f2 = lnsig[i + 1], f3 = lnsig[i + 2];
    double l0 = -t * (t - 1.0) * (t - 2.0) / 6.0;
    double l1 = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
    double l2 = -(t + 1.0) * t * (t - 2.0) / 2.0;
    double l3 = (t + 1.0) * t * (t - 1.0) / 6.0;
    return exp(l0 * f0 + l1 * f1 + l2 * f2 + l3 * f3);
}

// Halo mass of virial temperature 10^logt at redshift z (Sec. 2.1.3, after Barkana & Loeb 2001).
__device__ double virial_mass(double logt, double z, double h, double om, double ol, double mu) {
    const double zp = 1.0 + z;
    const double om_z = om * zp * zp * zp / (om * zp * zp * zp + ol);
    const double d = om_z - 1.0;
    const double dc = 18.0 * kPi * kPi + 82.0 * d - 39.0 * d * d;
    return 1e8 / h * pow(mu / 0.6, -1.5) * pow(om / om_z * dc / (18.0 * kPi * kPi), -0.5) *
           pow(pow(10.0, logt) / 1.98e4, 1.5) * pow(zp / 10.0, -1.5);
}

struct WalkerTableArgs {
    const double* params;
    const double* growth;
    const double* lnsig;
    double lnr_lo, dlnr;
    double z[EOR21_MAX_Z];
    int n_z, n_walkers, max_radii;
    double r_cell, r_factor, r_mfp_max, delta_c, mu;
    double h, omega_m, omega_l, omega_b, rho_mean;
    WalkerInfo* walkers;
    PairInfo* pairs;
    int* err;
};

// One thread per (walker, redshift): M_min (Sec. 2.1.3), ladder (Sec. 2.1), sigma^2 of
// each radius, the threshold overdensity of Eq. 1 and the partial-ionization constants.
// One warp per (walker, redshift): lane j takes radii j and j + 32 of the ladder. Every lane
// forms the ladder by the same sequence of FP64 divisions (so that radius j is bitwise the
// serial ladder's), the walker's M_min and erfcinv(1/zeta); the lanes then fill their radii's
// thresholds of Eq. 1 and the last lane to hold a radius sets the R_cell quantities.
__global__ void k_walker_tables(WalkerTableArgs a) {
    const int pid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (pid >= a.n_walkers * a.n_z) return;
    const int w = pid / a.n_z, zi = pid % a.n_z;
    const double zeta = a.params[3 * w], r_mfp = a.params[3 * w + 1], logt = a.params[3 * w + 2];
    PairInfo& P = a.pairs[pid];
    const bool ok = isfinite(zeta) && isfinite(r_mfp) && isfinite(logt) && zeta > 0.0 && r_mfp > 0.0 &&
                    r_mfp <= a.r_mfp_max && logt > 0.0 && logt < 12.0;
    if (!ok) {
        if (lane == 0) {
            atomicOr(a.err, kErrParam);
            P.w = w; P.zi = zi; P.pad = 0;
            P.n_r = 0;
            if (zi == 0) a.walkers[w].n_r = 0;
        }
        return;
    }
    // radius ladder: R_mfp, R_mfp / f, ... while above R_cell, then R_cell once
    double rj[2] = {0.0, 0.0};
    int nr = 0;
    bool over = false;
    {
        double r = r_mfp;
        while (r > a.r_cell) {
            if (nr >= a.max_radii - 1) { over = true; break; }
            if (nr == lane) rj[0] = r;
            if (nr == lane + 32) rj[1] = r;
            nr++;
            r = r / a.r_factor;
        }
        if (nr == lane) rj[0] = a.r_cell;
        if (nr == lane + 32) rj[1] = a.r_cell;
        nr++;
    }
    if (over && lane == 0) atomicOr(a.err, kErrLadder);
    // virial temperature -> minimum halo mass at z
    const double zp = 1.0 + a.z[zi];
    const double m_min = virial_mass(logt, a.z[zi], a.h, a.omega_m, a.omega_l, a.mu);
    const double r_min = cbrt(3.0 * m_min / (4.0 * kPi * a.rho_mean));
    const double g2 = a.growth[zi] * a.growth[zi];
    const double s2_min = g2 * interp_lnsig(a.lnsig, a.lnr_lo, a.dlnr, r_min, a.err);
    // zeta erfc((delta_c - delta_R) / sqrt(2 s2)) >= 1  <=>  delta_R >= delta_c - sqrt(2 s2) erfcinv(1/zeta)
    const double u_star = zeta >= 1.0 ? erfcinv(1.0 / zeta) : 0.0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int j = lane + 32 * h;
        if (j < nr) {
            const double s2 = s2_min - g2 * interp_lnsig(a.lnsig, a.lnr_lo, a.dlnr, rj[h], a.err);
            const double dcrit = (s2 > 0.0 && zeta >= 1.0) ? a.delta_c - sqrt(2.0 * s2) * u_star : INFINITY;
            P.delta_crit[j] = (float)dcrit;
            if (zi == 0) a.walkers[w].radii[j] = rj[h];
            if (j == nr - 1) {   // R_cell
                P.cell_ok = s2 > 0.0 ? 1.0f : 0.0f;
                P.inv_sqrt2s2_cell = s2 > 0.0 ? (float)(1.0 / sqrt(2.0 * s2)) : 0.0f;
            }
        } else if (j < kMaxRadii) {
            P.delta_crit[j] = INFINITY;
        }
        if (j < kMaxRadii) P.delta_hi[j] = INFINITY;
    }
    if (lane == 0) {
        P.w = w; P.zi = zi; P.pad = 0;
        P.n_r = nr;
        if (zi == 0) a.walkers[w].n_r = nr;
        P.f_inv_h = 0.0f;
        P.zeta = (float)zeta;
        const double h2 = a.h * a.h;
        P.t0 = (float)(27.0 * sqrt(zp / 10.0 * 0.15 / (a.omega_m * h2)) * (a.omega_b * h2 / 0.023));
    }
}

// ------------------------------------------------ mass-dependent efficiency (Sec. 5)
//
// F(delta_R) = sum_i Int zeta_i(M) f(S(M) | delta_R, S_R) dS over population i's masses below
// M_R, f the extended Press-Schechter first-crossing distribution
//     f(S) dS = nu / sqrt(2 pi) (S - S_R)^(-3/2) exp(-nu^2 / (2 (S - S_R))) dS,  nu = delta_c - delta_R.
// In y = ln(S - S_R) this is Int zeta(M(y)) K(t) dy with t = nu e^(-y/2) / sqrt(2) and the
// smooth bump K = t e^(-t^2) / sqrt(pi) (unit integral over y), so composite Gauss-Legendre on
// unit panels in y resolves every nu; M(y) comes from inverting the sigma^2 table once per
// node. Below the last panel (masses within e^-36 of M_R in variance) zeta is zeta(M_R) and
// the bump integrates to erfc(t). One warp per (walker, redshift, radius).

constexpr int kPopMax = 2;                   // populations of an efficiency model
constexpr int kPopPanels = 36;               // unit panels in y per population
constexpr int kPopGL = 4;                    // Gauss-Legendre nodes per panel
constexpr int kPopNodes = kPopMax * kPopPanels * kPopGL;
constexpr int kPopWarps = 4;                 // tasks per block
constexpr int kPopScan = 64;                 // scan of nu: geometric from nu_max down by 1e-7
constexpr int kPopRounds = 5;                // 33-way multisection rounds per crossing

__constant__ double kGL4x[kPopGL] = {-0.86113631159405258, -0.33998104358485626, 0.33998104358485626,
                                     0.86113631159405258};
__constant__ double kGL4w[kPopGL] = {0.34785484513745386, 0.65214515486254614, 0.65214515486254614,
                                     0.34785484513745386};

// ln R where interp_lnsig's cubic equals L: bisection over the decreasing table for the
// cell, then Newton steps on that cell's 4-point Lagrange cubic.
__device__ double lnr_of_lnsig(const double* lnsig, double lnr_lo, double dlnr, double L, int* err) {
    if (!(L <= lnsig[1] && L >= lnsig[kSigmaTable - 2])) {
        atomicOr(err, kErrSigmaRange);
        L = fmin(fmax(L, lnsig[kSigmaTable - 2]), lnsig[1]);
    }
    int lo = 1, hi = kSigmaTable - 2;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (lnsig[mid] >= L) lo = mid; else hi = mid;
    }
    const double f0 = lnsig[lo - 1], f1 = lnsig[lo], f2 = lnsig[lo + 1], f3 = lnsig[lo + 2];
    double t = f1 > f2 ? (f1 - L) / (f1 - f2) : 0.0;
    for (int it = 0; it < 6; it++) {
        const double t2 = t * t;
        const double p = -t * (t - 1.0) * (t - 2.0) / 6.0 * f0 + (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0 * f1 -
                         (t + 1.0) * t * (t - 2.0) / 2.0 * f2 + (t + 1.0) * t * (t - 1.0) / 6.0 * f3 - L;
        const double dp = -(3.0 * t2 - 6.0 * t + 2.0) / 6.0 * f0 + (3.0 * t2 - 4.0 * t - 1.0) / 2.0 * f1 -
                          (3.0 * t2 - 2.0 * t - 2.0) / 2.0 * f2 + (3.0 * t2 - 1.0) / 6.0 * f3;
        if (dp == 0.0) break;
        t = fmin(fmax(t - p / dp, -0.5), 1.5);
    }
    return lnr_lo + (lo + t) * dlnr;
}

struct Pop {
    double zeta0, lnmp, slope, lnm_lo, lnm_hi;   // zeta0 (M / M_p)^slope on [M_lo, M_hi)
};

struct PopArgs {
    const double* params;   // [walker][3]
    const double* effp;     // [walker][4]
    const double* growth;
    const double* lnsig;
    double lnr_lo, dlnr;
    double z[EOR21_MAX_Z];
    int n_z, n_walkers, max_radii, model;
    double delta_c, mu, h, omega_m, omega_l, rho_mean;
    const WalkerInfo* walkers;
    PairInfo* pairs;
    float* ftab;            // [pair][kFTab]
    int* err;
};

__device__ int make_pops(const PopArgs& a, const double* p, const double* q, double z, Pop* out) {
    const double ln1e10 = 23.025850929940457;
    if (a.model == 1) {
        int n = 0;
        out[n++] = Pop{p[0], ln1e10, q[0], log(virial_mass(p[2], z, a.h, a.omega_m, a.omega_l, a.mu)), INFINITY};
        if (q[1] > 0.0)
            out[n++] = Pop{q[1], ln1e10, q[2], log(virial_mass(q[3], z, a.h, a.omega_m, a.omega_l, a.mu)), INFINITY};
        return n;
    }
    // Sec. 5: zeta0 (T / T_F)^alpha on [10^4 K, T_F), zeta0 (T / T_F)^beta above; T ~ M^(2/3)
    const double lmf = log(virial_mass(p[2], z, a.h, a.omega_m, a.omega_l, a.mu));
    const double lmc = log(virial_mass(4.0, z, a.h, a.omega_m, a.omega_l, a.mu));
    int n = 0;
    if (lmc < lmf) out[n++] = Pop{p[0], lmf, 2.0 * q[0] / 3.0, lmc, lmf};
    out[n++] = Pop{p[0], lmf, 2.0 * q[1] / 3.0, fmax(lmf, lmc), INFINITY};
    return n;
}

__global__ void __launch_bounds__(32 * kPopWarps) k_pop_tables(PopArgs a) {
    __shared__ double s_c[kPopWarps][kPopNodes];   // e^(-y/2) / sqrt(2) of each node
    __shared__ double s_a[kPopWarps][kPopNodes];   // Gauss-Legendre weight x zeta(M(y)) / sqrt(pi)
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long task = (long long)blockIdx.x * kPopWarps + wid;
    const int pair = (int)(task / a.max_radii), j = (int)(task % a.max_radii);
    if (pair >= a.n_walkers * a.n_z) return;   // warp-uniform exits
    PairInfo& P = a.pairs[pair];
    const int n_r = P.n_r;
    if (j >= n_r) return;
    const int w = pair / a.n_z, zi = pair % a.n_z;
    const double* p = a.params + 3 * w;
    const double* q = a.effp + 4 * w;
    bool ok = true;
    for (int i = 0; i < 4; i++) ok = ok && isfinite(q[i]);
    ok = ok && fabs(q[0]) <= 10.0 && fabs(q[a.model == 1 ? 2 : 1]) <= 10.0;
    if (a.model == 1) ok = ok && q[1] >= 0.0 && q[3] > 0.0 && q[3] < 12.0;
    if (!ok) {
        if (lane == 0) {
            atomicOr(a.err, kErrParam);
            P.delta_crit[j] = INFINITY;
            P.delta_hi[j] = INFINITY;
        }
        return;
    }
    Pop pops[kPopMax];
    const int np = make_pops(a, p, q, a.z[zi], pops);
    const double g2 = a.growth[zi] * a.growth[zi];
    const double ln_mass_r3 = log(4.0 / 3.0 * kPi * a.rho_mean);   // ln M = this + 3 ln R
    const double r = a.walkers[w].radii[j];
    const double lnm_r = ln_mass_r3 + 3.0 * log(r);
    const double s_r = g2 * interp_lnsig(a.lnsig, a.lnr_lo, a.dlnr, r, a.err);
    double f_c = 0.0, ds_max = 0.0;
    double tail_z[kPopMax] = {0.0, 0.0}, tail_c[kPopMax] = {0.0, 0.0};
    int nb[kPopMax] = {0, 0}, ne[kPopMax] = {0, 0};
    int base = 0;
    for (int i = 0; i < np; i++) {
        const Pop pp = pops[i];
        nb[i] = ne[i] = base;
        if (lnm_r >= pp.lnm_lo && lnm_r < pp.lnm_hi) f_c += pp.zeta0 * exp(pp.slope * (lnm_r - pp.lnmp));
        if (pp.lnm_lo >= lnm_r) continue;
        const double ds_lo = g2 * interp_lnsig(a.lnsig, a.lnr_lo, a.dlnr, exp((pp.lnm_lo - ln_mass_r3) / 3.0), a.err) - s_r;
        if (!(ds_lo > 0.0)) continue;
        const double y_lo = log(ds_lo);
        double y_bot = y_lo - kPopPanels;
        bool tail = true;
        if (pp.lnm_hi < lnm_r) {
            const double ds_top =
                g2 * interp_lnsig(a.lnsig, a.lnr_lo, a.dlnr, exp((pp.lnm_hi - ln_mass_r3) / 3.0), a.err) - s_r;
            if (ds_top > 0.0 && log(ds_top) > y_bot) {
                y_bot = log(ds_top);
                tail = false;
            }
        }
        if (!(y_lo > y_bot)) continue;
        ds_max = fmax(ds_max, ds_lo);
        const int panels = max(1, min(kPopPanels, (int)ceil(y_lo - y_bot - 1e-9)));
        const double hp = (y_lo - y_bot) / panels;
        const int nn = panels * kPopGL;
        for (int k = lane; k < nn; k += 32) {
            const int pan = k / kPopGL, g = k % kPopGL;
            const double y = y_bot + (pan + 0.5 * (kGL4x[g] + 1.0)) * hp;
            const double lnr = lnr_of_lnsig(a.lnsig, a.lnr_lo, a.dlnr, log((s_r + exp(y)) / g2), a.err);
            const double lnm = ln_mass_r3 + 3.0 * lnr;
            s_c[wid][base + k] = exp(-0.5 * y) * 0.70710678118654752;
            s_a[wid][base + k] = 0.5 * hp * kGL4w[g] * pp.zeta0 * exp(pp.slope * (lnm - pp.lnmp)) * 0.56418958354775628;
        }
        if (tail) {
            tail_z[i] = pp.zeta0 * exp(pp.slope * (fmin(lnm_r, pp.lnm_hi) - pp.lnmp));
            tail_c[i] = exp(-0.5 * y_bot) * 0.70710678118654752;
        }
        ne[i] = base + nn;
        base += nn;
    }
    __syncwarp();
    auto F = [&](double nu) {   // efficiency-weighted collapsed fraction at nu > 0 (one lane)
        double f = 0.0;
        for (int i = 0; i < np; i++) {
            for (int k = nb[i]; k < ne[i]; k++) {
                const double t = nu * s_c[wid][k];
                if (t < 6.0) f += s_a[wid][k] * t * exp(-t * t);
            }
            if (tail_z[i] != 0.0) f += tail_z[i] * erfc(nu * tail_c[i]);
        }
        return f;
    };
    // scan nu_k = nu_max q^k (k < 64), then nu = 0 (the collapsed value)
    const double nu_max = ds_max > 0.0 ? 8.0 * sqrt(2.0 * ds_max) : 1.0;
    const double ratio = pow(1e-7, 1.0 / (kPopScan - 1));
    const unsigned full = 0xffffffffu;
    const bool s0 = F(nu_max * pow(ratio, lane)) >= 1.0, s1 = F(nu_max * pow(ratio, lane + 32)) >= 1.0;
    const unsigned long long bits =
        (unsigned long long)__ballot_sync(full, s0) | ((unsigned long long)__ballot_sync(full, s1) << 32);
    const bool sc = f_c >= 1.0;
    int ncross = 0, kc[2] = {0, 0};
    for (int k = 0; k < kPopScan; k++) {
        const bool bk = (bits >> k) & 1ull, bn = k + 1 < kPopScan ? ((bits >> (k + 1)) & 1ull) != 0 : sc;
        if (bk != bn) {
            if (ncross < 2) kc[ncross] = k;
            ncross++;
        }
    }
    double root[2] = {INFINITY, INFINITY};
    if ((bits & 1ull) || ncross > 2) {
        if (lane == 0) atomicOr(a.err, kErrShape);
        ncross = 0;
    }
    for (int c = 0; c < ncross; c++) {
        const int k = kc[c];
        const bool sa = (bits >> k) & 1ull;
        double nu_a = nu_max * pow(ratio, k), nu_b = k + 1 < kPopScan ? nu_max * pow(ratio, k + 1) : 0.0;
        for (int it = 0; it < kPopRounds; it++) {
            const double hh = (nu_a - nu_b) / 33.0;
            const bool sx = F(nu_b + (lane + 1) * hh) >= 1.0;
            const unsigned m = __ballot_sync(full, sx == sa);
            if (m == 0u) {
                nu_b = nu_b + 32.0 * hh;
            } else {
                const int l = __ffs(m) - 1;
                const double na = nu_b + (l + 1) * hh;
                nu_b = l == 0 ? nu_b : nu_b + l * hh;
                nu_a = na;
            }
        }
        root[c] = a.delta_c - 0.5 * (nu_a + nu_b);
    }
    if (lane == 0) {
        P.delta_crit[j] = ncross >= 1 ? (float)root[0] : INFINITY;
        P.delta_hi[j] = ncross == 2 ? (float)root[1] : INFINITY;
    }
    if (j == n_r - 1) {   // R_cell: the table of F for the partial ionization
        float* tab = a.ftab + (size_t)pair * kFTab;
        const double ht = nu_max / (kFTab - 1);
        for (int i = lane; i < kFTab; i += 32) tab[i] = (float)(i == 0 ? f_c : F(i * ht));
        if (lane == 0) {
            P.f_inv_h = (float)(1.0 / ht);
            P.zeta = 1.0f;
            P.cell_ok = 1.0f;
            P.inv_sqrt2s2_cell = 0.0f;
        }
    }
}

// W(kR) of each walker's radii on the grid's |m|^2 values, FP32: a 12-term series below
// x = 2 (the closed form cancels there in single precision), the closed form above.
__device__ __forceinline__ float tophat_f32(float x) {
    if (x < 2.0f) {
        float x2 = x * x, term = 1.0f, sum = 1.0f;
#pragma unroll
        for (int n = 0; n < 12; n++) {
            term *= -x2 / (float)((2 * n + 2) * (2 * n + 5));
            sum += term;
        }
        return sum;
    }
    float s, c;
    sincosf(x, &s, &c);
    return 3.0f * (s - x * c) / (x * x * x);
}

__global__ void k_window_tables(const WalkerInfo* walkers, int max_radii, int n_m2, float kf, float* wtab) {
    int m2 = blockIdx.x * blockDim.x + threadIdx.x;
    int wj = blockIdx.y;
    int w = wj / max_radii, j = wj % max_radii;
    if (m2 >= n_m2 || j >= walkers[w].n_r) return;
    float r = (float)walkers[w].radii[j];
    wtab[(size_t)wj * n_m2 + m2] = tophat_f32(kf * sqrtf((float)m2) * r);
}

__global__ void k_window_single(double r, int n_m2, float kf, float* wtab) {
    int m2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (m2 < n_m2) wtab[m2] = tophat_f32(kf * sqrtf((float)m2) * (float)r);
}

}  // namespace

cudaError_t build_cosmology_tables(eor_ctx* c) {
    const eor_config& g = c->cfg;
    double om_h2 = g.omega_m * g.h * g.h;
    double lnr_lo = log(kSigmaRlo), dlnr = (log(kSigmaRhi) - log(kSigmaRlo)) / (kSigmaTable - 1);
    trace_begin(c, kKOther);
    k_sigma2_shape<<<kSigmaTable + 1, 256, 0, c->stream>>>(lnr_lo, dlnr, kSigmaTable, 8.0 / g.h, om_h2,
                                                           g.n_s, c->d_lnsig);
    trace_end(c);
    trace_begin(c, kKOther);
    k_sigma2_normalise<<<1, 256, 0, c->stream>>>(c->d_lnsig, kSigmaTable, g.sigma8, c->d_cosmo_amp);
    trace_end(c);
    double* d_z = nullptr;
    cudaError_t e = cudaMallocAsync(&d_z, sizeof(double) * g.n_z, c->stream);
    if (e != cudaSuccess) return e;
    cudaMemcpyAsync(d_z, g.z, sizeof(double) * g.n_z, cudaMemcpyHostToDevice, c->stream);
    trace_begin(c, kKOther);
    k_growth<<<g.n_z, 128, 0, c->stream>>>(d_z, g.n_z, g.omega_m, 1.0 - g.omega_m, c->d_growth);
    trace_end(c);
    cudaFreeAsync(d_z, c->stream);
    double kf = 2.0 * kPi / g.box_mpc;
    // every mode of plane kz has |k| >= kf kz, so planes with kf kz >= k_hi hold no binned mode
    c->ps_planes = 0;
    while (c->ps_planes < c->nh && kf * c->ps_planes < g.k_hi) c->ps_planes++;
    trace_begin(c, kKOther);
    k_bin_table<<<(c->n_m2 + 255) / 256, 256, 0, c->stream>>>(c->n_m2, kf, g.k_lo, g.k_hi, g.n_bins,
                                                              c->d_bin_of_m2);
    trace_end(c);
    trace_begin(c, kKOther);
    k_chi2_bins<<<1, 64, 0, c->stream>>>(g.n_bins, g.k_lo, g.k_hi, g.chi2_k_lo, g.chi2_k_hi, c->d_chi2_use);
    trace_end(c);
    cudaMemsetAsync(c->d_nmodes, 0, sizeof(long long) * g.n_bins, c->stream);
    cudaMemsetAsync(c->d_ksum, 0, sizeof(double) * g.n_bins, c->stream);
    trace_begin(c, kKOther);
    k_mode_counts<<<256, 256, 0, c->stream>>>(c->n, kf, c->d_bin_of_m2, g.n_bins, c->d_nmodes, c->d_ksum);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t build_walker_tables(eor_ctx* c, int n_walkers) {
    const eor_config& g = c->cfg;
    WalkerTableArgs a{};
    a.params = c->d_params;
    a.growth = c->d_growth;
    a.lnsig = c->d_lnsig;
    a.lnr_lo = log(kSigmaRlo);
    a.dlnr = (log(kSigmaRhi) - log(kSigmaRlo)) / (kSigmaTable - 1);
    for (int j = 0; j < g.n_z; j++) a.z[j] = g.z[j];
    a.n_z = g.n_z;
    a.n_walkers = n_walkers;
    a.max_radii = c->max_radii;
    double dx = g.box_mpc / g.n;
    a.r_cell = g.r_cell_rule == 1 ? dx : cbrt(3.0 / (4.0 * kPi)) * dx;
    a.r_factor = g.r_factor;
    a.r_mfp_max = g.r_mfp_max;
    a.delta_c = g.delta_c;
    a.mu = g.mu;
    a.h = g.h; a.omega_m = g.omega_m; a.omega_l = 1.0 - g.omega_m; a.omega_b = g.omega_b;
    a.rho_mean = g.omega_m * kRhoCritH2 * g.h * g.h;
    a.walkers = c->d_walkers;
    a.pairs = c->d_pairs;
    a.err = c->d_err;
    int np = n_walkers * g.n_z;
    trace_begin(c, kKTables);
    k_walker_tables<<<(np + 3) / 4, 128, 0, c->stream>>>(a);   // one warp per (walker, redshift)
    trace_end(c);
    if (g.efficiency_model) {
        PopArgs pa{};
        pa.params = c->d_params;
        pa.effp = c->d_effp;
        pa.growth = c->d_growth;
        pa.lnsig = c->d_lnsig;
        pa.lnr_lo = a.lnr_lo;
        pa.dlnr = a.dlnr;
        for (int j = 0; j < g.n_z; j++) pa.z[j] = g.z[j];
        pa.n_z = g.n_z;
        pa.n_walkers = n_walkers;
        pa.max_radii = c->max_radii;
        pa.model = g.efficiency_model;
        pa.delta_c = g.delta_c;
        pa.mu = g.mu;
        pa.h = g.h; pa.omega_m = g.omega_m; pa.omega_l = 1.0 - g.omega_m;
        pa.rho_mean = a.rho_mean;
        pa.walkers = c->d_walkers;
        pa.pairs = c->d_pairs;
        pa.ftab = c->d_ftab;
        pa.err = c->d_err;
        const long long tasks = (long long)np * c->max_radii;
        trace_begin(c, kKTables);
        k_pop_tables<<<(unsigned)((tasks + kPopWarps - 1) / kPopWarps), 32 * kPopWarps, 0, c->stream>>>(pa);
        trace_end(c);
    }
    if (c->tune.method == kMethodDirect) {   // the per-radius windows only the direct method reads
        dim3 grid((c->n_m2 + 255) / 256, n_walkers * c->max_radii);
        trace_begin(c, kKTables);
        k_window_tables<<<grid, 256, 0, c->stream>>>(c->d_walkers, c->max_radii, c->n_m2,
                                                      (float)(2.0 * kPi / g.box_mpc), c->d_wtab);
        trace_end(c);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if ((e = build_walker_coefs(c, n_walkers)) != cudaSuccess) return e;
    if (c->tune.method == kMethodBasisTf32 && c->d_tcB) return build_columns(c, n_walkers);
    if (c->f16) return build_columns_f16(c, n_walkers);
    return cudaSuccess;
}

cudaError_t launch_window_table(eor_ctx* c, double r, float* wtab) {
    trace_begin(c, kKOther);
    k_window_single<<<(c->n_m2 + 255) / 256, 256, 0, c->stream>>>(r, c->n_m2,
                                                                  (float)(2.0 * kPi / c->cfg.box_mpc), wtab);
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
