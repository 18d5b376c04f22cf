/*
 * eor_oracle.h — plain FP64 CPU oracle of the excursion-set 21-cm likelihood path
 * (Greig & Mesinger 2015, "21CMMC", arXiv:1501.06576).
 *
 * TEST INFRASTRUCTURE ONLY. This header and eor_oracle.c exist to check the CUDA
 * path. Only tests/, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load them. They share no code, header, table or constant generator with the
 * CUDA library, and the CUDA library never calls them.
 *
 * Every step is written in the order the paper states it, in double precision,
 * with a textbook radix-2 FFT (brute-force DFT for other sizes). Nothing is
 * blocked, fused or reordered for speed beyond the OpenMP loops over
 * independent FFT lines and cells.
 *
 * Pins (tests/test_oracle_*.py check each against something other than itself):
 *   or_fft1d / or_fft3d      brute-force DFT (numpy matrix sums), Parseval, round trip
 *   or_tophat_w              scipy spherical Bessel j1: W(x) = 3 j1(x)/x, W(0) = 1
 *   or_sigma2                closed form for a white spectrum (sigma^2 = A / V_R),
 *                            scipy quadrature of j1 for n_s = 1, sigma(8/h) = sigma8
 *   or_growth                Einstein-de Sitter limit D = 1/(1+z); Carroll-Press-Turner
 *                            growth suppression within 1 %
 *   or_growth_rate           Einstein-de Sitter f = 1; the numerical derivative of ln D;
 *                            Linder's Omega_m(z)^0.55 within 1 %
 *   or_los_gradient          plane waves: along the line of sight the field itself, across
 *                            it zero, at 45 degrees half of it
 *   or_mmin                  the three halo masses printed in Sec. 3.1 / 4.1 (10^8.06,
 *                            10^8.78, 10^9.11 Msun at z = 8), tests/golden/mmin_paper.txt
 *   or_t0_mk                 27 mK at (1+z)/10 = 1, Omega_m h^2 = 0.15, Omega_b h^2 = 0.023
 *   or_ionize                brute force 8^3 (direct DFT sums), uniform-box closed form,
 *                            plane-wave closed form, x_HI in [0,1], monotone in zeta and T_vir
 *   or_power_spectrum        plane-wave single-bin closed form, Parseval, GRF P(k) recovery
 *   or_chi2                  closed-form bin selection (bins 2..11) and unit contributions
 *   or_dsigma2_dlnr          central differences of or_sigma2
 *   or_var_table / or_var_s  exact or_sigma2 at off-grid masses
 *   or_fcoll_pops            slope 0: zeta erfc (or_fcoll); a split mass range adds up to the
 *                            whole; delta_R -> delta_c: zeta(M_R); a pure power-law spectrum
 *                            without a region: the incomplete-gamma closed form
 *   or_ionize_pops           one slope-0 population: or_ionize's flags and x_HI
 *   or_bbks_transfer         parity unpinned beyond its q -> 0 limit: the coefficients are
 *                            Bardeen et al. (1986) App. G, which the paper does not print.
 */
#ifndef EOR_ORACLE_H
#define EOR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Flat LCDM cosmology (Sec. 1 lists the paper's values; workloads use their own). */
typedef struct {
    double h, omega_m, omega_l, omega_b, n_s, sigma8;
    int use_transfer;   /* 1: BBKS transfer function; 0: T(q) = 1 (pure power law, for pins) */
    double amp;         /* P(k) amplitude A, set by or_cosmo_init so sigma(8/h Mpc) = sigma8 */
} or_cosmo;

/* Knobs of the excursion-set step whose values the paper does not state. */
typedef struct {
    double r_factor;    /* ladder ratio R_j / R_{j+1} (1.1) */
    int r_cell_rule;    /* 0: R_cell = (3/(4 pi))^(1/3) dx (sphere of a cell's volume); 1: R_cell = dx */
    double delta_c;     /* linear collapse threshold (1.686) */
    double mu;          /* mean molecular weight in M_min (0.6) */
} or_ion_cfg;

void   or_set_threads(int n);          /* OpenMP threads (0 = library default) */
int    or_get_threads(void);

/* FFT: in place, unnormalised, sign -1 forward / +1 inverse; data as interleaved (re, im). */
void   or_fft1d(double* a, int n, int sign);
void   or_fft3d(double* a, int n, int sign);             /* n^3 row-major, z fastest */

/* Cosmology, all in Mpc (not Mpc/h) and solar masses. */
double or_bbks_transfer(double q);
void   or_cosmo_init(or_cosmo* c);
double or_pk(const or_cosmo* c, double k);               /* linear P(k) at z = 0, Mpc^3 */
double or_tophat_w(double x);                            /* 3 (sin x - x cos x) / x^3 */
double or_sigma2(const or_cosmo* c, double r);           /* sigma^2 of the top-hat radius r at z = 0 */
double or_growth(const or_cosmo* c, double z);           /* D(z), D(0) = 1 */
double or_growth_rate(const or_cosmo* c, double z);      /* f = d ln D / d ln a */
double or_rho_mean(const or_cosmo* c);                   /* mean matter density, Msun / Mpc^3 */
double or_mass_to_radius(const or_cosmo* c, double m);
double or_mmin(const or_cosmo* c, double tvir, double z, double mu);
double or_t0_mk(const or_cosmo* c, double z);            /* 21-cm brightness prefactor, mK */

/* R ladder R_mfp, R_mfp/f, ... down to R_cell; returns its length (writes at most cap radii). */
int    or_radius_ladder(const or_ion_cfg* cfg, int n, double box_mpc, double r_mfp, double* radii, int cap);
double or_r_cell(const or_ion_cfg* cfg, int n, double box_mpc);

/* Conditional collapsed fraction of Eq. 1 for one smoothed overdensity. */
double or_fcoll(double delta_r, double sigma2_min, double sigma2_r, double delta_c);

/* Mass-dependent ionizing efficiency (Sec. 5): a population of sources with
 * zeta(M) = zeta0 (M / m_pivot)^slope for m_lo <= M < m_hi (m_hi <= 0: no upper limit). */
typedef struct {
    double zeta0, m_pivot, slope, m_lo, m_hi;
} or_pop;

/* S(M) = D^2 sigma^2(R(M)) and dS/d ln M on a uniform ln M grid at one redshift (growth D),
 * interpolated by cubic Hermite polynomials. */
typedef struct {
    int n;
    double lnm0, dlnm;
    double* s;
    double* ds;
} or_var_table;

double or_dsigma2_dlnr(const or_cosmo* c, double r);      /* d sigma^2 / d ln R at z = 0 */
or_var_table* or_var_table_new(const or_cosmo* c, double growth, double m_lo, double m_hi, double dlnm);
void   or_var_table_free(or_var_table* t);
double or_var_s(const or_var_table* t, double lnm, double* dsdlnm);

/* sum_i Int zeta_i(M) dn/dM(M | delta_R, M_R) M / rho dM over population i's mass range below
 * M_R, with the extended Press-Schechter conditional mass function (first-crossing form);
 * delta_R >= delta_c gives sum_i zeta_i(M_R) over populations whose range holds M_R.
 * m_r <= 0: no region (S_R = 0; the unconditional fraction, delta_R < delta_c only). */
double or_fcoll_pops(const or_var_table* t, const or_pop* pops, int n_pops, double m_r, double delta_r,
                     double delta_c);

/* or_ionize with the populations' efficiency: flagged where the efficiency-weighted
 * collapsed fraction reaches 1 at some radius; partial ionization min(1, that fraction) at
 * R_cell. */
int    or_ionize_pops(const or_cosmo* c, const or_ion_cfg* cfg, int n, double box_mpc, double z,
                      const float* delta, const or_pop* pops, int n_pops, double r_mfp,
                      double* xhi, uint8_t* flag, double* dtb, double* xhi_mean);

/* delta_R = IDFT(W(kR) DFT(delta)) / n^3 for one radius; out: n^3 doubles. */
void   or_filter_box(int n, double box_mpc, const float* delta, double r, double* out);

/* IDFT(k_z^2/k^2 DFT(delta)) / n^3 along the last axis (line of sight); out: n^3 doubles.
 * Linear theory: dv_r/dr = -f H times this field (velocity-gradient term of delta T_b). */
void   or_los_gradient(int n, double box_mpc, const float* delta, double* out);

/* Excursion-set ionization of one box at redshift z for parameters (zeta, R_mfp, log10 T_vir).
 * Any output pointer may be NULL. Returns the ladder length. */
int    or_ionize(const or_cosmo* c, const or_ion_cfg* cfg, int n, double box_mpc, double z,
                 const float* delta, double zeta, double r_mfp, double log10_tvir,
                 double* xhi, uint8_t* flag, double* dtb, double* xhi_mean);

/* Spherically averaged power spectrum Delta^2(k) of a real n^3 box (Sec. 2.2), nbins
 * logarithmic bins on [k_lo, k_hi). Empty bins give NaN with nmodes 0. */
void   or_power_spectrum(int n, double box_mpc, const double* box, int nbins, double k_lo, double k_hi,
                         double* d2, double* kmean, int64_t* nmodes);

/* chi^2 over one redshift's bins whose geometric centre lies in [chi_lo, chi_hi] (Sec. 2.5). */
double or_chi2(int nbins, double k_lo, double k_hi, double chi_lo, double chi_hi,
               const double* d2, const int64_t* nmodes, const double* mock, const double* sigma);

#ifdef __cplusplus
}
#endif
#endif
