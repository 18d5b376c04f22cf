/*
 * eor21.h — C ABI of libeor21, the GB300 (sm_103a) implementation of the data-parallel
 * hot path inside every likelihood call of 21CMMC (Greig & Mesinger 2015,
 * arXiv:1501.06576): the seminumerical excursion-set reionization step on fixed
 * density boxes, the 21-cm brightness temperature, its spherically averaged power
 * spectrum and the chi^2 against a mock.
 *
 * Call order (EOR_ESTATE otherwise):
 *   eor_create -> eor_init_boxes -> eor_set_params -> eor_run_ionization
 *              -> eor_power_spectrum -> eor_chi2
 * eor_likelihood runs set_params .. chi2 as one call (one CUDA-graph replay). With a
 * mass-dependent efficiency (eor_config.efficiency_model 1 or 2), eor_set_efficiency
 * comes before eor_set_params / eor_likelihood.
 *
 * Memory: the caller owns every pointer it passes; the library copies inputs and
 * never keeps a caller pointer past the call. The library owns its device memory
 * (cudaMalloc, or the allocator given in eor_config). A `mem` argument says where a
 * caller buffer lives: EOR_HOST (the call returns when the data is copied and the
 * outputs are ready) or EOR_DEVICE (a device pointer on the context's device; the
 * work is ordered on the context's stream and the call returns without waiting).
 *
 * Errors: every int-returning call gives EOR_OK (0) or a code below, and
 * eor_last_error() gives the message. No exception crosses the ABI, nothing aborts,
 * and no kernel traps: device-side checks set an error word that the host reads.
 *
 * Layouts (row-major, last index fastest):
 *   density boxes   float [n_z][n][n][n]      (x, y, z), box j at redshift cfg.z[j]
 *   walker params   double [n_walkers][3]     (zeta, R_mfp [Mpc], log10 T_vir [K])
 *   efficiency      double [n_walkers][4]     (efficiency_model 1 and 2, see eor_config)
 *   x_HI boxes      float [n_walkers][n_z][n][n][n]
 *   x_HI means      double [n_walkers][n_z]
 *   spectra         double [n_walkers][n_z][n_bins]  (Delta^2 in mK^2, mean |k| in 1/Mpc)
 *   mode counts     long long [n_walkers][n_z][n_bins]
 *   mock, sigma     double [n_z][n_bins]
 *   chi^2           double [n_walkers]
 */
#ifndef EOR21_H
#define EOR21_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define EOR21_MAX_Z 8
#define EOR21_MAX_BINS 64
#define EOR21_MAX_RADII 64

enum {
    EOR_OK = 0,
    EOR_EINVAL = 1,    /* bad size, NaN or out-of-range value, NULL where one is required */
    EOR_ENOMEM = 2,    /* device or host allocation failed */
    EOR_ECUDA = 3,     /* a CUDA call failed (message holds cudaGetErrorString) */
    EOR_ETIMEOUT = 4,  /* a bounded device-side wait ran out */
    EOR_ESTATE = 5,    /* call out of order */
    EOR_ENOTSUP = 6    /* grid size or option this build does not provide */
};

enum { EOR_HOST = 0, EOR_DEVICE = 1 };

typedef struct eor_ctx eor_ctx;   /* opaque, library-owned */

/* Problem description. eor_default_config fills the 128^3, 250 Mpc, z = 8, 9, 10
 * workload with the readings the library takes where the paper is silent. */
typedef struct {
    int n;                       /* grid side: 16, 32, 64, 128 or 256 */
    double box_mpc;              /* comoving box side L [Mpc] */
    int n_z;                     /* redshifts, 1..EOR21_MAX_Z */
    double z[EOR21_MAX_Z];
    double h, omega_m, omega_b, n_s, sigma8;   /* flat LCDM, Omega_Lambda = 1 - Omega_m */
    double r_factor;             /* ratio between successive filter radii (1.1) */
    int r_cell_rule;             /* 0: R_cell = radius of a sphere of one cell's volume; 1: cell side */
    double delta_c;              /* linear collapse threshold (1.686) */
    double mu;                   /* mean molecular weight in the T_vir -> M relation (0.6) */
    int n_bins;                  /* logarithmic k bins (14) */
    double k_lo, k_hi;           /* bin range [k_lo, k_hi) [1/Mpc] (0.1, 1.5) */
    double chi2_k_lo, chi2_k_hi; /* bins whose geometric centre lies here enter chi^2 (0.15, 1.0) */
    int max_walkers;             /* largest n_walkers passed to eor_set_params */
    double r_mfp_max;            /* largest R_mfp passed to eor_set_params [Mpc] (sizes tables) */
    /* Optional device allocator (both or neither); NULL: cudaMalloc / cudaFree. */
    void* (*dev_alloc)(size_t bytes, void* user);
    void (*dev_free)(void* ptr, void* user);
    void* alloc_user;
    /* Velocity-gradient factor of delta T_b (Sec. 2.2): 1 multiplies delta T_b by
     * H / (dv_r/dr + H) with linear peculiar velocities along the last box axis,
     * dv_r/dr / H = -f IDFT(k_z^2/k^2 delta_hat) (f = d ln D / d ln a), clipped to
     * [-rsd_max_dvdr, rsd_max_dvdr]; 0 (default) leaves the factor at 1. The factor is a
     * per-box field, formed once at eor_init_boxes. */
    int rsd;
    double rsd_max_dvdr;         /* 0.2 */
    /* 1: eor_init_boxes takes its boxes as linear density fields and evolves each with the
     * Zel'dovich approximation (Sec. 2.1): one unit-mass particle per cell displaced by
     * psi = IDFT(i k / k^2 delta_hat) and deposited back by cloud-in-cell weights (FP32
     * atomics: the evolved box can differ between loads in the last bits); the excursion set
     * and delta T_b then use the evolved field. 0 (default): the boxes are used as given. */
    int zeldovich;
    /* Ionizing efficiency. 0 (default): the step function of Sec. 3, zeta for every halo
     * above M_min(T_vir). 1 and 2: a mass-dependent efficiency (Sec. 5), Eq. 1 applied to
     * the efficiency-weighted collapsed fraction
     *     F(delta_R) = sum_i Int zeta_i(M) dn/dM(M | delta_R, R) M / rho dM
     * over each population's mass range below M_R = 4 pi R^3 rho / 3, with the extended
     * Press-Schechter conditional mass function (first-crossing form; F = sum_i zeta_i(M_R)
     * once delta_R >= delta_c); x_HII = min(1, F) at R_cell. Per walker the params of
     * eor_set_params and four numbers q of eor_set_efficiency:
     *   1: two populations zeta_i0 (M / 1e10 Msun)^alpha_i above M_min(T_vir,i):
     *      params (zeta_10, R_mfp, log10 T_vir,1), q (alpha_1, zeta_20, alpha_2, log10 T_vir,2);
     *   2: Sec. 5's feedback form zeta0 (T_vir / T_F)^alpha for 10^4 K <= T_vir < T_F and
     *      zeta0 (T_vir / T_F)^beta above T_F, mass slopes 2 alpha / 3 and 2 beta / 3 (T_vir ~
     *      M^(2/3) at fixed z): params (zeta0, R_mfp, log10 T_F), q (alpha, beta, 0, 0).
     * Per (walker, redshift, radius) FP64 on the GPU: the delta_R where F = 1 (Eq. 1 holds on
     * the interval between them), and at R_cell a table of F in delta_R. */
    int efficiency_model;
} eor_config;

/* Defaults: n = 128, L = 250 Mpc, z = {8, 9, 10}, (h, Omega_m, Omega_b, n_s, sigma_8) =
 * (0.68, 0.31, 0.02254/0.68^2, 0.96, 0.82), r_factor 1.1, r_cell_rule 0, delta_c 1.686,
 * mu 0.6 (the value that reproduces the halo masses printed in Sec. 3.1 and 4.1),
 * 14 bins on [0.1, 1.5), chi^2 bins 0.15..1.0 (Sec. 2.5), max_walkers 1, r_mfp_max 20,
 * rsd 0 (rsd_max_dvdr 0.2). */
void eor_default_config(eor_config* cfg);

/* Create a context on the current CUDA device, ordered on `cuda_stream` (a cudaStream_t;
 * NULL: a stream the context creates). Builds the FP64 cosmology tables on the GPU:
 * growth D(z), the top-hat mass variance sigma^2(R) (Sec. 2.1 via the collapsed fraction),
 * and the k-bin tables. *out is NULL on failure. */
int eor_create(const eor_config* cfg, void* cuda_stream, eor_ctx** out);

/* Load the fixed density boxes (Sec. 2.5: the likelihood samples one fixed realization)
 * and Fourier transform each once (R2C, FP32). delta: float [n_z][n][n][n], used as
 * given (delta T_b is proportional to 1 + delta). */
int eor_init_boxes(eor_ctx* ctx, const float* delta, int mem);

/* Set the walkers for the next run: params double [n_walkers][3] = (zeta, R_mfp [Mpc],
 * log10 T_vir [K]) with zeta > 0, 0 < R_mfp <= r_mfp_max, n_walkers <= max_walkers.
 * Builds per walker and redshift, in FP64 on the GPU: M_min(T_vir, z) (Sec. 2.1.3),
 * the radius ladder from R_mfp down to R_cell (Sec. 2.1), sigma^2 of every radius and
 * the overdensity at which zeta f_coll = 1 (Eq. 1); and per radius the FP32 top-hat
 * window W(kR) on the grid. */
int eor_set_params(eor_ctx* ctx, const double* params, int n_walkers, int mem);

/* Efficiency parameters of the walkers (efficiency_model 1 or 2; EOR_ESTATE otherwise):
 * q double [n_walkers][4] as eor_config.efficiency_model describes, host (mem EOR_HOST) or
 * device memory; copied. They stay in force for later eor_set_params / eor_likelihood calls
 * of up to n_walkers walkers (EOR_ESTATE for more). EOR_EINVAL for non-finite values,
 * |alpha| > 10, zeta_20 < 0 or log10 T_vir,2 outside (0, 12). */
int eor_set_efficiency(eor_ctx* ctx, const double* q, int n_walkers, int mem);

/* Excursion-set ionization (Eq. 1 and the partial ionization at R_cell of Sec. 2.1) of
 * every (walker, redshift): for each radius, filter the density spectrum with W(kR),
 * inverse-FFT and flag cells where zeta f_coll >= 1; cells never flagged get
 * x_HII = zeta f_coll(R_cell). Then delta T_b = T0(z) x_HI (1 + delta) (Sec. 2.2, with
 * T_S >> T_gamma and no velocity term). xhi (optional, float [n_walkers][n_z][n^3]) and
 * xhi_mean (optional, double [n_walkers][n_z]) receive the neutral fraction. The Fourier
 * transform and shell sums of delta T_b run here too, fused behind the last radius, so
 * delta T_b never goes to memory; eor_power_spectrum then only normalises the sums. */
int eor_run_ionization(eor_ctx* ctx, float* xhi, double* xhi_mean, int mem);

/* Spherically averaged 21-cm power spectrum Delta^2(k) = k^3 P(k) / (2 pi^2) of delta T_b
 * (Sec. 2.2): FFT (FP32), then per bin the mean over its modes (k != 0) of
 * k^3 |dx^3 DFT|^2 / (2 pi^2 V), accumulated in FP64. Bins with no mode give NaN.
 * d2 and kmean double [n_walkers][n_z][n_bins]; nmodes long long, same shape; each
 * pointer optional. */
int eor_power_spectrum(eor_ctx* ctx, double* d2, double* kmean, long long* nmodes, int mem);

/* chi^2 = sum over redshifts (Sec. 3.4) and over bins with geometric centre in
 * [chi2_k_lo, chi2_k_hi] (Sec. 2.5) of ((Delta^2 - mock) / sigma)^2, FP64. mock_d2 and
 * sigma double [n_z][n_bins] (sigma > 0 on the used bins); chi2 double [n_walkers]. */
int eor_chi2(eor_ctx* ctx, const double* mock_d2, const double* sigma, double* chi2, int mem);

/* set_params + run_ionization + power_spectrum + chi2 for a batch of walkers, replayed
 * as one captured CUDA graph per batch size. Same argument rules as those calls; d2
 * (optional) receives the spectra. */
int eor_likelihood(eor_ctx* ctx, const double* params, int n_walkers, const double* mock_d2,
                   const double* sigma, double* chi2, double* d2, int mem);

/* Diagnostics through the same kernels. eor_filtered_density: the density of box
 * z_index smoothed by the top-hat of radius r_mpc, float [n][n][n].
 * eor_density_spectrum: the box's R2C half spectrum as float pairs (re, im) in the
 * layout [kz][kx][ky] with kz = 0..n/2. eor_walker_ladder: walker w's radii (double,
 * up to EOR21_MAX_RADII) and their count, after eor_set_params. */
int eor_filtered_density(eor_ctx* ctx, int z_index, double r_mpc, float* out, int mem);
int eor_density_spectrum(eor_ctx* ctx, int z_index, float* out, int mem);
/* The density box z_index the likelihood uses (the evolved one with zeldovich = 1),
 * float [n][n][n]. */
int eor_density_box(eor_ctx* ctx, int z_index, float* out, int mem);
int eor_walker_ladder(eor_ctx* ctx, int walker, double* radii, int* n_radii);

/* Power spectrum of any real box on the context's grid (Sec. 2.2 definition, the same
 * kernels as eor_power_spectrum): box float [n][n][n]; d2, kmean double [n_bins] and
 * nmodes long long [n_bins], each optional. Needs only eor_create. */
int eor_box_power_spectrum(eor_ctx* ctx, const float* box, double* d2, double* kmean, long long* nmodes,
                           int mem);

/* Total uncertainty of mock spectra per bin (Sec. 2.4's T+S equation, Sec. 2.5's modelling
 * error): sigma_b^2 = (sum over the bin's modes i of 1 / (N_i + mock_b)^2)^-1
 * + (model_frac mock_b)^2, over the modes of the full grid (k != 0) in the context's bins.
 * mock_d2 double [n_z][n_bins]; thermal (optional, NULL = no thermal noise) float
 * [n_z][n/2 + 1][n][n]: the per-mode thermal noise Delta^2_N in the half-spectrum layout
 * [kz][kx][ky], shared by each mode's conjugate; sigma double [n_z][n_bins], NaN where a bin
 * has no mode. Uses only the context's grid and bins (needs only eor_create). */
int eor_noise_sigma(eor_ctx* ctx, const double* mock_d2, const float* thermal, double model_frac, double* sigma,
                    int mem);

/* Launch schedule of eor_run_ionization / eor_likelihood (results do not depend on it):
 * group = radii per pencil launch (1..16), pairs = (walker, redshift) pairs in flight
 * (1..64; scratch memory grows with pairs, and with group * pairs while EOR_METHOD_DIRECT
 * is chosen), plane_threads = CTA size of the
 * 128^3 plane kernels (512 or 1024; ignored for smaller grids). Defaults 8, 16, 512.
 * Reallocates the scratch buffers and drops the captured graph. */
int eor_set_tuning(eor_ctx* ctx, int group, int pairs, int plane_threads);

/* The tiling of the power spectrum's 3D transform. split 0 (default; n <= 128, the basis
 * methods) = slab passes: one CTA per x slab forms the real input (delta T_b from the flag
 * contraction's flags, or the stored boxes), transforms it along z and y in shared memory
 * (about 68 KB at n = 128, three CTAs per SM), then one CTA per (kz plane, 32 y slots)
 * transforms along x and adds the shell sums. split 1 = a pencil pass along z, then one CTA
 * per n x n kz plane (132 KB at n = 128); split 2 (n = 128) = the same with a cluster of two
 * CTAs per plane (each holds 64 rows, transforms them, then 64 columns reading the other half
 * through distributed shared memory). The direct method always runs split 1 or 2 (0 reads as
 * 1 there); n = 256 runs its own row and column passes. EOR_ENOTSUP for 2 at n != 128 and for
 * 0 at n > 128; EOR_EINVAL outside 0..2. Drops the captured graph. eor_get_tuning reads the
 * current schedule (each pointer optional; ps_split reads 1 where the choice does not apply). */
int eor_set_ps_split(eor_ctx* ctx, int split);
/* Streams of the basis methods' power spectrum: 2 (default) = the plane pass of a batch of
 * (walker, redshift) pairs runs on a second stream of the context while the pencil pass of the
 * next batch runs (a double-buffered intermediate; the two streams fork and join by events,
 * also inside the captured graph); 1 = the two passes in turn on the context's stream. Drops
 * the captured graph. */
int eor_set_ps_streams(eor_ctx* ctx, int streams);
int eor_get_tuning(const eor_ctx* ctx, int* group, int* pairs, int* plane_threads, int* ps_split, int* ps_streams);

/* Autotuner of the launch schedule (results depend on it only through the FP32 rounding of
 * the spectrum's transforms and partial sums): times eor_likelihood on
 * these walkers (arguments as there, n_walkers <= max_walkers) with CUDA events on the
 * context's stream, `reps` graph replays per candidate after one warm-up, over the
 * candidates of the current method -- pairs in {4, 8, 16, 32} (and 64 for the basis methods
 * with more than 32 (walker, redshift) pairs) x the spectrum's tiling
 * (split 0 at n <= 128; 128^3 grids also split 2, and split 1 with plane_threads 512 or
 * 1024; split 1 and 512 otherwise) x ps_streams in {2, 1}, and for EOR_METHOD_DIRECT (one
 * stream, splits 1 and 2) also group in {4, 8, 16} and plane_threads -- and keeps the
 * fastest (eor_set_tuning,
 * eor_set_ps_split, eor_set_ps_streams). group, pairs, plane_threads and ms (mean
 * milliseconds of one call) receive the choice, each optional; eor_get_tuning gives the
 * rest. Tracing is off while it runs and is restored afterwards. */
int eor_autotune(eor_ctx* ctx, const double* params, int n_walkers, const double* mock_d2, const double* sigma,
                 int reps, int* group, int* pairs, int* plane_threads, double* ms, int mem);

/* How the radius loop is evaluated (results agree to FP32 rounding; see the parity tests):
 * EOR_METHOD_BASIS (default): every walker's filtered fields are assembled from a small
 *   set of basis fields F_b = IDFT(phi_b delta_hat), built once per density box, with the
 *   top-hat W(kR) = sum_b c_b(R) phi_b(k) to 1e-6 on the grid's |k| for every R in
 *   [R_cell, r_mfp_max]; the threshold and the OR over radii are fused into that
 *   contraction, which runs on the tensor cores (tcgen05, FP32 accumulation) on
 *   power-of-two-scaled FP16 operands split into hi + lo parts (three products side by side
 *   along K) when the basis has at most 31 functions, else on the FP32 units; it yields the
 *   Eq. 1 flags, and x_HI, delta T_b and the spectrum follow in the spectrum's passes
 *   (eor_set_ps_split), delta T_b never stored.
 * EOR_METHOD_BASIS_TF32: the same contraction on TF32 hi + lo operands (three products per
 *   K step of 8, x_HI and delta T_b in its epilogue): the previous form, kept for comparison
 *   (its operands are allocated when it is chosen).
 * EOR_METHOD_BASIS_SIMT: the same contraction on the FP32 units only.
 * EOR_METHOD_DIRECT: a filter and inverse FFT of the density spectrum for every radius
 *   (its group x pairs half spectra of scratch are allocated when it is chosen and released
 *   when another method is, its per-radius window tables on its first choice; EOR_ENOMEM
 *   leaves the method unchanged).
 * eor_basis_info gives the basis size and its largest residual |W - sum c phi|. A bounded
 * tensor-core wait that runs out makes the call return EOR_ETIMEOUT. */
enum { EOR_METHOD_BASIS = 0, EOR_METHOD_DIRECT = 1, EOR_METHOD_BASIS_SIMT = 2, EOR_METHOD_BASIS_TF32 = 3 };
int eor_set_method(eor_ctx* ctx, int method);
int eor_basis_info(const eor_ctx* ctx, int* rank, double* max_residual);
/* The contraction the current method runs: *kind = EOR_CONTRACT_NONE (the direct method),
 * EOR_CONTRACT_FP32 (FP32 units), EOR_CONTRACT_TF32 (tcgen05, TF32 hi/lo) or
 * EOR_CONTRACT_FP16 (tcgen05, FP16 hi/lo along K); *k_slots = the K extent of its MMA operands
 * (0 for the first two). */
enum { EOR_CONTRACT_NONE = 0, EOR_CONTRACT_FP32 = 1, EOR_CONTRACT_TF32 = 2, EOR_CONTRACT_FP16 = 3 };
int eor_contraction_info(const eor_ctx* ctx, int* kind, int* k_slots);
/* Test-only failure injection (off by default; not part of the method). With step >= 0,
 * every CTA of the tensor-core contraction withholds the epilogue's release of the
 * accumulator buffer of its step-th accumulator tile (a step is one coefficient chunk against
 * one tile of cells; each CTA counts its steps over all the cells it takes), and the MMA
 * thread's wait for that release (before step + 2, the same buffer) gives up after about
 * wait_ms milliseconds (counted in SM clock cycles at the highest SM clock; longer in wall
 * time at a lower clock) instead of 2 s. The wait that gives up records role 2 (MMA),
 * barrier 7 (accumulator free) and the step; the CTA then stops issuing, waits for its MMAs
 * and copies already in flight, frees its tensor memory and exits, and the next call that
 * reads the context's error word (eor_set_params, or eor_likelihood with host buffers)
 * returns EOR_ETIMEOUT, its message naming the first role, barrier and step that gave up. No
 * asynchronous copy or MMA is made to time out. step < 0 switches the injection off. The
 * captured likelihood graph is rebuilt at the next call. */
int eor_debug_withhold(eor_ctx* ctx, int step, double wait_ms);

/* Diagnostic of the basis reformulation: w[m2] = sum_b c_b(R) phi_b(k) for R = r_mpc and
 * k = (2 pi / box_mpc) sqrt(m2), m2 = 0 .. 3 (n/2)^2 (double [3 (n/2)^2 + 1]; NaN where no
 * mode of the grid has that |m|^2), from the FP64 basis and coefficient table, so that a
 * caller can compare it with the top-hat W(kR) = 3 (sin x - x cos x)/x^3 of Sec. 2.1.
 * r_mpc must lie in [R_cell, r_mfp_max] (EOR_EINVAL otherwise). Host output needs
 * 8 (3 (n/2)^2 + 1) <= 4 n^3 bytes (every n >= 16 here). */
int eor_basis_window(eor_ctx* ctx, double r_mpc, double* w, int mem);

/* Tracing (not part of the method). With tracing on, every kernel launch of the
 * following calls is bracketed by CUDA events on the context's stream, also inside the
 * captured graph of eor_likelihood (switching tracing re-captures it). eor_trace_read
 * waits for the stream and sums, per kernel class, the event-timed milliseconds and the
 * launches of the last call: classes 0..EOR21_KERNEL_CLASSES-1 are named by
 * eor_kernel_class_name. eor_launch_count: kernels the last call launched (for
 * eor_likelihood, the kernels of one graph replay), traced or not. */
#define EOR21_KERNEL_CLASSES 8
int eor_trace(eor_ctx* ctx, int enable);
int eor_trace_read(eor_ctx* ctx, double* total_ms, long long* launches, int n_classes);
const char* eor_kernel_class_name(int cls);
long long eor_launch_count(const eor_ctx* ctx);

/* Allocation-free power spectrum of one box. The paper has no counterpart: this is a
 * service for callers that cannot allocate GPU memory where they need the result, such as
 * applications that give all device memory to their own pool or budget (a cudaMalloc
 * outside it fails or breaks their accounting) and code that must not synchronize the
 * device (cudaMalloc and cudaFree can). It needs no context and calls no cudaMalloc,
 * cudaFree or allocating library routine: its scratch (the box's half spectrum, the bin of
 * every |m|^2, the shell sums and mode counts) is one static device array of
 * EOR21_NOALLOC_SCRATCH_BYTES bytes, held by every GPU that loads the library until the
 * process exits; n is at most EOR21_NOALLOC_MAX_N (larger n gives EOR_EINVAL). Same
 * definition as eor_box_power_spectrum: box is a device pointer to float [n][n][n]; d2
 * (double [n_bins]) and nmodes (long long [n_bins], optional) are device pointers; bins
 * are n_bins logarithmic bins on [k_lo, k_hi) for a box of side box_mpc. The library sees
 * only raw pointers, so the caller must pass buffers of those types and sizes on the
 * current device (the Python binding checks them). The work is ordered on cuda_stream
 * (NULL: the legacy default stream) and the call returns without waiting. The first call
 * on a device looks up the array's device address, and the first call for each n on a
 * device sets the shared-memory limits of its two FFT kernels, with that device current:
 * make those first calls before any stream capture. All calls share the array and the
 * last call's contents stay in it (each call clears what it accumulates): calls that
 * overlap on the GPU race, so issue them on one stream. Errors: EOR_EINVAL, EOR_ECUDA;
 * message via eor_last_error(NULL). */
#define EOR21_NOALLOC_MAX_N 128
#define EOR21_NOALLOC_SCRATCH_BYTES (9u << 20)
int eor_box_power_spectrum_noalloc(int n, double box_mpc, int n_bins, double k_lo, double k_hi, const float* box,
                                   double* d2, long long* nmodes, void* cuda_stream);

/* Check of the tensor-core (tcgen05, TF32) path on the current device: D = A B^T with
 * A float [128][32], B float [n][32] (n a multiple of 16, 16..256) and D float [128][n],
 * all device pointers, through the same operand layout, descriptors and tensor-memory
 * reads as the tensor-core contraction; err (device int) gets bit 0 set if the MMA did not
 * complete within its bounded wait. Ordered on cuda_stream, no wait. Not part of the
 * method: a diagnostic of the build on this GPU. */
int eor_tensor_core_check(const float* a, const float* b, float* d, int n, int* err, void* cuda_stream);

/* ------------------------------------------------------------------------------------
 * Learned surrogate of the power spectrum (not in the paper: a service around it).
 *
 * An ensemble of multilayer perceptrons maps a walker's (zeta, R_mfp, log10 T_vir) and a
 * redshift to log10 Delta^2 in the n_bins bins of Sec. 2.2, so that a likelihood call can
 * skip the simulation for walkers where the ensemble is trusted; every other walker runs
 * the full excursion-set simulation above (the "fallback"), which also generates the
 * training set and judges the surrogate's error.
 *
 * Network of each member: inputs x = (zeta, R_mfp, log10 T_vir, z), each mapped linearly
 * from its prior interval onto [-1, 1] (z from [min z, max z]); hidden layers
 * h = GELU(W h' + b), GELU(u) = u Phi(u); output y = W h' + b, with
 * log10 Delta^2_b = mean_b + std_b y_b (mean and std of the training targets per bin).
 * Weights are used rounded to bfloat16 (round to nearest even); sums and activations are
 * FP32. Training: mean squared error of y over samples and bins, Adam (beta 0.9, 0.999,
 * eps 1e-8) on FP32 master weights, the gradient passing the bf16 rounding unchanged.
 *
 * Parameter vector of one member (float, eor_emu_n_params values): layer by layer from
 * the input, W [fan_out][fan_in] then b [fan_out]; members follow one another.
 *
 * Fallback rule: a walker is simulated instead of emulated when, at any redshift, the
 * largest per-bin standard deviation of the members' log10 Delta^2 exceeds the threshold
 * tau (set by eor_emu_calibrate or eor_emu_set_threshold; +infinity before), when a
 * predicted bin lies below 10 x d2_floor, or when its parameters leave the prior box.
 * The network's inputs are (zeta, R_mfp, log10 T_vir, z): it emulates the step-function
 * efficiency only, and eor_emu_likelihood returns EOR_ENOTSUP for a context with
 * efficiency_model 1 or 2.
 * -------------------------------------------------------------------------------------- */
#define EOR21_EMU_MAX_HIDDEN 8
#define EOR21_EMU_MAX_MEMBERS 8

typedef struct eor_emu eor_emu;   /* opaque, library-owned */

typedef struct {
    int n_z;                     /* redshifts covered (the z input), 1..EOR21_MAX_Z */
    double z[EOR21_MAX_Z];
    int n_bins;                  /* outputs: log10 Delta^2 per bin, 1..EOR21_MAX_BINS */
    int hidden;                  /* width of every hidden layer, 4..1024 (256) */
    int n_hidden;                /* hidden layers, 1..EOR21_EMU_MAX_HIDDEN (3) */
    int members;                 /* ensemble size, 1..EOR21_EMU_MAX_MEMBERS (4) */
    int max_rows;                /* largest minibatch, and largest walkers x n_z of one prediction (16384) */
    int max_samples;             /* largest training set in samples = walkers x n_z (65536) */
    double prior_lo[3], prior_hi[3];   /* box of (zeta, R_mfp, log10 T_vir): (5, 5, 4) .. (100, 20, 6) */
    double d2_floor;             /* Delta^2 floor before log10 [mK^2] (1e-2) */
    double err_tol;              /* per-bin relative error the fallback guards (0.05) */
    unsigned long long seed;     /* weight initialisation */
} eor_emu_config;

/* Defaults above for the 128^3, z = 8, 9, 10 workload's 14 bins. */
void eor_emu_default_config(eor_emu_config* cfg);

/* Create on the current device, ordered on cuda_stream (NULL: own stream); weights are
 * initialised uniform in +-sqrt(3 / fan_in) (biases 0) from a counter-based SplitMix64
 * stream keyed by cfg.seed and the member. */
int eor_emu_create(const eor_emu_config* cfg, void* cuda_stream, eor_emu** out);
long long eor_emu_n_params(const eor_emu* emu);   /* per member */

/* Training set: params double [n_walkers][3] and the simulated spectra d2 double
 * [n_walkers][n_z][n_bins] (eor_likelihood's d2). Targets are log10 max(d2, d2_floor)
 * (NaN -> floor); their per-bin mean and standard deviation (FP64) become the output
 * normalisation. n_walkers x n_z <= max_samples. */
int eor_emu_set_data(eor_emu* emu, const double* params, const double* d2, int n_walkers, int mem);

/* `steps` Adam steps of every member on minibatches of `batch` samples drawn with
 * replacement (SplitMix64 keyed by seed, member and step), learning rate lr decaying by
 * a cosine from lr to lr / 50 over the call. One captured CUDA graph per step, replayed.
 * loss (optional, double [members], host): mean minibatch loss of the last min(steps, 64)
 * steps. */
int eor_emu_train(eor_emu* emu, int steps, int batch, double lr, unsigned long long seed, double* loss);

/* Diagnostics of the training kernels on a caller batch shared by all members:
 * x float [n][4] (network inputs), t float [n][n_bins] (standardised targets), n <= max_rows.
 * eor_emu_forward: y float [members][n][n_bins]. eor_emu_loss_grad: loss double [members]
 * and grad float [members][n_params]. eor_emu_train_batch: `steps` full-batch Adam steps at
 * the constant rate lr; loss (optional) double [members] of the last step. */
int eor_emu_forward(eor_emu* emu, const float* x, int n, float* y, int mem);
int eor_emu_loss_grad(eor_emu* emu, const float* x, const float* t, int n, double* loss, float* grad, int mem);
int eor_emu_train_batch(eor_emu* emu, const float* x, const float* t, int n, int steps, double lr, double* loss,
                        int mem);

/* Master weights float [members][n_params] out or in (set resets Adam's moments and step
 * count), and the output normalisation double [2][n_bins] = (mean, std), std > 0. */
int eor_emu_get_weights(eor_emu* emu, float* w, int mem);
int eor_emu_set_weights(eor_emu* emu, const float* w, int mem);
int eor_emu_get_normalization(eor_emu* emu, double* mean_std);
int eor_emu_set_normalization(eor_emu* emu, const double* mean_std);

/* Ensemble prediction for walkers params double [n_walkers][3] at every redshift
 * (n_walkers x n_z <= max_rows): log10_d2 double [n_walkers][n_z][n_bins] (members'
 * mean), spread double [n_walkers][n_z] (largest per-bin standard deviation over members,
 * in dex) and fallback int [n_walkers] (1: the rule above sends it to the simulation);
 * each output optional. */
int eor_emu_predict(eor_emu* emu, const double* params, int n_walkers, double* log10_d2, double* spread,
                    int* fallback, int mem);

/* Choose tau on validation walkers with simulated spectra d2 (as in eor_emu_set_data): the
 * largest threshold (capped at the largest score seen) such that at least `recall` of
 * the walkers whose emulated Delta^2 misses the simulated one by more than err_tol in some
 * bin with modes are sent to the simulation. tau (optional) and frac (optional: fraction
 * of these walkers sent to the simulation) are host doubles. */
int eor_emu_calibrate(eor_emu* emu, const double* params, const double* d2, int n_walkers, double recall,
                      double* tau, double* frac, int mem);
int eor_emu_set_threshold(eor_emu* emu, double tau);

/* Likelihood of walkers (as eor_likelihood, whose arguments these follow) with the
 * surrogate: emulated walkers get Delta^2 = 10^prediction (NaN in bins without modes) and
 * chi^2 over them; the others run eor_likelihood on ctx (which must cover the same
 * redshifts and bins; its max_walkers bounds one simulation batch) and get its results.
 * fallback (optional) int [n_walkers]. The call reads the number of fallback walkers back
 * to the host once; n_walkers x n_z <= max_rows. */
int eor_emu_likelihood(eor_emu* emu, eor_ctx* ctx, const double* params, int n_walkers, const double* mock_d2,
                       const double* sigma, double* chi2, double* d2, int* fallback, int mem);

/* Where predictions (eor_emu_predict, eor_emu_calibrate, eor_emu_likelihood) run: 1 = the
 * 5th-generation tensor cores (tcgen05 BF16 x BF16, FP32 accumulation; every layer input,
 * activations included, rounded to BF16), the default when the network has 3 hidden layers
 * of 256 and at most 16 bins; 0 = the FP32 units (BF16-rounded weights, FP32 activations,
 * the arithmetic of training). EOR_ENOTSUP for 1 with another shape. eor_emu_inference
 * gives the current choice. */
int eor_emu_set_inference(eor_emu* emu, int tensor_cores);
int eor_emu_inference(const eor_emu* emu);

const char* eor_emu_last_error(const eor_emu* emu);
void eor_emu_destroy(eor_emu* emu);

/* ------------------------------------------------------------------------------------
 * Affine-invariant ensemble sampler on the device (Sec. 2.4: Goodman & Weare 2010, as in
 * emcee / CosmoHammer), with the optional neutral-fraction prior of Sec. 3.3.
 *
 * One step updates the two halves of the ensemble in turn: walker k of the active half picks
 * a partner j of the other half, draws z from g(z) ~ 1/sqrt(z) on [1/a, a], proposes
 * Y = X_j + z (X_k - X_j) and accepts with probability min(1, z^2 p(Y) / p(X_k)), where
 * log p = -chi^2 / 2 (eor_likelihood's chi^2 on the context) inside the flat prior box and,
 * when xhi_prior_z >= 0, only where the mean neutral fraction at redshift index xhi_prior_z
 * is >= xhi_prior_min; -infinity elsewhere. A half's proposals are evaluated as one batch by
 * the context's captured likelihood graph; between steps nothing goes to the host.
 * Random numbers: SplitMix64 keyed by seed; draw c (partner, stretch, accept) of walker k in
 * half h of step s is output ((2 s + h) n_walkers + k) 3 + c, uniform = top 53 bits / 2^53.
 * Without a context (ctx NULL) the target is the Gaussian log p = -(y - mean)^T P (y - mean)/2
 * given in the config (gauss_target = 1): a check of the sampler itself.
 * -------------------------------------------------------------------------------------- */
typedef struct eor_mcmc eor_mcmc;   /* opaque, library-owned */

typedef struct {
    int n_walkers;                       /* even, >= 4; n_walkers / 2 <= the context's max_walkers */
    double a;                            /* stretch scale > 1 (2) */
    double prior_lo[3], prior_hi[3];     /* flat prior box of (zeta, R_mfp, log10 T_vir) */
    int xhi_prior_z;                     /* redshift index of the neutral-fraction prior, -1: none */
    double xhi_prior_min;                /* its lower limit (0.05, Sec. 3.3) */
    unsigned long long seed;
    int gauss_target;                    /* 1: Gaussian test target (ctx NULL) */
    double gauss_mean[3], gauss_precision[9];
} eor_mcmc_config;

void eor_mcmc_default_config(eor_mcmc_config* cfg);   /* 128 walkers, a = 2, the workloads' prior box */
/* ctx: the likelihood (boxes loaded); it must outlive the sampler, which runs on its stream.
 * The sampled parameters are (zeta, R_mfp, log10 T_vir). With a mass-dependent efficiency
 * (efficiency_model 1 or 2) the four efficiency parameters are held fixed: the
 * likelihood of proposal slot i (of each half-ensemble call) uses row i of
 * eor_set_efficiency, which must cover n_walkers / 2 rows (equal rows fix them for all). */
int eor_mcmc_create(const eor_mcmc_config* cfg, eor_ctx* ctx, eor_mcmc** out);
/* Starting walkers params double [n_walkers][3], mock and sigma as for eor_likelihood
 * (ignored without a context); lnp (optional) double [n_walkers] receives their log
 * posteriors. Resets the step count. */
int eor_mcmc_start(eor_mcmc* m, const double* params, const double* mock_d2, const double* sigma, double* lnp,
                   int mem);
/* `steps` steps; each optional output gets one row per step after both halves moved:
 * chain double [steps][n_walkers][3], lnp double [steps][n_walkers], accepted int
 * [steps][n_walkers] (1 where the walker's last proposal was accepted). */
int eor_mcmc_run(eor_mcmc* m, int steps, double* chain, double* lnp, int* accepted, int mem);
/* Current walkers (double [n_walkers][3]) and their log posteriors, each optional. */
int eor_mcmc_walkers(eor_mcmc* m, double* params, double* lnp, int mem);
const char* eor_mcmc_last_error(const eor_mcmc* m);
void eor_mcmc_destroy(eor_mcmc* m);

/* Message of the last failed call on ctx. With ctx NULL: the message of the calling host
 * thread's last failed call that has no context (eor_create, eor_box_power_spectrum_noalloc,
 * eor_tensor_core_check); that message is kept per thread, so threads that fail such calls
 * at the same time do not overwrite each other's. */
const char* eor_last_error(const eor_ctx* ctx);
const char* eor_version(void);
void eor_destroy(eor_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
