// eor_internal.cuh — data shared by the translation units of libeor21 (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/eor21.h"

namespace eor {

constexpr int kMaxRadii = EOR21_MAX_RADII;
constexpr int kSigmaTable = 1024;          // ln R grid of the sigma^2(R) table
constexpr double kSigmaRlo = 0.005;        // [Mpc]
constexpr double kSigmaRhi = 1000.0;       // [Mpc]
constexpr double kPi = 3.14159265358979323846;
constexpr double kRhoCritH2 = 2.775e11;    // 3 H0^2 / (8 pi G) in h^2 Msun / Mpc^3
constexpr int kBasisCand = 512;            // candidate radii of the filter basis
constexpr int kBasisMax = 48;              // largest filter basis
constexpr double kBasisTol = 1e-6;         // max |W - projection| over candidates and |k| (FP32 level)
constexpr int kCoefGrid = 8192;            // uniform R grid of the basis coefficient table
constexpr int kFTab = 1024;                // entries of a walker's partial-ionization table in nu

// Device error word bits (set by kernels, read by the host).
enum : int {
    kErrLadder = 1,       // a walker's ladder exceeds the table size
    kErrSigmaRange = 2,   // a radius outside the sigma^2 table
    kErrParam = 4,        // non-finite or out-of-range walker parameter
    kErrTimeout = 8,      // a bounded tensor-core wait ran out
    kErrShape = 16,       // a mass-dependent efficiency whose zeta f_coll crosses 1 more than twice
};

// Per (walker, redshift): everything the fused kernels need.
struct PairInfo {
    int w, zi, n_r, pad;
    float zeta;              // ionizing efficiency
    float t0;                // brightness prefactor T0(z) [mK]
    float inv_sqrt2s2_cell;  // 1 / sqrt(2 (sigma^2_min - sigma^2(R_cell))) or 0 when <= 0
    float cell_ok;           // 1 when R_cell's mass exceeds M_min, else 0
    float f_inv_h;           // > 0: partial ionization from the pair's table in nu (step 1 / f_inv_h)
    float pad2[3];
    float delta_crit[kMaxRadii];   // delta_R >= delta_crit  <=>  zeta f_coll >= 1 (+inf: never)
    float delta_hi[kMaxRadii];     // ... and delta_R <= delta_hi (+inf except for a falling efficiency)
};

// erfc(x) for x >= 0 from the Chebyshev fit of Numerical Recipes (Press et al. 1992, Sec. 6.2,
// "erfcc"; fractional error below 1.2e-7 everywhere): t = 1 / (1 + x/2) and
// erfc(x) = t exp(-x^2 + P(t)) with P a degree-9 polynomial. Branch-free. The exponential is
// CUDA's fast __expf (a few ulp, and |-x^2 + P| of at most ~30 for the arguments that matter:
// below 2e-6 relative in erfc, 2e-6 of x_HI at most) and the reciprocal CUDA's fast
// __fdividef (about 2 ulp in t: a few 1e-7 relative in erfc). The correctly rounded
// reciprocal made this function about a third of the pencil pass's instructions.
__device__ __forceinline__ float erfc_cheb(float x) {
    const float t = __fdividef(1.0f, fmaf(0.5f, x, 1.0f));
    float p = 0.17087277f;
    p = fmaf(p, t, -0.82215223f);
    p = fmaf(p, t, 1.48851587f);
    p = fmaf(p, t, -1.13520398f);
    p = fmaf(p, t, 0.27886807f);
    p = fmaf(p, t, -0.18628806f);
    p = fmaf(p, t, 0.09678418f);
    p = fmaf(p, t, 0.37409196f);
    p = fmaf(p, t, 1.00002368f);
    p = fmaf(p, t, -1.26551223f);
    return t * __expf(fmaf(-x, x, p));
}

// Efficiency-weighted collapsed fraction at nu = delta_c - delta_R from a pair's table
// (kFTab values at nu = i / inv_h; nu <= 0: the collapsed-region value in entry 0), by
// Catmull-Rom cubic interpolation (end intervals use a linearly extrapolated neighbour),
// clamped at 0.
__device__ __forceinline__ float pop_table_f(const float* tab, float nu, float inv_h) {
    if (!(nu > 0.0f)) return tab[0];
    const float x = nu * inv_h;
    if (x >= (float)(kFTab - 1)) return tab[kFTab - 1];
    const int i = (int)x;
    const float t = x - (float)i;
    const float p1 = tab[i], p2 = tab[i + 1];
    const float p0 = i > 0 ? tab[i - 1] : 2.0f * p1 - p2;
    const float p3 = i + 2 < kFTab ? tab[i + 2] : 2.0f * p2 - p1;
    const float c3 = 3.0f * (p1 - p2) + p3 - p0, c2 = 2.0f * p0 - 5.0f * p1 + 4.0f * p2 - p3;
    return fmaxf(0.0f, fmaf(0.5f * t, p2 - p0 + t * (c2 + t * c3), p1));
}

// Per walker (FP64 ladder, kept for diagnostics).
struct WalkerInfo {
    int n_r, pad[3];
    double radii[kMaxRadii];
};

// Cosmology constants the table kernels need.
struct CosmoParams {
    double h, omega_m, omega_l, omega_b, n_s, sigma8;
    double amp;          // P(k) amplitude (set after the sigma_8 integral)
    double rho_mean;     // Msun / Mpc^3
};

// Kernel classes of the tracing facility (eor_trace).
enum KernelClass : int {
    kKTables = 0,      // per-walker tables and window tables
    kKFilterPlane = 1, // pass 1: filter + inverse plane FFT
    kKPencil = 2,      // pass 2: C2R pencils + flag (+ x_HI, delta T_b, R2C)
    kKPsPlane = 3,     // forward plane FFT + shell sums
    kKFinish = 4,      // x_HI means, spectra, chi^2
    kKForward = 5,     // density spectrum (once per box)
    kKOther = 6,       // cosmology tables and diagnostics
    kKBasis = 7,       // basis contraction + flag + x_HI + delta T_b
    kKClasses = 8
};

enum Method : int { kMethodBasis = 0, kMethodDirect = 1, kMethodBasisSimt = 2, kMethodBasisTf32 = 3 };

struct Tuning {
    int group;          // radii per pencil launch (G)
    int pairs;          // (walker, redshift) pairs in flight (P)
    int plane_threads;  // CTA size of the 128^3 plane kernels (512 or 1024)
    int method;         // kMethodBasis, kMethodDirect, kMethodBasisSimt or kMethodBasisTf32
    int ps_split;       // spectrum tiling: 0 slab + x-line passes (n <= 128), 1 one CTA per plane, 2 a cluster (n = 128)
    int ps_streams;     // 2: the spectrum's plane passes overlap the next batch's pencil pass; 1: in turn
};

}  // namespace eor

struct eor_ctx {
    eor_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // the power spectrum's plane passes run on stream2, overlapping the next batch's pencil pass
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_pencil[2] = {nullptr, nullptr}, ev_plane[2] = {nullptr, nullptr};
    int device = 0;
    int n = 0, nh = 0, n_m2 = 0, max_radii = 0;
    size_t n3 = 0, nspec = 0;
    eor::CosmoParams cosmo{};
    eor::Tuning tune{8, 16, 512, eor::kMethodBasis, 0, 2};

    // device buffers
    float* d_delta = nullptr;        // [n_z][n^3]
    float* d_bright = nullptr;       // [n_z][n^3] (1 + delta) H/(dv_r/dr + H) - 1 when cfg.rsd, else unused
    float2* d_spec = nullptr;        // [n_z][nh][n][n]
    double* d_lnsig = nullptr;       // ln sigma^2(R) at z = 0 on the ln R grid
    double* d_growth = nullptr;      // [2][n_z]: D(z), then f = d ln D / d ln a
    double* d_cosmo_amp = nullptr;   // [1] P(k) amplitude
    signed char* d_bin_of_m2 = nullptr;   // [n_m2] bin of |m|^2 or -1
    signed char* d_chi2_use = nullptr;    // [n_bins] 1 where the bin enters chi^2
    long long* d_nmodes = nullptr;   // [n_bins]
    double* d_ksum = nullptr;        // [n_bins]
    double* d_params = nullptr;      // [max_walkers][3]
    double* d_effp = nullptr;        // [max_walkers][4] efficiency-model parameters (eor_set_efficiency)
    float* d_ftab = nullptr;         // [max_walkers][n_z][kFTab] partial-ionization tables (models 1, 2)
    int eff_walkers = 0;             // walkers whose efficiency parameters are set
    eor::WalkerInfo* d_walkers = nullptr;
    eor::PairInfo* d_pairs = nullptr;
    float* d_wtab = nullptr;         // [max_walkers][max_radii][n_m2]
    float2* d_inter = nullptr;       // [G*P][nspec]
    uint32_t* d_flags = nullptr;     // [P][flag words per pair]
    float2* d_psinter = nullptr;     // [2][P][nspec] (two halves: pencil and plane passes overlap)
    double* d_ps_sum = nullptr;      // [max_walkers][n_z][n_bins]
    double* d_xhi_sum = nullptr;     // [max_walkers][n_z]
    double* d_chi2 = nullptr;        // [max_walkers]
    double* d_mock = nullptr;        // [n_z][n_bins] x 2 (mock, sigma)
    double* d_d2 = nullptr;          // [max_walkers][n_z][n_bins]
    double* d_kmean = nullptr;       // [max_walkers][n_z][n_bins]
    long long* d_nmodes_pair = nullptr;   // [max_walkers][n_z][n_bins]
    double* d_xhi_mean = nullptr;    // [max_walkers][n_z]
    float* d_xhi_out = nullptr;      // optional [max_walkers][n_z][n^3]
    float* d_scratch_box = nullptr;  // [n^3] diagnostics
    eor::PairInfo* d_diag_pair = nullptr;   // one-task table for diagnostics
    float* d_diag_wtab = nullptr;    // [n_m2] window of one radius
    double* d_diag_ps = nullptr;     // [4][n_bins] sums, d2, kmean, (counts as double)
    long long* d_diag_cnt = nullptr; // [n_bins]
    int* d_err = nullptr;
    size_t flag_words = 0;

    // filter basis (radius-batched method)
    int n_kd = 0, basis_rank = 0, kb = 0, ncc = 1;
    double basis_residual = 0.0, coef_h = 0.0, coef_r_lo = 0.0;
    int* d_kd_m2 = nullptr;          // [n_m2] distinct |m|^2, ascending
    int* d_m2_to_kd = nullptr;       // [n_m2] index into the distinct list or -1
    double* d_basis = nullptr;       // [kBasisMax][n_m2] orthonormal basis on the distinct |k|
    double* d_coef_tab = nullptr;    // [kBasisMax][kCoefGrid] c_b(R)
    float* d_phi_m2 = nullptr;       // [kBasisMax][n_m2] FP32 basis on the |m|^2 index
    float* d_F = nullptr;            // [n_z][kb][n^3] basis fields
    float* d_coef = nullptr;         // [max_walkers][max_radii][kb] walker coefficients
    float* d_dtb = nullptr;          // [max_walkers][n_z][n^3] delta T_b
    float* d_xpart = nullptr;        // [max_walkers][n_z][n^3/128] partial x_HI sums
    int* d_cols = nullptr;           // tensor-core column slots: (walker << 8 | radius) or -1
    int* d_gmeta = nullptr;          // per group of 32 column slots: walker << 2 | first << 1 | last
    int* d_goff = nullptr;           // [max_walkers + 1] first group of each walker
    unsigned char* d_tcA = nullptr;  // tensor-core A operands of every CTA (TF32 hi/lo core matrices)
    unsigned char* d_tcB = nullptr;  // tensor-core coefficient chunks per redshift
    unsigned long long* d_xq = nullptr;   // [pairs] fixed-point x_HI sums of the tensor-core path
    // FP16 split contraction (step-function efficiency, basis rank <= 31)
    bool f16 = false;                // the tensor-core contraction runs on FP16 split operands
    int k16 = 0;                     // its K slots: 3 (rank + 1) rounded up to 16
    int num_sms = 0;                 // persistent grid size
    unsigned char* d_a16 = nullptr;  // [n_z][n^3 / 128][128 x k16 FP16] A operands
    unsigned char* d_b16 = nullptr;  // [n_z][chunk][256 x k16 FP16 + group records]
    float* d_fscale = nullptr;       // [n_z][32] power-of-two bound of |F_b|, then [n_z][32] scratch
    float* d_dcell = nullptr;        // [n_z][n^3] delta at R_cell
    uint32_t* d_fwords = nullptr;    // [max_walkers][n_z][n^3 / 32] Eq. 1 flags above R_cell
    int* d_ncols = nullptr;          // [1] number of columns
    int n_ready_tables = 0;
    int ps_planes = 0;               // kz planes holding a binned mode: kf kz < k_hi

    // state
    int stage = 0;                   // 0 created, 1 boxes, 2 params, 3 ionized, 4 spectra
    int n_walkers = 0;
    std::string err;

    // tracing: event pairs around each launch of the last call (or captured graph)
    bool trace_on = false;
    std::vector<cudaEvent_t> trace_events;
    std::vector<int> trace_class;
    int trace_used = 0;
    long long launches = 0;          // kernels launched by the last call
    long long graph_launches = 0;    // kernels in the captured graph

    // test-only failure injection of the tensor-core contraction (eor_debug_withhold)
    int dbg_withhold = -1;
    unsigned long long dbg_wait_ns = 0;

    // captured likelihood graphs, keyed by walker count
    cudaGraphExec_t graph_exec = nullptr;
    int graph_walkers = -1;
    bool graph_traced = false;
};

namespace eor {

// api.cu (tracing)
void trace_begin(eor_ctx* c, int cls);
void trace_end(eor_ctx* c);
void trace_begin_on(eor_ctx* c, int cls, cudaStream_t s);
void trace_end_on(eor_ctx* c, cudaStream_t s);
size_t estimate_launches(const eor_ctx* c);

// tables.cu
cudaError_t build_cosmology_tables(eor_ctx* c);
cudaError_t build_walker_tables(eor_ctx* c, int n_walkers);
// the partial-ionization tables when a mass-dependent efficiency is on, else nullptr
inline const float* pop_tables(const eor_ctx* c) { return c->cfg.efficiency_model ? c->d_ftab : nullptr; }

// basis.cu
cudaError_t build_basis(eor_ctx* c);
cudaError_t build_walker_coefs(eor_ctx* c, int n_walkers);
cudaError_t launch_basis_window(eor_ctx* c, double r, double* out);
cudaError_t launch_basis_ionize(eor_ctx* c, float* xhi_out);
cudaError_t prepare_basis_kernel(eor_ctx* c);
size_t basis_ionize_smem(int kb, int max_radii);
int basis_cells_per_cta();

// tcgen05.cu
size_t basis_tc_smem(bool pops);
bool basis_tc_fits(int rank);
size_t basis_tc_a_bytes(long long n3, int n_z);
size_t basis_tc_b_bytes(const eor_ctx* c);
size_t basis_tc_column_slots(const eor_ctx* c);
cudaError_t prepare_basis_tc(eor_ctx* c);
cudaError_t format_basis_tc(eor_ctx* c);
cudaError_t build_columns(eor_ctx* c, int n_walkers);
cudaError_t launch_basis_ionize_tc(eor_ctx* c, float* xhi_out);
bool basis_f16_fits(int rank);
int basis_f16_kslots(int rank);
size_t basis_f16_a_bytes(long long n3, int n_z, int rank);
size_t basis_f16_b_bytes(const eor_ctx* c);
size_t basis_f16_column_slots(const eor_ctx* c);
cudaError_t prepare_basis_f16(eor_ctx* c);
cudaError_t format_basis_f16(eor_ctx* c);
cudaError_t build_columns_f16(eor_ctx* c, int n_walkers);
cudaError_t launch_basis_ionize_f16(eor_ctx* c);
void launch_xq_finish(const unsigned long long* xq, int pairs, double* xhi_sum, cudaStream_t s);

// kernels.cu
cudaError_t prepare_kernels(int n);
cudaError_t launch_ps_from_boxes(eor_ctx* c, float* xhi_out);
cudaError_t prepare_box_ps_raw(int n);
cudaError_t launch_box_ps_raw(int n, const float* box, float2* spec, const signed char* bins, double* sums, int n_bins,
                              float kf3, const PairInfo* pair_info, cudaStream_t stream);

// api.cu: message returned by eor_last_error(NULL)
void set_global_error(const std::string& msg);
size_t flag_words_per_pair(int n);
cudaError_t launch_forward_spectrum(eor_ctx* c, int zi);
cudaError_t launch_ionization(eor_ctx* c, float* xhi_out);
cudaError_t launch_xhi_mean(eor_ctx* c);
cudaError_t launch_power_spectrum(eor_ctx* c);
cudaError_t launch_chi2(eor_ctx* c);
cudaError_t launch_filtered_density(eor_ctx* c, int zi, float* out, const float* wtab);
cudaError_t launch_window_table(eor_ctx* c, double r, float* wtab);
cudaError_t launch_box_power_spectrum(eor_ctx* c, const float* box);
cudaError_t launch_brightness_weight(eor_ctx* c, int zi);
cudaError_t launch_zeldovich(eor_ctx* c, int zi, float* work);
cudaError_t launch_noise_sigma(eor_ctx* c, const double* mock, const float* thermal, double model_frac, double* sums,
                               double* sigma);
// the field multiplying T0 x_HI in delta T_b, minus 1: delta, or the velocity-weighted form
inline const float* brightness_base(const eor_ctx* c) { return c->cfg.rsd ? c->d_bright : c->d_delta; }
bool grid_supported(int n);

}  // namespace eor
