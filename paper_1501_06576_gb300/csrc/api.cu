// api.cu — the extern "C" boundary of libeor21: context lifetime, argument checks,
// host <-> device copies and the order of kernel launches. No step of the method runs
// on the host; the host only sizes buffers and sequences launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "eor_internal.cuh"

using eor::kPi;

namespace {

const char* kVersion = "libeor21 0.1 (sm_103a)";
thread_local std::string g_create_error;

int fail(eor_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

int cuda_fail(eor_ctx* c, cudaError_t e, const char* what) {
    return fail(c, EOR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
    } while (0)

void* dev_alloc(eor_ctx* c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (c->cfg.dev_alloc) return c->cfg.dev_alloc(bytes, c->cfg.alloc_user);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(eor_ctx* c, void* p) {
    if (!p) return;
    if (c->cfg.dev_free) c->cfg.dev_free(p, c->cfg.alloc_user);
    else cudaFree(p);
}

template <class T>
bool alloc_n(eor_ctx* c, T** out, size_t count) {
    *out = static_cast<T*>(dev_alloc(c, sizeof(T) * count));
    return *out != nullptr;
}

// Half spectra held by d_inter: the direct method filters group x pairs of them per launch;
// the other methods use one (the filtered-density and box diagnostics).
size_t inter_slots(int method, int pairs, int group) {
    return method == eor::kMethodDirect ? (size_t)pairs * group : 1;
}

// Number of radii of the ladder that starts at r_mfp: used only to size tables and the
// launch schedule (the ladders themselves are built on the device).
int ladder_bound(const eor_config& g, double r_mfp) {
    double dx = g.box_mpc / g.n;
    double r_cell = g.r_cell_rule == 1 ? dx : cbrt(3.0 / (4.0 * kPi)) * dx;
    int count = 0;
    double r = r_mfp;
    while (r > r_cell && count <= EOR21_MAX_RADII) {
        count++;
        r = r / g.r_factor;
    }
    return count + 1;
}

int copy_in(eor_ctx* c, void* dst, const void* src, size_t bytes, int mem) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, mem == EOR_DEVICE ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy in");
    return EOR_OK;
}

int copy_out(eor_ctx* c, void* dst, const void* src, size_t bytes, int mem) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, mem == EOR_DEVICE ? cudaMemcpyDeviceToDevice
                                                                        : cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "copy out");
    return EOR_OK;
}

int finish(eor_ctx* c, int mem) {
    if (mem == EOR_HOST) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
    return EOR_OK;
}

int check_device_error(eor_ctx* c) {
    int words[2] = {0, 0};
    cudaError_t e = cudaMemcpy(words, c->d_err, sizeof(words), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "read error word");
    const int err = words[0];
    if (err & eor::kErrParam) return fail(c, EOR_EINVAL, "walker parameter non-finite or out of range "
                                                         "(zeta > 0, 0 < R_mfp <= r_mfp_max, 0 < log10 T_vir < 12)");
    if (err & eor::kErrLadder) return fail(c, EOR_EINVAL, "radius ladder longer than the tables (raise r_mfp_max)");
    if (err & eor::kErrSigmaRange) return fail(c, EOR_EINVAL, "radius or halo mass outside the sigma^2 table range");
    if (err & eor::kErrShape)
        return fail(c, EOR_ENOTSUP, "mass-dependent efficiency: zeta f_coll crosses 1 more than twice in delta_R "
                                    "(Eq. 1 is then not one interval; not supported)");
    if (err & eor::kErrTimeout) {
        char where[96];
        snprintf(where, sizeof(where), " (first: role %d, barrier %d, step %d)", (words[1] >> 28) & 15,
                 (words[1] >> 20) & 255, words[1] & 0xFFFFF);
        return fail(c, EOR_ETIMEOUT, std::string("a bounded tensor-core wait ran out") + where);
    }
    return EOR_OK;
}

bool valid_mem(int mem) { return mem == EOR_HOST || mem == EOR_DEVICE; }

int run_params_to_chi2(eor_ctx* c) {
    cudaError_t e;
    if ((e = eor::build_walker_tables(c, c->n_walkers)) != cudaSuccess) return cuda_fail(c, e, "walker tables");
    if ((e = eor::launch_ionization(c, nullptr)) != cudaSuccess) return cuda_fail(c, e, "ionization");
    if ((e = eor::launch_xhi_mean(c)) != cudaSuccess) return cuda_fail(c, e, "x_HI mean");
    if ((e = eor::launch_power_spectrum(c)) != cudaSuccess) return cuda_fail(c, e, "power spectrum");
    if ((e = eor::launch_chi2(c)) != cudaSuccess) return cuda_fail(c, e, "chi2");
    return EOR_OK;
}

void trace_reset(eor_ctx* c) {
    c->trace_used = 0;
    c->trace_class.clear();
    c->launches = 0;
}

cudaError_t trace_reserve(eor_ctx* c, size_t pairs) {
    if (!c->trace_on) return cudaSuccess;
    while (c->trace_events.size() < 2 * pairs) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        c->trace_events.push_back(e);
    }
    return cudaSuccess;
}

}  // namespace

namespace eor {

void set_global_error(const std::string& msg) { g_create_error = msg; }

// Record on the context's stream; while the stream is being captured, as an external event
// node so the graph records it on every replay.
static void trace_record(cudaStream_t s, cudaEvent_t e) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &st);
    if (st == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else cudaEventRecord(e, s);
}

// The pair of events of one launch on stream s (the launch it brackets runs between them).
void trace_begin_on(eor_ctx* c, int cls, cudaStream_t s) {
    if (!c->trace_on) return;
    const size_t i = 2 * (size_t)c->trace_used;
    if (i + 1 >= c->trace_events.size()) return;   // pool sized beforehand; beyond it, untraced
    trace_record(s, c->trace_events[i]);
    c->trace_class.push_back(cls);
}

void trace_end_on(eor_ctx* c, cudaStream_t s) {
    c->launches++;
    if (!c->trace_on) return;
    const size_t i = 2 * (size_t)c->trace_used;
    if (i + 1 >= c->trace_events.size() || c->trace_class.size() != (size_t)c->trace_used + 1) return;
    trace_record(s, c->trace_events[i + 1]);
    c->trace_used++;
}

void trace_begin(eor_ctx* c, int cls) { trace_begin_on(c, cls, c->stream); }
void trace_end(eor_ctx* c) { trace_end_on(c, c->stream); }

}  // namespace eor

extern "C" {

void eor_default_config(eor_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->n = 128;
    cfg->box_mpc = 250.0;
    cfg->n_z = 3;
    cfg->z[0] = 8.0; cfg->z[1] = 9.0; cfg->z[2] = 10.0;
    cfg->h = 0.68; cfg->omega_m = 0.31; cfg->omega_b = 0.02254 / (0.68 * 0.68);
    cfg->n_s = 0.96; cfg->sigma8 = 0.82;
    cfg->r_factor = 1.1;
    cfg->r_cell_rule = 0;
    cfg->delta_c = 1.686;
    cfg->mu = 0.6;
    cfg->n_bins = 14; cfg->k_lo = 0.1; cfg->k_hi = 1.5;
    cfg->chi2_k_lo = 0.15; cfg->chi2_k_hi = 1.0;
    cfg->max_walkers = 1;
    cfg->r_mfp_max = 20.0;
    cfg->rsd = 0;
    cfg->rsd_max_dvdr = 0.2;
    cfg->zeldovich = 0;
    cfg->efficiency_model = 0;
}

const char* eor_version(void) { return kVersion; }

const char* eor_last_error(const eor_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void eor_destroy(eor_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    for (cudaEvent_t e : c->trace_events) cudaEventDestroy(e);
    void* bufs[] = {c->d_delta, c->d_bright, c->d_spec, c->d_lnsig, c->d_growth, c->d_cosmo_amp, c->d_bin_of_m2,
                    c->d_nmodes, c->d_ksum, c->d_params, c->d_walkers, c->d_pairs, c->d_wtab, c->d_inter,
                    c->d_flags, c->d_psinter, c->d_ps_sum, c->d_xhi_sum, c->d_chi2, c->d_mock, c->d_d2,
                    c->d_kmean, c->d_nmodes_pair, c->d_xhi_out, c->d_xhi_mean, c->d_scratch_box,
                    c->d_diag_pair, c->d_diag_wtab, c->d_diag_ps, c->d_diag_cnt, c->d_chi2_use, c->d_kd_m2,
                    c->d_m2_to_kd, c->d_basis, c->d_coef_tab, c->d_phi_m2, c->d_F, c->d_coef, c->d_dtb, c->d_xpart,
                    c->d_cols, c->d_gmeta, c->d_goff, c->d_ncols, c->d_tcA, c->d_tcB, c->d_xq, c->d_err,
                    c->d_a16, c->d_b16, c->d_fscale, c->d_dcell, c->d_fwords, c->d_effp, c->d_ftab};
    for (void* p : bufs) dev_free(c, p);
    for (cudaEvent_t e : {c->ev_fork, c->ev_pencil[0], c->ev_pencil[1], c->ev_plane[0], c->ev_plane[1]})
        if (e) cudaEventDestroy(e);
    if (c->stream2) cudaStreamDestroy(c->stream2);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int eor_create(const eor_config* cfg, void* cuda_stream, eor_ctx** out) {
    if (!out) return fail(nullptr, EOR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, EOR_EINVAL, "cfg is NULL");
    const eor_config& g = *cfg;
    if (!eor::grid_supported(g.n)) return fail(nullptr, EOR_ENOTSUP, "n must be 16, 32, 64, 128 or 256");
    if (!(g.box_mpc > 0.0) || !isfinite(g.box_mpc)) return fail(nullptr, EOR_EINVAL, "box_mpc must be > 0");
    if (g.n_z < 1 || g.n_z > EOR21_MAX_Z) return fail(nullptr, EOR_EINVAL, "n_z out of range");
    for (int j = 0; j < g.n_z; j++)
        if (!(g.z[j] >= 0.0) || !isfinite(g.z[j])) return fail(nullptr, EOR_EINVAL, "redshift must be >= 0");
    if (!(g.h > 0.0) || !(g.omega_m > 0.0 && g.omega_m <= 1.0) || !(g.omega_b > 0.0) || !(g.sigma8 > 0.0) ||
        !isfinite(g.n_s))
        return fail(nullptr, EOR_EINVAL, "cosmology out of range");
    if (!(g.r_factor > 1.0) || !(g.delta_c > 0.0) || !(g.mu > 0.0) || (g.r_cell_rule != 0 && g.r_cell_rule != 1))
        return fail(nullptr, EOR_EINVAL, "ionization settings out of range");
    if (g.n_bins < 1 || g.n_bins > EOR21_MAX_BINS || !(g.k_lo > 0.0) || !(g.k_hi > g.k_lo))
        return fail(nullptr, EOR_EINVAL, "bin settings out of range");
    if (g.max_walkers < 1 || !(g.r_mfp_max > 0.0)) return fail(nullptr, EOR_EINVAL, "max_walkers/r_mfp_max");
    if ((g.dev_alloc == nullptr) != (g.dev_free == nullptr))
        return fail(nullptr, EOR_EINVAL, "dev_alloc and dev_free come together");
    if ((g.rsd != 0 && g.rsd != 1) || (g.rsd && !(g.rsd_max_dvdr > 0.0 && g.rsd_max_dvdr < 1.0)))
        return fail(nullptr, EOR_EINVAL, "rsd must be 0 or 1, with 0 < rsd_max_dvdr < 1");
    if (g.zeldovich != 0 && g.zeldovich != 1) return fail(nullptr, EOR_EINVAL, "zeldovich must be 0 or 1");
    if (g.efficiency_model < 0 || g.efficiency_model > 2)
        return fail(nullptr, EOR_EINVAL, "efficiency_model must be 0, 1 or 2");

    eor_ctx* c = new (std::nothrow) eor_ctx();
    if (!c) return fail(nullptr, EOR_ENOMEM, "host allocation");
    c->cfg = g;
    cudaGetDevice(&c->device);
    if (cuda_stream) {
        c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("stream create: ") + cudaGetErrorString(e);
            delete c;
            return EOR_ECUDA;
        }
        c->own_stream = true;
    }
    {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream2, cudaStreamNonBlocking);
        for (cudaEvent_t* ev : {&c->ev_fork, &c->ev_pencil[0], &c->ev_pencil[1], &c->ev_plane[0], &c->ev_plane[1]})
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            g_create_error = std::string("second stream: ") + cudaGetErrorString(e);
            eor_destroy(c);
            return EOR_ECUDA;
        }
    }
    c->n = g.n;
    c->nh = g.n / 2 + 1;
    c->n3 = (size_t)g.n * g.n * g.n;
    c->nspec = (size_t)c->nh * g.n * g.n;
    c->n_m2 = 3 * (g.n / 2) * (g.n / 2) + 1;
    c->max_radii = ladder_bound(g, g.r_mfp_max);
    if (c->max_radii > EOR21_MAX_RADII) {
        eor_destroy(c);
        return fail(nullptr, EOR_EINVAL, "r_mfp_max gives more radii than EOR21_MAX_RADII");
    }
    const int P = c->tune.pairs, G = c->tune.group, W = g.max_walkers, Z = g.n_z, B = g.n_bins;
    const size_t pairs = (size_t)W * Z;
    c->flag_words = eor::flag_words_per_pair(g.n);
    bool ok = alloc_n(c, &c->d_delta, (size_t)Z * c->n3) && alloc_n(c, &c->d_spec, (size_t)Z * c->nspec) &&
              alloc_n(c, &c->d_lnsig, eor::kSigmaTable + 1) && alloc_n(c, &c->d_growth, 2 * (size_t)Z) &&
              alloc_n(c, &c->d_cosmo_amp, 1) && alloc_n(c, &c->d_bin_of_m2, c->n_m2) &&
              alloc_n(c, &c->d_nmodes, B) && alloc_n(c, &c->d_ksum, B) && alloc_n(c, &c->d_params, 3 * W) &&
              alloc_n(c, &c->d_walkers, W) && alloc_n(c, &c->d_pairs, pairs) &&
              alloc_n(c, &c->d_inter, inter_slots(c->tune.method, P, G) * c->nspec) &&
              alloc_n(c, &c->d_flags, (size_t)P * c->flag_words) && alloc_n(c, &c->d_psinter, 2 * (size_t)P * c->nspec) &&
              alloc_n(c, &c->d_ps_sum, pairs * B) && alloc_n(c, &c->d_xhi_sum, pairs) &&
              alloc_n(c, &c->d_xhi_mean, pairs) && alloc_n(c, &c->d_chi2, W) && alloc_n(c, &c->d_mock, 2 * Z * B) &&
              alloc_n(c, &c->d_d2, pairs * B) && alloc_n(c, &c->d_kmean, pairs * B) &&
              alloc_n(c, &c->d_nmodes_pair, pairs * B) && alloc_n(c, &c->d_scratch_box, c->n3) &&
              alloc_n(c, &c->d_diag_pair, 1) && alloc_n(c, &c->d_diag_wtab, c->n_m2) &&
              alloc_n(c, &c->d_diag_ps, 4 * B) && alloc_n(c, &c->d_diag_cnt, B) && alloc_n(c, &c->d_chi2_use, B) &&
              alloc_n(c, &c->d_kd_m2, c->n_m2) && alloc_n(c, &c->d_m2_to_kd, c->n_m2) &&
              alloc_n(c, &c->d_basis, (size_t)eor::kBasisMax * c->n_m2) &&
              alloc_n(c, &c->d_coef_tab, (size_t)eor::kBasisMax * eor::kCoefGrid) &&
              alloc_n(c, &c->d_phi_m2, (size_t)eor::kBasisMax * c->n_m2) && alloc_n(c, &c->d_err, 2);
    if (!ok) {
        eor_destroy(c);
        return fail(nullptr, EOR_ENOMEM, "device allocation failed");
    }
    cudaError_t e = eor::prepare_kernels(c->n);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int), c->stream);
    if (e == cudaSuccess) e = eor::build_cosmology_tables(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = eor::build_basis(c);
    if (e != cudaSuccess) {
        g_create_error = std::string("cosmology tables: ") + cudaGetErrorString(e);
        eor_destroy(c);
        return EOR_ECUDA;
    }
    c->ncc = (c->max_radii + 31) / 32;
    const size_t parts = c->n3 / 128;   // the finest x_HI partial sums (per warp of 128 cells)
    ok = alloc_n(c, &c->d_F, (size_t)Z * c->kb * c->n3) && alloc_n(c, &c->d_coef, (size_t)W * c->max_radii * c->kb) &&
         alloc_n(c, &c->d_dtb, pairs * c->n3) && alloc_n(c, &c->d_xpart, pairs * parts) &&
         alloc_n(c, &c->d_ncols, 1);
    // the tensor-core contraction: FP16 split operands for the step-function efficiency, TF32
    // split operands with a mass-dependent efficiency (interval flags, partial-ionization tables)
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (c->num_sms < 1) c->num_sms = 1;
    c->f16 = eor::basis_f16_fits(c->basis_rank);
    if (ok && c->f16) {   // (the TF32 contraction's operands are allocated when that method is chosen)
        c->k16 = eor::basis_f16_kslots(c->basis_rank);
        ok = alloc_n(c, &c->d_a16, eor::basis_f16_a_bytes((long long)c->n3, Z, c->basis_rank)) &&
             alloc_n(c, &c->d_b16, eor::basis_f16_b_bytes(c)) && alloc_n(c, &c->d_xq, pairs) &&
             alloc_n(c, &c->d_fscale, 2 * 32 * (size_t)Z) && alloc_n(c, &c->d_dcell, (size_t)Z * c->n3) &&
             alloc_n(c, &c->d_fwords, pairs * (c->n3 / 32)) &&
             alloc_n(c, &c->d_cols, eor::basis_f16_column_slots(c)) &&
             alloc_n(c, &c->d_gmeta, eor::basis_f16_column_slots(c) / 32) && alloc_n(c, &c->d_goff, (size_t)W + 1);
    }
    if (ok && g.rsd) ok = alloc_n(c, &c->d_bright, (size_t)Z * c->n3);
    if (ok && g.efficiency_model)
        ok = alloc_n(c, &c->d_effp, 4 * (size_t)W) && alloc_n(c, &c->d_ftab, pairs * eor::kFTab);
    if (!ok) {
        eor_destroy(c);
        return fail(nullptr, EOR_ENOMEM, "device allocation failed (basis fields)");
    }
    if ((e = eor::prepare_basis_kernel(c)) != cudaSuccess || (e = eor::prepare_basis_tc(c)) != cudaSuccess ||
        (e = eor::prepare_basis_f16(c)) != cudaSuccess) {
        g_create_error = std::string("basis kernel: ") + cudaGetErrorString(e);
        eor_destroy(c);
        return EOR_ECUDA;
    }
    *out = c;
    return EOR_OK;
}

int eor_init_boxes(eor_ctx* c, const float* delta, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (!delta || !valid_mem(mem)) return fail(c, EOR_EINVAL, "delta is NULL or bad mem");
    int r = copy_in(c, c->d_delta, delta, sizeof(float) * c->cfg.n_z * c->n3, mem);
    if (r) return r;
    float* zwork = nullptr;   // Zel'dovich displacement fields and deposit
    if (c->cfg.zeldovich && !alloc_n(c, &zwork, 4 * c->n3)) return fail(c, EOR_ENOMEM, "Zel'dovich work space");
    for (int zi = 0; zi < c->cfg.n_z; zi++) {
        cudaError_t e;
        if (c->cfg.zeldovich) {
            // linear spectrum -> displaced particles -> evolved box, then its spectrum below
            if ((e = eor::launch_forward_spectrum(c, zi)) != cudaSuccess ||
                (e = eor::launch_zeldovich(c, zi, zwork)) != cudaSuccess) {
                dev_free(c, zwork);
                return cuda_fail(c, e, "Zel'dovich evolution");
            }
        }
        e = eor::launch_forward_spectrum(c, zi);
        if (e != cudaSuccess) { dev_free(c, zwork); return cuda_fail(c, e, "forward spectrum"); }
        if (c->cfg.rsd && (e = eor::launch_brightness_weight(c, zi)) != cudaSuccess)
        {
            dev_free(c, zwork);
            return cuda_fail(c, e, "velocity-gradient factor");
        }
        // basis fields F_b = IDFT(phi_b delta_hat) of this box
        for (int b = 0; b < c->kb; b++) {
            e = eor::launch_filtered_density(c, zi, c->d_F + ((size_t)zi * c->kb + b) * c->n3,
                                             c->d_phi_m2 + (size_t)b * c->n_m2);
            if (e != cudaSuccess) {
                dev_free(c, zwork);
                return cuda_fail(c, e, "basis fields");
            }
        }
    }
    if (c->d_tcA || c->f16) {
        cudaError_t e = c->f16 ? eor::format_basis_f16(c) : cudaSuccess;
        if (e == cudaSuccess && c->d_tcA) e = eor::format_basis_tc(c);
        if (e != cudaSuccess) {
            dev_free(c, zwork);
            return cuda_fail(c, e, "tensor-core operands");
        }
    }
    r = finish(c, EOR_HOST);
    dev_free(c, zwork);
    if (r) return r;
    c->stage = 1;
    return EOR_OK;
}

int eor_set_efficiency(eor_ctx* c, const double* q, int n_walkers, int mem) {
    if (!c) return EOR_EINVAL;
    if (!c->cfg.efficiency_model) return fail(c, EOR_ESTATE, "efficiency_model is 0: no efficiency parameters");
    if (!q || !valid_mem(mem) || n_walkers < 1 || n_walkers > c->cfg.max_walkers)
        return fail(c, EOR_EINVAL, "q NULL, bad mem or n_walkers outside 1..max_walkers");
    if (mem == EOR_HOST) {
        for (int w = 0; w < n_walkers; w++) {
            const double* v = q + 4 * w;
            bool ok = isfinite(v[0]) && isfinite(v[1]) && isfinite(v[2]) && isfinite(v[3]) && fabs(v[0]) <= 10.0;
            if (c->cfg.efficiency_model == 1) ok = ok && fabs(v[2]) <= 10.0 && v[1] >= 0.0 && v[3] > 0.0 && v[3] < 12.0;
            else ok = ok && fabs(v[1]) <= 10.0;
            if (!ok)
                return fail(c, EOR_EINVAL, "efficiency parameter non-finite or out of range (|alpha| <= 10, "
                                           "zeta_20 >= 0, 0 < log10 T_vir,2 < 12)");
        }
    }
    int r = copy_in(c, c->d_effp, q, sizeof(double) * 4 * n_walkers, mem);
    if (r) return r;
    c->eff_walkers = n_walkers;
    if (c->stage > 1) c->stage = 1;   // the tables follow at the next eor_set_params
    return EOR_OK;
}

int eor_set_params(eor_ctx* c, const double* params, int n_walkers, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (c->stage < 1) return fail(c, EOR_ESTATE, "eor_init_boxes first");
    if (!params || !valid_mem(mem) || n_walkers < 1 || n_walkers > c->cfg.max_walkers)
        return fail(c, EOR_EINVAL, "params NULL, bad mem or n_walkers outside 1..max_walkers");
    if (c->cfg.efficiency_model && n_walkers > c->eff_walkers)
        return fail(c, EOR_ESTATE, "eor_set_efficiency for these walkers first");
    int r = copy_in(c, c->d_params, params, sizeof(double) * 3 * n_walkers, mem);
    if (r) return r;
    CK(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int), c->stream), "memset");
    c->n_walkers = n_walkers;
    CK(eor::build_walker_tables(c, n_walkers), "walker tables");
    CK(cudaStreamSynchronize(c->stream), "walker tables");
    r = check_device_error(c);
    if (r) { c->stage = 1; return r; }
    c->stage = 2;
    return EOR_OK;
}

int eor_run_ionization(eor_ctx* c, float* xhi, double* xhi_mean, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (c->stage < 2) return fail(c, EOR_ESTATE, "eor_set_params first");
    if (!valid_mem(mem)) return fail(c, EOR_EINVAL, "bad mem");
    const size_t pairs = (size_t)c->n_walkers * c->cfg.n_z;
    float* xhi_dev = nullptr;
    if (xhi) {
        if (mem == EOR_DEVICE) {
            xhi_dev = xhi;
        } else {
            if (!c->d_xhi_out && !alloc_n(c, &c->d_xhi_out, (size_t)c->cfg.max_walkers * c->cfg.n_z * c->n3))
                return fail(c, EOR_ENOMEM, "x_HI output buffer");
            xhi_dev = c->d_xhi_out;
        }
    }
    CK(eor::launch_ionization(c, xhi_dev), "ionization");
    CK(eor::launch_xhi_mean(c), "x_HI mean");
    int r;
    if (xhi && mem == EOR_HOST && (r = copy_out(c, xhi, xhi_dev, sizeof(float) * pairs * c->n3, mem))) return r;
    if (xhi_mean && (r = copy_out(c, xhi_mean, c->d_xhi_mean, sizeof(double) * pairs, mem))) return r;
    r = finish(c, mem);
    if (r) return r;
    c->stage = 3;
    return EOR_OK;
}

int eor_power_spectrum(eor_ctx* c, double* d2, double* kmean, long long* nmodes, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (c->stage < 3) return fail(c, EOR_ESTATE, "eor_run_ionization first");
    if (!valid_mem(mem)) return fail(c, EOR_EINVAL, "bad mem");
    CK(eor::launch_power_spectrum(c), "power spectrum");
    const size_t cnt = (size_t)c->n_walkers * c->cfg.n_z * c->cfg.n_bins;
    int r;
    if (d2 && (r = copy_out(c, d2, c->d_d2, sizeof(double) * cnt, mem))) return r;
    if (kmean && (r = copy_out(c, kmean, c->d_kmean, sizeof(double) * cnt, mem))) return r;
    if (nmodes && (r = copy_out(c, nmodes, c->d_nmodes_pair, sizeof(long long) * cnt, mem))) return r;
    r = finish(c, mem);
    if (r) return r;
    c->stage = 4;
    return EOR_OK;
}

int eor_chi2(eor_ctx* c, const double* mock_d2, const double* sigma, double* chi2, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (c->stage < 4) return fail(c, EOR_ESTATE, "eor_power_spectrum first");
    if (!mock_d2 || !sigma || !chi2 || !valid_mem(mem)) return fail(c, EOR_EINVAL, "NULL argument or bad mem");
    const size_t zb = (size_t)c->cfg.n_z * c->cfg.n_bins;
    int r;
    if ((r = copy_in(c, c->d_mock, mock_d2, sizeof(double) * zb, mem))) return r;
    if ((r = copy_in(c, c->d_mock + zb, sigma, sizeof(double) * zb, mem))) return r;
    CK(eor::launch_chi2(c), "chi2");
    if ((r = copy_out(c, chi2, c->d_chi2, sizeof(double) * c->n_walkers, mem))) return r;
    return finish(c, mem);
}

int eor_likelihood(eor_ctx* c, const double* params, int n_walkers, const double* mock_d2, const double* sigma,
                   double* chi2, double* d2, int mem) {
    if (!c) return EOR_EINVAL;
    if (c->stage < 1) return fail(c, EOR_ESTATE, "eor_init_boxes first");
    if (!params || !mock_d2 || !sigma || !chi2 || !valid_mem(mem) || n_walkers < 1 ||
        n_walkers > c->cfg.max_walkers)
        return fail(c, EOR_EINVAL, "NULL argument, bad mem or n_walkers outside 1..max_walkers");
    if (c->cfg.efficiency_model && n_walkers > c->eff_walkers)
        return fail(c, EOR_ESTATE, "eor_set_efficiency for these walkers first");
    const size_t zb = (size_t)c->cfg.n_z * c->cfg.n_bins;
    int r;
    if ((r = copy_in(c, c->d_params, params, sizeof(double) * 3 * n_walkers, mem))) return r;
    if ((r = copy_in(c, c->d_mock, mock_d2, sizeof(double) * zb, mem))) return r;
    if ((r = copy_in(c, c->d_mock + zb, sigma, sizeof(double) * zb, mem))) return r;
    CK(cudaMemsetAsync(c->d_err, 0, 2 * sizeof(int), c->stream), "memset");
    c->n_walkers = n_walkers;
    if (c->graph_walkers != n_walkers || c->graph_traced != c->trace_on) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
            c->graph_walkers = -1;
        }
        cudaGraph_t graph = nullptr;
        trace_reset(c);
        CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        int rr = run_params_to_chi2(c);
        cudaError_t ec = cudaStreamEndCapture(c->stream, &graph);
        if (rr) {
            if (graph) cudaGraphDestroy(graph);
            return rr;
        }
        if (ec != cudaSuccess) return cuda_fail(c, ec, "end capture");
        ec = cudaGraphInstantiate(&c->graph_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ec != cudaSuccess) return cuda_fail(c, ec, "graph instantiate");
        c->graph_walkers = n_walkers;
        c->graph_traced = c->trace_on;
        c->graph_launches = c->launches;
    }
    c->launches = c->graph_launches;
    CK(cudaGraphLaunch(c->graph_exec, c->stream), "graph launch");
    if ((r = copy_out(c, chi2, c->d_chi2, sizeof(double) * n_walkers, mem))) return r;
    if (d2 && (r = copy_out(c, d2, c->d_d2, sizeof(double) * n_walkers * zb, mem))) return r;
    r = finish(c, mem);
    if (r) return r;
    if (mem == EOR_HOST && (r = check_device_error(c))) return r;
    c->stage = 4;
    return EOR_OK;
}

int eor_filtered_density(eor_ctx* c, int z_index, double r_mpc, float* out, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (c->stage < 1) return fail(c, EOR_ESTATE, "eor_init_boxes first");
    if (!out || !valid_mem(mem) || z_index < 0 || z_index >= c->cfg.n_z || !(r_mpc >= 0.0) || !isfinite(r_mpc))
        return fail(c, EOR_EINVAL, "bad argument");
    CK(eor::launch_window_table(c, r_mpc, c->d_diag_wtab), "window table");
    float* dst = mem == EOR_DEVICE ? out : c->d_scratch_box;
    CK(eor::launch_filtered_density(c, z_index, dst, c->d_diag_wtab), "filtered density");
    int r;
    if (mem == EOR_HOST && (r = copy_out(c, out, dst, sizeof(float) * c->n3, mem))) return r;
    return finish(c, mem);
}

int eor_density_spectrum(eor_ctx* c, int z_index, float* out, int mem) {
    if (!c) return EOR_EINVAL;
    if (c->stage < 1) return fail(c, EOR_ESTATE, "eor_init_boxes first");
    if (!out || !valid_mem(mem) || z_index < 0 || z_index >= c->cfg.n_z) return fail(c, EOR_EINVAL, "bad argument");
    int r = copy_out(c, out, c->d_spec + (size_t)z_index * c->nspec, sizeof(float2) * c->nspec, mem);
    if (r) return r;
    return finish(c, mem);
}

int eor_density_box(eor_ctx* c, int z_index, float* out, int mem) {
    if (!c) return EOR_EINVAL;
    if (c->stage < 1) return fail(c, EOR_ESTATE, "eor_init_boxes first");
    if (!out || !valid_mem(mem) || z_index < 0 || z_index >= c->cfg.n_z) return fail(c, EOR_EINVAL, "bad argument");
    int r = copy_out(c, out, c->d_delta + (size_t)z_index * c->n3, sizeof(float) * c->n3, mem);
    if (r) return r;
    return finish(c, mem);
}

int eor_walker_ladder(eor_ctx* c, int walker, double* radii, int* n_radii) {
    if (!c) return EOR_EINVAL;
    if (c->stage < 2) return fail(c, EOR_ESTATE, "eor_set_params first");
    if (walker < 0 || walker >= c->n_walkers || !radii || !n_radii) return fail(c, EOR_EINVAL, "bad argument");
    eor::WalkerInfo wi;
    CK(cudaMemcpyAsync(&wi, c->d_walkers + walker, sizeof(wi), cudaMemcpyDeviceToHost, c->stream), "copy ladder");
    CK(cudaStreamSynchronize(c->stream), "copy ladder");
    *n_radii = wi.n_r;
    for (int j = 0; j < wi.n_r && j < EOR21_MAX_RADII; j++) radii[j] = wi.radii[j];
    return EOR_OK;
}

int eor_box_power_spectrum(eor_ctx* c, const float* box, double* d2, double* kmean, long long* nmodes, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (!box || !valid_mem(mem)) return fail(c, EOR_EINVAL, "box is NULL or bad mem");
    const float* src = box;
    int r;
    if (mem == EOR_HOST) {
        if ((r = copy_in(c, c->d_scratch_box, box, sizeof(float) * c->n3, mem))) return r;
        src = c->d_scratch_box;
    }
    CK(eor::launch_box_power_spectrum(c, src), "box power spectrum");
    const int nb = c->cfg.n_bins;
    if (d2 && (r = copy_out(c, d2, c->d_diag_ps + nb, sizeof(double) * nb, mem))) return r;
    if (kmean && (r = copy_out(c, kmean, c->d_diag_ps + 2 * nb, sizeof(double) * nb, mem))) return r;
    if (nmodes && (r = copy_out(c, nmodes, c->d_diag_cnt, sizeof(long long) * nb, mem))) return r;
    return finish(c, mem);
}

int eor_noise_sigma(eor_ctx* c, const double* mock_d2, const float* thermal, double model_frac, double* sigma,
                    int mem) {
    if (!c) return EOR_EINVAL;
    if (!mock_d2 || !sigma || !valid_mem(mem) || !(model_frac >= 0.0) || !isfinite(model_frac))
        return fail(c, EOR_EINVAL, "mock_d2/sigma NULL, bad mem or model_frac < 0");
    const size_t zb = (size_t)c->cfg.n_z * c->cfg.n_bins;
    double* buf = nullptr;     // mock, sums, sigma
    float* th = nullptr;
    if (!alloc_n(c, &buf, 3 * zb)) return fail(c, EOR_ENOMEM, "noise buffers");
    int r = copy_in(c, buf, mock_d2, sizeof(double) * zb, mem);
    if (!r && thermal) {
        if (mem == EOR_DEVICE) {
            th = const_cast<float*>(thermal);
        } else if (!alloc_n(c, &th, (size_t)c->cfg.n_z * c->nspec)) {
            r = fail(c, EOR_ENOMEM, "thermal noise buffer");
        } else {
            r = copy_in(c, th, thermal, sizeof(float) * c->cfg.n_z * c->nspec, mem);
        }
    }
    if (!r) {
        cudaError_t e = eor::launch_noise_sigma(c, buf, th, model_frac, buf + zb, buf + 2 * zb);
        if (e != cudaSuccess) r = cuda_fail(c, e, "noise sigma");
    }
    if (!r) r = copy_out(c, sigma, buf + 2 * zb, sizeof(double) * zb, mem);
    if (!r) r = finish(c, EOR_HOST);   // the scratch is freed below
    if (thermal && mem == EOR_HOST) dev_free(c, th);
    dev_free(c, buf);
    return r;
}

int eor_set_tuning(eor_ctx* c, int group, int pairs, int plane_threads) {
    if (!c) return EOR_EINVAL;
    if (group < 1 || group > 16 || pairs < 1 || pairs > 64 || (plane_threads != 512 && plane_threads != 1024))
        return fail(c, EOR_EINVAL, "tuning out of range (group 1..16, pairs 1..64, plane_threads 512|1024)");
    CK(cudaStreamSynchronize(c->stream), "tuning");
    float2* inter = nullptr;
    uint32_t* flags = nullptr;
    float2* psinter = nullptr;
    if (!alloc_n(c, &inter, inter_slots(c->tune.method, pairs, group) * c->nspec) ||
        !alloc_n(c, &flags, (size_t)pairs * c->flag_words) ||
        !alloc_n(c, &psinter, 2 * (size_t)pairs * c->nspec)) {
        dev_free(c, inter);
        dev_free(c, flags);
        dev_free(c, psinter);
        return fail(c, EOR_ENOMEM, "tuning scratch");
    }
    dev_free(c, c->d_inter);
    dev_free(c, c->d_flags);
    dev_free(c, c->d_psinter);
    c->d_inter = inter;
    c->d_flags = flags;
    c->d_psinter = psinter;
    c->tune = eor::Tuning{group, pairs, plane_threads, c->tune.method, c->tune.ps_split, c->tune.ps_streams};
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_walkers = -1;
    }
    return EOR_OK;
}

int eor_autotune(eor_ctx* c, const double* params, int n_walkers, const double* mock_d2, const double* sigma,
                 int reps, int* group, int* pairs, int* plane_threads, double* ms, int mem) {
    if (!c) return EOR_EINVAL;
    if (c->stage < 1) return fail(c, EOR_ESTATE, "eor_init_boxes first");
    if (reps < 1 || reps > 1000) return fail(c, EOR_EINVAL, "reps outside 1..1000");
    struct Cand { int group, pairs, threads, split, streams; };
    std::vector<Cand> cands;
    const int groups_direct[] = {4, 8, 16};
    const int pairs_list[] = {4, 8, 16, 32, 64};
    const bool direct = c->tune.method == eor::kMethodDirect;
    const int n_pairs = n_walkers * c->cfg.n_z;
    for (int streams : {2, 1}) {
        if (streams == 2 && direct) continue;   // the direct method's passes run in one stream
        for (int split : {0, 2, 1}) {
            if (split == 0 && (direct || c->n > 128)) continue;   // slab passes: the basis methods' spectrum
            if (split == 2 && c->n != 128) continue;   // the cluster form of the spectrum's plane pass
            for (int th : {512, 1024}) {
                if (th == 1024 && c->n != 128) continue;
                if (th == 1024 && split != 1 && !direct) continue;   // the CTA size then changes no kernel of the step
                for (int p : pairs_list) {
                    // 64 pairs in flight: the basis methods, and only with more than 32 pairs to run
                    if (p == 64 && (direct || n_pairs <= 32)) continue;
                    if (direct)
                        for (int gsz : groups_direct) cands.push_back({gsz, p, th, split, streams});
                    else
                        cands.push_back({c->tune.group, p, th, split, streams});
                }
            }
        }
    }
    const bool traced = c->trace_on;
    c->trace_on = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        c->trace_on = traced;
        return fail(c, EOR_ECUDA, "autotune events");
    }
    const Cand start{c->tune.group, c->tune.pairs, c->tune.plane_threads, c->tune.ps_split, c->tune.ps_streams};
    Cand best = start;
    double best_ms = INFINITY;
    std::vector<double> chi2_host;
    double* chi2 = nullptr;   // chi^2 of the warm-up calls, where the caller's buffers live
    if (mem == EOR_DEVICE) {
        if (n_walkers >= 1 && !alloc_n(c, &chi2, (size_t)n_walkers)) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            c->trace_on = traced;
            return fail(c, EOR_ENOMEM, "autotune buffer");
        }
    } else {
        chi2_host.resize(n_walkers >= 1 ? (size_t)n_walkers : 1);
        chi2 = chi2_host.data();
    }
    int r = EOR_OK;
    for (const Cand& k : cands) {
        if ((r = eor_set_tuning(c, k.group, k.pairs, k.threads)) != EOR_OK) break;
        c->tune.ps_split = k.split;
        c->tune.ps_streams = k.streams;
        // warm-up: captures this schedule's graph and checks the arguments
        if ((r = eor_likelihood(c, params, n_walkers, mock_d2, sigma, chi2, nullptr, mem)) != EOR_OK) break;
        cudaEventRecord(e0, c->stream);
        for (int i = 0; i < reps && r == EOR_OK; i++) {
            cudaError_t e = cudaGraphLaunch(c->graph_exec, c->stream);
            if (e != cudaSuccess) r = cuda_fail(c, e, "autotune replay");
        }
        cudaEventRecord(e1, c->stream);
        if (r != EOR_OK) break;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) { r = cuda_fail(c, e, "autotune timing"); break; }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        const double per = (double)t / reps;
        if (per < best_ms) {
            best_ms = per;
            best = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (mem == EOR_DEVICE) dev_free(c, chi2);
    c->trace_on = traced;
    if (r != EOR_OK) {
        const std::string msg = c->err;
        eor_set_tuning(c, start.group, start.pairs, start.threads);
        c->tune.ps_split = start.split;
        c->tune.ps_streams = start.streams;
        return fail(c, r, "autotune: " + msg);
    }
    if ((r = eor_set_tuning(c, best.group, best.pairs, best.threads)) != EOR_OK) return r;
    c->tune.ps_split = best.split;
    c->tune.ps_streams = best.streams;
    if (group) *group = best.group;
    if (pairs) *pairs = best.pairs;
    if (plane_threads) *plane_threads = best.threads;
    if (ms) *ms = best_ms;
    return EOR_OK;
}

int eor_set_ps_split(eor_ctx* c, int split) {
    if (!c) return EOR_EINVAL;
    if (split < 0 || split > 2) return fail(c, EOR_EINVAL, "ps_split must be 0, 1 or 2");
    if (split == 2 && c->n != 128) return fail(c, EOR_ENOTSUP, "the two-CTA plane pass serves n = 128 only");
    if (split == 0 && c->n > 128) return fail(c, EOR_ENOTSUP, "the slab passes serve n <= 128 only");
    CK(cudaStreamSynchronize(c->stream), "ps split");
    c->tune.ps_split = split;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_walkers = -1;
    }
    return EOR_OK;
}

int eor_set_ps_streams(eor_ctx* c, int streams) {
    if (!c) return EOR_EINVAL;
    if (streams != 1 && streams != 2) return fail(c, EOR_EINVAL, "ps_streams must be 1 or 2");
    CK(cudaStreamSynchronize(c->stream), "ps streams");
    c->tune.ps_streams = streams;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_walkers = -1;
    }
    return EOR_OK;
}

int eor_get_tuning(const eor_ctx* c, int* group, int* pairs, int* plane_threads, int* ps_split, int* ps_streams) {
    if (!c) return EOR_EINVAL;
    if (group) *group = c->tune.group;
    if (pairs) *pairs = c->tune.pairs;
    if (plane_threads) *plane_threads = c->tune.plane_threads;
    if (ps_split) *ps_split = c->n > 128 || (c->n < 128 && c->tune.ps_split == 2) ? 1 : c->tune.ps_split;
    if (ps_streams) *ps_streams = c->tune.ps_streams;
    return EOR_OK;
}

int eor_set_method(eor_ctx* c, int method) {
    if (!c) return EOR_EINVAL;
    if (method != EOR_METHOD_BASIS && method != EOR_METHOD_DIRECT && method != EOR_METHOD_BASIS_SIMT &&
        method != EOR_METHOD_BASIS_TF32)
        return fail(c, EOR_EINVAL, "unknown method");
    CK(cudaStreamSynchronize(c->stream), "method");
    const int internal = method == EOR_METHOD_BASIS        ? eor::kMethodBasis
                         : method == EOR_METHOD_DIRECT     ? eor::kMethodDirect
                         : method == EOR_METHOD_BASIS_SIMT ? eor::kMethodBasisSimt
                                                           : eor::kMethodBasisTf32;
    if (method == EOR_METHOD_BASIS_TF32 && !c->d_tcA && eor::basis_tc_fits(c->basis_rank)) {
        // the TF32 contraction's operands, formatted now if the boxes are already in place
        if (!alloc_n(c, &c->d_tcA, eor::basis_tc_a_bytes((long long)c->n3, c->cfg.n_z)) ||
            !alloc_n(c, &c->d_tcB, eor::basis_tc_b_bytes(c))) {
            dev_free(c, c->d_tcA);
            c->d_tcA = nullptr;
            return fail(c, EOR_ENOMEM, "TF32 contraction operands");
        }
        if (!c->d_xq && !alloc_n(c, &c->d_xq, (size_t)c->cfg.max_walkers * c->cfg.n_z))
            return fail(c, EOR_ENOMEM, "TF32 contraction sums");
        if (!c->d_cols &&
            !(alloc_n(c, &c->d_cols, eor::basis_tc_column_slots(c)) &&
              alloc_n(c, &c->d_gmeta, eor::basis_tc_column_slots(c) / 32) &&
              alloc_n(c, &c->d_goff, (size_t)c->cfg.max_walkers + 1)))
            return fail(c, EOR_ENOMEM, "TF32 contraction columns");
        if (c->stage >= 1) CK(eor::format_basis_tc(c), "TF32 contraction operands");
    }
    // the direct method's per-radius window tables, allocated on its first choice and kept
    if (internal == eor::kMethodDirect && !c->d_wtab &&
        !alloc_n(c, &c->d_wtab, (size_t)c->cfg.max_walkers * c->max_radii * c->n_m2))
        return fail(c, EOR_ENOMEM, "direct-method window tables");
    // the direct method's scratch, resized last: every failure above leaves the method and its
    // buffers as they were
    const size_t slots = inter_slots(internal, c->tune.pairs, c->tune.group);
    if (slots != inter_slots(c->tune.method, c->tune.pairs, c->tune.group)) {
        float2* inter = nullptr;
        if (!alloc_n(c, &inter, slots * c->nspec)) return fail(c, EOR_ENOMEM, "direct-method scratch");
        dev_free(c, c->d_inter);
        c->d_inter = inter;
    }
    c->tune.method = internal;
    if (c->graph_exec) {
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_walkers = -1;
    }
    if (c->stage >= 2) {   // the walker tables of the chosen contraction (column layout)
        CK(eor::build_walker_tables(c, c->n_walkers), "walker tables");
        CK(cudaStreamSynchronize(c->stream), "walker tables");
        if (c->stage > 2) c->stage = 2;
    }
    return EOR_OK;
}

int eor_basis_info(const eor_ctx* c, int* rank, double* max_residual) {
    if (!c || !rank || !max_residual) return EOR_EINVAL;
    *rank = c->basis_rank;
    *max_residual = c->basis_residual;
    return EOR_OK;
}

int eor_contraction_info(const eor_ctx* c, int* kind, int* k_slots) {
    if (!c || !kind || !k_slots) return EOR_EINVAL;
    *k_slots = 0;
    if (c->tune.method == eor::kMethodDirect) {
        *kind = EOR_CONTRACT_NONE;
    } else if (c->tune.method == eor::kMethodBasis && c->f16) {
        *kind = EOR_CONTRACT_FP16;
        *k_slots = c->k16;
    } else if (c->tune.method == eor::kMethodBasisTf32 && c->d_tcA) {
        *kind = EOR_CONTRACT_TF32;
        *k_slots = (c->basis_rank + 1 + 7) / 8 * 8;
    } else {
        *kind = EOR_CONTRACT_FP32;
    }
    return EOR_OK;
}

int eor_basis_window(eor_ctx* c, double r_mpc, double* w, int mem) {
    if (!c) return EOR_EINVAL;
    trace_reset(c);
    CK(trace_reserve(c, eor::estimate_launches(c)), "trace events");
    if (!w || !valid_mem(mem) || !(r_mpc > 0.0) || !isfinite(r_mpc)) return fail(c, EOR_EINVAL, "bad argument");
    const double dx = c->cfg.box_mpc / c->n;
    const double r_cell = c->cfg.r_cell_rule == 1 ? dx : cbrt(3.0 / (4.0 * kPi)) * dx;
    if (r_mpc < r_cell * (1.0 - 1e-12) || r_mpc > fmax(c->cfg.r_mfp_max, r_cell) * (1.0 + 1e-12))
        return fail(c, EOR_EINVAL, "r_mpc outside [R_cell, r_mfp_max], the basis's radius range");
    double* dst = mem == EOR_DEVICE ? w : reinterpret_cast<double*>(c->d_scratch_box);
    if (mem == EOR_HOST && sizeof(double) * c->n_m2 > sizeof(float) * c->n3)
        return fail(c, EOR_ENOTSUP, "grid too small for the host copy of the window");
    CK(eor::launch_basis_window(c, r_mpc, dst), "basis window");
    int r;
    if (mem == EOR_HOST && (r = copy_out(c, w, dst, sizeof(double) * c->n_m2, mem))) return r;
    return finish(c, mem);
}

int eor_debug_withhold(eor_ctx* c, int step, double wait_ms) {
    if (!c) return EOR_EINVAL;
    if (step >= 0 && !(wait_ms > 0.0 && wait_ms <= 2000.0))
        return fail(c, EOR_EINVAL, "wait_ms must be in (0, 2000]");
    CK(cudaStreamSynchronize(c->stream), "debug withhold");
    c->dbg_withhold = step >= 0 ? step : -1;
    c->dbg_wait_ns = step >= 0 ? (unsigned long long)(wait_ms * 1e6) : 0ull;
    if (c->graph_exec) {   // the captured graph holds the kernel's arguments
        cudaGraphExecDestroy(c->graph_exec);
        c->graph_exec = nullptr;
        c->graph_walkers = -1;
    }
    return EOR_OK;
}

int eor_trace(eor_ctx* c, int enable) {
    if (!c) return EOR_EINVAL;
    c->trace_on = enable != 0;
    return EOR_OK;
}

int eor_trace_read(eor_ctx* c, double* total_ms, long long* launches, int n_classes) {
    if (!c) return EOR_EINVAL;
    if (n_classes < 0 || (n_classes > 0 && (!total_ms || !launches))) return fail(c, EOR_EINVAL, "bad argument");
    CK(cudaStreamSynchronize(c->stream), "trace read");
    for (int k = 0; k < n_classes; k++) { total_ms[k] = 0.0; launches[k] = 0; }
    for (int i = 0; i < c->trace_used; i++) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, c->trace_events[2 * i], c->trace_events[2 * i + 1]), "event time");
        int k = c->trace_class[i];
        if (k < n_classes) {
            total_ms[k] += ms;
            launches[k] += 1;
        }
    }
    return EOR_OK;
}

const char* eor_kernel_class_name(int cls) {
    static const char* names[] = {"tables", "filter_plane", "pencil_ionize", "ps_plane", "finish", "forward_fft",
                                  "other", "basis_ionize"};
    return (cls >= 0 && cls < eor::kKClasses) ? names[cls] : "";
}

long long eor_launch_count(const eor_ctx* c) { return c ? c->launches : -1; }

}  // extern "C"
