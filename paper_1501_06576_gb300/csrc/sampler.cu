// sampler.cu — the affine-invariant ensemble sampler (stretch move) on the device.
//
// 21CMMC samples its likelihood with the affine-invariant ensemble sampler of Goodman &
// Weare (2010), as packaged by Foreman-Mackey et al. (2013) (Sec. 2.4), optionally with a
// lower limit on the neutral fraction at one redshift (Sec. 3.3). Here the whole chain
// runs on the GPU: per step, each half of the ensemble proposes stretch moves against the
// other half (k_mcmc_propose), the batched likelihood graph of the context evaluates the
// half's proposals (eor_likelihood's captured graph, replayed on the device parameters),
// and k_mcmc_accept takes the Metropolis decision. The host only enqueues launches: no
// copy or synchronisation between steps.
//
// Random numbers: SplitMix64 (Steele, Lea & Flood 2014); for step s, half h, walker k and
// draw c (partner, stretch, accept) the output ((2 s + h) W + k) 3 + c of the stream keyed
// by the seed, a uniform being its top 53 bits over 2^53.
#include <math.h>
#include <string.h>

#include <new>
#include <string>

#include "eor_internal.cuh"

namespace {

constexpr int kDim = 3;   // (zeta, R_mfp, log10 T_vir)

struct McState {
    double a;                // stretch scale
    double lo[kDim], hi[kDim];
    int prior_z;             // redshift index of the neutral-fraction prior or -1
    double xhi_min;
    unsigned long long seed;
    int n_walkers, n_z;
    // Gaussian test target (no context): log p = -(y - mu)^T P (y - mu) / 2
    int gauss;
    double mu[kDim], prec[kDim * kDim];
};

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform_at(unsigned long long seed, unsigned long long n) {
    const unsigned long long u = mix64(mix64(seed) + 0x9E3779B97F4A7C15ull * (n + 1));
    return (double)(u >> 11) * (1.0 / 9007199254740992.0);
}

__device__ __forceinline__ double gauss_lnp(const McState& st, const double* y) {
    double d[kDim], q = 0.0;
    for (int i = 0; i < kDim; i++) d[i] = y[i] - st.mu[i];
    for (int i = 0; i < kDim; i++)
        for (int j = 0; j < kDim; j++) q += d[i] * st.prec[i * kDim + j] * d[j];
    return -0.5 * q;
}

// Proposals of half h at step s: walker k = h W/2 + i stretches from a partner j of the other
// half. Inside the prior box the proposal goes to the likelihood's parameter slot i; outside
// it the slot gets the walker's own (valid) position and the proposal is marked rejected.
__global__ void k_mcmc_propose(McState st, long long step, int h, const double* x, double* y, double* zs,
                               unsigned char* inside, double* lik_params) {
    const int half = st.n_walkers / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    const int k = h * half + i;
    const unsigned long long base = ((unsigned long long)(2 * step + h) * st.n_walkers + k) * 3ull;
    const int j = (1 - h) * half + min((int)(uniform_at(st.seed, base) * half), half - 1);
    const double u = uniform_at(st.seed, base + 1);
    const double z = ((st.a - 1.0) * u + 1.0) * ((st.a - 1.0) * u + 1.0) / st.a;
    bool in = true;
    double p[kDim];
    for (int c = 0; c < kDim; c++) {
        p[c] = x[3 * j + c] + z * (x[3 * k + c] - x[3 * j + c]);
        if (!(p[c] >= st.lo[c] && p[c] <= st.hi[c])) in = false;
    }
    for (int c = 0; c < kDim; c++) {
        y[3 * i + c] = p[c];
        if (lik_params) lik_params[3 * i + c] = in ? p[c] : x[3 * k + c];
    }
    zs[i] = z;
    inside[i] = in ? 1 : 0;
}

// Metropolis decision of half h: log p(Y) = -chi^2 / 2 inside the priors (-inf outside),
// accept when u < z^(d-1) p(Y) / p(X_k). After the second half the ensemble is recorded as
// chain row `step` (positions, log posteriors, acceptances).
__global__ void k_mcmc_accept(McState st, long long step, int h, const double* y, const double* zs,
                              const unsigned char* inside, const double* chi2, const double* xhi_mean, double* x,
                              double* lnp, unsigned char* acc) {
    const int half = st.n_walkers / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    const int k = h * half + i;
    const unsigned long long base = ((unsigned long long)(2 * step + h) * st.n_walkers + k) * 3ull;
    double lny = -INFINITY;
    if (inside[i]) {
        lny = st.gauss ? gauss_lnp(st, y + 3 * i) : -0.5 * chi2[i];
        if (!st.gauss && st.prior_z >= 0 && !(xhi_mean[(size_t)i * st.n_z + st.prior_z] >= st.xhi_min))
            lny = -INFINITY;
    }
    bool take = false;
    if (isfinite(lny)) {
        const double q = (kDim - 1) * log(zs[i]) + lny - lnp[k];
        const double u = uniform_at(st.seed, base + 2);
        take = u == 0.0 || log(u) < q;
    }
    if (take) {
        for (int c = 0; c < kDim; c++) x[3 * k + c] = y[3 * i + c];
        lnp[k] = lny;
    }
    acc[k] = take ? 1 : 0;
}

__global__ void k_mcmc_record(int n_walkers, const double* x, const double* lnp, const unsigned char* acc,
                              double* chain_row, double* lnp_row, int* acc_row) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_walkers) return;
    if (chain_row)
        for (int c = 0; c < kDim; c++) chain_row[3 * k + c] = x[3 * k + c];
    if (lnp_row) lnp_row[k] = lnp[k];
    if (acc_row) acc_row[k] = acc[k];
}

// Log posterior of the starting walkers of one half (slot i = walker h W/2 + i).
__global__ void k_mcmc_start_lnp(McState st, int h, const double* x, const double* chi2, const double* xhi_mean,
                                 double* lnp) {
    const int half = st.n_walkers / 2;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= half) return;
    const int k = h * half + i;
    bool in = true;
    for (int c = 0; c < kDim; c++)
        if (!(x[3 * k + c] >= st.lo[c] && x[3 * k + c] <= st.hi[c])) in = false;
    double v = -INFINITY;
    if (in) {
        v = st.gauss ? gauss_lnp(st, x + 3 * k) : -0.5 * chi2[i];
        if (!st.gauss && st.prior_z >= 0 && !(xhi_mean[(size_t)i * st.n_z + st.prior_z] >= st.xhi_min)) v = -INFINITY;
    }
    lnp[k] = v;
}

}  // namespace

struct eor_mcmc {
    eor_mcmc_config cfg{};
    eor_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    McState st{};
    double *d_x = nullptr, *d_lnp = nullptr, *d_y = nullptr, *d_z = nullptr, *d_mock = nullptr;
    double* d_chi2_out = nullptr;   // output slot of the set-up likelihood calls (results stay in the context)
    unsigned char *d_inside = nullptr, *d_acc = nullptr;
    double *d_chain = nullptr, *d_lnp_rows = nullptr;
    int* d_acc_rows = nullptr;
    size_t rows_cap = 0;
    long long steps_done = 0;
    bool started = false;
    std::string err;
};

namespace {

thread_local std::string g_mcmc_create_error;

int mfail(eor_mcmc* m, int code, const std::string& msg) {
    if (m) m->err = msg;
    else g_mcmc_create_error = msg;
    return code;
}

#define MK(call, what)                                                                                \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return mfail(m, EOR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
bool malloc_n(T** p, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

cudaMemcpyKind kin(int mem) { return mem == EOR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kout(int mem) { return mem == EOR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

unsigned blocks_for(int n) { return (unsigned)((n + 127) / 128); }

// Makes sure the context's captured likelihood graph is the one for half the ensemble, with
// this sampler's mock and sigma in place (one eor_likelihood call on the current walkers of
// half 0 when it is not).
int ensure_graph(eor_mcmc* m) {
    eor_ctx* c = m->ctx;
    const int half = m->st.n_walkers / 2;
    const size_t zb = (size_t)c->cfg.n_z * c->cfg.n_bins;
    if (c->graph_exec == nullptr || c->graph_walkers != half) {
        int r = eor_likelihood(c, m->d_x, half, m->d_mock, m->d_mock + zb, m->d_chi2_out, nullptr, EOR_DEVICE);
        if (r) return mfail(m, r, std::string("likelihood: ") + eor_last_error(c));
    }
    MK(cudaMemcpyAsync(c->d_mock, m->d_mock, sizeof(double) * 2 * zb, cudaMemcpyDeviceToDevice, c->stream), "mock");
    return EOR_OK;
}

// chi^2 and x_HI means of the parameters now in the context's parameter slots.
int evaluate(eor_mcmc* m) {
    MK(cudaGraphLaunch(m->ctx->graph_exec, m->ctx->stream), "likelihood graph");
    return EOR_OK;
}

}  // namespace

extern "C" {

void eor_mcmc_default_config(eor_mcmc_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->n_walkers = 128;
    cfg->a = 2.0;
    cfg->prior_lo[0] = 5.0;
    cfg->prior_lo[1] = 5.0;
    cfg->prior_lo[2] = 4.0;
    cfg->prior_hi[0] = 100.0;
    cfg->prior_hi[1] = 20.0;
    cfg->prior_hi[2] = 6.0;
    cfg->xhi_prior_z = -1;
    cfg->xhi_prior_min = 0.05;
    cfg->seed = 1;
}

void eor_mcmc_destroy(eor_mcmc* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    void* bufs[] = {m->d_x, m->d_lnp, m->d_y, m->d_z, m->d_mock, m->d_inside, m->d_acc, m->d_chain, m->d_lnp_rows,
                    m->d_acc_rows, m->d_chi2_out};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

int eor_mcmc_create(const eor_mcmc_config* cfg, eor_ctx* ctx, eor_mcmc** out) {
    if (!out) return mfail(nullptr, EOR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return mfail(nullptr, EOR_EINVAL, "cfg is NULL");
    const eor_mcmc_config& g = *cfg;
    if (g.n_walkers < 4 || g.n_walkers % 2 != 0 || !(g.a > 1.0) || !isfinite(g.a))
        return mfail(nullptr, EOR_EINVAL, "n_walkers must be even and >= 4, a > 1");
    for (int c = 0; c < kDim; c++)
        if (!(g.prior_hi[c] > g.prior_lo[c]) || !isfinite(g.prior_lo[c]) || !isfinite(g.prior_hi[c]))
            return mfail(nullptr, EOR_EINVAL, "prior box must have hi > lo, finite");
    if (ctx) {
        if (g.n_walkers / 2 > ctx->cfg.max_walkers)
            return mfail(nullptr, EOR_EINVAL, "half the ensemble must fit the context's max_walkers");
        // every point of the prior box must be a valid likelihood argument
        if (!(g.prior_lo[0] > 0.0) || !(g.prior_lo[1] > 0.0) || !(g.prior_hi[1] <= ctx->cfg.r_mfp_max) ||
            !(g.prior_lo[2] > 0.0) || !(g.prior_hi[2] < 12.0))
            return mfail(nullptr, EOR_EINVAL, "prior box outside the valid parameters (zeta > 0, 0 < R_mfp <= "
                                              "r_mfp_max, 0 < log10 T_vir < 12)");
        if (g.xhi_prior_z >= ctx->cfg.n_z) return mfail(nullptr, EOR_EINVAL, "xhi_prior_z beyond the context's redshifts");
    } else {
        if (g.gauss_target == 0) return mfail(nullptr, EOR_EINVAL, "no context: only the Gaussian test target");
    }
    eor_mcmc* m = new (std::nothrow) eor_mcmc();
    if (!m) return mfail(nullptr, EOR_ENOMEM, "host allocation");
    m->cfg = g;
    m->ctx = ctx;
    McState& st = m->st;
    st.a = g.a;
    for (int c = 0; c < kDim; c++) {
        st.lo[c] = g.prior_lo[c];
        st.hi[c] = g.prior_hi[c];
        st.mu[c] = g.gauss_mean[c];
    }
    for (int i = 0; i < kDim * kDim; i++) st.prec[i] = g.gauss_precision[i];
    st.gauss = ctx ? 0 : 1;
    st.prior_z = g.xhi_prior_z;
    st.xhi_min = g.xhi_prior_min;
    st.seed = g.seed;
    st.n_walkers = g.n_walkers;
    st.n_z = ctx ? ctx->cfg.n_z : 1;
    if (ctx) {
        m->stream = ctx->stream;
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete m;
            return mfail(nullptr, EOR_ECUDA, "stream create");
        }
        m->own_stream = true;
    }
    const int W = g.n_walkers, half = W / 2;
    const size_t zb = ctx ? (size_t)ctx->cfg.n_z * ctx->cfg.n_bins : 1;
    if (!malloc_n(&m->d_x, 3 * (size_t)W) || !malloc_n(&m->d_lnp, (size_t)W) || !malloc_n(&m->d_y, 3 * (size_t)half) ||
        !malloc_n(&m->d_z, (size_t)half) || !malloc_n(&m->d_mock, 2 * zb) || !malloc_n(&m->d_inside, (size_t)half) ||
        !malloc_n(&m->d_acc, (size_t)W) || !malloc_n(&m->d_chi2_out, (size_t)half)) {
        eor_mcmc_destroy(m);
        return mfail(nullptr, EOR_ENOMEM, "device allocation failed");
    }
    *out = m;
    return EOR_OK;
}

int eor_mcmc_start(eor_mcmc* m, const double* params, const double* mock_d2, const double* sigma, double* lnp,
                   int mem) {
    if (!m) return EOR_EINVAL;
    if (!params || (mem != EOR_HOST && mem != EOR_DEVICE)) return mfail(m, EOR_EINVAL, "params NULL or bad mem");
    const int W = m->st.n_walkers, half = W / 2;
    MK(cudaMemcpyAsync(m->d_x, params, sizeof(double) * 3 * W, kin(mem), m->stream), "copy params");
    MK(cudaMemsetAsync(m->d_acc, 0, (size_t)W, m->stream), "memset");
    if (m->ctx) {
        eor_ctx* c = m->ctx;
        if (c->stage < 1) return mfail(m, EOR_ESTATE, "the context has no density boxes");
        if (!mock_d2 || !sigma) return mfail(m, EOR_EINVAL, "mock_d2 and sigma are required with a context");
        const size_t zb = (size_t)c->cfg.n_z * c->cfg.n_bins;
        MK(cudaMemcpyAsync(m->d_mock, mock_d2, sizeof(double) * zb, kin(mem), m->stream), "copy mock");
        MK(cudaMemcpyAsync(m->d_mock + zb, sigma, sizeof(double) * zb, kin(mem), m->stream), "copy sigma");
        for (int h = 0; h < 2; h++) {
            // full likelihood call for each half (checks parameters, captures the graph)
            int r = eor_likelihood(c, m->d_x + 3 * (size_t)h * half, half, m->d_mock, m->d_mock + zb,
                                   m->d_chi2_out, nullptr, EOR_DEVICE);
            if (r) return mfail(m, r, std::string("likelihood: ") + eor_last_error(c));
            k_mcmc_start_lnp<<<blocks_for(half), 128, 0, m->stream>>>(m->st, h, m->d_x, c->d_chi2, c->d_xhi_mean,
                                                                      m->d_lnp);
            MK(cudaGetLastError(), "start lnp");
        }
        MK(cudaStreamSynchronize(m->stream), "start");
        int dev_err = 0;
        MK(cudaMemcpy(&dev_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
        if (dev_err) return mfail(m, EOR_EINVAL, "starting walkers rejected by the likelihood's parameter checks");
    } else {
        for (int h = 0; h < 2; h++) {
            k_mcmc_start_lnp<<<blocks_for(half), 128, 0, m->stream>>>(m->st, h, m->d_x, nullptr, nullptr, m->d_lnp);
            MK(cudaGetLastError(), "start lnp");
        }
    }
    if (lnp) MK(cudaMemcpyAsync(lnp, m->d_lnp, sizeof(double) * W, kout(mem), m->stream), "copy lnp");
    MK(cudaStreamSynchronize(m->stream), "start");
    m->steps_done = 0;
    m->started = true;
    return EOR_OK;
}

int eor_mcmc_run(eor_mcmc* m, int steps, double* chain, double* lnp, int* accepted, int mem) {
    if (!m) return EOR_EINVAL;
    if (!m->started) return mfail(m, EOR_ESTATE, "eor_mcmc_start first");
    if (steps < 1 || (mem != EOR_HOST && mem != EOR_DEVICE)) return mfail(m, EOR_EINVAL, "steps < 1 or bad mem");
    const int W = m->st.n_walkers, half = W / 2;
    const size_t rows = (size_t)steps;
    // row buffers: the caller's device buffers, else staging on the device
    double* chain_d = nullptr;
    double* lnp_d = nullptr;
    int* acc_d = nullptr;
    if (mem == EOR_DEVICE) {
        chain_d = chain;
        lnp_d = lnp;
        acc_d = accepted;
    } else if (chain || lnp || accepted) {
        if (m->rows_cap < rows) {
            cudaFree(m->d_chain);
            cudaFree(m->d_lnp_rows);
            cudaFree(m->d_acc_rows);
            m->d_chain = m->d_lnp_rows = nullptr;
            m->d_acc_rows = nullptr;
            m->rows_cap = 0;
            if (!malloc_n(&m->d_chain, rows * 3 * W) || !malloc_n(&m->d_lnp_rows, rows * W) ||
                !malloc_n(&m->d_acc_rows, rows * W))
                return mfail(m, EOR_ENOMEM, "chain buffers");
            m->rows_cap = rows;
        }
        chain_d = chain ? m->d_chain : nullptr;
        lnp_d = lnp ? m->d_lnp_rows : nullptr;
        acc_d = accepted ? m->d_acc_rows : nullptr;
    }
    eor_ctx* c = m->ctx;
    if (c) {
        int r = ensure_graph(m);
        if (r) return r;
    }
    for (int s = 0; s < steps; s++) {
        const long long step = m->steps_done + s;
        for (int h = 0; h < 2; h++) {
            k_mcmc_propose<<<blocks_for(half), 128, 0, m->stream>>>(m->st, step, h, m->d_x, m->d_y, m->d_z,
                                                                    m->d_inside, c ? c->d_params : nullptr);
            MK(cudaGetLastError(), "propose");
            if (c) {
                int r = evaluate(m);
                if (r) return r;
            }
            k_mcmc_accept<<<blocks_for(half), 128, 0, m->stream>>>(m->st, step, h, m->d_y, m->d_z, m->d_inside,
                                                                   c ? c->d_chi2 : nullptr,
                                                                   c ? c->d_xhi_mean : nullptr, m->d_x, m->d_lnp,
                                                                   m->d_acc);
            MK(cudaGetLastError(), "accept");
        }
        if (chain_d || lnp_d || acc_d) {
            k_mcmc_record<<<blocks_for(W), 128, 0, m->stream>>>(W, m->d_x, m->d_lnp, m->d_acc,
                                                                chain_d ? chain_d + (size_t)s * 3 * W : nullptr,
                                                                lnp_d ? lnp_d + (size_t)s * W : nullptr,
                                                                acc_d ? acc_d + (size_t)s * W : nullptr);
            MK(cudaGetLastError(), "record");
        }
    }
    m->steps_done += steps;
    if (mem == EOR_HOST) {
        if (chain) MK(cudaMemcpyAsync(chain, m->d_chain, sizeof(double) * rows * 3 * W, kout(mem), m->stream), "copy");
        if (lnp) MK(cudaMemcpyAsync(lnp, m->d_lnp_rows, sizeof(double) * rows * W, kout(mem), m->stream), "copy");
        if (accepted) MK(cudaMemcpyAsync(accepted, m->d_acc_rows, sizeof(int) * rows * W, kout(mem), m->stream), "copy");
        MK(cudaStreamSynchronize(m->stream), "run");
    }
    return EOR_OK;
}

int eor_mcmc_walkers(eor_mcmc* m, double* params, double* lnp, int mem) {
    if (!m) return EOR_EINVAL;
    if (mem != EOR_HOST && mem != EOR_DEVICE) return mfail(m, EOR_EINVAL, "bad mem");
    const int W = m->st.n_walkers;
    if (params) MK(cudaMemcpyAsync(params, m->d_x, sizeof(double) * 3 * W, kout(mem), m->stream), "copy");
    if (lnp) MK(cudaMemcpyAsync(lnp, m->d_lnp, sizeof(double) * W, kout(mem), m->stream), "copy");
    if (mem == EOR_HOST) MK(cudaStreamSynchronize(m->stream), "walkers");
    return EOR_OK;
}

const char* eor_mcmc_last_error(const eor_mcmc* m) { return m ? m->err.c_str() : g_mcmc_create_error.c_str(); }

}  // extern "C"
