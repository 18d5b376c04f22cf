// emulator.cu — the learned surrogate of the 21-cm power spectrum and its training.
//
// The paper has no surrogate: every likelihood call runs the excursion-set simulation.
// This unit adds an ensemble of small multilayer perceptrons that predict log10 Delta^2
// (Sec. 2.2's spectrum in logarithmic k bins) from (zeta, R_mfp, log10 T_vir, z), trained
// on spectra the simulation produced, and a likelihood call that emulates the walkers the
// ensemble agrees on and sends every other walker to the simulation (eor_likelihood).
//
// All arithmetic runs in the kernels below: the dense layers are one tiled FP32 GEMM
// kernel (64 x 64 tiles, 4 x 4 outputs per thread, bf16-rounded weights, FP32 sums) with
// the bias, GELU, GELU-derivative or plain store fused into its epilogue; column sums,
// the loss, Adam, minibatch gathering, normalisation and the fallback rule are kernels
// too. Every reduction runs in a fixed order, so results do not depend on scheduling.
// The host sizes buffers, sequences launches and picks the calibration threshold.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "eor_internal.cuh"
#include "tc.cuh"

namespace {

namespace tc = eor::tc;

constexpr int kIn = 4;                                 // zeta, R_mfp, log10 T_vir, z
constexpr int kMaxLayers = EOR21_EMU_MAX_HIDDEN + 1;
constexpr int kLossHist = 64;                          // ring of per-step minibatch losses
constexpr float kAdamB1 = 0.9f, kAdamB2 = 0.999f, kAdamEps = 1e-8f;

// Parameter layout of one member.
struct Layout {
    int n_layers;
    int fin[kMaxLayers], fout[kMaxLayers];
    long long off_w[kMaxLayers], off_b[kMaxLayers];
    long long n_params;
};

// Training state on the device (read by the step graph's kernels, advanced by k_emu_tick).
struct StepState {
    long long t;                // Adam steps taken since the weights were set
    int call_step, call_steps;  // position in the current eor_emu_train call
    int schedule;               // 1: cosine decay over the call; 0: constant rate
    float lr0;
    unsigned long long seed;
    int n_samples, batch;
    float lr, c1, c2;           // rate and bias corrections 1 - beta^(t+1) of the next Adam step
};

enum Epi : int { kEpiLinear = 0, kEpiGelu = 1, kEpiGeluGrad = 2, kEpiPlain = 3 };

// C(m, n) = sum_k A(m, k) B(k, n) for member blockIdx.z, with A(m, k) = A[e ae + m am + k ak]
// and B(k, n) = B[e be + k bk + n bn]; C[e ce + m cm + n]. Epilogues: + bias (kEpiLinear);
// z = acc + bias stored to pre_out and GELU(z) to C (kEpiGelu); acc * GELU'(pre) (kEpiGeluGrad);
// acc (kEpiPlain).
struct GemmArgs {
    const float* A;
    long long ae, am, ak;
    const float* B;
    long long be, bk, bn;
    float* C;
    long long ce, cm;
    const float* bias;
    long long bias_e;
    const float* pre;
    float* pre_out;
    long long pre_e, pre_m;
    int M, N, K;
    int* flag;                  // tensor-core form: bit 1 set when a bounded wait ran out
};

__device__ __forceinline__ float gelu_f(float u) { return 0.5f * u * (1.0f + erff(u * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad_f(float u) {
    return 0.5f * (1.0f + erff(u * 0.70710678118654752f)) + u * expf(-0.5f * u * u) * 0.39894228040143268f;
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// The same GEMM on the 5th-generation tensor cores: one CTA computes a 128 x NT tile of C
// (MMA M = 128, N = NT) for member blockIdx.z with tcgen05 kind::tf32 MMAs accumulating in
// tensor memory. K advances in stages of 32: all 128 threads load the stage's A (128 x 32)
// and B (NT x 32) values through their strides, split each into TF32 hi + lo (hi = TF32
// rounding, lo = TF32 rounding of the remainder) and store them K-major in the no-swizzle
// core-matrix layout; thread 0 then issues per K step of 8 the products hi*hi + lo*hi and,
// unless B is exact in TF32 (B_EXACT: the bf16-rounded weights, whose 8 significant bits
// TF32 holds), hi*lo: FP32-level products, FP32 accumulation, as the FP32-unit kernel. Two
// stages alternate, so the loads of one overlap the MMAs of the other. The epilogue
// (warp w: rows 32 w .. 32 w + 31) reads the accumulators back with tcgen05.ld and applies
// the same bias / GELU / GELU-derivative / plain store. Every wait is bounded in GPU time;
// a wait that gives up sets bit 1 of g.flag, and the CTA waits for its MMAs before freeing
// its tensor memory.
constexpr int kGtM = 128, kGtK = 32, kGtThreads = 128;
constexpr uint64_t kGtWaitNs = 2000000000ull;            // 2 s of GPU time per bounded wait
constexpr uint32_t kGtABytes = kGtM * kGtK * 4;          // one 128 x 32 TF32 operand (16 KB)

template <int NT>
constexpr uint32_t gt_stage_bytes(bool b_exact) {
    return 2 * kGtABytes + (b_exact ? 1u : 2u) * (uint32_t)NT * kGtK * 4;
}

template <int NT>
constexpr size_t gt_smem(bool b_exact) {
    return 2 * (size_t)gt_stage_bytes<NT>(b_exact) + 4 * sizeof(uint64_t) + 16;
}

// One stage's operand values in registers: core row (row, quad) = the 4 values k = 4 quad ..
// 4 quad + 3 of one row, 16 bytes of the K-major core-matrix layout. Core row index cr maps
// to row (cr >> 6) * 8 + (cr & 7) and quad (cr >> 3) & 7, so that a warp's 32 lanes write 8
// rows x 4 quads: 512 contiguous-in-banks bytes, no bank conflict.
template <int ROWS>
struct GtStage {
    static constexpr int PER = ROWS * 8 / kGtThreads;   // core rows per thread
    float4 v[PER];
};

__device__ __forceinline__ int gt_row(int cr) { return (cr >> 6) * 8 + (cr & 7); }
__device__ __forceinline__ int gt_quad(int cr) { return (cr >> 3) & 7; }

// Operand (row, k) = P[row * rs + k * ks] for row < rows and k < K, else 0.
template <int ROWS>
__device__ __forceinline__ void gt_load(GtStage<ROWS>& st, const float* P, long long rs, long long ks, int row0,
                                        int rows, int k0, int K) {
#pragma unroll
    for (int i = 0; i < GtStage<ROWS>::PER; i++) {
        const int cr = threadIdx.x + i * kGtThreads, r = row0 + gt_row(cr), k = k0 + 4 * gt_quad(cr);
        float x[4];
#pragma unroll
        for (int c = 0; c < 4; c++) x[c] = (r < rows && k + c < K) ? P[r * rs + (k + c) * ks] : 0.0f;
        st.v[i] = make_float4(x[0], x[1], x[2], x[3]);
    }
}

// hi (and with LO the remainder's TF32 rounding) of the stage into the core-matrix layout.
template <int ROWS, bool LO>
__device__ __forceinline__ void gt_store(const GtStage<ROWS>& st, unsigned char* hi, unsigned char* lo) {
#pragma unroll
    for (int i = 0; i < GtStage<ROWS>::PER; i++) {
        const int cr = threadIdx.x + i * kGtThreads;
        const uint32_t off = tc::core_offset(gt_row(cr), 4 * gt_quad(cr));
        const float x[4] = {st.v[i].x, st.v[i].y, st.v[i].z, st.v[i].w};
        uint32_t h[4], l[4];
#pragma unroll
        for (int c = 0; c < 4; c++) {
            h[c] = tc::to_tf32(x[c]);
            l[c] = tc::to_tf32(x[c] - __uint_as_float(h[c]));
        }
        *reinterpret_cast<uint4*>(hi + off) = make_uint4(h[0], h[1], h[2], h[3]);
        if constexpr (LO) *reinterpret_cast<uint4*>(lo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

template <int EPI, bool B_EXACT, int NT>
__global__ void __launch_bounds__(kGtThreads) k_emu_gemm_tc(GemmArgs g) {
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256 && (NT * 8) % kGtThreads == 0, "MMA N");
    constexpr uint32_t kStage = gt_stage_bytes<NT>(B_EXACT);
    constexpr uint32_t kBBytes = (uint32_t)NT * kGtK * 4;
    constexpr uint32_t kCols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kStage);   // [2] MMAs of a stage done
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
    const int e = blockIdx.z, m0 = blockIdx.y * kGtM, n0 = blockIdx.x * NT;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const float* A = g.A + e * g.ae;
    const float* B = g.B + e * g.be;
    if (warp == 0) tc::tmem_alloc(tslot, kCols);
    if (t == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_init(bar + 1, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const int nk = (g.K + kGtK - 1) / kGtK;
    // B(n, k) = B[k bk + n bn]: rows n, stride bn; k stride bk
    GtStage<kGtM> ra;
    GtStage<NT> rb;
    gt_load<kGtM>(ra, A, g.am, g.ak, m0, g.M, 0, g.K);
    gt_load<NT>(rb, B, g.bn, g.bk, n0, g.N, 0, g.K);
    bool ok = true;
    int last = -1;   // the last stage whose MMAs were issued (every thread tracks it)
    for (int kc = 0; kc < nk; kc++) {
        const int st = kc & 1;
        // the MMAs that read this stage two steps ago are done (a timeout stops every thread)
        if (kc >= 2 && !__syncthreads_and(tc::mbar_wait(bar + st, (uint32_t)((kc - 2) >> 1) & 1u, kGtWaitNs))) {
            ok = false;
            break;
        }
        unsigned char* Ah = sm + st * kStage;
        unsigned char* Al = Ah + kGtABytes;
        unsigned char* Bh = Al + kGtABytes;
        unsigned char* Bl = Bh + kBBytes;   // unused with B_EXACT
        gt_store<kGtM, true>(ra, Ah, Al);
        gt_store<NT, !B_EXACT>(rb, Bh, Bl);
        if (kc + 1 < nk) {   // the next stage's loads are in flight during the barrier and the MMAs
            gt_load<kGtM>(ra, A, g.am, g.ak, m0, g.M, (kc + 1) * kGtK, g.K);
            gt_load<NT>(rb, B, g.bn, g.bk, n0, g.N, (kc + 1) * kGtK, g.K);
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            const uint32_t idesc = tc::idesc_tf32(kGtM, NT);
            for (int ks = 0; ks < kGtK / 8; ks++) {
                const uint32_t ko = (uint32_t)ks * 2 * tc::kLBO;
                const uint64_t ah = tc::smem_desc(tc::smem_addr(Ah) + ko, tc::kLBO, tc::kSBO);
                const uint64_t al = tc::smem_desc(tc::smem_addr(Al) + ko, tc::kLBO, tc::kSBO);
                const uint64_t bh = tc::smem_desc(tc::smem_addr(Bh) + ko, tc::kLBO, tc::kSBO);
                tc::mma_tf32(tmem, ah, bh, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                tc::mma_tf32(tmem, al, bh, idesc, 1u);
                if constexpr (!B_EXACT) {
                    const uint64_t bl = tc::smem_desc(tc::smem_addr(Bl) + ko, tc::kLBO, tc::kSBO);
                    tc::mma_tf32(tmem, ah, bl, idesc, 1u);
                }
            }
            tc::mma_commit(bar + st);
        }
        last = kc;
    }
    // the last issued stage's commit completes once every MMA issued before it has finished
    bool done = last < 0 || tc::mbar_wait(bar + (last & 1), (uint32_t)(last >> 1) & 1u, kGtWaitNs);
    if (!done) done = tc::mbar_wait(bar + (last & 1), (uint32_t)(last >> 1) & 1u, kGtWaitNs);
    tc::fence_after_sync();
    const bool good = __syncthreads_and(ok && done);
    if (good) {
        const int m = m0 + warp * 32 + lane;
        const uint32_t base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float v[16];
            tc::tmem_ld16(base + (uint32_t)c0, v);
            if (m >= g.M) continue;
#pragma unroll
            for (int j = 0; j < 16; j++) {
                const int n = n0 + c0 + j;
                if (n >= g.N) continue;
                float x = v[j];
                if (EPI == kEpiLinear) {
                    x += g.bias[e * g.bias_e + n];
                } else if (EPI == kEpiGelu) {
                    x += g.bias[e * g.bias_e + n];
                    g.pre_out[e * g.pre_e + m * g.pre_m + n] = x;
                    x = gelu_f(x);
                } else if (EPI == kEpiGeluGrad) {
                    x *= gelu_grad_f(g.pre[e * g.pre_e + m * g.pre_m + n]);
                }
                g.C[e * g.ce + m * g.cm + n] = x;
            }
        }
    } else if (t == 0 && g.flag) {
        atomicOr(g.flag, 2);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

// out[e oe + n] = sum over rows of dz[e ze + r zm + n] (bias gradients). Block: 32 columns x
// 8 row slices; slice s sums rows s, s + 8, ... in order, then the slices add in order.
constexpr int kColSlices = 8;
__global__ void __launch_bounds__(32 * kColSlices) k_emu_colsum(const float* dz, long long ze, long long zm, int rows,
                                                                int n_cols, float* out, long long oe) {
    __shared__ float part[kColSlices][32];
    const int e = blockIdx.y, c = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + c;
    float s = 0.0f;
    if (n < n_cols) {
        const float* p = dz + e * ze + n;
#pragma unroll 4
        for (int r = sl; r < rows; r += kColSlices) s += p[(long long)r * zm];
    }
    part[sl][c] = s;
    __syncthreads();
    if (sl == 0 && n < n_cols) {
        float tot = part[0][c];
#pragma unroll
        for (int k = 1; k < kColSlices; k++) tot += part[k][c];
        out[e * oe + n] = tot;
    }
}

// Mean squared error of member blockIdx.x and dL/dy = 2 (y - t) / (rows n_out). t may be
// shared by all members (te = 0). The loss goes to loss[slot * members + e] with
// slot = (state->t mod kLossHist) when state is given, else slot 0.
__global__ void __launch_bounds__(256) k_emu_loss(const float* y, long long ye, const float* t, long long te,
                                                  int rows, int n_out, float* dy, double* loss,
                                                  const StepState* state, int members) {
    __shared__ double red[256];
    const int e = blockIdx.x;
    const long long cnt = (long long)rows * n_out;
    const float scale = 2.0f / (float)cnt;
    double part = 0.0;
    for (long long i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float d = y[e * ye + i] - t[e * te + i];
        dy[e * ye + i] = scale * d;
        part += (double)d * d;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int slot = state ? (int)(state->t % kLossHist) : 0;
        loss[slot * members + e] = red[0] / (double)cnt;
    }
}

__device__ __forceinline__ bool is_weight(const Layout& lay, long long p) {
    for (int l = 0; l < lay.n_layers; l++)
        if (p >= lay.off_w[l] && p < lay.off_b[l]) return true;
    return false;
}

// One Adam step (Kingma & Ba 2015) of every parameter of every member, then the bf16
// rounding of the updated weights into wq (biases are copied unrounded). The rate and the
// bias corrections come from the step state.
__global__ void k_emu_adam(float* w, float* wq, float* m, float* v, const float* g, long long total, Layout lay,
                           const StepState* st) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const float lr = st->lr, c1 = st->c1, c2 = st->c2;
    const float gi = g[i];
    const float mi = kAdamB1 * m[i] + (1.0f - kAdamB1) * gi;
    const float vi = kAdamB2 * v[i] + (1.0f - kAdamB2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + kAdamEps);
    w[i] = wi;
    wq[i] = is_weight(lay, i % lay.n_params) ? bf16_round(wi) : wi;
}

// Rate (cosine decay from lr0 to lr0 / 50 over the call, or constant) and bias corrections
// of the Adam step that follows t steps.
__device__ void next_step_constants(StepState* st) {
    float lr = st->lr0;
    if (st->schedule) {
        const double f = 0.5 * (1.0 + cos(eor::kPi * (double)st->call_step / (double)max(st->call_steps, 1)));
        lr = (float)(st->lr0 * (0.02 + 0.98 * f));
    }
    st->lr = lr;
    st->c1 = (float)(1.0 - pow((double)kAdamB1, (double)(st->t + 1)));
    st->c2 = (float)(1.0 - pow((double)kAdamB2, (double)(st->t + 1)));
}

__global__ void k_emu_tick(StepState* st) {
    st->t += 1;
    st->call_step += 1;
    next_step_constants(st);
}

__global__ void k_emu_begin(StepState* st, int steps, float lr0, int schedule, unsigned long long seed,
                            int n_samples, int batch, int reset_t) {
    if (reset_t) st->t = 0;
    st->call_step = 0;
    st->call_steps = steps;
    st->schedule = schedule;
    st->lr0 = lr0;
    st->seed = seed;
    st->n_samples = n_samples;
    st->batch = batch;
    next_step_constants(st);
}

// SplitMix64 (Steele, Lea & Flood 2014): output n of the stream with state seed + n * golden.
__device__ __forceinline__ unsigned long long splitmix_mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long splitmix_at(unsigned long long seed, unsigned long long stream,
                                                          unsigned long long n) {
    const unsigned long long key = splitmix_mix(seed + 0x9E3779B97F4A7C15ull * (2 * stream + 1));
    return splitmix_mix(key + 0x9E3779B97F4A7C15ull * (n + 1));
}

// Minibatch of member blockIdx.y: sample index drawn uniformly (multiply-shift of the top
// 32 bits) with replacement, keyed by (seed, member, step, row).
__global__ void k_emu_gather(const float* dx, const float* dt, int n_out, const StepState* st, long long xe,
                             long long te, float* x, float* t) {
    const int e = blockIdx.y, i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st->batch) return;
    const unsigned long long u =
        splitmix_at(st->seed, (unsigned long long)e, (unsigned long long)st->t * st->batch + i);
    const long long idx = (long long)(((u >> 32) * (unsigned long long)st->n_samples) >> 32);
#pragma unroll
    for (int c = 0; c < kIn; c++) x[e * xe + (long long)i * kIn + c] = dx[idx * kIn + c];
    for (int b = 0; b < n_out; b++) t[e * te + (long long)i * n_out + b] = dt[idx * n_out + b];
}

// Initial weights: uniform on +-sqrt(3 / fan_in), biases 0; Adam moments 0.
__global__ void k_emu_init(float* w, float* wq, float* m, float* v, long long total, Layout lay,
                           unsigned long long seed) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const long long e = i / lay.n_params, p = i % lay.n_params;
    float val = 0.0f;
    for (int l = 0; l < lay.n_layers; l++)
        if (p >= lay.off_w[l] && p < lay.off_b[l]) {
            const double u = (double)(splitmix_at(seed, 1000 + e, p) >> 11) * (1.0 / 9007199254740992.0);
            val = (float)((2.0 * u - 1.0) * sqrt(3.0 / lay.fin[l]));
        }
    w[i] = val;
    wq[i] = bf16_round(val);
    m[i] = 0.0f;
    v[i] = 0.0f;
}

// Master weights -> rounded working copy (after eor_emu_set_weights).
__global__ void k_emu_requant(const float* w, float* wq, float* m, float* v, long long total, Layout lay) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    wq[i] = is_weight(lay, i % lay.n_params) ? bf16_round(w[i]) : w[i];
    m[i] = 0.0f;
    v[i] = 0.0f;
}

struct FeatureMap {
    double lo[3], hi[3];
    double z_lo, z_hi;
    double z[EOR21_MAX_Z];
    int n_z;
};

__device__ __forceinline__ float feature(double v, double lo, double hi) {
    return (float)(2.0 * (v - lo) / (hi - lo) - 1.0);
}

// Inputs of row w n_z + j: walker w's parameters and redshift j mapped onto [-1, 1].
__global__ void k_emu_features(const double* params, int n_walkers, FeatureMap fm, float* x) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_walkers * fm.n_z) return;
    const int w = r / fm.n_z, j = r % fm.n_z;
#pragma unroll
    for (int c = 0; c < 3; c++) x[(long long)r * kIn + c] = feature(params[3 * w + c], fm.lo[c], fm.hi[c]);
    x[(long long)r * kIn + 3] = fm.z_hi > fm.z_lo ? feature(fm.z[j], fm.z_lo, fm.z_hi) : 0.0f;
}

// Training targets of row r: log10 max(d2, floor), NaN -> floor (FP64).
__global__ void k_emu_targets(const double* d2, long long count, double floor_v, double* raw) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double d = d2[i];
    raw[i] = log10(isfinite(d) ? fmax(d, floor_v) : floor_v);
}

// Per-bin mean and standard deviation of the targets (block per bin, FP64, fixed-order
// tree reduction; two passes). std is floored at 1e-6 dex.
__global__ void __launch_bounds__(256) k_emu_stats(const double* raw, int n_rows, int n_out, double* norm) {
    __shared__ double red[256];
    const int b = blockIdx.x;
    double s = 0.0;
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) s += raw[(long long)r * n_out + b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    const double mean = red[0] / n_rows;
    __syncthreads();
    s = 0.0;
    for (int r = threadIdx.x; r < n_rows; r += blockDim.x) {
        const double d = raw[(long long)r * n_out + b] - mean;
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        norm[b] = mean;
        norm[n_out + b] = fmax(sqrt(red[0] / n_rows), 1e-6);
    }
}

__global__ void k_emu_standardize(const double* raw, long long count, int n_out, const double* norm, float* t) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int b = (int)(i % n_out);
    t[i] = (float)((raw[i] - norm[b]) / norm[n_out + b]);
}

// Ensemble combination and fallback rule, one thread per walker: per row and bin the
// members' log10 Delta^2 = mean + std y, their average (pred) and population standard
// deviation; spread = largest standard deviation over bins; score = largest spread over
// redshifts, +inf when a predicted bin is below log10(10 floor) or a parameter leaves
// the prior box. fallback = !(score <= tau).
__global__ void k_emu_combine(const float* y, long long ye, int members, int n_walkers, int n_z, int n_out,
                              const double* norm, const double* params, FeatureMap fm, double log_floor10,
                              double tau, double* pred, double* spread, double* score, int* fallback) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_walkers) return;
    bool outside = false;
    for (int c = 0; c < 3; c++) {
        const double p = params[3 * w + c];
        if (!(p >= fm.lo[c] && p <= fm.hi[c])) outside = true;
    }
    double sc = 0.0;
    bool low = false;
    for (int j = 0; j < n_z; j++) {
        const long long r = (long long)w * n_z + j;
        double sp = 0.0;
        for (int b = 0; b < n_out; b++) {
            double p[EOR21_EMU_MAX_MEMBERS];
            double avg = 0.0;
            for (int e = 0; e < members; e++) {
                p[e] = norm[b] + norm[n_out + b] * (double)y[e * ye + r * n_out + b];
                avg += p[e];
            }
            avg /= members;
            double var = 0.0;
            for (int e = 0; e < members; e++) var += (p[e] - avg) * (p[e] - avg);
            sp = fmax(sp, sqrt(var / members));
            pred[r * n_out + b] = avg;
            if (!(avg >= log_floor10)) low = true;
        }
        spread[r] = sp;
        sc = fmax(sc, sp);
    }
    if (outside || low) sc = INFINITY;
    score[w] = sc;
    fallback[w] = !(sc <= tau);
}

// Largest relative error |10^pred / d2 - 1| of walker w over its redshifts and the bins
// with modes (d2 finite and above the floor); 0 when there are none.
__global__ void k_emu_error(const double* pred, const double* d2, int n_walkers, int n_z, int n_out,
                            double floor_v, double* err) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_walkers) return;
    double m = 0.0;
    for (long long i = (long long)w * n_z * n_out; i < (long long)(w + 1) * n_z * n_out; i++) {
        const double d = d2[i];
        if (!(isfinite(d) && d > floor_v)) continue;
        m = fmax(m, fabs(pow(10.0, pred[i]) / d - 1.0));
    }
    err[w] = m;
}

// Indices of the fallback walkers in ascending order and their count (one block).
__global__ void __launch_bounds__(1024) k_emu_compact(const int* fallback, int n_walkers, int* list, int* count) {
    __shared__ int base;
    __shared__ int warp_tot[32];
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w0 = 0; w0 < n_walkers; w0 += blockDim.x) {
        const int w = w0 + threadIdx.x;
        const int f = (w < n_walkers && fallback[w]) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, f);
        if (lane == 0) warp_tot[warp] = __popc(bal);
        __syncthreads();
        int before = 0;
        for (int k = 0; k < warp; k++) before += warp_tot[k];
        if (f) list[base + before + __popc(bal & ((1u << lane) - 1u))] = w;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < (int)(blockDim.x >> 5); k++) tot += warp_tot[k];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

// Parameters of fallback walkers list[first .. first + n_pad) (the tail repeats the last
// listed walker so a simulation batch keeps a fixed size).
__global__ void k_emu_gather_params(const double* params, const int* list, int first, int n_real, int n_pad,
                                    double* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    const int w = list[first + min(i, n_real - 1)];
    for (int c = 0; c < 3; c++) out[3 * i + c] = params[3 * w + c];
}

__global__ void k_emu_scatter(const int* list, int first, int n_real, const double* sim_chi2, const double* sim_d2,
                              int zb, double* chi2, double* d2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_real) return;
    const int w = list[first + i];
    chi2[w] = sim_chi2[i];
    for (int k = 0; k < zb; k++) d2[(long long)w * zb + k] = sim_d2[(long long)i * zb + k];
}

// Emulated walkers: Delta^2 = 10^pred (NaN in bins without modes) and chi^2 as in the
// simulation's chi^2 (Sec. 2.5 bins, summed over redshifts, Sec. 3.4).
__global__ void k_emu_chi2(const double* pred, const int* fallback, int n_walkers, int n_z, int n_out,
                           const signed char* use, const long long* nmodes, const double* mock, const double* sigma,
                           double* chi2, double* d2) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= n_walkers || fallback[w]) return;
    double acc = 0.0;
    for (int j = 0; j < n_z; j++)
        for (int b = 0; b < n_out; b++) {
            const long long i = ((long long)w * n_z + j) * n_out + b;
            const double v = nmodes[b] > 0 ? pow(10.0, pred[i]) : (double)NAN;
            d2[i] = v;
            if (!use[b] || nmodes[b] == 0) continue;
            const double r = (v - mock[j * n_out + b]) / sigma[j * n_out + b];
            acc += r * r;
        }
    chi2[w] = acc;
}

// ------------------------------------------------------------------ tensor-core inference
//
// The 256-wide hidden layers as BF16 x BF16 tcgen05 MMAs (kind::f16, FP32 accumulation in
// tensor memory): one CTA carries 128 rows of one member through the whole network, the
// activations staying in shared memory as the next layer's A operand and the weights of
// one layer at a time arriving by bulk copy. Operands are K-major without swizzle: an
// 8-row x 16-byte core matrix holds 8 BF16 values along K; core (g, kc) of a 256-wide
// operand sits at g * 4096 + kc * 128 bytes. Every layer input is rounded to BF16 (the
// first, the four features, too), the products and sums are FP32.
constexpr int kTcHidden = 256;                          // the only width this path serves
constexpr uint32_t kTcSbo16 = (kTcHidden / 8) * 128;    // bytes between 8-row groups (4096)
constexpr uint32_t kTcActBytes = 128 * kTcHidden * 2;   // activations of a tile (64 KB)
constexpr uint32_t kTcWBytes = kTcHidden * kTcHidden * 2;  // one hidden layer's weights (128 KB)
constexpr int kTcOutN = 16;                             // MMA N of the output layer (>= n_bins)
constexpr uint32_t kTcW3Bytes = kTcOutN * kTcHidden * 2;   // output layer's weights (8 KB)
constexpr uint32_t kTcMemberBytes = 2 * kTcWBytes + kTcW3Bytes;
constexpr uint64_t kTcWaitNs = 2000000000ull;           // 2 s of GPU time per bounded wait

__device__ __forceinline__ uint32_t core16(int row, int k) {
    return (uint32_t)((row >> 3) * kTcSbo16 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Instruction descriptor of kind::f16 with BF16 operands and FP32 accumulation, K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

// Weights of hidden layers 1, 2 and the output layer of every member in the BF16 core-matrix
// layout: [member][W1 | W2 | W3 padded to kTcOutN rows with zeros].
__global__ void k_emu_format_tc(const float* wq, Layout lay, int members, unsigned char* out) {
    const long long per = (long long)(2 * kTcHidden + kTcOutN) * kTcHidden;
    const long long total = per * members;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)(i / per);
        const long long r = i % per;
        const int layer = r < (long long)kTcHidden * kTcHidden ? 1 : (r < 2LL * kTcHidden * kTcHidden ? 2 : 3);
        const long long rl = r - (long long)(layer - 1) * kTcHidden * kTcHidden;
        const int o = (int)(rl / kTcHidden), k = (int)(rl % kTcHidden);
        float v = 0.0f;
        if (o < lay.fout[layer]) v = wq[(size_t)e * lay.n_params + lay.off_w[layer] + (size_t)o * kTcHidden + k];
        unsigned char* base = out + (size_t)e * kTcMemberBytes + (size_t)(layer - 1) * kTcWBytes;
        *reinterpret_cast<__nv_bfloat16*>(base + core16(o, k)) = __float2bfloat16_rn(v);
    }
}

// Forward pass of 128 rows (blockIdx.x) of member blockIdx.y: layer 0 (4 inputs) on the FP32
// units, hidden layers 1-2 and the output layer on the tensor cores. y [member][rows][n_out].
__global__ void __launch_bounds__(128, 1) k_emu_infer_tc(const float* x, int rows, const float* wq, Layout lay,
                                                         const unsigned char* wfmt, int n_out, float* y,
                                                         long long ye, int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                        // activations, 64 KB
    unsigned char* Bs = sm + kTcActBytes;          // weights of the current layer, 128 KB
    uint64_t* barW = reinterpret_cast<uint64_t*>(Bs + kTcWBytes);
    uint64_t* barD = barW + 1;
    uint64_t* barF = barW + 2;   // final drain on the failure path
    uint32_t* tslot = reinterpret_cast<uint32_t*>(barW + 3);
    const int t = threadIdx.x, warp = t >> 5, e = blockIdx.y;
    const int row = blockIdx.x * 128 + t;
    const float* w = wq + (size_t)e * lay.n_params;
    const unsigned char* wm = wfmt + (size_t)e * kTcMemberBytes;

    if (warp == 0) tc::tmem_alloc(tslot, 256);
    if (t == 0) {
        tc::mbar_init(barW, 1);
        tc::mbar_init(barD, 1);
        tc::mbar_init(barF, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    int owed = -1;   // thread 0: barW phase of a weight copy not yet seen to land
    if (t == 0) {    // layer 1's weights arrive while layer 0 runs
        tc::mbar_expect_tx(barW, kTcWBytes);
        tc::bulk_g2s(Bs, wm, kTcWBytes, barW);
        owed = 0;
    }
    // layer 0 on the FP32 units: h = GELU(W0 bf16(x) + b0), stored as BF16 (row t of the tile)
    {
        float xin[4];
#pragma unroll
        for (int c = 0; c < 4; c++)
            xin[c] = row < rows ? __bfloat162float(__float2bfloat16_rn(x[(size_t)row * 4 + c])) : 0.0f;
        const float* w0 = w + lay.off_w[0];
        const float* b0 = w + lay.off_b[0];
        for (int o0 = 0; o0 < kTcHidden; o0 += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; q++) {
                float hv[2];
#pragma unroll
                for (int u = 0; u < 2; u++) {
                    const int o = o0 + 2 * q + u;
                    float z = b0[o];
#pragma unroll
                    for (int c = 0; c < 4; c++) z = fmaf(w0[o * 4 + c], xin[c], z);
                    hv[u] = gelu_f(z);
                }
                pk[q] = pack_bf16(hv[0], hv[1]);
            }
            *reinterpret_cast<uint4*>(As + core16(t, o0)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    bool ok = true;
    uint32_t phase = 0;
    for (int layer = 1; layer <= 3; layer++) {
        const int n = layer == 3 ? kTcOutN : kTcHidden;
        if (t == 0) {
            ok = ok && tc::mbar_wait(barW, phase, kTcWaitNs);
            if (ok) owed = -1;
            if (ok) {
                tc::fence_after_sync();
                const uint32_t idesc = idesc_bf16(128, n);
                for (int ks = 0; ks < kTcHidden / 16; ks++) {
                    const uint64_t ad = tc::smem_desc(tc::smem_addr(As) + ks * 256, 128, kTcSbo16);
                    const uint64_t bd = tc::smem_desc(tc::smem_addr(Bs) + ks * 256, 128, kTcSbo16);
                    mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                }
            }
            tc::mma_commit(barD);   // also when skipped: completes once the MMAs issued so far are done
        }
        const bool done = tc::mbar_wait(barD, phase, kTcWaitNs);
        tc::fence_after_sync();
        phase ^= 1u;
        const bool good = __syncthreads_and(done && (t != 0 || ok));
        if (!good) {
            if (t == 0) atomicOr(err, 1);
            break;
        }
        if (t == 0 && layer < 3) {   // the MMAs are done with B: the next layer's weights
            const uint32_t bytes = layer == 1 ? kTcWBytes : kTcW3Bytes;
            tc::mbar_expect_tx(barW, bytes);
            tc::bulk_g2s(Bs, wm + (size_t)layer * kTcWBytes, bytes, barW);
            owed = (int)phase;
        }
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        const float* bias = w + lay.off_b[layer];
        if (layer < 3) {
            for (int c0 = 0; c0 < kTcHidden; c0 += 32) {
                float v[32];
                tc::tmem_ld32(lane_base + (uint32_t)c0, v);
#pragma unroll
                for (int g = 0; g < 4; g++) {
                    uint32_t pk[4];
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        pk[q] = pack_bf16(gelu_f(v[8 * g + 2 * q] + bias[c0 + 8 * g + 2 * q]),
                                          gelu_f(v[8 * g + 2 * q + 1] + bias[c0 + 8 * g + 2 * q + 1]));
                    *reinterpret_cast<uint4*>(As + core16(t, c0 + 8 * g)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                }
            }
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        } else {
            float v[16];
            tc::tmem_ld16(lane_base, v);
            if (row < rows)
                for (int b = 0; b < n_out; b++) y[(size_t)e * ye + (size_t)row * n_out + b] = v[b] + bias[b];
        }
    }
    // failure path: no MMA may run and no copy may land after the CTA is gone
    if (t == 0) {
        if (owed >= 0) tc::mbar_wait(barW, (uint32_t)owed, kTcWaitNs);
        tc::mma_commit(barF);
        tc::mbar_wait(barF, 0, kTcWaitNs);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

size_t emu_tc_smem() { return kTcActBytes + kTcWBytes + 3 * sizeof(uint64_t) + 16; }

}  // namespace

struct eor_emu {
    eor_emu_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Layout lay{};
    int E = 0, H = 0, B = 0, Z = 0, rows = 0;
    FeatureMap fm{};
    float *d_w = nullptr, *d_wq = nullptr, *d_m = nullptr, *d_v = nullptr, *d_grad = nullptr;
    float *d_x = nullptr, *d_t = nullptr, *d_act = nullptr, *d_pre = nullptr, *d_y = nullptr, *d_dy = nullptr;
    float *d_da = nullptr, *d_db = nullptr;
    double* d_loss = nullptr;            // [kLossHist][E]
    float *d_data_x = nullptr, *d_data_t = nullptr;
    double* d_data_raw = nullptr;
    double* d_norm = nullptr;            // [2][B]
    StepState* d_state = nullptr;
    double *d_params = nullptr, *d_d2in = nullptr;
    double *d_pred = nullptr, *d_spread = nullptr, *d_score = nullptr, *d_err = nullptr;
    int *d_fallback = nullptr, *d_list = nullptr, *d_count = nullptr;
    double *d_mock = nullptr, *d_chi2 = nullptr, *d_d2out = nullptr;
    double *d_fparams = nullptr, *d_fchi2 = nullptr, *d_fd2 = nullptr;
    int fcap = 0;                        // walkers the fallback buffers hold
    int n_samples = 0;
    bool has_norm = false;
    double tau = INFINITY;
    long long t_host = 0;                // Adam steps taken (host mirror)
    cudaGraphExec_t step_graph = nullptr;
    int graph_batch = -1;
    cudaEvent_t ev_emu = nullptr, ev_sim = nullptr;
    bool tc_ok = false;                  // the network's shape fits the tensor-core inference
    bool use_tc = false;                 // predictions on the tensor cores (else the FP32 units)
    unsigned char* d_wfmt = nullptr;     // BF16 core-matrix weights of every member
    int* d_flag = nullptr;               // bit 0: a bounded wait of the inference ran out, bit 1: of a GEMM
    std::string err;
};

namespace {

thread_local std::string g_emu_create_error;

int efail(eor_emu* m, int code, const std::string& msg) {
    if (m) m->err = msg;
    else g_emu_create_error = msg;
    return code;
}

#define EK(call, what)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return efail(m, EOR_ECUDA, std::string(what) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
bool ealloc(T** p, size_t count) {
    if (count == 0) count = 1;
    if (cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

unsigned grid_for(long long n, int block) { return (unsigned)((n + block - 1) / block); }

template <int EPI, bool B_EXACT, int NT>
cudaError_t gemm_tc(cudaStream_t s, const GemmArgs& g, int members) {
    dim3 grid(grid_for(g.N, NT), grid_for(g.M, kGtM), members);
    k_emu_gemm_tc<EPI, B_EXACT, NT><<<grid, kGtThreads, gt_smem<NT>(B_EXACT), s>>>(g);
    return cudaGetLastError();
}

// C = A B with the epilogue EPI on the tensor cores; b_exact: B holds the bf16-rounded
// weights (exact in TF32, two products); N tiles of 16, 32 or 64 columns.
template <int EPI>
cudaError_t gemm(cudaStream_t s, const GemmArgs& g, int members, bool b_exact) {
    if (b_exact) {
        if (g.N <= 16) return gemm_tc<EPI, true, 16>(s, g, members);
        if (g.N <= 32) return gemm_tc<EPI, true, 32>(s, g, members);
        return gemm_tc<EPI, true, 64>(s, g, members);
    }
    if (g.N <= 16) return gemm_tc<EPI, false, 16>(s, g, members);
    if (g.N <= 32) return gemm_tc<EPI, false, 32>(s, g, members);
    return gemm_tc<EPI, false, 64>(s, g, members);
}

template <int EPI, bool B_EXACT>
cudaError_t prepare_gemm_tc_epi() {
    cudaError_t e = cudaFuncSetAttribute(k_emu_gemm_tc<EPI, B_EXACT, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gt_smem<16>(B_EXACT));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_emu_gemm_tc<EPI, B_EXACT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gt_smem<32>(B_EXACT));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_emu_gemm_tc<EPI, B_EXACT, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gt_smem<64>(B_EXACT));
    return e;
}

cudaError_t prepare_gemm_tc() {
    cudaError_t e;
    if ((e = prepare_gemm_tc_epi<kEpiLinear, true>()) != cudaSuccess) return e;
    if ((e = prepare_gemm_tc_epi<kEpiGelu, true>()) != cudaSuccess) return e;
    if ((e = prepare_gemm_tc_epi<kEpiGeluGrad, true>()) != cudaSuccess) return e;
    if ((e = prepare_gemm_tc_epi<kEpiPlain, false>()) != cudaSuccess) return e;
    if ((e = prepare_gemm_tc_epi<kEpiLinear, false>()) != cudaSuccess) return e;
    if ((e = prepare_gemm_tc_epi<kEpiGelu, false>()) != cudaSuccess) return e;
    if ((e = prepare_gemm_tc_epi<kEpiGeluGrad, false>()) != cudaSuccess) return e;
    return prepare_gemm_tc_epi<kEpiPlain, true>();
}

long long act_stride(const eor_emu* m) { return (long long)m->rows * m->H; }
long long out_stride(const eor_emu* m) { return (long long)m->rows * m->B; }
float* act(const eor_emu* m, int l) { return m->d_act + (size_t)l * m->E * act_stride(m); }
float* pre(const eor_emu* m, int l) { return m->d_pre + (size_t)l * m->E * act_stride(m); }

// Forward pass of every member on `rows` rows of inputs x (member stride xe: 0 when the
// members share one input batch). Hidden layers keep their pre-activations for backward.
cudaError_t forward(eor_emu* m, const float* x, long long xe, int rows) {
    const Layout& L = m->lay;
    cudaError_t e = cudaSuccess;
    for (int l = 0; l < L.n_layers && e == cudaSuccess; l++) {
        GemmArgs g{};
        const bool first = l == 0, last = l == L.n_layers - 1;
        g.A = first ? x : act(m, l - 1);
        g.ae = first ? xe : act_stride(m);
        g.am = first ? kIn : m->H;
        g.ak = 1;
        g.B = m->d_wq + L.off_w[l];
        g.be = L.n_params;
        g.bk = 1;
        g.bn = L.fin[l];
        g.bias = m->d_wq + L.off_b[l];
        g.bias_e = L.n_params;
        g.M = rows;
        g.N = L.fout[l];
        g.K = L.fin[l];
        if (last) {
            g.C = m->d_y;
            g.ce = out_stride(m);
            g.cm = m->B;
            g.flag = m->d_flag;
            e = gemm<kEpiLinear>(m->stream, g, m->E, true);
        } else {
            g.C = act(m, l);
            g.ce = act_stride(m);
            g.cm = m->H;
            g.pre_out = pre(m, l);
            g.pre_e = act_stride(m);
            g.pre_m = m->H;
            g.flag = m->d_flag;
            e = gemm<kEpiGelu>(m->stream, g, m->E, true);
        }
    }
    return e;
}

// Gradients of every member into d_grad, from dL/dy in d_dy (after forward on the same x).
cudaError_t backward(eor_emu* m, const float* x, long long xe, int rows) {
    const Layout& L = m->lay;
    const float* dz = m->d_dy;
    long long dz_e = out_stride(m), dz_m = m->B;
    cudaError_t e = cudaSuccess;
    for (int l = L.n_layers - 1; l >= 0 && e == cudaSuccess; l--) {
        const bool first = l == 0;
        const float* in = first ? x : act(m, l - 1);
        const long long in_e = first ? xe : act_stride(m), in_m = first ? kIn : m->H;
        // dW_l[o][i] = sum_r dz[r][o] in[r][i]
        GemmArgs g{};
        g.A = dz;
        g.ae = dz_e;
        g.am = 1;
        g.ak = dz_m;
        g.B = in;
        g.be = in_e;
        g.bk = in_m;
        g.bn = 1;
        g.C = m->d_grad + L.off_w[l];
        g.ce = L.n_params;
        g.cm = L.fin[l];
        g.M = L.fout[l];
        g.N = L.fin[l];
        g.K = rows;
        g.flag = m->d_flag;
        e = gemm<kEpiPlain>(m->stream, g, m->E, false);
        if (e != cudaSuccess) break;
        // db_l[o] = sum_r dz[r][o]
        k_emu_colsum<<<dim3(grid_for(L.fout[l], 32), m->E), 32 * kColSlices, 0, m->stream>>>(
            dz, dz_e, dz_m, rows, L.fout[l], m->d_grad + L.off_b[l], L.n_params);
        e = cudaGetLastError();
        if (e != cudaSuccess || first) break;
        // dz_{l-1}[r][i] = (sum_o dz[r][o] W_l[o][i]) GELU'(pre_{l-1}[r][i])
        float* next = (dz == m->d_da) ? m->d_db : m->d_da;
        GemmArgs d{};
        d.A = dz;
        d.ae = dz_e;
        d.am = dz_m;
        d.ak = 1;
        d.B = m->d_wq + L.off_w[l];
        d.be = L.n_params;
        d.bk = L.fin[l];
        d.bn = 1;
        d.C = next;
        d.ce = act_stride(m);
        d.cm = m->H;
        d.pre = pre(m, l - 1);
        d.pre_e = act_stride(m);
        d.pre_m = m->H;
        d.M = rows;
        d.N = L.fin[l];
        d.K = L.fout[l];
        d.flag = m->d_flag;
        e = gemm<kEpiGeluGrad>(m->stream, d, m->E, true);
        dz = next;
        dz_e = act_stride(m);
        dz_m = m->H;
    }
    return e;
}

cudaError_t adam(eor_emu* m) {
    const long long total = (long long)m->E * m->lay.n_params;
    k_emu_adam<<<grid_for(total, 256), 256, 0, m->stream>>>(m->d_w, m->d_wq, m->d_m, m->d_v, m->d_grad, total,
                                                           m->lay, m->d_state);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_emu_tick<<<1, 1, 0, m->stream>>>(m->d_state);
    return cudaGetLastError();
}

// One minibatch training step of every member (the body of the captured step graph).
cudaError_t train_step(eor_emu* m, int batch) {
    const long long xe = (long long)m->rows * kIn, te = out_stride(m);
    k_emu_gather<<<dim3(grid_for(batch, 128), m->E), 128, 0, m->stream>>>(m->d_data_x, m->d_data_t, m->B,
                                                                          m->d_state, xe, te, m->d_x, m->d_t);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = forward(m, m->d_x, xe, batch);
    if (e == cudaSuccess) {
        k_emu_loss<<<m->E, 256, 0, m->stream>>>(m->d_y, out_stride(m), m->d_t, te, batch, m->B, m->d_dy, m->d_loss,
                                                m->d_state, m->E);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = backward(m, m->d_x, xe, batch);
    if (e == cudaSuccess) e = adam(m);
    return e;
}

bool valid_mem(int mem) { return mem == EOR_HOST || mem == EOR_DEVICE; }

cudaMemcpyKind kind_in(int mem) { return mem == EOR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }
cudaMemcpyKind kind_out(int mem) { return mem == EOR_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }

int finish(eor_emu* m, int mem) {
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem == EOR_HOST) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return efail(m, EOR_ECUDA, std::string("emulator: ") + cudaGetErrorString(e));
    if (mem == EOR_HOST) {   // a bounded wait of a tensor-core GEMM that ran out
        int flag = 0;
        EK(cudaMemcpy(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost), "flag");
        if (flag & 2) return efail(m, EOR_ETIMEOUT, "a bounded wait of a tensor-core GEMM ran out");
    }
    return EOR_OK;
}

// Copy the caller batch (x [n][4], t [n][B], optional) into member 0's slots.
int load_batch(eor_emu* m, const float* x, const float* t, int n, int mem) {
    if (!x || n < 1 || n > m->rows || !valid_mem(mem)) return efail(m, EOR_EINVAL, "batch NULL, bad mem or n outside 1..max_rows");
    EK(cudaMemcpyAsync(m->d_x, x, sizeof(float) * kIn * n, kind_in(mem), m->stream), "copy x");
    if (t) EK(cudaMemcpyAsync(m->d_t, t, sizeof(float) * m->B * n, kind_in(mem), m->stream), "copy t");
    return EOR_OK;
}

// Prediction of n_walkers walkers whose parameters are already in d_params.
cudaError_t predict_device(eor_emu* m, int n_walkers) {
    const int rows = n_walkers * m->Z;
    k_emu_features<<<grid_for(rows, 128), 128, 0, m->stream>>>(m->d_params, n_walkers, m->fm, m->d_x);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        if (m->use_tc) {
            const long long total = (long long)(2 * kTcHidden + kTcOutN) * kTcHidden * m->E;
            k_emu_format_tc<<<grid_for(total, 256), 256, 0, m->stream>>>(m->d_wq, m->lay, m->E, m->d_wfmt);
            e = cudaGetLastError();
            if (e == cudaSuccess) {
                k_emu_infer_tc<<<dim3(grid_for(rows, 128), m->E), 128, emu_tc_smem(), m->stream>>>(
                    m->d_x, rows, m->d_wq, m->lay, m->d_wfmt, m->B, m->d_y, out_stride(m), m->d_flag);
                e = cudaGetLastError();
            }
        } else {
            e = forward(m, m->d_x, 0, rows);
        }
    }
    if (e == cudaSuccess) {
        k_emu_combine<<<grid_for(n_walkers, 128), 128, 0, m->stream>>>(
            m->d_y, out_stride(m), m->E, n_walkers, m->Z, m->B, m->d_norm, m->d_params, m->fm,
            log10(10.0 * m->cfg.d2_floor), m->tau, m->d_pred, m->d_spread, m->d_score, m->d_fallback);
        e = cudaGetLastError();
    }
    return e;
}

int copy_params(eor_emu* m, const double* params, int n_walkers, int mem) {
    if (!params || !valid_mem(mem) || n_walkers < 1 || (long long)n_walkers * m->Z > m->rows)
        return efail(m, EOR_EINVAL, "params NULL, bad mem or n_walkers x n_z outside 1..max_rows");
    EK(cudaMemcpyAsync(m->d_params, params, sizeof(double) * 3 * n_walkers, kind_in(mem), m->stream), "copy params");
    return EOR_OK;
}

}  // namespace

extern "C" {

void eor_emu_default_config(eor_emu_config* cfg) {
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->n_z = 3;
    cfg->z[0] = 8.0;
    cfg->z[1] = 9.0;
    cfg->z[2] = 10.0;
    cfg->n_bins = 14;
    cfg->hidden = 256;
    cfg->n_hidden = 3;
    cfg->members = 4;
    cfg->max_rows = 16384;
    cfg->max_samples = 65536;
    cfg->prior_lo[0] = 5.0;
    cfg->prior_lo[1] = 5.0;
    cfg->prior_lo[2] = 4.0;
    cfg->prior_hi[0] = 100.0;
    cfg->prior_hi[1] = 20.0;
    cfg->prior_hi[2] = 6.0;
    cfg->d2_floor = 1e-2;
    cfg->err_tol = 0.05;
    cfg->seed = 1;
}

void eor_emu_destroy(eor_emu* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    if (m->step_graph) cudaGraphExecDestroy(m->step_graph);
    if (m->ev_emu) cudaEventDestroy(m->ev_emu);
    if (m->ev_sim) cudaEventDestroy(m->ev_sim);
    void* bufs[] = {m->d_w, m->d_wq, m->d_m, m->d_v, m->d_grad, m->d_x, m->d_t, m->d_act, m->d_pre, m->d_y,
                    m->d_dy, m->d_da, m->d_db, m->d_loss, m->d_data_x, m->d_data_t, m->d_data_raw, m->d_norm,
                    m->d_state, m->d_params, m->d_d2in, m->d_pred, m->d_spread, m->d_score, m->d_err,
                    m->d_fallback, m->d_list, m->d_count, m->d_mock, m->d_chi2, m->d_d2out, m->d_fparams,
                    m->d_fchi2, m->d_fd2, m->d_wfmt, m->d_flag};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (m->own_stream && m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

int eor_emu_create(const eor_emu_config* cfg, void* cuda_stream, eor_emu** out) {
    eor_emu* m = nullptr;
    if (!out) return efail(nullptr, EOR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return efail(nullptr, EOR_EINVAL, "cfg is NULL");
    const eor_emu_config& g = *cfg;
    if (g.n_z < 1 || g.n_z > EOR21_MAX_Z || g.n_bins < 1 || g.n_bins > EOR21_MAX_BINS || g.hidden < 4 ||
        g.hidden > 1024 || g.n_hidden < 1 || g.n_hidden > EOR21_EMU_MAX_HIDDEN || g.members < 1 ||
        g.members > EOR21_EMU_MAX_MEMBERS || g.max_rows < 1 || g.max_samples < 1 || !(g.d2_floor > 0.0) ||
        !(g.err_tol > 0.0))
        return efail(nullptr, EOR_EINVAL, "emulator configuration out of range");
    for (int c = 0; c < 3; c++)
        if (!(g.prior_hi[c] > g.prior_lo[c]) || !isfinite(g.prior_lo[c]) || !isfinite(g.prior_hi[c]))
            return efail(nullptr, EOR_EINVAL, "prior box must have hi > lo, finite");
    for (int j = 0; j < g.n_z; j++)
        if (!isfinite(g.z[j])) return efail(nullptr, EOR_EINVAL, "redshift not finite");
    if ((long long)g.max_rows * g.members * g.hidden > (1LL << 31))
        return efail(nullptr, EOR_EINVAL, "max_rows x members x hidden too large");
    m = new (std::nothrow) eor_emu();
    if (!m) return efail(nullptr, EOR_ENOMEM, "host allocation");
    m->cfg = g;
    m->E = g.members;
    m->H = g.hidden;
    m->B = g.n_bins;
    m->Z = g.n_z;
    m->rows = g.max_rows;
    Layout& L = m->lay;
    L.n_layers = g.n_hidden + 1;
    long long p = 0;
    for (int l = 0; l < L.n_layers; l++) {
        L.fin[l] = l == 0 ? kIn : g.hidden;
        L.fout[l] = l == L.n_layers - 1 ? g.n_bins : g.hidden;
        L.off_w[l] = p;
        p += (long long)L.fin[l] * L.fout[l];
        L.off_b[l] = p;
        p += L.fout[l];
    }
    L.n_params = p;
    FeatureMap& fm = m->fm;
    for (int c = 0; c < 3; c++) {
        fm.lo[c] = g.prior_lo[c];
        fm.hi[c] = g.prior_hi[c];
    }
    fm.n_z = g.n_z;
    fm.z_lo = fm.z_hi = g.z[0];
    for (int j = 0; j < g.n_z; j++) {
        fm.z[j] = g.z[j];
        fm.z_lo = std::min(fm.z_lo, g.z[j]);
        fm.z_hi = std::max(fm.z_hi, g.z[j]);
    }
    if (cuda_stream) {
        m->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            eor_emu_destroy(m);
            return efail(nullptr, EOR_ECUDA, "stream create");
        }
        m->own_stream = true;
    }
    const size_t EP = (size_t)m->E * L.n_params, R = (size_t)m->rows, E = (size_t)m->E;
    const size_t S = (size_t)g.max_samples;
    bool ok = ealloc(&m->d_w, EP) && ealloc(&m->d_wq, EP) && ealloc(&m->d_m, EP) && ealloc(&m->d_v, EP) &&
              ealloc(&m->d_grad, EP) && ealloc(&m->d_x, E * R * kIn) && ealloc(&m->d_t, E * R * m->B) &&
              ealloc(&m->d_act, (size_t)g.n_hidden * E * R * m->H) &&
              ealloc(&m->d_pre, (size_t)g.n_hidden * E * R * m->H) && ealloc(&m->d_y, E * R * m->B) &&
              ealloc(&m->d_dy, E * R * m->B) && ealloc(&m->d_da, E * R * m->H) && ealloc(&m->d_db, E * R * m->H) &&
              ealloc(&m->d_loss, (size_t)kLossHist * E) && ealloc(&m->d_data_x, S * kIn) &&
              ealloc(&m->d_data_t, S * m->B) && ealloc(&m->d_data_raw, S * m->B) && ealloc(&m->d_norm, 2 * m->B) &&
              ealloc(&m->d_state, 1) && ealloc(&m->d_params, 3 * std::max(R, S)) &&
              ealloc(&m->d_d2in, std::max(R, S) * m->B) && ealloc(&m->d_pred, R * m->B) &&
              ealloc(&m->d_spread, R) && ealloc(&m->d_score, R) && ealloc(&m->d_err, R) &&
              ealloc(&m->d_fallback, R) && ealloc(&m->d_list, R) && ealloc(&m->d_count, 1) &&
              ealloc(&m->d_mock, 2 * (size_t)m->Z * m->B) && ealloc(&m->d_chi2, R) && ealloc(&m->d_d2out, R * m->B);
    if (!ok) {
        eor_emu_destroy(m);
        return efail(nullptr, EOR_ENOMEM, "device allocation failed");
    }
    if (!ealloc(&m->d_flag, 1) || cudaMemsetAsync(m->d_flag, 0, sizeof(int), m->stream) != cudaSuccess ||
        prepare_gemm_tc() != cudaSuccess) {
        cudaGetLastError();
        eor_emu_destroy(m);
        return efail(nullptr, EOR_ENOMEM, "tensor-core GEMM set-up");
    }
    m->tc_ok = g.hidden == kTcHidden && g.n_hidden == 3 && g.n_bins <= kTcOutN;
    if (m->tc_ok) {
        if (!ealloc(&m->d_wfmt, (size_t)m->E * kTcMemberBytes) ||
            cudaFuncSetAttribute(k_emu_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)emu_tc_smem()) !=
                cudaSuccess) {
            cudaGetLastError();
            eor_emu_destroy(m);
            return efail(nullptr, EOR_ENOMEM, "tensor-core inference buffers");
        }
        m->use_tc = true;
    }
    if (cudaEventCreateWithFlags(&m->ev_emu, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->ev_sim, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        eor_emu_destroy(m);
        return efail(nullptr, EOR_ECUDA, "event create");
    }
    std::vector<double> norm(2 * m->B, 0.0);
    for (int b = 0; b < m->B; b++) norm[m->B + b] = 1.0;
    cudaError_t e = cudaMemcpyAsync(m->d_norm, norm.data(), sizeof(double) * norm.size(), cudaMemcpyHostToDevice,
                                    m->stream);
    if (e == cudaSuccess) {
        k_emu_init<<<grid_for((long long)EP, 256), 256, 0, m->stream>>>(m->d_w, m->d_wq, m->d_m, m->d_v,
                                                                        (long long)EP, L, g.seed);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_emu_begin<<<1, 1, 0, m->stream>>>(m->d_state, 0, 0.0f, 0, g.seed, 0, 0, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        g_emu_create_error = std::string("emulator init: ") + cudaGetErrorString(e);
        eor_emu_destroy(m);
        return EOR_ECUDA;
    }
    *out = m;
    return EOR_OK;
}

long long eor_emu_n_params(const eor_emu* m) { return m ? m->lay.n_params : -1; }

const char* eor_emu_last_error(const eor_emu* m) { return m ? m->err.c_str() : g_emu_create_error.c_str(); }

int eor_emu_set_data(eor_emu* m, const double* params, const double* d2, int n_walkers, int mem) {
    if (!m) return EOR_EINVAL;
    const long long S = (long long)n_walkers * m->Z;
    if (!params || !d2 || !valid_mem(mem) || n_walkers < 1 || S > m->cfg.max_samples)
        return efail(m, EOR_EINVAL, "params/d2 NULL, bad mem or n_walkers x n_z outside 1..max_samples");
    EK(cudaMemcpyAsync(m->d_params, params, sizeof(double) * 3 * n_walkers, kind_in(mem), m->stream), "copy params");
    EK(cudaMemcpyAsync(m->d_d2in, d2, sizeof(double) * S * m->B, kind_in(mem), m->stream), "copy d2");
    k_emu_features<<<grid_for(S, 128), 128, 0, m->stream>>>(m->d_params, n_walkers, m->fm, m->d_data_x);
    k_emu_targets<<<grid_for(S * m->B, 256), 256, 0, m->stream>>>(m->d_d2in, S * m->B, m->cfg.d2_floor,
                                                                  m->d_data_raw);
    k_emu_stats<<<m->B, 256, 0, m->stream>>>(m->d_data_raw, (int)S, m->B, m->d_norm);
    k_emu_standardize<<<grid_for(S * m->B, 256), 256, 0, m->stream>>>(m->d_data_raw, S * m->B, m->B, m->d_norm,
                                                                      m->d_data_t);
    m->n_samples = (int)S;
    m->has_norm = true;
    return finish(m, EOR_HOST);
}

int eor_emu_train(eor_emu* m, int steps, int batch, double lr, unsigned long long seed, double* loss) {
    if (!m) return EOR_EINVAL;
    if (m->n_samples < 1) return efail(m, EOR_ESTATE, "eor_emu_set_data first");
    if (steps < 1 || batch < 1 || batch > m->rows || !(lr > 0.0) || !isfinite(lr))
        return efail(m, EOR_EINVAL, "steps >= 1, 1 <= batch <= max_rows, lr > 0");
    k_emu_begin<<<1, 1, 0, m->stream>>>(m->d_state, steps, (float)lr, 1, seed, m->n_samples, batch, 0);
    EK(cudaGetLastError(), "train begin");
    if (m->graph_batch != batch) {
        if (m->step_graph) {
            cudaGraphExecDestroy(m->step_graph);
            m->step_graph = nullptr;
            m->graph_batch = -1;
        }
        cudaGraph_t graph = nullptr;
        EK(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        cudaError_t es = train_step(m, batch);
        cudaError_t ec = cudaStreamEndCapture(m->stream, &graph);
        if (es != cudaSuccess || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return efail(m, EOR_ECUDA, std::string("capture training step: ") +
                                           cudaGetErrorString(es != cudaSuccess ? es : ec));
        }
        ec = cudaGraphInstantiate(&m->step_graph, graph, 0);
        cudaGraphDestroy(graph);
        EK(ec, "instantiate training step");
        m->graph_batch = batch;
    }
    for (int s = 0; s < steps; s++) EK(cudaGraphLaunch(m->step_graph, m->stream), "training step");
    m->t_host += steps;
    if (loss) {
        std::vector<double> hist((size_t)kLossHist * m->E);
        EK(cudaMemcpyAsync(hist.data(), m->d_loss, sizeof(double) * hist.size(), cudaMemcpyDeviceToHost, m->stream),
           "copy losses");
        int r = finish(m, EOR_HOST);
        if (r) return r;
        const int last = std::min(steps, kLossHist);
        for (int e = 0; e < m->E; e++) {
            double s = 0.0;
            for (int k = 1; k <= last; k++) s += hist[(size_t)((m->t_host - k) % kLossHist) * m->E + e];
            loss[e] = s / last;
        }
        return EOR_OK;
    }
    return finish(m, EOR_HOST);
}

int eor_emu_forward(eor_emu* m, const float* x, int n, float* y, int mem) {
    if (!m) return EOR_EINVAL;
    if (!y) return efail(m, EOR_EINVAL, "y is NULL");
    int r = load_batch(m, x, nullptr, n, mem);
    if (r) return r;
    EK(forward(m, m->d_x, 0, n), "forward");
    for (int e = 0; e < m->E; e++)
        EK(cudaMemcpyAsync(y + (size_t)e * n * m->B, m->d_y + (size_t)e * out_stride(m), sizeof(float) * n * m->B,
                           kind_out(mem), m->stream),
           "copy y");
    return finish(m, mem);
}

int eor_emu_loss_grad(eor_emu* m, const float* x, const float* t, int n, double* loss, float* grad, int mem) {
    if (!m) return EOR_EINVAL;
    if (!t || !loss || !grad) return efail(m, EOR_EINVAL, "t, loss or grad is NULL");
    int r = load_batch(m, x, t, n, mem);
    if (r) return r;
    EK(forward(m, m->d_x, 0, n), "forward");
    k_emu_loss<<<m->E, 256, 0, m->stream>>>(m->d_y, out_stride(m), m->d_t, 0, n, m->B, m->d_dy, m->d_loss, nullptr,
                                            m->E);
    EK(cudaGetLastError(), "loss");
    EK(backward(m, m->d_x, 0, n), "backward");
    EK(cudaMemcpyAsync(grad, m->d_grad, sizeof(float) * m->E * m->lay.n_params, kind_out(mem), m->stream),
       "copy grad");
    EK(cudaMemcpyAsync(loss, m->d_loss, sizeof(double) * m->E, kind_out(mem), m->stream), "copy loss");
    return finish(m, mem);
}

int eor_emu_train_batch(eor_emu* m, const float* x, const float* t, int n, int steps, double lr, double* loss,
                        int mem) {
    if (!m) return EOR_EINVAL;
    if (!t || steps < 1 || !(lr > 0.0) || !isfinite(lr)) return efail(m, EOR_EINVAL, "t NULL, steps < 1 or lr <= 0");
    int r = load_batch(m, x, t, n, mem);
    if (r) return r;
    k_emu_begin<<<1, 1, 0, m->stream>>>(m->d_state, steps, (float)lr, 0, 0, 0, n, 0);
    EK(cudaGetLastError(), "begin");
    for (int s = 0; s < steps; s++) {
        EK(forward(m, m->d_x, 0, n), "forward");
        k_emu_loss<<<m->E, 256, 0, m->stream>>>(m->d_y, out_stride(m), m->d_t, 0, n, m->B, m->d_dy, m->d_loss,
                                                nullptr, m->E);
        EK(cudaGetLastError(), "loss");
        EK(backward(m, m->d_x, 0, n), "backward");
        EK(adam(m), "adam");
    }
    m->t_host += steps;
    if (loss) EK(cudaMemcpyAsync(loss, m->d_loss, sizeof(double) * m->E, kind_out(mem), m->stream), "copy loss");
    return finish(m, mem);
}

int eor_emu_get_weights(eor_emu* m, float* w, int mem) {
    if (!m) return EOR_EINVAL;
    if (!w || !valid_mem(mem)) return efail(m, EOR_EINVAL, "w NULL or bad mem");
    EK(cudaMemcpyAsync(w, m->d_w, sizeof(float) * m->E * m->lay.n_params, kind_out(mem), m->stream), "copy weights");
    return finish(m, mem);
}

int eor_emu_set_weights(eor_emu* m, const float* w, int mem) {
    if (!m) return EOR_EINVAL;
    if (!w || !valid_mem(mem)) return efail(m, EOR_EINVAL, "w NULL or bad mem");
    const long long total = (long long)m->E * m->lay.n_params;
    EK(cudaMemcpyAsync(m->d_w, w, sizeof(float) * total, kind_in(mem), m->stream), "copy weights");
    k_emu_requant<<<grid_for(total, 256), 256, 0, m->stream>>>(m->d_w, m->d_wq, m->d_m, m->d_v, total, m->lay);
    k_emu_begin<<<1, 1, 0, m->stream>>>(m->d_state, 0, 0.0f, 0, 0, 0, 0, 1);
    m->t_host = 0;
    return finish(m, mem);
}

int eor_emu_get_normalization(eor_emu* m, double* mean_std) {
    if (!m) return EOR_EINVAL;
    if (!mean_std) return efail(m, EOR_EINVAL, "mean_std is NULL");
    EK(cudaMemcpyAsync(mean_std, m->d_norm, sizeof(double) * 2 * m->B, cudaMemcpyDeviceToHost, m->stream), "copy");
    return finish(m, EOR_HOST);
}

int eor_emu_set_normalization(eor_emu* m, const double* mean_std) {
    if (!m) return EOR_EINVAL;
    if (!mean_std) return efail(m, EOR_EINVAL, "mean_std is NULL");
    for (int b = 0; b < m->B; b++)
        if (!isfinite(mean_std[b]) || !(mean_std[m->B + b] > 0.0) || !isfinite(mean_std[m->B + b]))
            return efail(m, EOR_EINVAL, "normalisation: finite means and std > 0");
    EK(cudaMemcpyAsync(m->d_norm, mean_std, sizeof(double) * 2 * m->B, cudaMemcpyHostToDevice, m->stream), "copy");
    if (m->n_samples > 0) {
        const long long cnt = (long long)m->n_samples * m->B;
        k_emu_standardize<<<grid_for(cnt, 256), 256, 0, m->stream>>>(m->d_data_raw, cnt, m->B, m->d_norm,
                                                                    m->d_data_t);
    }
    m->has_norm = true;
    return finish(m, EOR_HOST);
}

int eor_emu_predict(eor_emu* m, const double* params, int n_walkers, double* log10_d2, double* spread, int* fallback,
                    int mem) {
    if (!m) return EOR_EINVAL;
    int r = copy_params(m, params, n_walkers, mem);
    if (r) return r;
    EK(predict_device(m, n_walkers), "predict");
    const size_t rows = (size_t)n_walkers * m->Z;
    if (log10_d2)
        EK(cudaMemcpyAsync(log10_d2, m->d_pred, sizeof(double) * rows * m->B, kind_out(mem), m->stream), "copy");
    if (spread) EK(cudaMemcpyAsync(spread, m->d_spread, sizeof(double) * rows, kind_out(mem), m->stream), "copy");
    if (fallback)
        EK(cudaMemcpyAsync(fallback, m->d_fallback, sizeof(int) * n_walkers, kind_out(mem), m->stream), "copy");
    r = finish(m, mem);
    if (r || !m->use_tc || mem != EOR_HOST) return r;
    int flag = 0;
    EK(cudaMemcpy(&flag, m->d_flag, sizeof(int), cudaMemcpyDeviceToHost), "flag");
    return flag ? efail(m, EOR_ETIMEOUT, "a bounded tensor-core wait of the inference ran out") : EOR_OK;
}

int eor_emu_set_inference(eor_emu* m, int tensor_cores) {
    if (!m) return EOR_EINVAL;
    if (tensor_cores && !m->tc_ok)
        return efail(m, EOR_ENOTSUP, "tensor-core inference needs 3 hidden layers of 256 and at most 16 bins");
    m->use_tc = tensor_cores != 0;
    return EOR_OK;
}

int eor_emu_inference(const eor_emu* m) { return m ? (m->use_tc ? 1 : 0) : -1; }

int eor_emu_set_threshold(eor_emu* m, double tau) {
    if (!m) return EOR_EINVAL;
    if (isnan(tau)) return efail(m, EOR_EINVAL, "tau is NaN");
    m->tau = tau;
    return EOR_OK;
}

int eor_emu_calibrate(eor_emu* m, const double* params, const double* d2, int n_walkers, double recall, double* tau,
                      double* frac, int mem) {
    if (!m) return EOR_EINVAL;
    if (!d2 || !(recall > 0.0 && recall <= 1.0)) return efail(m, EOR_EINVAL, "d2 NULL or recall outside (0, 1]");
    int r = copy_params(m, params, n_walkers, mem);
    if (r) return r;
    const size_t zb = (size_t)m->Z * m->B;
    EK(cudaMemcpyAsync(m->d_d2in, d2, sizeof(double) * n_walkers * zb, kind_in(mem), m->stream), "copy d2");
    EK(predict_device(m, n_walkers), "predict");
    k_emu_error<<<grid_for(n_walkers, 128), 128, 0, m->stream>>>(m->d_pred, m->d_d2in, n_walkers, m->Z, m->B,
                                                                 m->cfg.d2_floor, m->d_err);
    EK(cudaGetLastError(), "error");
    std::vector<double> score(n_walkers), err(n_walkers);
    EK(cudaMemcpyAsync(score.data(), m->d_score, sizeof(double) * n_walkers, cudaMemcpyDeviceToHost, m->stream), "copy");
    EK(cudaMemcpyAsync(err.data(), m->d_err, sizeof(double) * n_walkers, cudaMemcpyDeviceToHost, m->stream), "copy");
    r = finish(m, EOR_HOST);
    if (r) return r;
    // host: the threshold from the scores of the walkers the surrogate gets wrong
    std::vector<double> bad;
    double max_finite = 0.0;
    for (int w = 0; w < n_walkers; w++) {
        if (isfinite(score[w])) max_finite = std::max(max_finite, score[w]);
        if (!(err[w] <= m->cfg.err_tol)) bad.push_back(score[w]);
    }
    double t = max_finite;
    if (!bad.empty()) {
        std::sort(bad.begin(), bad.end(), [](double a, double b) { return a > b; });
        const size_t k = (size_t)ceil(recall * (double)bad.size() - 1e-12);
        const double sk = bad[std::max<size_t>(k, 1) - 1];
        // walkers fall back when score > tau: tau just below the k-th largest bad score
        if (isfinite(sk)) t = std::min(max_finite, nextafter(sk, -INFINITY));
    }
    m->tau = t;
    if (tau) *tau = t;
    if (frac) {
        int nf = 0;
        for (int w = 0; w < n_walkers; w++) nf += !(score[w] <= t);
        *frac = (double)nf / n_walkers;
    }
    return EOR_OK;
}

int eor_emu_likelihood(eor_emu* m, eor_ctx* ctx, const double* params, int n_walkers, const double* mock_d2,
                       const double* sigma, double* chi2, double* d2, int* fallback, int mem) {
    if (!m) return EOR_EINVAL;
    if (!ctx || !mock_d2 || !sigma || !chi2) return efail(m, EOR_EINVAL, "ctx, mock_d2, sigma or chi2 is NULL");
    if (ctx->stage < 1) return efail(m, EOR_ESTATE, "the simulation context has no density boxes");
    if (ctx->cfg.efficiency_model != 0)
        return efail(m, EOR_ENOTSUP, "the surrogate emulates the step-function efficiency (efficiency_model 0) only");
    if (ctx->cfg.n_z != m->Z || ctx->cfg.n_bins != m->B)
        return efail(m, EOR_EINVAL, "the simulation context covers other redshifts or bins");
    for (int j = 0; j < m->Z; j++)
        if (ctx->cfg.z[j] != m->cfg.z[j]) return efail(m, EOR_EINVAL, "the simulation context covers other redshifts");
    int r = copy_params(m, params, n_walkers, mem);
    if (r) return r;
    const size_t zb = (size_t)m->Z * m->B;
    EK(cudaMemcpyAsync(m->d_mock, mock_d2, sizeof(double) * zb, kind_in(mem), m->stream), "copy mock");
    EK(cudaMemcpyAsync(m->d_mock + zb, sigma, sizeof(double) * zb, kind_in(mem), m->stream), "copy sigma");
    EK(predict_device(m, n_walkers), "predict");
    k_emu_compact<<<1, 1024, 0, m->stream>>>(m->d_fallback, n_walkers, m->d_list, m->d_count);
    EK(cudaGetLastError(), "compact");
    int nf = 0;
    EK(cudaMemcpyAsync(&nf, m->d_count, sizeof(int), cudaMemcpyDeviceToHost, m->stream), "copy count");
    EK(cudaStreamSynchronize(m->stream), "count");
    // emulated walkers
    k_emu_chi2<<<grid_for(n_walkers, 128), 128, 0, m->stream>>>(m->d_pred, m->d_fallback, n_walkers, m->Z, m->B,
                                                                ctx->d_chi2_use, ctx->d_nmodes, m->d_mock,
                                                                m->d_mock + zb, m->d_chi2, m->d_d2out);
    EK(cudaGetLastError(), "emulated chi2");
    // fallback walkers: simulation batches of at most max_walkers, padded to a multiple of
    // 32 walkers so that repeated calls replay the same captured graph
    const int cap = ctx->cfg.max_walkers;
    if (nf > 0 && m->fcap < cap) {
        cudaFree(m->d_fparams);
        cudaFree(m->d_fchi2);
        cudaFree(m->d_fd2);
        m->d_fparams = m->d_fchi2 = m->d_fd2 = nullptr;
        m->fcap = 0;
        if (!ealloc(&m->d_fparams, 3 * (size_t)cap) || !ealloc(&m->d_fchi2, (size_t)cap) ||
            !ealloc(&m->d_fd2, (size_t)cap * zb))
            return efail(m, EOR_ENOMEM, "fallback buffers");
        m->fcap = cap;
    }
    for (int first = 0; first < nf; first += cap) {
        const int n_real = std::min(cap, nf - first);
        const int n_pad = std::min(cap, (n_real + 31) / 32 * 32);
        k_emu_gather_params<<<grid_for(n_pad, 128), 128, 0, m->stream>>>(m->d_params, m->d_list, first, n_real,
                                                                         n_pad, m->d_fparams);
        EK(cudaGetLastError(), "gather params");
        EK(cudaEventRecord(m->ev_emu, m->stream), "event");
        EK(cudaStreamWaitEvent(ctx->stream, m->ev_emu, 0), "event wait");
        r = eor_likelihood(ctx, m->d_fparams, n_pad, m->d_mock, m->d_mock + zb, m->d_fchi2, m->d_fd2, EOR_DEVICE);
        if (r) return efail(m, r, std::string("simulation: ") + eor_last_error(ctx));
        EK(cudaEventRecord(m->ev_sim, ctx->stream), "event");
        EK(cudaStreamWaitEvent(m->stream, m->ev_sim, 0), "event wait");
        k_emu_scatter<<<grid_for(n_real, 128), 128, 0, m->stream>>>(m->d_list, first, n_real, m->d_fchi2, m->d_fd2,
                                                                    (int)zb, m->d_chi2, m->d_d2out);
        EK(cudaGetLastError(), "scatter");
    }
    EK(cudaMemcpyAsync(chi2, m->d_chi2, sizeof(double) * n_walkers, kind_out(mem), m->stream), "copy chi2");
    if (d2) EK(cudaMemcpyAsync(d2, m->d_d2out, sizeof(double) * n_walkers * zb, kind_out(mem), m->stream), "copy d2");
    if (fallback)
        EK(cudaMemcpyAsync(fallback, m->d_fallback, sizeof(int) * n_walkers, kind_out(mem), m->stream), "copy");
    r = finish(m, mem);
    if (r) return r;
    if (nf > 0 && mem == EOR_HOST) {
        // device-side checks of the simulation (parameters, ladders, bounded waits)
        int dev_err = 0;
        EK(cudaMemcpy(&dev_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
        if (dev_err) return efail(m, dev_err & eor::kErrTimeout ? EOR_ETIMEOUT : EOR_EINVAL,
                                  "simulation of fallback walkers reported a device-side error");
    }
    return EOR_OK;
}

}  // extern "C"
