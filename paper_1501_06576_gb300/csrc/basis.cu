// basis.cu — the radius-batched form of the excursion-set filter (sm_103a).
//
// Filtering is linear, so delta_R = IDFT(W(|k| R) delta_hat) can be assembled from any
// set of fields F_b = IDFT(phi_b(|k|) delta_hat) whose span holds W(. R) on the grid's
// |k| values: if W(k R) = sum_b c_b(R) phi_b(k) there, then delta_R = sum_b c_b(R) F_b.
// On a discrete grid the top-hat family {W(k R) : R_cell <= R <= R_max} is numerically
// low-rank (about 30 functions reproduce it to 1e-9 for the 64^3 and 128^3 grids).
//
// At eor_create (FP64): the distinct |m|^2 of the grid; a greedy pivoted Gram-Schmidt
// over W(k R) at candidate radii picks an orthonormal basis phi_b until every candidate
// is reproduced to kBasisTol; a table of c_b(R) = <phi_b, W(. R)> on a fine uniform R grid.
// At eor_init_boxes: the FP32 basis fields F_b of every box (one inverse FFT each, the
// same plane and pencil kernels as the per-radius path). At eor_set_params: c_b(R_j) of
// every walker radius by 4-point interpolation in the FP64 table.
// Per likelihood: one contraction over b for every (cell, walker, radius) with the
// threshold of Eq. 1, the OR over radii, the partial ionization at R_cell and
// delta T_b = T0 x_HI (1 + delta) fused into its epilogue.
#include <math.h>

#include "eor_internal.cuh"

namespace eor {

namespace {

__device__ double window_tophat_f64(double x) {
    if (x < 0.05) {
        double x2 = x * x;
        return 1.0 - x2 * (0.1 - x2 * (1.0 / 280.0 - x2 / 15120.0));
    }
    double s, c;
    sincos(x, &s, &c);
    return 3.0 * (s - x * c) / (x * x * x);
}

__device__ double block_reduce_sum(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; i++) s += red[i];
    return s;   // every thread
}

__device__ double block_reduce_max(double v, double* red) {
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; i++) s = fmax(s, red[i]);
    return s;
}

// 1 where |m|^2 occurs on the half-spectrum grid.
__global__ void k_mark_m2(int n, int* present) {
    const int nh = n / 2 + 1;
    const long long total = (long long)n * n * nh;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
        const int iz = (int)(e % nh), iy = (int)((e / nh) % n), ix = (int)(e / ((long long)nh * n));
        const int mx = ix < n / 2 ? ix : ix - n, my = iy < n / 2 ? iy : iy - n;
        present[mx * mx + my * my + iz * iz] = 1;
    }
}

// Ordered list of the present |m|^2 and the inverse map (one block, chunked scan).
__global__ void k_compact_m2(int n_m2, const int* present, int* kd_m2, int* m2_to_kd, int* n_kd) {
    __shared__ int s_cnt[1024];
    const int t = threadIdx.x, per = (n_m2 + blockDim.x - 1) / blockDim.x;
    const int lo = t * per, hi = min(n_m2, lo + per);
    int cnt = 0;
    for (int i = lo; i < hi; i++) cnt += present[i] ? 1 : 0;
    s_cnt[t] = cnt;
    __syncthreads();
    if (t == 0) {
        int run = 0;
        for (int i = 0; i < (int)blockDim.x; i++) { int v = s_cnt[i]; s_cnt[i] = run; run += v; }
        *n_kd = run;
    }
    __syncthreads();
    int pos = s_cnt[t];
    for (int i = lo; i < hi; i++) {
        if (present[i]) { kd_m2[pos] = i; m2_to_kd[i] = pos; pos++; }
        else m2_to_kd[i] = -1;
    }
}

// res[c][k] = W(k_k R_c) for the candidate radii.
__global__ void k_init_candidates(const int* kd_m2, int n_kd, double kf, const double* cand, double* res) {
    const int c = blockIdx.y;
    const double r = cand[c];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n_kd; k += gridDim.x * blockDim.x)
        res[(size_t)c * n_kd + k] = window_tophat_f64(kf * sqrt((double)kd_m2[k]) * r);
}

__global__ void k_col_absmax(const double* res, int n_kd, double* colmax) {
    __shared__ double red[32];
    double m = 0.0;
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) m = fmax(m, fabs(res[(size_t)blockIdx.x * n_kd + k]));
    m = block_reduce_max(m, red);
    if (threadIdx.x == 0) colmax[blockIdx.x] = m;
}

// Pivot = candidate with the largest residual; its residual, orthogonalised twice against
// the basis so far and normalised, becomes basis vector `rank`.
__global__ void k_pivot_orthonormalise(const double* colmax, int n_cand, const double* res, int n_kd, double* basis,
                                       int rank, double* pivmax) {
    __shared__ double red[32];
    __shared__ int s_piv;
    if (threadIdx.x == 0) {
        int best = 0;
        for (int c = 1; c < n_cand; c++)
            if (colmax[c] > colmax[best]) best = c;
        s_piv = best;
        pivmax[0] = colmax[best];
    }
    __syncthreads();
    const double* col = res + (size_t)s_piv * n_kd;
    double* v = basis + (size_t)rank * n_kd;
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) v[k] = col[k];
    __syncthreads();
    for (int pass = 0; pass < 2; pass++) {
        for (int p = 0; p < rank; p++) {
            const double* u = basis + (size_t)p * n_kd;
            double d = 0.0;
            for (int k = threadIdx.x; k < n_kd; k += blockDim.x) d += u[k] * v[k];
            d = block_reduce_sum(d, red);
            for (int k = threadIdx.x; k < n_kd; k += blockDim.x) v[k] -= d * u[k];
            __syncthreads();
        }
    }
    double nn = 0.0;
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) nn += v[k] * v[k];
    nn = block_reduce_sum(nn, red);
    const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) v[k] *= inv;
}

// res[c] -= <v, res[c]> v for every candidate (one block per candidate).
__global__ void k_deflate(double* res, int n_kd, const double* v) {
    __shared__ double red[32];
    double* col = res + (size_t)blockIdx.x * n_kd;
    double d = 0.0;
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) d += v[k] * col[k];
    d = block_reduce_sum(d, red);
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) col[k] -= d * v[k];
}

// c_b(R_g) = <phi_b, W(. R_g)> on the uniform grid R_g = r_lo + g h (one block per radius).
__global__ void __launch_bounds__(256) k_coef_table(const double* basis, int rank, const int* kd_m2, int n_kd,
                                                    double kf, double r_lo, double h, int n_grid, double* tab) {
    __shared__ double red[32];
    const double r = r_lo + h * blockIdx.x;
    double acc[kBasisMax];
#pragma unroll
    for (int b = 0; b < kBasisMax; b++) acc[b] = 0.0;
    for (int k = threadIdx.x; k < n_kd; k += blockDim.x) {
        const double w = window_tophat_f64(kf * sqrt((double)kd_m2[k]) * r);
#pragma unroll
        for (int b = 0; b < kBasisMax; b++)
            if (b < rank) acc[b] += basis[(size_t)b * n_kd + k] * w;
    }
    for (int b = 0; b < rank; b++) {
        const double s = block_reduce_sum(acc[b], red);
        if (threadIdx.x == 0) tab[(size_t)b * n_grid + blockIdx.x] = s;
    }
}

// FP32 basis functions on the |m|^2 index, for building the basis fields.
__global__ void k_basis_m2(const double* basis, int n_kd, const int* m2_to_kd, int n_m2, int kb, int rank,
                           float* phi) {
    const int b = blockIdx.y;
    for (int m2 = blockIdx.x * blockDim.x + threadIdx.x; m2 < n_m2; m2 += gridDim.x * blockDim.x) {
        const int k = m2_to_kd[m2];
        phi[(size_t)b * n_m2 + m2] = (b < rank && k >= 0) ? (float)basis[(size_t)b * n_kd + k] : 0.0f;
    }
}

// Walker radius j -> coefficients c_b(R_j), 4-point Lagrange in the FP64 table, stored FP32
// as [walker][radius][b]; zero beyond the ladder and beyond the rank.
__global__ void k_walker_coefs(const WalkerInfo* walkers, const double* tab, int rank, int kb, int max_radii,
                               double r_lo, double h, int n_grid, float* coef, int* err) {
    const int w = blockIdx.y;
    const int j = blockIdx.x;             // radius slot 0 .. max_radii-1
    const int b = threadIdx.x;            // basis index
    if (b >= kb) return;
    const int n_r = walkers[w].n_r;
    float out = 0.0f;
    if (j < n_r && b < rank) {
        const double u = (walkers[w].radii[j] - r_lo) / h;
        int i = (int)floor(u);
        if (i < 1 || i > n_grid - 3) {
            atomicOr(err, kErrLadder);
            i = i < 1 ? 1 : n_grid - 3;
        }
        const double t = u - i;
        const double* f = tab + (size_t)b * n_grid + (i - 1);
        const double l0 = -t * (t - 1.0) * (t - 2.0) / 6.0;
        const double l1 = (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0;
        const double l2 = -(t + 1.0) * t * (t - 2.0) / 2.0;
        const double l3 = (t + 1.0) * t * (t - 1.0) / 6.0;
        out = (float)(l0 * f[0] + l1 * f[1] + l2 * f[2] + l3 * f[3]);
    }
    coef[((size_t)w * max_radii + j) * kb + b] = out;
}

// Diagnostic: the basis's reconstruction sum_b c_b(R) phi_b(|m|^2) of the top-hat window at
// radius r on every |m|^2 index (NaN where no grid mode has that |m|^2), in FP64 with the
// coefficients interpolated from the table as the walker coefficients are.
__global__ void k_basis_window(const double* basis, int n_kd, const int* m2_to_kd, int n_m2, int rank,
                               const double* tab, double r_lo, double h, int n_grid, double r, double* out) {
    __shared__ double s_c[kBasisMax];
    if (threadIdx.x < rank) {
        const double u = (r - r_lo) / h;
        int i = (int)floor(u);
        i = i < 1 ? 1 : (i > n_grid - 3 ? n_grid - 3 : i);
        const double t = u - i;
        const double* f = tab + (size_t)threadIdx.x * n_grid + (i - 1);
        s_c[threadIdx.x] = -t * (t - 1.0) * (t - 2.0) / 6.0 * f[0] + (t + 1.0) * (t - 1.0) * (t - 2.0) / 2.0 * f[1] -
                           (t + 1.0) * t * (t - 2.0) / 2.0 * f[2] + (t + 1.0) * t * (t - 1.0) / 6.0 * f[3];
    }
    __syncthreads();
    for (int m2 = blockIdx.x * blockDim.x + threadIdx.x; m2 < n_m2; m2 += gridDim.x * blockDim.x) {
        const int k = m2_to_kd[m2];
        double w = k >= 0 ? 0.0 : nan("");
        if (k >= 0)
            for (int b = 0; b < rank; b++) w += s_c[b] * basis[(size_t)b * n_kd + k];
        out[m2] = w;
    }
}

// ------------------------------------------------------------------ the contraction

constexpr int kCPL = 2;                 // cells per thread
constexpr int kBThreads = 256;          // 8 warps
constexpr int kTC = kCPL * kBThreads;   // cells per CTA
constexpr int kWCH = 16;                // walkers per coefficient chunk

struct BasisArgs {
    const float* F;             // [n_z][kb][n3] basis fields
    const float* coef;          // [walker][max_radii][kb] coefficients c_b(R_j)
    const PairInfo* pairs;      // [walker * n_z + zi]
    const float* delta;         // [n_z][n3]
    float* dtb;                 // [pair][n3]
    float* xhi_out;             // optional [pair][n3]
    float* xpart;               // [pair][n3 / kTC] per-CTA neutral-fraction sums
    const float* ftab;          // [pair][kFTab] with a mass-dependent efficiency, else nullptr
    int n_walkers, n_z, max_radii;
    long long n3;
    float delta_c;
};

// Per-walker constants of a chunk, staged in shared memory.
struct WalkerConst {
    float zeta, t0, inv, cell_ok;
};

// One CTA: kTC cells of one redshift against every walker. Each thread keeps the KB basis
// values of its kCPL cells in registers; the block walks the flattened list of (walker,
// radius) columns of a chunk of walkers, each column a shared-memory record
// [c_0 .. c_{KB-1}, delta_crit, last, slot, -] read by every lane at the same address.
// Per column: delta_R = sum_b c_b F_b, flag |= delta_R >= delta_crit (Eq. 1). At a walker's
// last column (R_cell, warp-uniform): x_HI = 1 - (flag ? 1 : min(1, zeta f_coll(R_cell))),
// delta T_b = T0 x_HI (1 + delta) stored for the thread's cells (coalesced), flag reset.
template <int KB>
__global__ void __launch_bounds__(kBThreads) k_basis_ionize(BasisArgs a) {
    constexpr int REC = KB + 4;                          // floats per column record
    extern __shared__ __align__(16) float sm[];
    float* Rc = sm;                                      // [kWCH * max_radii][REC]
    WalkerConst* Wc = reinterpret_cast<WalkerConst*>(Rc + (size_t)kWCH * a.max_radii * REC);   // [kWCH]
    float* Xs = reinterpret_cast<float*>(Wc + kWCH);     // [kWCH][8 warps]
    int* Off = reinterpret_cast<int*>(Xs + kWCH * (kBThreads / 32));   // [kWCH + 1] column offsets
    const int zi = blockIdx.y;
    const long long cell0 = (long long)blockIdx.x * kTC;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const long long mycell = cell0 + (long long)kCPL * t;

    float f[kCPL][KB];
#pragma unroll
    for (int b = 0; b < KB; b++) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(a.F + ((size_t)zi * KB + b) * a.n3 + mycell));
        f[0][b] = v.x;
        f[1][b] = v.y;
    }
    const float2 dens = __ldg(reinterpret_cast<const float2*>(a.delta + (size_t)zi * a.n3 + mycell));

    for (int w0 = 0; w0 < a.n_walkers; w0 += kWCH) {
        const int nw = min(kWCH, a.n_walkers - w0);
        __syncthreads();   // the previous chunk is done with the shared buffers
        if (t == 0) {
            int run = 0;
            for (int wl = 0; wl < nw; wl++) {
                Off[wl] = run;
                run += a.pairs[(size_t)(w0 + wl) * a.n_z + zi].n_r;
            }
            Off[nw] = run;
        }
        if (t < nw) {
            const PairInfo& pi = a.pairs[(size_t)(w0 + t) * a.n_z + zi];
            Wc[t] = WalkerConst{pi.zeta, pi.t0, a.ftab ? pi.f_inv_h : pi.inv_sqrt2s2_cell, pi.cell_ok};
        }
        __syncthreads();
        const int ncols = Off[nw];
        // column records: coefficients (KB floats) + threshold, last flag, walker slot
        for (int e = t; e < nw * a.max_radii; e += kBThreads) {
            const int wl = e / a.max_radii, j = e % a.max_radii;
            const int n_r = Off[wl + 1] - Off[wl];
            if (j >= n_r) continue;
            float* rec = Rc + (size_t)(Off[wl] + j) * REC;
            const float4* src = reinterpret_cast<const float4*>(a.coef + ((size_t)(w0 + wl) * a.max_radii + j) * KB);
#pragma unroll
            for (int q = 0; q < KB / 4; q++) reinterpret_cast<float4*>(rec)[q] = __ldg(src + q);
            rec[KB] = a.pairs[(size_t)(w0 + wl) * a.n_z + zi].delta_crit[j];
            rec[KB + 1] = (j == n_r - 1) ? 1.0f : 0.0f;
            rec[KB + 2] = (float)wl;
            rec[KB + 3] = a.pairs[(size_t)(w0 + wl) * a.n_z + zi].delta_hi[j];
        }
        __syncthreads();
        bool fl[kCPL] = {false, false};
        for (int col = 0; col < ncols; col++) {
            const float* rec = Rc + (size_t)col * REC;
            float acc[kCPL], acc2[kCPL];   // two partial sums per cell for instruction-level parallelism
#pragma unroll
            for (int ci = 0; ci < kCPL; ci++) acc[ci] = acc2[ci] = 0.0f;
#pragma unroll
            for (int q = 0; q < KB / 4; q++) {
                const float4 c = *reinterpret_cast<const float4*>(rec + 4 * q);
#pragma unroll
                for (int ci = 0; ci < kCPL; ci++) {
                    acc[ci] = fmaf(f[ci][4 * q + 0], c.x, acc[ci]);
                    acc2[ci] = fmaf(f[ci][4 * q + 1], c.y, acc2[ci]);
                    acc[ci] = fmaf(f[ci][4 * q + 2], c.z, acc[ci]);
                    acc2[ci] = fmaf(f[ci][4 * q + 3], c.w, acc2[ci]);
                }
            }
#pragma unroll
            for (int ci = 0; ci < kCPL; ci++) acc[ci] += acc2[ci];
            const float4 tail = *reinterpret_cast<const float4*>(rec + KB);   // threshold, last, slot, upper
#pragma unroll
            for (int ci = 0; ci < kCPL; ci++) fl[ci] |= acc[ci] >= tail.x && acc[ci] <= tail.w;
            if (tail.y != 0.0f) {   // R_cell of walker `slot`: same column for the whole block
                const int wl = (int)tail.z;
                const WalkerConst w = Wc[wl];
                const float* tab = a.ftab ? a.ftab + ((size_t)(w0 + wl) * a.n_z + zi) * kFTab : nullptr;
                float xh[kCPL], xsum = 0.0f;
#pragma unroll
                for (int ci = 0; ci < kCPL; ci++) {
                    float fc = 0.0f;
                    if (tab) fc = pop_table_f(tab, a.delta_c - acc[ci], w.inv);   // efficiency-weighted f_coll
                    else if (w.cell_ok > 0.5f) fc = acc[ci] >= a.delta_c ? 1.0f : erfcf((a.delta_c - acc[ci]) * w.inv);
                    xh[ci] = fl[ci] ? 0.0f : 1.0f - fminf(1.0f, w.zeta * fc);
                    xsum += xh[ci];
                    fl[ci] = false;
                }
                const size_t pair = (size_t)(w0 + wl) * a.n_z + zi;
                reinterpret_cast<float2*>(a.dtb + pair * a.n3 + mycell)[0] =
                    make_float2(w.t0 * xh[0] * (1.0f + dens.x), w.t0 * xh[1] * (1.0f + dens.y));
                if (a.xhi_out) reinterpret_cast<float2*>(a.xhi_out + pair * a.n3 + mycell)[0] = make_float2(xh[0], xh[1]);
                for (int off = 16; off > 0; off >>= 1) xsum += __shfl_xor_sync(0xffffffffu, xsum, off);
                if (lane == 0) Xs[wl * (kBThreads / 32) + warp] = xsum;
            }
        }
        __syncthreads();
        if (t < nw) {   // fixed-order sum: the result does not depend on scheduling
            double sum = 0.0;
            for (int i = 0; i < kBThreads / 32; i++) sum += Xs[t * (kBThreads / 32) + i];
            const int n_r = Off[t + 1] - Off[t];
            a.xpart[((size_t)(w0 + t) * a.n_z + zi) * (a.n3 / kTC) + blockIdx.x] = n_r > 0 ? (float)sum : 0.0f;
        }
    }
}

// Sum of the per-CTA partials of one (walker, redshift) in FP64.
__global__ void k_xpart_reduce(const float* xpart, int parts, double* xhi_sum) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < parts; i += blockDim.x) s += (double)xpart[(size_t)blockIdx.x * parts + i];
    s = block_reduce_sum(s, red);
    if (threadIdx.x == 0) xhi_sum[blockIdx.x] = s;
}

}  // namespace

size_t basis_ionize_smem(int kb, int max_radii) {
    return sizeof(float) * ((size_t)kWCH * max_radii * (kb + 4)) + sizeof(WalkerConst) * kWCH +
           sizeof(float) * kWCH * (kBThreads / 32) + sizeof(int) * (kWCH + 1);
}

int basis_cells_per_cta() { return kTC; }

// Build the basis, its coefficient table and the FP32 per-|m|^2 basis functions.
cudaError_t build_basis(eor_ctx* c) {
    const eor_config& g = c->cfg;
    const double kf = 2.0 * kPi / g.box_mpc;
    const double dx = g.box_mpc / g.n;
    const double r_cell = g.r_cell_rule == 1 ? dx : cbrt(3.0 / (4.0 * kPi)) * dx;
    const double r_max = g.r_mfp_max > r_cell ? g.r_mfp_max : r_cell * 1.0001;
    cudaError_t e;
    int *present = nullptr, *d_nkd = nullptr;
    double *cand = nullptr, *res = nullptr, *colmax = nullptr, *pivmax = nullptr;
    const size_t n_cand = kBasisCand;
    if ((e = cudaMalloc(&present, sizeof(int) * c->n_m2)) != cudaSuccess) return e;
    cudaMemsetAsync(present, 0, sizeof(int) * c->n_m2, c->stream);
    trace_begin(c, kKOther);
    k_mark_m2<<<512, 256, 0, c->stream>>>(c->n, present);
    trace_end(c);
    if ((e = cudaMalloc(&d_nkd, sizeof(int))) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_compact_m2<<<1, 1024, 0, c->stream>>>(c->n_m2, present, c->d_kd_m2, c->d_m2_to_kd, d_nkd);
    trace_end(c);
    int n_kd = 0;
    cudaMemcpyAsync(&n_kd, d_nkd, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
    c->n_kd = n_kd;
    // candidate radii, log-spaced over [R_cell, R_max]
    double hc[kBasisCand];
    for (size_t i = 0; i < n_cand; i++) hc[i] = exp(log(r_cell) + (log(r_max) - log(r_cell)) * i / (n_cand - 1));
    if ((e = cudaMalloc(&cand, sizeof(double) * n_cand)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&res, sizeof(double) * n_cand * n_kd)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&colmax, sizeof(double) * n_cand)) != cudaSuccess) return e;
    if ((e = cudaMalloc(&pivmax, sizeof(double))) != cudaSuccess) return e;
    cudaMemcpyAsync(cand, hc, sizeof(double) * n_cand, cudaMemcpyHostToDevice, c->stream);
    trace_begin(c, kKOther);
    k_init_candidates<<<dim3((n_kd + 255) / 256, n_cand), 256, 0, c->stream>>>(c->d_kd_m2, n_kd, kf, cand, res);
    trace_end(c);
    int rank = 0;
    double worst = 0.0;
    while (rank < kBasisMax) {
        trace_begin(c, kKOther);
        k_col_absmax<<<n_cand, 256, 0, c->stream>>>(res, n_kd, colmax);
        trace_end(c);
        trace_begin(c, kKOther);
        k_pivot_orthonormalise<<<1, 1024, 0, c->stream>>>(colmax, n_cand, res, n_kd, c->d_basis, rank, pivmax);
        trace_end(c);
        cudaMemcpyAsync(&worst, pivmax, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return e;
        if (worst <= kBasisTol) break;
        trace_begin(c, kKOther);
        k_deflate<<<n_cand, 256, 0, c->stream>>>(res, n_kd, c->d_basis + (size_t)rank * n_kd);
        trace_end(c);
        rank++;
    }
    c->basis_rank = rank;
    c->basis_residual = worst;
    c->kb = (rank + 3) / 4 * 4;
    if (c->kb == 0) c->kb = 4;
    // coefficient table on a uniform grid with two spare points at each end
    c->coef_h = (r_max - r_cell) / (kCoefGrid - 5);
    c->coef_r_lo = r_cell - 2.0 * c->coef_h;
    trace_begin(c, kKOther);
    k_coef_table<<<kCoefGrid, 256, 0, c->stream>>>(c->d_basis, rank, c->d_kd_m2, n_kd, kf, c->coef_r_lo, c->coef_h,
                                                   kCoefGrid, c->d_coef_tab);
    trace_end(c);
    trace_begin(c, kKOther);
    k_basis_m2<<<dim3((c->n_m2 + 255) / 256, c->kb), 256, 0, c->stream>>>(c->d_basis, n_kd, c->d_m2_to_kd, c->n_m2,
                                                                          c->kb, rank, c->d_phi_m2);
    trace_end(c);
    e = cudaStreamSynchronize(c->stream);
    cudaFree(present);
    cudaFree(d_nkd);
    cudaFree(cand);
    cudaFree(res);
    cudaFree(colmax);
    cudaFree(pivmax);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t build_walker_coefs(eor_ctx* c, int n_walkers) {
    trace_begin(c, kKTables);
    k_walker_coefs<<<dim3(c->max_radii, n_walkers), 64, 0, c->stream>>>(c->d_walkers, c->d_coef_tab, c->basis_rank,
                                                                       c->kb, c->max_radii, c->coef_r_lo, c->coef_h,
                                                                       kCoefGrid, c->d_coef, c->d_err);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_basis_window(eor_ctx* c, double r, double* out) {
    trace_begin(c, kKOther);
    k_basis_window<<<(c->n_m2 + 255) / 256, 256, 0, c->stream>>>(c->d_basis, c->n_kd, c->d_m2_to_kd, c->n_m2,
                                                                  c->basis_rank, c->d_coef_tab, c->coef_r_lo, c->coef_h,
                                                                  kCoefGrid, r, out);
    trace_end(c);
    return cudaGetLastError();
}

#define EOR_KB_DISPATCH(kb, FN, ...)          \
    switch (kb) {                             \
        case 4: return FN<4>(__VA_ARGS__);    \
        case 8: return FN<8>(__VA_ARGS__);    \
        case 12: return FN<12>(__VA_ARGS__);  \
        case 16: return FN<16>(__VA_ARGS__);  \
        case 20: return FN<20>(__VA_ARGS__);  \
        case 24: return FN<24>(__VA_ARGS__);  \
        case 28: return FN<28>(__VA_ARGS__);  \
        case 32: return FN<32>(__VA_ARGS__);  \
        case 36: return FN<36>(__VA_ARGS__);  \
        case 40: return FN<40>(__VA_ARGS__);  \
        case 44: return FN<44>(__VA_ARGS__);  \
        case 48: return FN<48>(__VA_ARGS__);  \
        default: return cudaErrorInvalidValue; \
    }

template <int KB>
cudaError_t prepare_kb(eor_ctx* c) {
    return cudaFuncSetAttribute(k_basis_ionize<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)basis_ionize_smem(KB, c->max_radii));
}

template <int KB>
cudaError_t launch_kb(eor_ctx* c, const BasisArgs& a, size_t smem) {
    k_basis_ionize<KB><<<dim3((unsigned)(c->n3 / kTC), c->cfg.n_z), kBThreads, smem, c->stream>>>(a);
    return cudaGetLastError();
}

cudaError_t prepare_basis_kernel(eor_ctx* c) { EOR_KB_DISPATCH(c->kb, prepare_kb, c) }

cudaError_t launch_kb_any(eor_ctx* c, const BasisArgs& a, size_t smem) { EOR_KB_DISPATCH(c->kb, launch_kb, c, a, smem) }

cudaError_t launch_basis_ionize(eor_ctx* c, float* xhi_out) {
    const int n_z = c->cfg.n_z;
    if (c->tune.method == kMethodBasis && c->f16) return launch_basis_ionize_f16(c);   // x_HI: pencil pass
    if (c->tune.method == kMethodBasisTf32 && c->d_tcA) return launch_basis_ionize_tc(c, xhi_out);
    BasisArgs a{c->d_F, c->d_coef, c->d_pairs, brightness_base(c), c->d_dtb, xhi_out, c->d_xpart, pop_tables(c), c->n_walkers, n_z,
                c->max_radii, (long long)c->n3, (float)c->cfg.delta_c};
    const size_t smem = basis_ionize_smem(c->kb, c->max_radii);
    const int parts = (int)(c->n3 / kTC);
    trace_begin(c, kKBasis);
    cudaError_t e = launch_kb_any(c, a, smem);
    trace_end(c);
    if (e != cudaSuccess) return e;
    trace_begin(c, kKFinish);
    k_xpart_reduce<<<c->n_walkers * n_z, 256, 0, c->stream>>>(c->d_xpart, parts, c->d_xhi_sum);
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
