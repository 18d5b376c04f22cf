// kernels.cu — the per-cell hot path of the excursion-set likelihood on sm_103a.
//
// A 3D real transform of an n^3 box is done in two kinds of pass:
//   plane pass  — one CTA per kz plane (n x n complex, shared-memory resident):
//                 2D complex FFT over (kx, ky), transform along kx first so both
//                 global sides of the CTA are coalesced;
//   pencil pass — one CTA per 32 (x, y) pencils: the real <-> half-complex transform
//                 along z, done as an n/2-point complex FFT plus a pre/post twist.
// Fused work:
//   pass 1 (plane, inverse)  multiplies the shared density spectrum by W(kR) on load;
//   pass 2 (pencil, C2R)     compares delta_R with the walker's threshold (Eq. 1) and
//                            ORs the ionization flag over a group of radii; at the last
//                            radius (R_cell) it adds the partial ionization, forms
//                            delta T_b = T0 x_HI (1 + delta) (Sec. 2.2) and runs the
//                            forward R2C along z of delta T_b;
//   PS pass (plane, forward) bins k^3 |X|^2 into the log-k shells in FP64 (Sec. 2.2).
// delta_R and delta T_b never touch global memory.
#include <math.h>

#include <cooperative_groups.h>

#include "eor_internal.cuh"
#include "fft_core.cuh"

namespace eor {

namespace {

__device__ __forceinline__ int signed_index(int i, int n) { return i < n / 2 ? i : i - n; }

// ------------------------------------------------------------------ plane pass

template <int N, int TMAX = 512>
struct Plane {
    static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
    static constexpr int S = N + 1;                        // padded row stride (float2)
    static constexpr int UNITS = N * R2;                   // (line, team member) pairs per pass
    static constexpr int THREADS = UNITS < TMAX ? UNITS : TMAX;
    static constexpr int LPT = UNITS / THREADS;            // lines per thread per pass
    static constexpr int NB = R1 / R2;                     // stage-B DFTs per unit
    static constexpr size_t SMEM = (size_t)N * S * sizeof(float2) + N * sizeof(float2) + 64 * sizeof(double);
    static constexpr size_t SMEM_PS = (size_t)N * S * sizeof(float2) + N * sizeof(float2) + 16 * THREADS * sizeof(float);
    // registers per thread of the shell-sum pass at 512 threads: 104 instead of the 128 that one
    // CTA per SM allows ran the 128^3 pass 5 % faster (4.1 against 4.35 us per plane set of a
    // pair); 96 and 88 were slower again, 80 spills
    static constexpr int PS_MAXREG = THREADS >= 1024 ? 64 : 104;
};

// 2D FFT of an n x n complex plane. load(r, c) gives the natural-order input; on return
// hold[l][q][k2] is the output at row rowOf(l) and column colOf(l, q, k2).
template <int N, int T, int DIR, class Load>
__device__ __forceinline__ void plane_fft(float2* buf, const float2* tw, Load load,
                                          float2 (&hold)[Plane<N, T>::LPT][Plane<N, T>::NB][Plane<N, T>::R2]) {
    using P = Plane<N, T>;
    const int t = threadIdx.x;
    // transform along the row index r, one line per column c
#pragma unroll
    for (int l = 0; l < P::LPT; l++) {
        const int u = t + P::THREADS * l, i = u / N, c = u % N;
        float2 a[P::R1];
#pragma unroll
        for (int j = 0; j < P::R1; j++) a[j] = load(j * P::R2 + i, c);
        dft_reg<P::R1, DIR>(a);
#pragma unroll
        for (int k1 = 1; k1 < P::R1; k1++) a[k1] = cmul(a[k1], tw_get<N, DIR>(tw, i * k1));
#pragma unroll
        for (int k1 = 0; k1 < P::R1; k1++) buf[(k1 * P::R2 + i) * P::S + c] = a[k1];
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < P::LPT; l++) {
        const int u = t + P::THREADS * l, i = u / N, c = u % N;
#pragma unroll
        for (int q = 0; q < P::NB; q++) {
            const int k1 = i + P::R2 * q;
#pragma unroll
            for (int i2 = 0; i2 < P::R2; i2++) hold[l][q][i2] = buf[(k1 * P::R2 + i2) * P::S + c];
            dft_reg<P::R2, DIR>(hold[l][q]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < P::LPT; l++) {
        const int u = t + P::THREADS * l, i = u / N, c = u % N;
#pragma unroll
        for (int q = 0; q < P::NB; q++)
#pragma unroll
            for (int k2 = 0; k2 < P::R2; k2++) buf[(i + P::R2 * q + P::R1 * k2) * P::S + c] = hold[l][q][k2];
    }
    __syncthreads();
    // transform along the column index, one line per row r
#pragma unroll
    for (int l = 0; l < P::LPT; l++) {
        const int u = t + P::THREADS * l, i = u / N, r = u % N;
        float2 a[P::R1];
#pragma unroll
        for (int j = 0; j < P::R1; j++) a[j] = buf[r * P::S + j * P::R2 + i];
        dft_reg<P::R1, DIR>(a);
#pragma unroll
        for (int k1 = 1; k1 < P::R1; k1++) a[k1] = cmul(a[k1], tw_get<N, DIR>(tw, i * k1));
#pragma unroll
        for (int k1 = 0; k1 < P::R1; k1++) buf[r * P::S + k1 * P::R2 + i] = a[k1];
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < P::LPT; l++) {
        const int u = t + P::THREADS * l, i = u / N, r = u % N;
#pragma unroll
        for (int q = 0; q < P::NB; q++) {
            const int k1 = i + P::R2 * q;
#pragma unroll
            for (int i2 = 0; i2 < P::R2; i2++) hold[l][q][i2] = buf[r * P::S + k1 * P::R2 + i2];
            dft_reg<P::R2, DIR>(hold[l][q]);
        }
    }
}

template <int N, int T>
__device__ __forceinline__ int plane_row(int l) { return (threadIdx.x + Plane<N, T>::THREADS * l) % N; }
template <int N, int T>
__device__ __forceinline__ int plane_col(int l, int q, int k2) {
    using P = Plane<N, T>;
    const int i = (threadIdx.x + P::THREADS * l) / N;
    return i + P::R2 * q + P::R1 * k2;
}

// After plane_fft: write hold to dst[r][c] (n x n, natural order) through shared memory.
template <int N, int T>
__device__ __forceinline__ void plane_store(float2* buf,
                                            const float2 (&hold)[Plane<N, T>::LPT][Plane<N, T>::NB][Plane<N, T>::R2],
                                            float2* dst) {
    using P = Plane<N, T>;
    __syncthreads();
#pragma unroll
    for (int l = 0; l < P::LPT; l++)
#pragma unroll
        for (int q = 0; q < P::NB; q++)
#pragma unroll
            for (int k2 = 0; k2 < P::R2; k2++) buf[plane_row<N, T>(l) * P::S + plane_col<N, T>(l, q, k2)] = hold[l][q][k2];
    __syncthreads();
    for (int e = threadIdx.x; e < N * N; e += P::THREADS) dst[e] = buf[(e / N) * P::S + (e % N)];
}

struct Pass1Args {
    const float2* spec;        // [n_z][nh][n][n]
    float2* inter;             // [P slots][G][nh][n][n]
    const PairInfo* pairs;
    const float* wtab;         // [walker][max_radii][n_m2]
    int max_radii, n_m2;
    int pair0, n_pairs, j0, G;
};

// Pass 1: delta_hat(k) W(|k| R) -> inverse 2D FFT over (kx, ky) for one kz plane of one
// (walker, redshift, radius) task.
template <int N, int T>
__global__ void __launch_bounds__(Plane<N, T>::THREADS, 1) k_plane_filter_inverse(Pass1Args a) {
    using P = Plane<N, T>;
    constexpr int NH = N / 2 + 1;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = smem + N * P::S;
    const int kz = blockIdx.x, tg = blockIdx.y, slot = blockIdx.z;
    const int pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return;
    const int n_r = a.pairs[pair].n_r, w = a.pairs[pair].w, zi = a.pairs[pair].zi;
    const int j = a.j0 + tg;
    if (j >= n_r) return;
    fill_twiddles<N>(tw);
    __syncthreads();
    const float2* src = a.spec + ((size_t)zi * NH + kz) * N * N;
    const float* wt = a.wtab + ((size_t)w * a.max_radii + j) * a.n_m2;
    const int mz2 = kz * kz;
    auto load = [&](int r, int c) {
        const int mx = signed_index(r, N), my = signed_index(c, N);
        const float wv = __ldg(wt + mx * mx + my * my + mz2);
        const float2 v = __ldg(src + r * N + c);
        return make_float2(v.x * wv, v.y * wv);
    };
    float2 hold[P::LPT][P::NB][P::R2];
    plane_fft<N, T, +1>(buf, tw, load, hold);
    float2* dst = a.inter + (((size_t)slot * a.G + tg) * NH + kz) * N * N;
    plane_store<N, T>(buf, hold, dst);
}

// Forward 2D FFT of plane kz of src ([nh][n][n], [x][y]) into dst ([nh][n][n], [kx][ky]).
template <int N, int T>
__global__ void __launch_bounds__(Plane<N, T>::THREADS, 1) k_plane_forward(const float2* src, float2* dst) {
    using P = Plane<N, T>;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = smem + N * P::S;
    const int kz = blockIdx.x;
    fill_twiddles<N>(tw);
    __syncthreads();
    const float2* s = src + (size_t)kz * N * N;
    auto load = [&](int r, int c) { return __ldg(s + r * N + c); };
    float2 hold[P::LPT][P::NB][P::R2];
    plane_fft<N, T, -1>(buf, tw, load, hold);
    plane_store<N, T>(buf, hold, dst + (size_t)kz * N * N);
}

struct PSArgs {
    const float2* ps_inter;    // [P slots][nh][n][n]  (z already transformed)
    const PairInfo* pairs;
    const signed char* bin_of_m2;
    double* ps_sum;            // [pair][n_bins]
    int pair0, n_pairs, n_bins;
    float kf3;                 // (2 pi / L)^3
};

constexpr int kPrivBins = 16;   // bins kept in per-thread shared-memory slots

// |m|^3 of a mode from m2 = |m|^2 >= 1 (every binned mode): m2^2 / sqrt(m2) with the fast
// reciprocal square root (a few 1e-7 relative; the correctly rounded sqrtf takes a longer
// instruction sequence, once per mode of every plane)
__device__ __forceinline__ float k3_of(float fm2) { return fm2 * fm2 * rsqrtf(fm2); }

// The CTA's shell sums from the per-thread slots priv[b][T]: warp w takes bins w, w + T/32,
// ...; each lane adds its slots, then a shuffle tree, in FP32 (this GPU issues FP64 at a few
// operations per clock per SM: a per-slot FP64 sum cost as much as the transforms), and the
// CTA's sum per bin goes to s_bins in FP64 for the global accumulation. The order is fixed, so
// the sums are reproducible; their rounding stays below 1e-5 relative per bin.
template <int T>
__device__ __forceinline__ void bin_sums(const float* priv, int n_bins, double* s_bins) {
    constexpr int WARPS = T / 32 > 0 ? T / 32 : 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x / 32;
    for (int b = warp; b < n_bins; b += WARPS) {
        float sum = 0.0f;
        for (int k = lane; k < T; k += 32) sum += priv[b * T + k];
        for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
        if (lane == 0) s_bins[b] = (double)sum;
    }
}

// Forward 2D FFT of one kz plane of delta T_b's z-transformed box, then the shell sums
// S_b += weight * k^3 |X|^2 (weight 2 for 0 < kz < n/2: the conjugate half). Each thread
// first sums its own modes per bin in FP32 (at most 32 modes each) in private shared-memory
// slots; bin_sums adds the slots of all threads in a fixed order, and the plane's sums go to
// the global FP64 shell sums.
template <int N, int T>
__global__ void __maxnreg__((Plane<N, T>::PS_MAXREG)) k_plane_ps(PSArgs a) {
    using P = Plane<N, T>;
    constexpr int NH = N / 2 + 1;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = smem + N * P::S;
    float* priv = reinterpret_cast<float*>(tw + N);          // [kPrivBins][THREADS]
    __shared__ double s_bins[EOR21_MAX_BINS];
    const int kz = blockIdx.x, slot = blockIdx.y;
    const int pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return;
    fill_twiddles<N>(tw);
    for (int e = threadIdx.x; e < kPrivBins * P::THREADS; e += P::THREADS) priv[e] = 0.0f;
    for (int e = threadIdx.x; e < EOR21_MAX_BINS; e += P::THREADS) s_bins[e] = 0.0;
    __syncthreads();
    const float2* s = a.ps_inter + ((size_t)slot * NH + kz) * N * N;
    auto load = [&](int r, int c) { return __ldg(s + r * N + c); };
    float2 hold[P::LPT][P::NB][P::R2];
    plane_fft<N, T, -1>(buf, tw, load, hold);
    const float weight = (kz == 0 || kz == N / 2) ? 1.0f : 2.0f;
    const int mz2 = kz * kz;
    const bool priv_ok = a.n_bins <= kPrivBins;
#pragma unroll
    for (int l = 0; l < P::LPT; l++) {
        const int mx = signed_index(plane_row<N, T>(l), N);
#pragma unroll
        for (int q = 0; q < P::NB; q++)
#pragma unroll
            for (int k2 = 0; k2 < P::R2; k2++) {
                const int my = signed_index(plane_col<N, T>(l, q, k2), N);
                const int m2 = mx * mx + my * my + mz2;
                const int b = a.bin_of_m2[m2];
                if (b >= 0) {
                    const float2 v = hold[l][q][k2];
                    const float fm2 = (float)m2;
                    const float val = weight * a.kf3 * k3_of(fm2) * (v.x * v.x + v.y * v.y);
                    if (priv_ok) priv[b * P::THREADS + threadIdx.x] += val;
                    else atomicAdd(&s_bins[b], (double)val);
                }
            }
    }
    __syncthreads();
    if (priv_ok) {
        bin_sums<P::THREADS>(priv, a.n_bins, s_bins);
        __syncthreads();
    }
    for (int b = threadIdx.x; b < a.n_bins; b += P::THREADS)
        if (s_bins[b] != 0.0) atomicAdd(&a.ps_sum[(size_t)pair * a.n_bins + b], s_bins[b]);
}

// The same pass for n = 128 as a cluster of two CTAs per plane: CTA h (the cluster rank)
// holds rows x = 64 h .. 64 h + 63 of the plane (66 KB instead of 132 KB, so two such CTAs
// share an SM and one's HBM load overlaps the other's transforms). Each CTA transforms its
// own rows along y, then, after a cluster barrier, columns y = 64 h .. 64 h + 63 along x,
// reading the other CTA's rows from its shared memory (distributed shared memory), and bins
// its outputs as k_plane_ps does. Transforms: the 16 x 8 two-step split of fft_core.cuh.
constexpr int kPs2Threads = 512;
constexpr int kPs2Rows = 64;                      // rows (and then columns) per CTA
constexpr int kPs2S = 129;                        // padded row stride (float2)
constexpr size_t kPs2Smem = (size_t)kPs2Rows * kPs2S * sizeof(float2) + 128 * sizeof(float2) +
                            (size_t)kPrivBins * kPs2Threads * sizeof(float);

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kPs2Threads, 2) k_plane_ps2(PSArgs a) {
    constexpr int N = 128, NH = N / 2 + 1, R1 = 16, R2 = 8;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;                                        // [64][kPs2S]
    float2* tw = smem + kPs2Rows * kPs2S;                      // [128]
    float* priv = reinterpret_cast<float*>(tw + N);            // [kPrivBins][threads]
    __shared__ double s_bins[EOR21_MAX_BINS];
    const int h = (int)cluster.block_rank();
    const int kz = blockIdx.x >> 1, slot = blockIdx.y;
    const int pair = a.pair0 + slot;
    const bool valid = pair < a.n_pairs;                       // uniform over the cluster
    const int t = threadIdx.x;
    fill_twiddles<N>(tw);
    for (int e = t; e < kPrivBins * kPs2Threads; e += kPs2Threads) priv[e] = 0.0f;
    for (int e = t; e < EOR21_MAX_BINS; e += kPs2Threads) s_bins[e] = 0.0;
    if (valid) {   // this CTA's 64 rows (contiguous in memory), two complex values per load
        const float4* src = reinterpret_cast<const float4*>(a.ps_inter + ((size_t)slot * NH + kz) * N * N +
                                                            (size_t)h * kPs2Rows * N);
        float4 v[kPs2Rows * N / 2 / kPs2Threads];
#pragma unroll
        for (int k = 0; k < kPs2Rows * N / 2 / kPs2Threads; k++) v[k] = __ldg(src + t + k * kPs2Threads);
#pragma unroll
        for (int k = 0; k < kPs2Rows * N / 2 / kPs2Threads; k++) {
            const int e = 2 * (t + k * kPs2Threads), r = e / N, c = e % N;
            buf[r * kPs2S + c] = make_float2(v[k].x, v[k].y);
            buf[r * kPs2S + c + 1] = make_float2(v[k].z, v[k].w);
        }
    }
    __syncthreads();
    // along y for each local row r: thread (i, r), i < R2
    const int i = t / kPs2Rows, r = t % kPs2Rows;
    if (valid) {
        float2 x[R1];
#pragma unroll
        for (int j = 0; j < R1; j++) x[j] = buf[r * kPs2S + j * R2 + i];
        dft_reg<R1, -1>(x);
#pragma unroll
        for (int k1 = 1; k1 < R1; k1++) x[k1] = cmul(x[k1], tw_get<N, -1>(tw, i * k1));
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) buf[r * kPs2S + k1 * R2 + i] = x[k1];
    }
    __syncthreads();
    float2 hold[R1 / R2][R2];
    if (valid) {
#pragma unroll
        for (int q = 0; q < R1 / R2; q++) {
            const int k1 = i + R2 * q;
#pragma unroll
            for (int i2 = 0; i2 < R2; i2++) hold[q][i2] = buf[r * kPs2S + k1 * R2 + i2];
            dft_reg<R2, -1>(hold[q]);
        }
    }
    __syncthreads();
    if (valid) {
#pragma unroll
        for (int q = 0; q < R1 / R2; q++)
#pragma unroll
            for (int k2 = 0; k2 < R2; k2++) buf[r * kPs2S + i + R2 * q + R1 * k2] = hold[q][k2];
    }
    cluster.sync();   // both halves transformed along y
    // along x for the cluster's columns y = 64 h + cl: thread (i, cl); rows 0..63 live in
    // CTA 0, rows 64..127 in CTA 1
    const int cl = t % kPs2Rows, c = h * kPs2Rows + cl;
    float2 x[R1];
    if (valid) {
        const float2* lo = cluster.map_shared_rank(buf, 0);
        const float2* hi = cluster.map_shared_rank(buf, 1);
#pragma unroll
        for (int j = 0; j < R1; j++) {
            const int row = j * R2 + i;
            x[j] = row < kPs2Rows ? lo[row * kPs2S + c] : hi[(row - kPs2Rows) * kPs2S + c];
        }
        dft_reg<R1, -1>(x);
#pragma unroll
        for (int k1 = 1; k1 < R1; k1++) x[k1] = cmul(x[k1], tw_get<N, -1>(tw, i * k1));
    }
    cluster.sync();   // every remote read is done: the buffer now holds this CTA's columns
    if (valid) {
#pragma unroll
        for (int k1 = 0; k1 < R1; k1++) buf[cl * kPs2S + k1 * R2 + i] = x[k1];
    }
    __syncthreads();
    if (valid) {
        const float weight = (kz == 0 || kz == N / 2) ? 1.0f : 2.0f;
        const int my = signed_index(c, N), mz2 = kz * kz;
#pragma unroll
        for (int q = 0; q < R1 / R2; q++) {
            const int k1 = i + R2 * q;
#pragma unroll
            for (int i2 = 0; i2 < R2; i2++) hold[q][i2] = buf[cl * kPs2S + k1 * R2 + i2];
            dft_reg<R2, -1>(hold[q]);
#pragma unroll
            for (int k2 = 0; k2 < R2; k2++) {   // mode (kx = k1 + R1 k2, ky = c, kz)
                const int mx = signed_index(k1 + R1 * k2, N);
                const int m2 = mx * mx + my * my + mz2;
                const int b = a.bin_of_m2[m2];
                if (b >= 0) {
                    const float2 u = hold[q][k2];
                    const float fm2 = (float)m2;
                    priv[b * kPs2Threads + t] += weight * a.kf3 * k3_of(fm2) * (u.x * u.x + u.y * u.y);
                }
            }
        }
    }
    __syncthreads();
    if (valid) bin_sums<kPs2Threads>(priv, a.n_bins, s_bins);
    __syncthreads();
    if (valid)
        for (int b = t; b < a.n_bins; b += kPs2Threads)
            if (s_bins[b] != 0.0) atomicAdd(&a.ps_sum[(size_t)pair * a.n_bins + b], s_bins[b]);
}

// ------------------------------------------------------------------ 256-point line passes
//
// A 256 x 256 complex plane (512 KB) does not fit one CTA's shared memory, so at n = 256 a
// plane pass becomes two line passes through global memory: 16 contiguous rows, or 16
// columns (stride 256), of 256 points per CTA, each line transformed by a team of 16 threads
// (256 = 16 x 16, the two-step split of fft_core.cuh). Lines sit in shared memory with one
// pad element per 16 (stage exchanges conflict-free) and an odd line stride (column loads
// conflict-free). Column-pass modes: plain store, density spectrum times a window on load
// (the inverse of pass 1), or the shell sums of the power spectrum (no store).

constexpr int kL = 256;
constexpr int kLLines = 16;                            // lines per CTA
constexpr int kLThreads = 16 * kLLines;                // a team of 16 threads per line
constexpr int kLStride = kL + kL / 16 + 1;             // 273 float2 per padded line
constexpr size_t kLSmemRows = (size_t)kLLines * kLStride * sizeof(float2) + kL * sizeof(float2);
constexpr size_t kLSmem = kLSmemRows + (size_t)kPrivBins * kLThreads * sizeof(float);   // column pass
__device__ __forceinline__ int lpad(int p) { return p + (p >> 4); }

enum LineMode : int { kLineStore = 0, kLineFilter = 1, kLinePs = 2 };

struct LineArgs {
    const float2* src;          // [task][NH][256][256], or the density spectra (kLineFilter)
    float2* dst;                // [task][NH][256][256] (kLineStore, kLineFilter)
    int G;                      // tasks per slot (radii of a launch); task = slot * G + tg
    // validity and windows (pass 1): pair = pair0 + slot, radius j0 + tg
    const PairInfo* pairs;      // nullptr: every task valid
    const float* wtab;          // [walker][max_radii][n_m2]
    int max_radii, n_m2, pair0, n_pairs, j0;
    // power spectrum
    const signed char* bin_of_m2;
    double* ps_sum;             // [pair][n_bins]
    int n_bins;
    float kf3;
};

// 256-point DFT of line `line` of buf in place (thread i of its team). On return thread i
// holds X[i + 16 k2] in hold[k2].
template <int DIR>
__device__ __forceinline__ void line_fft256(float2* buf, const float2* tw, int line, int i, float2 (&hold)[16]) {
    float2* L = buf + line * kLStride;
    float2 a[16];
#pragma unroll
    for (int j = 0; j < 16; j++) a[j] = L[lpad(j * 16 + i)];
    dft_reg<16, DIR>(a);
#pragma unroll
    for (int k1 = 1; k1 < 16; k1++) a[k1] = cmul(a[k1], tw_get<kL, DIR>(tw, i * k1));
    __syncthreads();
#pragma unroll
    for (int k1 = 0; k1 < 16; k1++) L[lpad(k1 * 16 + i)] = a[k1];
    __syncthreads();
#pragma unroll
    for (int i2 = 0; i2 < 16; i2++) hold[i2] = L[lpad(i * 16 + i2)];
    dft_reg<16, DIR>(hold);
}

__device__ __forceinline__ bool line_task_valid(const LineArgs& a, int slot, int tg) {
    if (!a.pairs) return true;
    const int pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return false;
    return a.wtab == nullptr || a.j0 + tg < a.pairs[pair].n_r;
}

// Rows of plane blockIdx.x / 16 (16 rows: blockIdx.x % 16) of task (blockIdx.z, blockIdx.y),
// transformed along the contiguous axis, src -> dst (may be the same buffer).
template <int DIR>
__global__ void __launch_bounds__(kLThreads) k_lines_rows(LineArgs a) {
    constexpr int NH = kL / 2 + 1;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = smem + kLLines * kLStride;
    const int plane = blockIdx.x / 16, rg = blockIdx.x % 16, tg = blockIdx.y, slot = blockIdx.z;
    if (!line_task_valid(a, slot, tg)) return;
    const size_t off = (((size_t)slot * a.G + tg) * NH + plane) * kL * kL + (size_t)rg * kLLines * kL;
    fill_twiddles<kL>(tw);
    const float2* src = a.src + off;
    for (int e = threadIdx.x; e < kLLines * kL; e += kLThreads) buf[(e / kL) * kLStride + lpad(e % kL)] = __ldg(src + e);
    __syncthreads();
    float2 hold[16];
    const int line = threadIdx.x / 16, i = threadIdx.x % 16;
    line_fft256<DIR>(buf, tw, line, i, hold);
    __syncthreads();
#pragma unroll
    for (int k2 = 0; k2 < 16; k2++) buf[line * kLStride + lpad(i + 16 * k2)] = hold[k2];
    __syncthreads();
    float2* dst = a.dst + off;
    for (int e = threadIdx.x; e < kLLines * kL; e += kLThreads) dst[e] = buf[(e / kL) * kLStride + lpad(e % kL)];
}

// Columns c0 .. c0 + 15 (c0 = 16 (blockIdx.x % 16)) of plane blockIdx.x / 16, transformed
// along the row index.
template <int DIR, int MODE>
__global__ void __launch_bounds__(kLThreads) k_lines_cols(LineArgs a) {
    constexpr int NH = kL / 2 + 1;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;
    float2* tw = smem + kLLines * kLStride;
    float* priv = reinterpret_cast<float*>(tw + kL);      // [kPrivBins][kLThreads]
    __shared__ double s_bins[EOR21_MAX_BINS];
    const int plane = blockIdx.x / 16, c0 = (blockIdx.x % 16) * kLLines, tg = blockIdx.y, slot = blockIdx.z;
    if (!line_task_valid(a, slot, tg)) return;
    fill_twiddles<kL>(tw);
    const size_t task_off = (((size_t)slot * a.G + tg) * NH + plane) * kL * kL;
    if constexpr (MODE == kLineFilter) {
        const int pair = a.pair0 + slot, j = a.j0 + tg;
        const PairInfo& pi = a.pairs[pair];
        const float2* spec = a.src + ((size_t)pi.zi * NH + plane) * kL * kL;
        const float* wt = a.wtab + ((size_t)pi.w * a.max_radii + j) * a.n_m2;
        const int mz2 = plane * plane;
        for (int e = threadIdx.x; e < kLLines * kL; e += kLThreads) {
            const int r = e / kLLines, cc = e % kLLines;
            const int mx = signed_index(r, kL), my = signed_index(c0 + cc, kL);
            const float wv = __ldg(wt + mx * mx + my * my + mz2);
            const float2 v = __ldg(spec + (size_t)r * kL + c0 + cc);
            buf[cc * kLStride + lpad(r)] = make_float2(v.x * wv, v.y * wv);
        }
    } else {
        const float2* src = a.src + task_off;
        for (int e = threadIdx.x; e < kLLines * kL; e += kLThreads) {
            const int r = e / kLLines, cc = e % kLLines;
            buf[cc * kLStride + lpad(r)] = __ldg(src + (size_t)r * kL + c0 + cc);
        }
    }
    if constexpr (MODE == kLinePs) {
        for (int e = threadIdx.x; e < kPrivBins * kLThreads; e += kLThreads) priv[e] = 0.0f;
        for (int e = threadIdx.x; e < EOR21_MAX_BINS; e += kLThreads) s_bins[e] = 0.0;
    }
    __syncthreads();
    float2 hold[16];
    const int line = threadIdx.x / 16, i = threadIdx.x % 16;
    line_fft256<DIR>(buf, tw, line, i, hold);
    if constexpr (MODE == kLinePs) {
        // row index r = i + 16 k2 (kx), column c0 + line (ky), plane kz: S_b += w k^3 |X|^2
        const float weight = (plane == 0 || plane == kL / 2) ? 1.0f : 2.0f;
        const int my = signed_index(c0 + line, kL), mz2 = plane * plane;
        const bool priv_ok = a.n_bins <= kPrivBins;
#pragma unroll
        for (int k2 = 0; k2 < 16; k2++) {
            const int mx = signed_index(i + 16 * k2, kL);
            const int m2 = mx * mx + my * my + mz2;
            const int b = a.bin_of_m2[m2];
            if (b >= 0) {
                const float2 v = hold[k2];
                const float fm2 = (float)m2;
                const float val = weight * a.kf3 * k3_of(fm2) * (v.x * v.x + v.y * v.y);
                if (priv_ok) priv[b * kLThreads + threadIdx.x] += val;
                else atomicAdd(&s_bins[b], (double)val);
            }
        }
        __syncthreads();
        if (priv_ok) {
            bin_sums<kLThreads>(priv, a.n_bins, s_bins);
            __syncthreads();
        }
        const int pair = a.pair0 + slot;
        for (int b = threadIdx.x; b < a.n_bins; b += kLThreads)
            if (s_bins[b] != 0.0) atomicAdd(&a.ps_sum[(size_t)pair * a.n_bins + b], s_bins[b]);
    } else {
        __syncthreads();
#pragma unroll
        for (int k2 = 0; k2 < 16; k2++) buf[line * kLStride + lpad(i + 16 * k2)] = hold[k2];
        __syncthreads();
        float2* dst = a.dst + task_off;
        for (int e = threadIdx.x; e < kLLines * kL; e += kLThreads) {
            const int r = e / kLLines, cc = e % kLLines;
            dst[(size_t)r * kL + c0 + cc] = buf[cc * kLStride + lpad(r)];
        }
    }
}

// ------------------------------------------------------------------ pencil pass

template <int N>
struct Pencil {
    static constexpr int M = N / 2;                      // complex length of the z transform
    static constexpr int P1 = Split<M>::R1, P2 = Split<M>::R2;
    static constexpr int TY = N < 32 ? N : 32;           // pencils per CTA (consecutive y)
    static constexpr int THREADS = TY * P2;
    static constexpr int NBp = P1 / P2;
    static constexpr int DS = N + 2;                     // density tile row stride (floats)
    static constexpr int TILES = N * N / TY;
    static constexpr size_t SMEM = (size_t)(M + 1) * TY * sizeof(float2) + (size_t)M * TY * sizeof(float2) +
                                   (size_t)TY * DS * sizeof(float) + N * sizeof(float2);
};

template <int N>
struct PencilSmem {
    float2* xs;   // [(M+1)][TY] half spectrum of the tile's pencils, or Z after a forward core
    float2* zs;   // [M][TY] exchange
    float* ds;    // [TY][DS] density / x_HI tile
    float2* tw;   // [N]
    __device__ PencilSmem(void* base) {
        using P = Pencil<N>;
        char* p = (char*)base;
        xs = (float2*)p; p += (size_t)(P::M + 1) * P::TY * sizeof(float2);
        zs = (float2*)p; p += (size_t)P::M * P::TY * sizeof(float2);
        tw = (float2*)p; p += N * sizeof(float2);
        ds = (float*)p;
    }
};

// Complex-to-real along z for the tile's pencils: xs holds X[k] (k = 0..M) per pencil.
// On return z[q][k2] = x[2m] + i x[2m+1] with m = i + P2 q + P1 k2 (unnormalised).
template <int N>
__device__ __forceinline__ void pencil_c2r(const PencilSmem<N>& s, int p, int i,
                                           float2 (&z)[Pencil<N>::NBp][Pencil<N>::P2]) {
    using P = Pencil<N>;
    float2 a[P::P1];
#pragma unroll
    for (int j = 0; j < P::P1; j++) {
        const int k = j * P::P2 + i;
        const float2 xk = s.xs[k * P::TY + p], xm = cconj(s.xs[(P::M - k) * P::TY + p]);
        const float2 sum = cadd(xk, xm), dif = cmul(csub(xk, xm), tw_get<N, +1>(s.tw, k));
        a[j] = make_float2(sum.x - dif.y, sum.y + dif.x);     // sum + i * dif
    }
    dft_reg<P::P1, +1>(a);
#pragma unroll
    for (int k1 = 1; k1 < P::P1; k1++) a[k1] = cmul(a[k1], tw_get<N, +1>(s.tw, 2 * i * k1));
#pragma unroll
    for (int k1 = 0; k1 < P::P1; k1++) s.zs[(k1 * P::P2 + i) * P::TY + p] = a[k1];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < P::NBp; q++) {
        const int k1 = i + P::P2 * q;
#pragma unroll
        for (int i2 = 0; i2 < P::P2; i2++) z[q][i2] = s.zs[(k1 * P::P2 + i2) * P::TY + p];
        dft_reg<P::P2, +1>(z[q]);
    }
}

// Real-to-complex along z: z[q][k2] = x[2m] + i x[2m+1] with m = i + P2 q + P1 k2.
// Writes X[k], k = 0..M, of every pencil to dst[k * kstride + p].
template <int N>
__device__ __forceinline__ void pencil_r2c(const PencilSmem<N>& s, int p, int i,
                                           const float2 (&z)[Pencil<N>::NBp][Pencil<N>::P2], float2* dst,
                                           size_t kstride) {
    using P = Pencil<N>;
    float2 a[P::P1];
#pragma unroll
    for (int q = 0; q < P::NBp; q++)
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) a[q + P::NBp * k2] = z[q][k2];   // element m = i + P2 * j
    dft_reg<P::P1, -1>(a);
#pragma unroll
    for (int k1 = 1; k1 < P::P1; k1++) a[k1] = cmul(a[k1], tw_get<N, -1>(s.tw, 2 * i * k1));
    __syncthreads();   // zs and xs may still be read by a previous step
#pragma unroll
    for (int k1 = 0; k1 < P::P1; k1++) s.zs[(k1 * P::P2 + i) * P::TY + p] = a[k1];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < P::NBp; q++) {
        const int k1 = i + P::P2 * q;
        float2 b[P::P2];
#pragma unroll
        for (int i2 = 0; i2 < P::P2; i2++) b[i2] = s.zs[(k1 * P::P2 + i2) * P::TY + p];
        dft_reg<P::P2, -1>(b);
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) s.xs[(k1 + P::P1 * k2) * P::TY + p] = b[k2];   // Z natural
    }
    __syncthreads();
    // the split in pairs (k, M - k), one pair per two loads and one twiddle:
    // X[k] = E - (i/2) D, X[M - k] = conj(E) - (i/2) conj(D), E = (Z[k] + conj Z[M-k]) / 2,
    // D = (Z[k] - conj Z[M-k]) w_N^k (Z[M] = Z[0]; X[M] = E + (i/2) D at k = 0)
    for (int k = i; 2 * k <= P::M; k += P::P2) {
        const float2 zk = s.xs[k * P::TY + p];
        const float2 zm = cconj(s.xs[((P::M - k) & (P::M - 1)) * P::TY + p]);
        const float2 e = cscale(cadd(zk, zm), 0.5f);
        const float2 d = cmul(csub(zk, zm), tw_get<N, -1>(s.tw, k));
        dst[(size_t)k * kstride + p] = make_float2(e.x + 0.5f * d.y, e.y - 0.5f * d.x);
        if (k == 0)
            dst[(size_t)P::M * kstride + p] = make_float2(e.x - 0.5f * d.y, e.y + 0.5f * d.x);
        else if (2 * k != P::M)
            dst[(size_t)(P::M - k) * kstride + p] = make_float2(e.x - 0.5f * d.y, -e.y - 0.5f * d.x);
    }
}

template <int N>
__device__ __forceinline__ void pencil_load_spectrum(const PencilSmem<N>& s, const float2* src, size_t kstride) {
    using P = Pencil<N>;
    const int p = threadIdx.x % P::TY;
    for (int row = threadIdx.x / P::TY; row <= P::M; row += P::THREADS / P::TY)
        s.xs[row * P::TY + p] = __ldg(src + (size_t)row * kstride + p);
}

// Load the tile's TY pencils of a real box (contiguous TY * N floats) into ds: every load of
// a thread is issued before the first store, so that enough bytes are in flight to cover the
// memory latency.
template <int N>
__device__ __forceinline__ void pencil_load_real(const PencilSmem<N>& s, const float* src) {
    using P = Pencil<N>;
    constexpr int V = P::TY * N / 4;                             // float4 per tile
    constexpr int PER = (V + P::THREADS - 1) / P::THREADS;
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4 v[PER];
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const int e = threadIdx.x + k * P::THREADS;
        if (e < V) v[k] = __ldg(s4 + e);
    }
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const int e = threadIdx.x + k * P::THREADS;
        if (e < V) {
            const int pp = (4 * e) / N, zz = (4 * e) % N;
            float2* d = reinterpret_cast<float2*>(s.ds + pp * P::DS + zz);
            d[0] = make_float2(v[k].x, v[k].y);
            d[1] = make_float2(v[k].z, v[k].w);
        }
    }
}

template <int N>
__device__ __forceinline__ void pencil_store_real(const PencilSmem<N>& s, float* dst) {
    using P = Pencil<N>;
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int e = threadIdx.x; e < P::TY * N / 4; e += P::THREADS) {
        const int pp = (4 * e) / N, zz = (4 * e) % N;
        const float2* sv = reinterpret_cast<const float2*>(s.ds + pp * P::DS + zz);
        const float2 u = sv[0], v = sv[1];
        d4[e] = make_float4(u.x, u.y, v.x, v.y);
    }
}

struct Pass2Args {
    const float2* inter;        // [P slots][G][nh][n][n]
    const PairInfo* pairs;
    uint32_t* flags;            // [P slots][TILES][THREADS]
    const float* delta;         // [n_z][n^3]
    float* xhi_out;             // optional [pair][n^3]
    double* xhi_sum;            // [pair]
    float2* ps_inter;           // [P slots][nh][n][n]
    const float* ftab;          // [pair][kFTab] with a mass-dependent efficiency, else nullptr
    int pair0, n_pairs, j0, G;
    float delta_c;
};

// Pass 2: for the group of radii j0 .. j0+G-1 of one (walker, redshift): C2R along z,
// flag |= delta_R >= delta_crit(R). The group that holds R_cell then forms x_HI, delta T_b
// and delta T_b's R2C along z.
template <int N>
__global__ void __launch_bounds__(Pencil<N>::THREADS) k_pencil_ionize(Pass2Args a) {
    using P = Pencil<N>;
    constexpr int NH = N / 2 + 1;
    extern __shared__ __align__(16) float2 smem[];
    const PencilSmem<N> s(smem);
    const int tile = blockIdx.x, slot = blockIdx.y;
    const int pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return;
    const PairInfo& pi = a.pairs[pair];
    const int n_r = pi.n_r;
    if (a.j0 >= n_r) return;
    const int jend = min(a.j0 + a.G, n_r);
    const bool last = (jend == n_r);
    const int t = threadIdx.x, p = t % P::TY, i = t / P::TY;
    const int x = tile / (N / P::TY), y0 = (tile % (N / P::TY)) * P::TY;
    fill_twiddles<N>(s.tw);
    const size_t fidx = ((size_t)slot * P::TILES + tile) * P::THREADS + t;
    uint32_t flags = a.j0 == 0 ? 0u : a.flags[fidx];
    const float scale = 1.0f / ((float)N * (float)N * (float)N);
    float2 z[P::NBp][P::P2];
    for (int j = a.j0; j < jend; j++) {
        const float2* src = a.inter + (((size_t)slot * a.G + (j - a.j0)) * NH) * N * N + (size_t)x * N + y0;
        pencil_load_spectrum<N>(s, src, (size_t)N * N);
        __syncthreads();
        pencil_c2r<N>(s, p, i, z);
        const float dcrit = pi.delta_crit[j], dhi = pi.delta_hi[j];
#pragma unroll
        for (int q = 0; q < P::NBp; q++)
#pragma unroll
            for (int k2 = 0; k2 < P::P2; k2++) {
                const int bit = 2 * (q * P::P2 + k2);
                const float d0 = z[q][k2].x * scale, d1 = z[q][k2].y * scale;
                flags |= (uint32_t)(d0 >= dcrit && d0 <= dhi) << bit;
                flags |= (uint32_t)(d1 >= dcrit && d1 <= dhi) << (bit + 1);
            }
    }
    if (!last) {
        a.flags[fidx] = flags;
        return;
    }
    // ---- R_cell reached: partial ionization, x_HI, delta T_b (z holds delta at R_cell)
    const size_t n3 = (size_t)N * N * N;
    pencil_load_real<N>(s, a.delta + (size_t)pi.zi * n3 + ((size_t)x * N + y0) * N);
    __syncthreads();
    const float zeta = pi.zeta, t0 = pi.t0, inv = pi.inv_sqrt2s2_cell, dc = a.delta_c;
    const bool cell_ok = pi.cell_ok > 0.5f;
    float xsum = 0.0f;
#pragma unroll
    for (int q = 0; q < P::NBp; q++)
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) {
            const int m = i + P::P2 * q + P::P1 * k2;
            const int bit = 2 * (q * P::P2 + k2);
            float out[2];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const float dr = (h ? z[q][k2].y : z[q][k2].x) * scale;
                float f = 0.0f;
                if (a.ftab) f = pop_table_f(a.ftab + (size_t)pair * kFTab, dc - dr, pi.f_inv_h);   // efficiency-weighted
                else if (cell_ok) f = dr >= dc ? 1.0f : erfcf((dc - dr) * inv);
                const float xhii = ((flags >> (bit + h)) & 1u) ? 1.0f : fminf(1.0f, zeta * f);
                const float xhi = 1.0f - xhii;
                float* cell = s.ds + p * P::DS + 2 * m + h;
                out[h] = t0 * xhi * (1.0f + *cell);
                *cell = xhi;
                xsum += xhi;
            }
            z[q][k2] = make_float2(out[0], out[1]);
        }
    // neutral-fraction sum (FP64 across the block)
    double v = (double)xsum;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((t & 31) == 0) atomicAdd(&a.xhi_sum[pair], v);
    if (a.xhi_out) {
        __syncthreads();
        pencil_store_real<N>(s, a.xhi_out + (size_t)pair * n3 + ((size_t)x * N + y0) * N);
    }
    float2* dst = a.ps_inter + (size_t)slot * NH * N * N + (size_t)x * N + y0;
    pencil_r2c<N>(s, p, i, z, dst, (size_t)N * N);
}

// Forward R2C along z of a real box: src [n^3] -> dst [nh][n][n] ([kz][x][y]).
template <int N>
__global__ void __launch_bounds__(Pencil<N>::THREADS) k_pencil_forward(const float* src, float2* dst) {
    using P = Pencil<N>;
    extern __shared__ __align__(16) float2 smem[];
    const PencilSmem<N> s(smem);
    const int tile = blockIdx.x;
    const int t = threadIdx.x, p = t % P::TY, i = t / P::TY;
    const int x = tile / (N / P::TY), y0 = (tile % (N / P::TY)) * P::TY;
    fill_twiddles<N>(s.tw);
    pencil_load_real<N>(s, src + ((size_t)x * N + y0) * N);
    __syncthreads();
    float2 z[P::NBp][P::P2];
#pragma unroll
    for (int q = 0; q < P::NBp; q++)
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) {
            const int m = i + P::P2 * q + P::P1 * k2;
            z[q][k2] = make_float2(s.ds[p * P::DS + 2 * m], s.ds[p * P::DS + 2 * m + 1]);
        }
    pencil_r2c<N>(s, p, i, z, dst + (size_t)x * N + y0, (size_t)N * N);
}

// Forward R2C along z of the real boxes of pairs pair0 .. pair0 + gridDim.y - 1:
// src [pair][n^3] -> dst [slot][nh][n][n].
template <int N>
__global__ void __launch_bounds__(Pencil<N>::THREADS) k_pencil_forward_batch(const float* src, float2* dst, int pair0,
                                                                            int n_pairs) {
    using P = Pencil<N>;
    constexpr int NH = N / 2 + 1;
    extern __shared__ __align__(16) float2 smem[];
    const PencilSmem<N> s(smem);
    const int tile = blockIdx.x, slot = blockIdx.y, pair = pair0 + slot;
    if (pair >= n_pairs) return;
    const int t = threadIdx.x, p = t % P::TY, i = t / P::TY;
    const int x = tile / (N / P::TY), y0 = (tile % (N / P::TY)) * P::TY;
    fill_twiddles<N>(s.tw);
    pencil_load_real<N>(s, src + (size_t)pair * N * N * N + ((size_t)x * N + y0) * N);
    __syncthreads();
    float2 z[P::NBp][P::P2];
#pragma unroll
    for (int q = 0; q < P::NBp; q++)
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) {
            const int m = i + P::P2 * q + P::P1 * k2;
            z[q][k2] = make_float2(s.ds[p * P::DS + 2 * m], s.ds[p * P::DS + 2 * m + 1]);
        }
    pencil_r2c<N>(s, p, i, z, dst + (size_t)slot * NH * N * N + (size_t)x * N + y0, (size_t)N * N);
}

// round(v 2^23) for v in [0, 1], as __float2int_rn(v * 2^23) gives it, without the
// conversion unit: v 2^23 + 2^23 lies in [2^23, 2^24], where the float spacing is 1, so the
// fused multiply-add rounds to the nearest integer (ties to even) and its bits minus those of
// 2^23 are that integer.
__device__ __forceinline__ int fixed23(float v) {
    return __float_as_int(fmaf(v, 8388608.0f, 8388608.0f)) - 0x4B000000;
}

// x_HI of four cells (Sec. 2.1): 0 where a radius above R_cell flagged the cell (bit h of
// `bits`), else 1 - min(1, zeta f_coll(R_cell)) with f_coll = erfc((delta_c - delta_Rcell) inv),
// inv = 1 / sqrt(2 s^2) (f_coll = 1 where delta_Rcell >= delta_c; x_HI = 1 where s^2 <= 0, inv
// = 0), or with a mass-dependent efficiency 1 - min(1, F) from the pair's table `ftab` of the
// efficiency-weighted collapsed fraction at nu = delta_c - delta_Rcell. The step-function form
// is branch-free, its four erfc evaluations independent: a per-cell branch around them cost
// more than the evaluations it skipped.
__device__ __forceinline__ void xhi4(uint32_t bits, const float (&dc)[4], float delta_c, float zeta, float inv,
                                     const float* ftab, float f_inv_h, float (&xh)[4]) {
    if (ftab) {
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const float nu = delta_c - dc[h];
            xh[h] = ((bits >> h) & 1u) ? 0.0f : 1.0f - fminf(1.0f, pop_table_f(ftab, nu, f_inv_h));
        }
    } else {
#pragma unroll
        for (int h = 0; h < 4; h++) {
            const float nu = delta_c - dc[h];
            const float fe = erfc_cheb(fmaxf(nu, 0.0f) * inv);
            const float v = inv > 0.0f ? 1.0f - fminf(1.0f, zeta * (nu <= 0.0f ? 1.0f : fe)) : 1.0f;
            xh[h] = ((bits >> h) & 1u) ? 0.0f : v;
        }
    }
}

struct BrightArgs {
    const uint32_t* fwords;     // [pair][n3 / 32] Eq. 1 flags above R_cell (bit = cell % 32)
    const PairInfo* pairs;
    const float* delta;         // brightness base [n_z][n3]
    const float* dcell;         // [n_z][n3] delta at R_cell
    float* xhi_out;             // optional [pair][n3]
    unsigned long long* xq;     // [pair] fixed-point (2^23) sums of x_HI
    float2* dst;                // [slot][nh][n][n]
    const float* ftab;          // [pair][kFTab] with a mass-dependent efficiency, else nullptr
    int pair0, n_pairs;
    float delta_c;
};

// The flag contraction's pencil pass, for pairs pair0 .. pair0 + gridDim.y - 1: per cell of
// the tile's pencils x_HI = 0 where a radius above R_cell flagged it (Eq. 1), else
// 1 - min(1, zeta f_coll(R_cell)) with f_coll = erfc((delta_c - delta_Rcell) / sqrt(2 s^2))
// (1 where delta_Rcell >= delta_c; x_HI = 1 where s^2 <= 0) (Sec. 2.1), or with a
// mass-dependent efficiency 1 - min(1, F) from the pair's table of the efficiency-weighted
// collapsed fraction F at nu = delta_c - delta_Rcell (staged in shared memory); delta T_b =
// T0 x_HI (1 + delta) (Sec. 2.2), never stored; then its R2C along z into dst. The x_HI sum
// of the pair is exact: fixed point 2^-23, integer warp sums and 64-bit atomics.
template <int N>
__global__ void __launch_bounds__(Pencil<N>::THREADS) k_pencil_brightness(BrightArgs a) {
    using P = Pencil<N>;
    constexpr int NH = N / 2 + 1;
    constexpr int V = P::TY * N / 4;                             // float4 per tile
    constexpr int PER = (V + P::THREADS - 1) / P::THREADS;
    extern __shared__ __align__(16) float2 smem[];
    const PencilSmem<N> s(smem);
    float* ftab = reinterpret_cast<float*>(reinterpret_cast<char*>(smem) + Pencil<N>::SMEM);   // [kFTab]
    const int tile = blockIdx.x, slot = blockIdx.y, pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return;
    const PairInfo& pi = a.pairs[pair];
    const int t = threadIdx.x, p = t % P::TY, i = t / P::TY;
    const int x = tile / (N / P::TY), y0 = (tile % (N / P::TY)) * P::TY;
    const size_t n3 = (size_t)N * N * N, cell0 = ((size_t)x * N + y0) * N;
    fill_twiddles<N>(s.tw);
    if (a.ftab) {
        for (int e = t; e < kFTab; e += P::THREADS) ftab[e] = __ldg(a.ftab + (size_t)pair * kFTab + e);
        __syncthreads();
    }
    const float4* d4 = reinterpret_cast<const float4*>(a.delta + (size_t)pi.zi * n3 + cell0);
    const float4* c4 = reinterpret_cast<const float4*>(a.dcell + (size_t)pi.zi * n3 + cell0);
    const uint32_t* fw = a.fwords + (size_t)pair * (n3 / 32) + cell0 / 32;
    float4 dv[PER], cv[PER];
    uint32_t bits[PER];
#pragma unroll
    for (int k = 0; k < PER; k++) {   // every load issued before the first use
        const int e = t + k * P::THREADS;
        if (e < V) {
            dv[k] = __ldg(d4 + e);
            cv[k] = __ldg(c4 + e);
            bits[k] = __ldg(fw + (4 * e) / 32) >> ((4 * e) % 32);
        }
    }
    const float zeta = pi.zeta, t0 = pi.t0, inv = pi.cell_ok > 0.5f ? pi.inv_sqrt2s2_cell : 0.0f;
    int xq = 0;   // at most 32 cells x 2^23 per thread
#pragma unroll
    for (int k = 0; k < PER; k++) {
        const int e = t + k * P::THREADS;
        if (e >= V) continue;
        const float dd[4] = {dv[k].x, dv[k].y, dv[k].z, dv[k].w}, dc[4] = {cv[k].x, cv[k].y, cv[k].z, cv[k].w};
        float xh[4], tb[4];
        xhi4(bits[k], dc, a.delta_c, zeta, inv, a.ftab ? ftab : nullptr, pi.f_inv_h, xh);
#pragma unroll
        for (int h = 0; h < 4; h++) {
            tb[h] = t0 * xh[h] * (1.0f + dd[h]);
            xq += fixed23(xh[h]);
        }
        const int pp = (4 * e) / N, zz = (4 * e) % N;
        float2* d = reinterpret_cast<float2*>(s.ds + pp * P::DS + zz);
        d[0] = make_float2(tb[0], tb[1]);
        d[1] = make_float2(tb[2], tb[3]);
        if (a.xhi_out)
            reinterpret_cast<float4*>(a.xhi_out + (size_t)pair * n3 + cell0)[e] = make_float4(xh[0], xh[1], xh[2], xh[3]);
    }
    unsigned long long wsum = (unsigned long long)xq;       // a warp's cells can reach 2^32 in 2^-23 units
    for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
    if ((t & 31) == 0) atomicAdd(a.xq + pair, wsum);
    __syncthreads();
    float2 z[P::NBp][P::P2];
#pragma unroll
    for (int q = 0; q < P::NBp; q++)
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) {
            const int m = i + P::P2 * q + P::P1 * k2;
            z[q][k2] = make_float2(s.ds[p * P::DS + 2 * m], s.ds[p * P::DS + 2 * m + 1]);
        }
    pencil_r2c<N>(s, p, i, z, a.dst + (size_t)slot * NH * N * N + (size_t)x * N + y0, (size_t)N * N);
}

// Inverse C2R along z of one task's plane-pass output, writing delta_R (normalised).
template <int N>
__global__ void __launch_bounds__(Pencil<N>::THREADS) k_pencil_density(const float2* src, float* out) {
    using P = Pencil<N>;
    extern __shared__ __align__(16) float2 smem[];
    const PencilSmem<N> s(smem);
    const int tile = blockIdx.x;
    const int t = threadIdx.x, p = t % P::TY, i = t / P::TY;
    const int x = tile / (N / P::TY), y0 = (tile % (N / P::TY)) * P::TY;
    fill_twiddles<N>(s.tw);
    pencil_load_spectrum<N>(s, src + (size_t)x * N + y0, (size_t)N * N);
    __syncthreads();
    float2 z[P::NBp][P::P2];
    pencil_c2r<N>(s, p, i, z);
    const float scale = 1.0f / ((float)N * (float)N * (float)N);
#pragma unroll
    for (int q = 0; q < P::NBp; q++)
#pragma unroll
        for (int k2 = 0; k2 < P::P2; k2++) {
            const int m = i + P::P2 * q + P::P1 * k2;
            s.ds[p * P::DS + 2 * m] = z[q][k2].x * scale;
            s.ds[p * P::DS + 2 * m + 1] = z[q][k2].y * scale;
        }
    __syncthreads();
    pencil_store_real<N>(s, out + ((size_t)x * N + y0) * N);
}

// ------------------------------------------------------------------ slab passes of the spectrum
//
// The power spectrum's 3D transform at n <= 128 as two passes, each CTA small enough that
// several share an SM (and the two passes of consecutive batches share SMs on two streams):
//   slab pass  — one CTA per (x slab, pair): the slab's n x n real values (rows y, columns z)
//                sit in shared memory as n rows of M + 1 complex values (M = n / 2; the odd
//                row stride keeps every column and row walk conflict-free). The CTA forms the
//                real input (delta T_b from the Eq. 1 flags, or a stored box), transforms
//                along z (an M-point complex FFT of the packed (even, odd) pairs, then the
//                real-to-half-complex split), then along y, all in place, and writes planes
//                kz < planes of [kz][x][y slot];
//   x-line pass — one CTA per (kz plane, 32 y slots, pair): the transform along x, then the
//                shell sums as in k_plane_ps.
// In-place two-step transforms leave their outputs in a permuted order, which only relabels
// the modes: after the z transform kz = k1 + P1 k2 sits in column P2 k1 + k2 (kz = M in the
// extra column M), after the y transform ky = k1 + R1 k2 in row slot R2 k1 + k2.

template <int N>
struct Slab {
    static constexpr int M = N / 2, ZS = M + 1;                   // row stride (float2), odd
    static constexpr int P1 = Split<M>::R1, P2 = Split<M>::R2;   // the z transform (M points)
    static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;   // the y transform (N points)
    static constexpr int THREADS = N * N / 4 < 256 ? N * N / 4 : 256;
    static constexpr size_t SMEM = (size_t)N * ZS * sizeof(float2) + N * sizeof(float2);
};

template <int N>
__device__ __forceinline__ int slab_col(int kz) {
    using S = Slab<N>;
    return kz == S::M ? S::M : S::P2 * (kz % S::P1) + kz / S::P1;
}

// ky (or kx) held by row slot r after an in-place two-step N-point transform
template <int N>
__device__ __forceinline__ int slot_k(int r) {
    return r / Split<N>::R2 + Split<N>::R1 * (r % Split<N>::R2);
}

struct SlabArgs {
    const uint32_t* fwords;     // flag contraction: [pair][n3 / 32] Eq. 1 flags above R_cell
    const PairInfo* pairs;
    const float* delta;         // brightness base [n_z][n3]
    const float* dcell;         // [n_z][n3] delta at R_cell
    float* xhi_out;             // optional [pair][n3]
    unsigned long long* xq;     // [pair] fixed-point (2^23) sums of x_HI
    const float* ftab;          // [pair][kFTab] with a mass-dependent efficiency, else nullptr
    const float* box;           // stored boxes [pair][n3] (the other methods' delta T_b)
    float2* dst;                // [slot][nh][n][n]: planes kz < planes, [kz][x][y slot]
    int pair0, n_pairs, planes;
    float delta_c;
};

// One radix step of an in-place two-step transform over the R elements e[s * stride]
// (s = first + step * j, j < R): DFT over j, then the twiddles w_N^(tw_mul * i * k1), the
// outputs back into the same slots (slot first + step * k1).
template <int N, int R, int DIR>
__device__ __forceinline__ void ip_stage1(float2* e, int stride, int step, const float2* tw, int i, int tw_mul) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; j++) v[j] = e[(step * j) * stride];
    dft_reg<R, DIR>(v);
#pragma unroll
    for (int k1 = 1; k1 < R; k1++) v[k1] = cmul(v[k1], tw_get<N, DIR>(tw, tw_mul * i * k1));
#pragma unroll
    for (int k1 = 0; k1 < R; k1++) e[(step * k1) * stride] = v[k1];
}

// The second step: DFT over the R consecutive slots e[j * stride], outputs back in place.
template <int R, int DIR>
__device__ __forceinline__ void ip_stage2(float2* e, int stride) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; j++) v[j] = e[j * stride];
    dft_reg<R, DIR>(v);
#pragma unroll
    for (int k = 0; k < R; k++) e[k * stride] = v[k];
}

// The slab pass for pairs pair0 .. pair0 + gridDim.y - 1, slab x = blockIdx.x. BRIGHT: per
// cell x_HI = 0 where a radius above R_cell flagged it (Eq. 1), else 1 - min(1, zeta f_coll(R_cell))
// with f_coll = erfc((delta_c - delta_Rcell) / sqrt(2 s^2)) (1 where delta_Rcell >= delta_c;
// x_HI = 1 where s^2 <= 0) (Sec. 2.1), or with a mass-dependent efficiency 1 - min(1, F) from
// the pair's table of the efficiency-weighted collapsed fraction at nu = delta_c - delta_Rcell;
// delta T_b = T0 x_HI (1 + delta) (Sec. 2.2), never stored; the pair's x_HI sum is exact (fixed
// point 2^-23, integer warp sums and 64-bit atomics). Otherwise the input is the pair's stored box.
template <int N, bool BRIGHT>
__global__ void __launch_bounds__(Slab<N>::THREADS, 3) k_slab_ps(SlabArgs a) {
    using S = Slab<N>;
    constexpr int T = S::THREADS, NH = S::M + 1, ZS = S::ZS;
    constexpr int V = N * N / 4;                     // float4 per slab
    constexpr int PER = V / T;                       // float4 per thread
    constexpr int BATCH = PER < 4 ? PER : 4;         // loads in flight per thread
    static_assert(PER * T == V && PER % BATCH == 0, "slab tiling");
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;                              // [N][ZS]
    float2* tw = smem + N * ZS;                      // [N]
    float* ftab = reinterpret_cast<float*>(tw + N);  // [kFTab]
    float* re = reinterpret_cast<float*>(buf);       // real view: row y at re + 2 ZS y
    const int x = blockIdx.x, slot = blockIdx.y, pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return;
    const int t = threadIdx.x;
    const size_t n3 = (size_t)N * N * N, cell0 = (size_t)x * N * N;
    fill_twiddles<N>(tw);
    if constexpr (BRIGHT) {
        const PairInfo& pi = a.pairs[pair];
        if (a.ftab) {
            for (int e = t; e < kFTab; e += T) ftab[e] = __ldg(a.ftab + (size_t)pair * kFTab + e);
            __syncthreads();
        }
        const float4* d4 = reinterpret_cast<const float4*>(a.delta + (size_t)pi.zi * n3 + cell0);
        const float4* c4 = reinterpret_cast<const float4*>(a.dcell + (size_t)pi.zi * n3 + cell0);
        const uint32_t* fw = a.fwords + (size_t)pair * (n3 / 32) + cell0 / 32;
        const float zeta = pi.zeta, t0 = pi.t0, inv = pi.cell_ok > 0.5f ? pi.inv_sqrt2s2_cell : 0.0f;
        int xq = 0;   // at most 64 cells x 2^23 per thread
#pragma unroll 1
        for (int k0 = 0; k0 < PER; k0 += BATCH) {
            float4 dv[BATCH], cv[BATCH];
            uint32_t bits[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; k++) {   // every load of the batch before the first use
                const int e = t + (k0 + k) * T;
                dv[k] = __ldg(d4 + e);
                cv[k] = __ldg(c4 + e);
                bits[k] = __ldg(fw + (4 * e) / 32) >> ((4 * e) % 32);
            }
#pragma unroll
            for (int k = 0; k < BATCH; k++) {
                const int e = t + (k0 + k) * T;
                const float dd[4] = {dv[k].x, dv[k].y, dv[k].z, dv[k].w}, dc[4] = {cv[k].x, cv[k].y, cv[k].z, cv[k].w};
                float xh[4], tb[4];
                xhi4(bits[k], dc, a.delta_c, zeta, inv, a.ftab ? ftab : nullptr, pi.f_inv_h, xh);
#pragma unroll
                for (int h = 0; h < 4; h++) {
                    tb[h] = t0 * xh[h] * (1.0f + dd[h]);
                    xq += fixed23(xh[h]);
                }
                const int y = (4 * e) / N, z = (4 * e) % N;
                float2* d = reinterpret_cast<float2*>(re + 2 * ZS * y + z);
                d[0] = make_float2(tb[0], tb[1]);
                d[1] = make_float2(tb[2], tb[3]);
                if (a.xhi_out)
                    reinterpret_cast<float4*>(a.xhi_out + (size_t)pair * n3 + cell0)[e] =
                        make_float4(xh[0], xh[1], xh[2], xh[3]);
            }
        }
        unsigned long long wsum = (unsigned long long)xq;
        for (int off = 16; off > 0; off >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, off);
        if ((t & 31) == 0) atomicAdd(a.xq + pair, wsum);
    } else {
        const float4* b4 = reinterpret_cast<const float4*>(a.box + (size_t)pair * n3 + cell0);
#pragma unroll 1
        for (int k0 = 0; k0 < PER; k0 += BATCH) {
            float4 v[BATCH];
#pragma unroll
            for (int k = 0; k < BATCH; k++) v[k] = __ldg(b4 + t + (k0 + k) * T);
#pragma unroll
            for (int k = 0; k < BATCH; k++) {
                const int e = t + (k0 + k) * T, y = (4 * e) / N, z = (4 * e) % N;
                float2* d = reinterpret_cast<float2*>(re + 2 * ZS * y + z);
                d[0] = make_float2(v[k].x, v[k].y);
                d[1] = make_float2(v[k].z, v[k].w);
            }
        }
    }
    __syncthreads();
    // along z: the M-point FFT of c[m] = x[2m] + i x[2m+1] per row y (lanes walk y)
#pragma unroll 1
    for (int u = t; u < N * S::P2; u += T) {
        const int y = u % N, i = u / N;
        ip_stage1<N, S::P1, -1>(buf + y * ZS + i, 1, S::P2, tw, i, 2);
    }
    __syncthreads();
#pragma unroll 1
    for (int u = t; u < N * S::P1; u += T) {
        const int y = u % N, k1 = u / N;
        ip_stage2<S::P2, -1>(buf + y * ZS + S::P2 * k1, 1);
    }
    __syncthreads();
    // the real-to-half-complex split, pair (k, M - k) in the two columns it read:
    // X[k] = E - (i/2) w_N^k D, X[M-k] = conj(E) - (i/2) conj(w_N^k D), E = (Z[k] + conj Z[M-k]) / 2,
    // D = Z[k] - conj Z[M-k]; X[0] = Re + Im of Z[0], X[M] = Re - Im of Z[0], X[M/2] = conj Z[M/2]
#pragma unroll 1
    for (int u = t; u < N * (S::M / 2 + 1); u += T) {
        const int y = u % N, k = u / N;
        float2* row = buf + y * ZS;
        if (k == 0) {
            const float2 z0 = row[0];
            row[0] = make_float2(z0.x + z0.y, 0.0f);
            row[S::M] = make_float2(z0.x - z0.y, 0.0f);
        } else if (2 * k == S::M) {
            const int ca = slab_col<N>(k);
            row[ca] = cconj(row[ca]);
        } else {
            const int ca = slab_col<N>(k), cb = slab_col<N>(S::M - k);
            const float2 zk = row[ca], zm = cconj(row[cb]);
            const float2 e = cscale(cadd(zk, zm), 0.5f);
            const float2 d = cmul(csub(zk, zm), tw_get<N, -1>(tw, k));
            row[ca] = make_float2(e.x + 0.5f * d.y, e.y - 0.5f * d.x);
            row[cb] = make_float2(e.x - 0.5f * d.y, -e.y - 0.5f * d.x);
        }
    }
    __syncthreads();
    // along y for each column (lanes walk the columns); column M (kz = M) only when binned
    const bool col_m = a.planes > S::M;
#pragma unroll 1
    for (int u = t; u < S::M * S::R2; u += T) {
        const int c = u % S::M, i = u / S::M;
        ip_stage1<N, S::R1, -1>(buf + i * ZS + c, ZS, S::R2, tw, i, 1);
    }
    if (col_m)
        for (int i = t; i < S::R2; i += T) ip_stage1<N, S::R1, -1>(buf + i * ZS + S::M, ZS, S::R2, tw, i, 1);
    __syncthreads();
#pragma unroll 1
    for (int u = t; u < S::M * S::R1; u += T) {
        const int c = u % S::M, k1 = u / S::M;
        ip_stage2<S::R2, -1>(buf + (S::R2 * k1) * ZS + c, ZS);
    }
    if (col_m)
        for (int k1 = t; k1 < S::R1; k1 += T) ip_stage2<S::R2, -1>(buf + (S::R2 * k1) * ZS + S::M, ZS);
    __syncthreads();
    // planes kz < planes: row x of plane kz, y slots in order (lanes walk the slots: the
    // column reads of stride ZS are conflict-free, the row stores coalesced)
    float2* out = a.dst + (size_t)slot * NH * N * N;
    for (int u = t; u < a.planes * N; u += T) {
        const int kz = u / N, r = u % N;
        out[((size_t)kz * N + x) * N + r] = buf[r * ZS + slab_col<N>(kz)];
    }
}

template <int N>
struct XLine {
    static constexpr int TG = N < 32 ? N : 32;                    // y slots per CTA
    static constexpr int GS = TG + 1;                             // row stride (float2)
    static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
    static constexpr int THREADS = TG * R2;
    static constexpr size_t SMEM =
        (size_t)N * GS * sizeof(float2) + N * sizeof(float2) + (size_t)kPrivBins * THREADS * sizeof(float);
};

// The x-line pass: plane kz = blockIdx.x / (N / TG), y slots g0 .. g0 + TG - 1, of the slab
// pass's output; the transform along x (first step straight from global memory), then the
// shell sums S_b += weight * k^3 |X|^2 (weight 2 for 0 < kz < n/2) in per-thread FP32 slots
// (at most R1 modes each), added by bin_sums in a fixed order.
template <int N>
__global__ void __launch_bounds__(XLine<N>::THREADS) k_xline_ps(PSArgs a) {
    using L = XLine<N>;
    constexpr int T = L::THREADS, TG = L::TG, GS = L::GS, NH = N / 2 + 1, NT = N / TG;
    extern __shared__ __align__(16) float2 smem[];
    float2* buf = smem;                                  // [N][GS]
    float2* tw = smem + N * GS;                          // [N]
    float* priv = reinterpret_cast<float*>(tw + N);      // [kPrivBins][T]
    __shared__ double s_bins[EOR21_MAX_BINS];
    const int kz = blockIdx.x / NT, g0 = (blockIdx.x % NT) * TG, slot = blockIdx.y;
    const int pair = a.pair0 + slot;
    if (pair >= a.n_pairs) return;
    const int t = threadIdx.x;
    const bool priv_ok = a.n_bins <= kPrivBins;
    // first step along x, loads first: task (column cc, i), rows x = i + R2 j
    const int cc = t % TG, i = t / TG;
    const float2* src = a.ps_inter + ((size_t)slot * NH + kz) * N * N + g0 + cc;
    float2 v[L::R1];
#pragma unroll
    for (int j = 0; j < L::R1; j++) v[j] = __ldg(src + (size_t)(i + L::R2 * j) * N);
    fill_twiddles<N>(tw);
    for (int e = t; e < kPrivBins * T; e += T) priv[e] = 0.0f;
    for (int e = t; e < EOR21_MAX_BINS; e += T) s_bins[e] = 0.0;
    __syncthreads();
    dft_reg<L::R1, -1>(v);
#pragma unroll
    for (int k1 = 1; k1 < L::R1; k1++) v[k1] = cmul(v[k1], tw_get<N, -1>(tw, i * k1));
#pragma unroll
    for (int k1 = 0; k1 < L::R1; k1++) buf[(i + L::R2 * k1) * GS + cc] = v[k1];
    __syncthreads();
    const float weight = (kz == 0 || 2 * kz == N) ? 1.0f : 2.0f;
    const int mz2 = kz * kz;
#pragma unroll
    for (int u = t; u < TG * L::R1; u += T) {
        const int c = u % TG, k1 = u / TG;
        float2 w[L::R2];
#pragma unroll
        for (int i2 = 0; i2 < L::R2; i2++) w[i2] = buf[(L::R2 * k1 + i2) * GS + c];
        dft_reg<L::R2, -1>(w);
        const int my = signed_index(slot_k<N>(g0 + c), N);
#pragma unroll
        for (int k2 = 0; k2 < L::R2; k2++) {   // mode (kx = k1 + R1 k2, ky, kz)
            const int mx = signed_index(k1 + L::R1 * k2, N);
            const int m2 = mx * mx + my * my + mz2;
            const int b = a.bin_of_m2[m2];
            if (b >= 0) {
                const float fm2 = (float)m2;
                const float val = weight * a.kf3 * k3_of(fm2) * (w[k2].x * w[k2].x + w[k2].y * w[k2].y);
                if (priv_ok) priv[b * T + t] += val;
                else atomicAdd(&s_bins[b], (double)val);
            }
        }
    }
    __syncthreads();
    if (priv_ok) {
        bin_sums<T>(priv, a.n_bins, s_bins);
        __syncthreads();
    }
    for (int b = t; b < a.n_bins; b += T)
        if (s_bins[b] != 0.0) atomicAdd(&a.ps_sum[(size_t)pair * a.n_bins + b], s_bins[b]);
}

// ------------------------------------------------------------------ spectra and chi^2

// Delta^2 = S_b dx^6 / (2 pi^2 V) / n_b and mean |k| per (pair, bin).
__global__ void k_finish_spectra(const double* ps_sum, const long long* nmodes, const double* ksum, int n_pairs,
                                 int n_bins, double scale, double* d2, double* kmean, long long* nmodes_pair) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_pairs * n_bins) return;
    int b = e % n_bins;
    long long n = nmodes[b];
    d2[e] = n > 0 ? ps_sum[e] * scale / (double)n : nan("");
    kmean[e] = n > 0 ? ksum[b] / (double)n : nan("");
    nmodes_pair[e] = n;
}

// Volume-weighted neutral fraction per (walker, redshift).
__global__ void k_xhi_mean(const double* xhi_sum, int n_pairs, double inv_n3, double* out) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n_pairs) out[e] = xhi_sum[e] * inv_n3;
}

struct Chi2Args {
    const double* d2;          // [walker][n_z][n_bins]
    const signed char* use;    // [n_bins] 1 where the bin enters chi^2
    const long long* nmodes;   // [n_bins]
    const double* mock;        // [n_z][n_bins]
    const double* sigma;       // [n_z][n_bins]
    double* chi2;              // [walker]
    int n_walkers, n_z, n_bins;
};

// chi^2 per walker, summed linearly over redshifts (Sec. 3.4) over the bins the table
// marks (geometric centre in [chi2_k_lo, chi2_k_hi], Sec. 2.5). FP64; one warp per walker,
// its lanes over the (redshift, bin) terms, then a shuffle tree (one thread per walker spent
// its time in a chain of dependent FP64 divisions).
__global__ void k_chi2(Chi2Args a) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= a.n_walkers) return;   // uniform over the warp
    double acc = 0.0;
    for (int e = lane; e < a.n_z * a.n_bins; e += 32) {
        const int zi = e / a.n_bins, b = e % a.n_bins;
        if (!a.use[b] || a.nmodes[b] == 0) continue;
        const double r = (a.d2[((size_t)w * a.n_z + zi) * a.n_bins + b] - a.mock[e]) / a.sigma[e];
        acc += r * r;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) a.chi2[w] = acc;
}

// ------------------------------------------------------------------ launch helpers

template <class K>
cudaError_t set_smem(K kernel, size_t bytes) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Plane passes of every grid size: at n <= 128 one shared-memory-resident plane per CTA; at
// n = 256 a row pass and a column pass (each its own traced launch).

// Forward 2D transform of the NH planes of src ([kz][x][y]) into dst ([kz][kx][ky]).
template <int N, int T>
cudaError_t plane_forward(eor_ctx* c, const float2* src, float2* dst) {
    constexpr int NH = N / 2 + 1;
    if constexpr (N == kL) {
        LineArgs la{};
        la.src = src; la.dst = dst; la.G = 1;
        trace_begin(c, kKForward);
        k_lines_rows<-1><<<dim3(NH * 16, 1, 1), kLThreads, kLSmemRows, c->stream>>>(la);
        trace_end(c);
        la.src = dst;
        trace_begin(c, kKForward);
        k_lines_cols<-1, kLineStore><<<dim3(NH * 16, 1, 1), kLThreads, kLSmem, c->stream>>>(la);
        trace_end(c);
    } else {
        trace_begin(c, kKForward);
        k_plane_forward<N, T><<<NH, Plane<N, T>::THREADS, Plane<N, T>::SMEM, c->stream>>>(src, dst);
        trace_end(c);
    }
    return cudaGetLastError();
}

// Pass 1 (filter + inverse 2D transform) of G radii x P slots, as k_plane_filter_inverse.
template <int N, int T>
cudaError_t plane_filter_inverse(eor_ctx* c, const Pass1Args& a1, int P, int cls) {
    constexpr int NH = N / 2 + 1;
    if constexpr (N == kL) {
        LineArgs la{};
        la.src = a1.spec; la.dst = a1.inter; la.G = a1.G;
        la.pairs = a1.pairs; la.wtab = a1.wtab; la.max_radii = a1.max_radii; la.n_m2 = a1.n_m2;
        la.pair0 = a1.pair0; la.n_pairs = a1.n_pairs; la.j0 = a1.j0;
        trace_begin(c, cls);
        k_lines_cols<+1, kLineFilter><<<dim3(NH * 16, a1.G, P), kLThreads, kLSmem, c->stream>>>(la);
        trace_end(c);
        la.src = a1.inter;
        trace_begin(c, cls);
        k_lines_rows<+1><<<dim3(NH * 16, a1.G, P), kLThreads, kLSmemRows, c->stream>>>(la);
        trace_end(c);
    } else {
        trace_begin(c, cls);
        k_plane_filter_inverse<N, T><<<dim3(NH, a1.G, P), Plane<N, T>::THREADS, Plane<N, T>::SMEM, c->stream>>>(a1);
        trace_end(c);
    }
    return cudaGetLastError();
}

// Shell sums of `planes` kz planes of P slots of z-transformed boxes, as k_plane_ps, on stream s.
template <int N, int T>
cudaError_t plane_ps(eor_ctx* c, const PSArgs& ap, int planes, int P, cudaStream_t s) {
    if constexpr (N == kL) {
        LineArgs la{};
        la.src = ap.ps_inter; la.dst = const_cast<float2*>(ap.ps_inter); la.G = 1;
        la.pairs = ap.pairs; la.pair0 = ap.pair0; la.n_pairs = ap.n_pairs;
        la.bin_of_m2 = ap.bin_of_m2; la.ps_sum = ap.ps_sum; la.n_bins = ap.n_bins; la.kf3 = ap.kf3;
        trace_begin_on(c, kKPsPlane, s);
        k_lines_rows<-1><<<dim3(planes * 16, 1, P), kLThreads, kLSmemRows, s>>>(la);
        trace_end_on(c, s);
        trace_begin_on(c, kKPsPlane, s);
        k_lines_cols<-1, kLinePs><<<dim3(planes * 16, 1, P), kLThreads, kLSmem, s>>>(la);
        trace_end_on(c, s);
    } else if (N == 128 && c->tune.ps_split == 2) {
        trace_begin_on(c, kKPsPlane, s);
        k_plane_ps2<<<dim3(2 * planes, P), kPs2Threads, kPs2Smem, s>>>(ap);
        trace_end_on(c, s);
    } else {
        trace_begin_on(c, kKPsPlane, s);
        k_plane_ps<N, T><<<dim3(planes, P), Plane<N, T>::THREADS, Plane<N, T>::SMEM_PS, s>>>(ap);
        trace_end_on(c, s);
    }
    return cudaGetLastError();
}

template <int N, int T>
cudaError_t prepare_n() {
    cudaError_t e;
    if ((e = set_smem(k_pencil_forward<N>, Pencil<N>::SMEM)) != cudaSuccess) return e;
    if constexpr (N == kL) {
        if ((e = set_smem(k_lines_rows<-1>, kLSmemRows)) != cudaSuccess) return e;
        if ((e = set_smem(k_lines_rows<+1>, kLSmemRows)) != cudaSuccess) return e;
        if ((e = set_smem(k_lines_cols<-1, kLineStore>, kLSmem)) != cudaSuccess) return e;
        if ((e = set_smem(k_lines_cols<+1, kLineFilter>, kLSmem)) != cudaSuccess) return e;
        if ((e = set_smem(k_lines_cols<-1, kLinePs>, kLSmem)) != cudaSuccess) return e;
    } else {
        if ((e = set_smem(k_plane_forward<N, T>, Plane<N, T>::SMEM)) != cudaSuccess) return e;
        if ((e = set_smem(k_plane_filter_inverse<N, T>, Plane<N, T>::SMEM)) != cudaSuccess) return e;
        if ((e = set_smem(k_plane_ps<N, T>, Plane<N, T>::SMEM_PS)) != cudaSuccess) return e;
        if constexpr (N == 128)
            if ((e = set_smem(k_plane_ps2, kPs2Smem)) != cudaSuccess) return e;
        if ((e = set_smem(k_slab_ps<N, true>, Slab<N>::SMEM + kFTab * sizeof(float))) != cudaSuccess) return e;
        if ((e = set_smem(k_slab_ps<N, false>, Slab<N>::SMEM)) != cudaSuccess) return e;
        if ((e = set_smem(k_xline_ps<N>, XLine<N>::SMEM)) != cudaSuccess) return e;
    }
    if ((e = set_smem(k_pencil_ionize<N>, Pencil<N>::SMEM)) != cudaSuccess) return e;
    if ((e = set_smem(k_pencil_density<N>, Pencil<N>::SMEM)) != cudaSuccess) return e;
    if ((e = set_smem(k_pencil_forward_batch<N>, Pencil<N>::SMEM)) != cudaSuccess) return e;
    if ((e = set_smem(k_pencil_brightness<N>, Pencil<N>::SMEM + kFTab * sizeof(float))) != cudaSuccess) return e;
    return cudaSuccess;
}

// Power spectra of the delta T_b boxes of every (walker, redshift) written by the basis
// contraction: batched R2C along z, then the plane pass with the shell sums.
template <int N, int T>
cudaError_t ps_from_boxes_n(eor_ctx* c, float* xhi_out) {
    const int n_pairs = c->n_walkers * c->cfg.n_z, P = c->tune.pairs;
    cudaMemsetAsync(c->d_ps_sum, 0, sizeof(double) * n_pairs * c->cfg.n_bins, c->stream);
    const bool flags = c->f16 && c->tune.method == kMethodBasis;   // the flag contraction's pencil pass
    if (flags) cudaMemsetAsync(c->d_xq, 0, sizeof(unsigned long long) * n_pairs, c->stream);
    const float kf = (float)(2.0 * kPi / c->cfg.box_mpc);
    // batches of P pairs: the pencil pass of batch b (c->stream) fills half b % 2 of the
    // intermediate buffer; with two streams the plane pass of batch b (stream2) reads it while
    // the pencil pass of batch b + 1 fills the other half, and batch b + 2 waits for the plane
    // pass of batch b; with one stream the passes run in turn
    const bool two = c->tune.ps_streams == 2;
    const bool slab = N != kL && c->tune.ps_split == 0;   // slab and x-line passes
    cudaStream_t ps = two ? c->stream2 : c->stream;   // the plane passes' stream
    cudaError_t e = cudaSuccess;
    if (two && ((e = cudaEventRecord(c->ev_fork, c->stream)) != cudaSuccess ||
                (e = cudaStreamWaitEvent(c->stream2, c->ev_fork, 0)) != cudaSuccess))
        return e;
    int b = 0;
    for (int pair0 = 0; pair0 < n_pairs; pair0 += P, b++) {
        const int h = b & 1;
        float2* half = c->d_psinter + (size_t)h * P * c->nspec;
        if (two && b >= 2 && (e = cudaStreamWaitEvent(c->stream, c->ev_plane[h], 0)) != cudaSuccess) return e;
        trace_begin(c, kKForward);
        if (slab) {
            if constexpr (N != kL) {
                SlabArgs sa{c->d_fwords, c->d_pairs, brightness_base(c), c->d_dcell, xhi_out, c->d_xq, pop_tables(c),
                            c->d_dtb, half, pair0, n_pairs, c->ps_planes, (float)c->cfg.delta_c};
                if (flags)
                    k_slab_ps<N, true><<<dim3(N, P), Slab<N>::THREADS,
                                         Slab<N>::SMEM + (sa.ftab ? kFTab * sizeof(float) : 0), c->stream>>>(sa);
                else
                    k_slab_ps<N, false><<<dim3(N, P), Slab<N>::THREADS, Slab<N>::SMEM, c->stream>>>(sa);
            }
        } else if (flags) {
            BrightArgs ba{c->d_fwords, c->d_pairs, brightness_base(c), c->d_dcell, xhi_out, c->d_xq, half,
                          pop_tables(c), pair0, n_pairs, (float)c->cfg.delta_c};
            k_pencil_brightness<N><<<dim3(Pencil<N>::TILES, P), Pencil<N>::THREADS,
                                     Pencil<N>::SMEM + (ba.ftab ? kFTab * sizeof(float) : 0), c->stream>>>(ba);
        } else {
            k_pencil_forward_batch<N><<<dim3(Pencil<N>::TILES, P), Pencil<N>::THREADS, Pencil<N>::SMEM, c->stream>>>(
                c->d_dtb, half, pair0, n_pairs);
        }
        trace_end(c);
        if (two && ((e = cudaEventRecord(c->ev_pencil[h], c->stream)) != cudaSuccess ||
                    (e = cudaStreamWaitEvent(c->stream2, c->ev_pencil[h], 0)) != cudaSuccess))
            return e;
        PSArgs ap{half, c->d_pairs, c->d_bin_of_m2, c->d_ps_sum, pair0, n_pairs, c->cfg.n_bins, kf * kf * kf};
        if (slab) {
            if constexpr (N != kL) {
                trace_begin_on(c, kKPsPlane, ps);
                k_xline_ps<N><<<dim3(c->ps_planes * (N / XLine<N>::TG), P), XLine<N>::THREADS, XLine<N>::SMEM, ps>>>(ap);
                trace_end_on(c, ps);
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        } else if ((e = plane_ps<N, T>(c, ap, c->ps_planes, P, ps)) != cudaSuccess) {
            return e;
        }
        if (two && (e = cudaEventRecord(c->ev_plane[h], c->stream2)) != cudaSuccess) return e;
    }
    // join: the last plane pass of each half
    for (int h = 0; two && h < 2 && h < b; h++)
        if ((e = cudaStreamWaitEvent(c->stream, c->ev_plane[(b - 1 - h) & 1], 0)) != cudaSuccess) return e;
    if (flags) {
        trace_begin(c, kKFinish);
        launch_xq_finish(c->d_xq, n_pairs, c->d_xhi_sum, c->stream);
        trace_end(c);
    }
    return cudaGetLastError();
}

template <int N, int T>
cudaError_t forward_spectrum_n(eor_ctx* c, int zi) {
    float2* tmp = c->d_psinter;   // slot 0 of the PS scratch
    trace_begin(c, kKForward);
    k_pencil_forward<N><<<Pencil<N>::TILES, Pencil<N>::THREADS, Pencil<N>::SMEM, c->stream>>>(
        c->d_delta + (size_t)zi * c->n3, tmp);
    trace_end(c);
    return plane_forward<N, T>(c, tmp, c->d_spec + (size_t)zi * c->nspec);
}

template <int N, int T>
cudaError_t ionization_n(eor_ctx* c, float* xhi_out) {
    const int n_pairs = c->n_walkers * c->cfg.n_z;
    const int G = c->tune.group, P = c->tune.pairs;
    const int groups = (c->max_radii + G - 1) / G;
    cudaMemsetAsync(c->d_ps_sum, 0, sizeof(double) * n_pairs * c->cfg.n_bins, c->stream);
    const float kf = (float)(2.0 * kPi / c->cfg.box_mpc);
    for (int pair0 = 0; pair0 < n_pairs; pair0 += P) {
        for (int g = 0; g < groups; g++) {
            Pass1Args a1{c->d_spec, c->d_inter, c->d_pairs, c->d_wtab, c->max_radii, c->n_m2,
                         pair0, n_pairs, g * G, G};
            cudaError_t e = plane_filter_inverse<N, T>(c, a1, P, kKFilterPlane);
            if (e != cudaSuccess) return e;
            Pass2Args a2{c->d_inter, c->d_pairs, c->d_flags, brightness_base(c), xhi_out,
                         c->d_xhi_sum, c->d_psinter, pop_tables(c), pair0, n_pairs, g * G, G,
                         (float)c->cfg.delta_c};
            trace_begin(c, kKPencil);
            k_pencil_ionize<N><<<dim3(Pencil<N>::TILES, P), Pencil<N>::THREADS, Pencil<N>::SMEM, c->stream>>>(a2);
            trace_end(c);
        }
        PSArgs ap{c->d_psinter, c->d_pairs, c->d_bin_of_m2, c->d_ps_sum, pair0, n_pairs, c->cfg.n_bins,
                  kf * kf * kf};
        cudaError_t e = plane_ps<N, T>(c, ap, c->ps_planes, P, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

template <int N, int T>
cudaError_t filtered_density_n(eor_ctx* c, int zi, float* out, const float* wtab) {
    cudaError_t e;
    // one task: walker 0 of a one-radius table at wtab, box zi
    PairInfo pi{};
    pi.w = 0; pi.zi = zi; pi.n_r = 1;
    if ((e = cudaMemcpyAsync(c->d_diag_pair, &pi, sizeof(PairInfo), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
        return e;
    Pass1Args a1{c->d_spec, c->d_inter, c->d_diag_pair, wtab, 1, c->n_m2, 0, 1, 0, 1};
    if ((e = plane_filter_inverse<N, T>(c, a1, 1, kKFilterPlane)) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_pencil_density<N><<<Pencil<N>::TILES, Pencil<N>::THREADS, Pencil<N>::SMEM, c->stream>>>(c->d_inter, out);
    trace_end(c);
    return cudaGetLastError();
}

// delta_hat k_z^2 / k^2 (0 at k = 0) of a half spectrum [kz][kx][ky]: the Fourier transform of
// the line-of-sight second derivative field that gives linear dv_r/dr (last box axis).
__global__ void k_los_weight(const float2* spec, int n, float2* out) {
    const long long total = (long long)(n / 2 + 1) * n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(e / ((long long)n * n)), kx = (int)((e / n) % n), ky = (int)(e % n);
        const int mx = signed_index(kx, n), my = signed_index(ky, n);
        const int m2 = mx * mx + my * my + kz * kz;
        const float w = m2 > 0 ? (float)(kz * kz) / (float)m2 : 0.0f;
        const float2 v = spec[e];
        out[e] = make_float2(v.x * w, v.y * w);
    }
}

// (1 + delta) H / (dv_r/dr + H) - 1 with dv_r/dr / H = -f g clipped to [-max_dvdr, max_dvdr].
__global__ void k_rsd_weight(const float* delta, const float* g, const double* f, float max_dvdr, long long n3,
                             float* out) {
    const float fz = (float)*f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        const float dvdr = fminf(fmaxf(-fz * g[i], -max_dvdr), max_dvdr);
        out[i] = (1.0f + delta[i]) / (1.0f + dvdr) - 1.0f;
    }
}

// Real box of a half spectrum held at spec ([kz][kx][ky], one box) through the plane and
// pencil inverse passes with the unit window at wtab; normalised by 1/n^3.
template <int N, int T>
cudaError_t spectrum_to_box_n(eor_ctx* c, const float2* spec, float* out, const float* wtab) {
    cudaError_t e;
    PairInfo pi{};
    pi.w = 0; pi.zi = 0; pi.n_r = 1;
    if ((e = cudaMemcpyAsync(c->d_diag_pair, &pi, sizeof(PairInfo), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
        return e;
    Pass1Args a1{spec, c->d_inter, c->d_diag_pair, wtab, 1, c->n_m2, 0, 1, 0, 1};
    if ((e = plane_filter_inverse<N, T>(c, a1, 1, kKOther)) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_pencil_density<N><<<Pencil<N>::TILES, Pencil<N>::THREADS, Pencil<N>::SMEM, c->stream>>>(c->d_inter, out);
    trace_end(c);
    return cudaGetLastError();
}

template <int N, int T>
cudaError_t box_power_spectrum_n(eor_ctx* c, const float* box) {
    constexpr int NH = N / 2 + 1;
    const int nb = c->cfg.n_bins;
    const float kf = (float)(2.0 * kPi / c->cfg.box_mpc);
    cudaError_t e;
    PairInfo pi{};
    if ((e = cudaMemcpyAsync(c->d_diag_pair, &pi, sizeof(PairInfo), cudaMemcpyHostToDevice, c->stream)) !=
        cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(c->d_diag_ps, 0, sizeof(double) * nb, c->stream)) != cudaSuccess) return e;
    trace_begin(c, kKForward);
    k_pencil_forward<N><<<Pencil<N>::TILES, Pencil<N>::THREADS, Pencil<N>::SMEM, c->stream>>>(box, c->d_psinter);
    trace_end(c);
    PSArgs ap{c->d_psinter, c->d_diag_pair, c->d_bin_of_m2, c->d_diag_ps, 0, 1, nb, kf * kf * kf};
    if ((e = plane_ps<N, T>(c, ap, NH, 1, c->stream)) != cudaSuccess) return e;
    const double dx = c->cfg.box_mpc / c->n;
    const double vol = c->cfg.box_mpc * c->cfg.box_mpc * c->cfg.box_mpc;
    const double scale = dx * dx * dx * dx * dx * dx / (2.0 * kPi * kPi * vol);
    trace_begin(c, kKFinish);
    k_finish_spectra<<<(nb + 255) / 256, 256, 0, c->stream>>>(c->d_diag_ps, c->d_nmodes, c->d_ksum, 1, nb, scale,
                                                              c->d_diag_ps + nb, c->d_diag_ps + 2 * nb,
                                                              c->d_diag_cnt);
    trace_end(c);
    return cudaGetLastError();
}

// Inverse-weighted mode sums of the T+S equation: sums[z][b] += w / (N_i + mock[z][b])^2 over
// the half-spectrum modes of bin b (w = 2 for 0 < kz < n/2: the conjugate mode, else 1).
// Block-private FP64 bins in shared memory, then one global add per bin and block.
__global__ void __launch_bounds__(256) k_noise_sums(int n, const signed char* bin, int n_bins, const double* mock,
                                                    const float* thermal, double* sums) {
    __shared__ double s[EOR21_MAX_BINS];
    const int zi = blockIdx.y;
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) s[b] = 0.0;
    __syncthreads();
    const int nh = n / 2 + 1;
    const long long total = (long long)nh * n * n;
    const float* th = thermal ? thermal + (size_t)zi * total : nullptr;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(e / ((long long)n * n)), kx = (int)((e / n) % n), ky = (int)(e % n);
        const int mx = signed_index(kx, n), my = signed_index(ky, n);
        const int b = bin[mx * mx + my * my + kz * kz];
        if (b < 0) continue;
        const double w = (kz == 0 || kz == n / 2) ? 1.0 : 2.0;
        const double d = (th ? (double)th[e] : 0.0) + mock[(size_t)zi * n_bins + b];
        atomicAdd(&s[b], w / (d * d));
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x)
        if (s[b] != 0.0) atomicAdd(&sums[(size_t)zi * n_bins + b], s[b]);
}

__global__ void k_noise_finish(const double* sums, const double* mock, const long long* nmodes, int n_bins, int count,
                               double model_frac, double* sigma) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int b = i % n_bins;
    const double m = model_frac * mock[i];
    sigma[i] = nmodes[b] > 0 ? sqrt(1.0 / sums[i] + m * m) : (double)NAN;
}

// Grid-size dispatch; the 128^3 plane kernels come in 512- and 1024-thread CTAs.
#define EOR_DISPATCH(c, FN, ...)                                                            \
    switch ((c)->n) {                                                                       \
        case 16: return FN<16, 512>(__VA_ARGS__);                                           \
        case 32: return FN<32, 512>(__VA_ARGS__);                                           \
        case 64: return FN<64, 512>(__VA_ARGS__);                                           \
        case 128:                                                                           \
            return (c)->tune.plane_threads >= 1024 ? FN<128, 1024>(__VA_ARGS__) : FN<128, 512>(__VA_ARGS__); \
        case 256: return FN<256, 512>(__VA_ARGS__);                                         \
        default: return cudaErrorInvalidValue;                                              \
    }

// Box power spectrum on caller-provided buffers (no context): R2C along z into spec, then
// the plane pass adding the shell sums into sums. pair_info points at one zeroed PairInfo.
template <int N, int T>
cudaError_t box_ps_raw_n(const float* box, float2* spec, const signed char* bins, double* sums, int n_bins,
                         float kf3, const PairInfo* pair_info, cudaStream_t stream) {
    constexpr int NH = N / 2 + 1;
    k_pencil_forward<N><<<Pencil<N>::TILES, Pencil<N>::THREADS, Pencil<N>::SMEM, stream>>>(box, spec);
    PSArgs ap{spec, pair_info, bins, sums, 0, 1, n_bins, kf3};
    k_plane_ps<N, T><<<dim3(NH, 1), Plane<N, T>::THREADS, Plane<N, T>::SMEM_PS, stream>>>(ap);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_box_ps_raw(int n, const float* box, float2* spec, const signed char* bins, double* sums, int n_bins,
                              float kf3, const PairInfo* pair_info, cudaStream_t stream) {
    switch (n) {
        case 16: return box_ps_raw_n<16, 512>(box, spec, bins, sums, n_bins, kf3, pair_info, stream);
        case 32: return box_ps_raw_n<32, 512>(box, spec, bins, sums, n_bins, kf3, pair_info, stream);
        case 64: return box_ps_raw_n<64, 512>(box, spec, bins, sums, n_bins, kf3, pair_info, stream);
        case 128: return box_ps_raw_n<128, 512>(box, spec, bins, sums, n_bins, kf3, pair_info, stream);
        default: return cudaErrorInvalidValue;
    }
}

// Shared-memory limits of the two kernels launch_box_ps_raw runs at grid size n (current device).
cudaError_t prepare_box_ps_raw(int n) {
    auto both = [](auto pencil, size_t ps, auto plane, size_t pls) {
        cudaError_t e = set_smem(pencil, ps);
        return e != cudaSuccess ? e : set_smem(plane, pls);
    };
    switch (n) {
        case 16: return both(k_pencil_forward<16>, Pencil<16>::SMEM, k_plane_ps<16, 512>, Plane<16, 512>::SMEM_PS);
        case 32: return both(k_pencil_forward<32>, Pencil<32>::SMEM, k_plane_ps<32, 512>, Plane<32, 512>::SMEM_PS);
        case 64: return both(k_pencil_forward<64>, Pencil<64>::SMEM, k_plane_ps<64, 512>, Plane<64, 512>::SMEM_PS);
        case 128:
            return both(k_pencil_forward<128>, Pencil<128>::SMEM, k_plane_ps<128, 512>, Plane<128, 512>::SMEM_PS);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_noise_sigma(eor_ctx* c, const double* mock, const float* thermal, double model_frac, double* sums,
                               double* sigma) {
    const int nb = c->cfg.n_bins, nz = c->cfg.n_z;
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(double) * nz * nb, c->stream);
    if (e != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_noise_sums<<<dim3(256, nz), 256, 0, c->stream>>>(c->n, c->d_bin_of_m2, nb, mock, thermal, sums);
    trace_end(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_noise_finish<<<(nz * nb + 127) / 128, 128, 0, c->stream>>>(sums, mock, c->d_nmodes, nb, nz * nb, model_frac,
                                                                 sigma);
    trace_end(c);
    return cudaGetLastError();
}

// Zel'dovich displacement along axis j of box zi in cells: i m_j / (kf |m|^2) delta_hat / dx, the
// Nyquist index of axis j set to zero (an odd derivative has no Nyquist value).
__global__ void k_za_weight(const float2* spec, int n, int axis, float inv_kf_dx, float2* out) {
    const long long total = (long long)(n / 2 + 1) * n * n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int kz = (int)(e / ((long long)n * n)), kx = (int)((e / n) % n), ky = (int)(e % n);
        const int mx = signed_index(kx, n), my = signed_index(ky, n);
        const int m2 = mx * mx + my * my + kz * kz;
        const int mj = axis == 0 ? mx : (axis == 1 ? my : kz);
        const bool nyq = axis == 2 ? kz == n / 2 : mj == -n / 2;
        const float w = (m2 > 0 && !nyq) ? (float)mj * inv_kf_dx / (float)m2 : 0.0f;
        const float2 v = spec[e];
        out[e] = make_float2(-v.y * w, v.x * w);   // i w delta_hat
    }
}

// Cloud-in-cell deposit of the unit-mass particle of every cell, displaced by psi [3][n^3]
// (cells), periodic; rho must start at zero.
__global__ void k_za_deposit(const float* psi, int n, float* rho) {
    const long long n3 = (long long)n * n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        const int qx = (int)(i / ((long long)n * n)), qy = (int)((i / n) % n), qz = (int)(i % n);
        const float px = qx + psi[i], py = qy + psi[n3 + i], pz = qz + psi[2 * n3 + i];
        const float fx = floorf(px), fy = floorf(py), fz = floorf(pz);
        const float tx = px - fx, ty = py - fy, tz = pz - fz;
        const int ix = (((int)fx % n) + n) % n, iy = (((int)fy % n) + n) % n, iz = (((int)fz % n) + n) % n;
#pragma unroll
        for (int cx = 0; cx < 2; cx++)
#pragma unroll
            for (int cy = 0; cy < 2; cy++)
#pragma unroll
                for (int cz = 0; cz < 2; cz++) {
                    const float w = (cx ? tx : 1.0f - tx) * (cy ? ty : 1.0f - ty) * (cz ? tz : 1.0f - tz);
                    const long long j = ((long long)((ix + cx) % n) * n + (iy + cy) % n) * n + (iz + cz) % n;
                    atomicAdd(rho + j, w);
                }
    }
}

__global__ void k_za_finish(const float* rho, long long n3, float* delta) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
        delta[i] = rho[i] - 1.0f;
}

// Zel'dovich evolution of box zi in place (its linear spectrum must be in d_spec): the three
// displacement fields, the deposit, delta = rho - 1. work: 4 n^3 floats.
cudaError_t launch_zeldovich(eor_ctx* c, int zi, float* work) {
    cudaError_t e;
    const size_t n3 = c->n3;
    const double dx = c->cfg.box_mpc / c->n, kf = 2.0 * kPi / c->cfg.box_mpc;
    if ((e = launch_window_table(c, 0.0, c->d_diag_wtab)) != cudaSuccess) return e;   // unit window
    for (int axis = 0; axis < 3; axis++) {
        trace_begin(c, kKOther);
        k_za_weight<<<1024, 256, 0, c->stream>>>(c->d_spec + (size_t)zi * c->nspec, c->n, axis,
                                                 (float)(1.0 / (kf * dx)), c->d_psinter);
        trace_end(c);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        float* out = work + (size_t)axis * n3;
        switch (c->n) {
            case 16: e = spectrum_to_box_n<16, 512>(c, c->d_psinter, out, c->d_diag_wtab); break;
            case 32: e = spectrum_to_box_n<32, 512>(c, c->d_psinter, out, c->d_diag_wtab); break;
            case 64: e = spectrum_to_box_n<64, 512>(c, c->d_psinter, out, c->d_diag_wtab); break;
            case 128:
                e = c->tune.plane_threads >= 1024 ? spectrum_to_box_n<128, 1024>(c, c->d_psinter, out, c->d_diag_wtab)
                                                  : spectrum_to_box_n<128, 512>(c, c->d_psinter, out, c->d_diag_wtab);
                break;
            case 256: e = spectrum_to_box_n<256, 512>(c, c->d_psinter, out, c->d_diag_wtab); break;
            default: return cudaErrorInvalidValue;
        }
        if (e != cudaSuccess) return e;
    }
    float* rho = work + 3 * n3;
    if ((e = cudaMemsetAsync(rho, 0, sizeof(float) * n3, c->stream)) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_za_deposit<<<2048, 256, 0, c->stream>>>(work, c->n, rho);
    trace_end(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_za_finish<<<1024, 256, 0, c->stream>>>(rho, (long long)n3, c->d_delta + (size_t)zi * n3);
    trace_end(c);
    return cudaGetLastError();
}

// The velocity-weighted brightness field of box zi (Sec. 2.2): k_z^2/k^2 delta_hat -> real
// field g (scratch box) -> (1 + delta) / (1 + clip(-f g)) - 1 into d_bright.
cudaError_t launch_brightness_weight(eor_ctx* c, int zi) {
    cudaError_t e;
    trace_begin(c, kKOther);
    k_los_weight<<<1024, 256, 0, c->stream>>>(c->d_spec + (size_t)zi * c->nspec, c->n, c->d_psinter);
    trace_end(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = launch_window_table(c, 0.0, c->d_diag_wtab)) != cudaSuccess) return e;   // W(0) = 1 everywhere
    switch (c->n) {
        case 16: e = spectrum_to_box_n<16, 512>(c, c->d_psinter, c->d_scratch_box, c->d_diag_wtab); break;
        case 32: e = spectrum_to_box_n<32, 512>(c, c->d_psinter, c->d_scratch_box, c->d_diag_wtab); break;
        case 64: e = spectrum_to_box_n<64, 512>(c, c->d_psinter, c->d_scratch_box, c->d_diag_wtab); break;
        case 128:
            e = c->tune.plane_threads >= 1024
                    ? spectrum_to_box_n<128, 1024>(c, c->d_psinter, c->d_scratch_box, c->d_diag_wtab)
                    : spectrum_to_box_n<128, 512>(c, c->d_psinter, c->d_scratch_box, c->d_diag_wtab);
            break;
        case 256: e = spectrum_to_box_n<256, 512>(c, c->d_psinter, c->d_scratch_box, c->d_diag_wtab); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_rsd_weight<<<1024, 256, 0, c->stream>>>(c->d_delta + (size_t)zi * c->n3, c->d_scratch_box,
                                              c->d_growth + c->cfg.n_z + zi, (float)c->cfg.rsd_max_dvdr,
                                              (long long)c->n3, c->d_bright + (size_t)zi * c->n3);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_box_power_spectrum(eor_ctx* c, const float* box) { EOR_DISPATCH(c, box_power_spectrum_n, c, box) }

size_t estimate_launches(const eor_ctx* c) {
    const int n_pairs = (c->n_walkers > 0 ? c->n_walkers : 1) * c->cfg.n_z;
    const int batches = (n_pairs + c->tune.pairs - 1) / c->tune.pairs;
    const int groups = (c->max_radii + c->tune.group - 1) / c->tune.group;
    return (size_t)batches * (2 * groups + 1) + 2 * (size_t)c->cfg.n_z * (c->kb + 1) + 64;
}

bool grid_supported(int n) { return n == 16 || n == 32 || n == 64 || n == 128 || n == 256; }

cudaError_t launch_forward_spectrum(eor_ctx* c, int zi) { EOR_DISPATCH(c, forward_spectrum_n, c, zi) }

cudaError_t launch_ionization(eor_ctx* c, float* xhi_out) {
    if (c->tune.method != kMethodDirect) {
        cudaError_t e = launch_basis_ionize(c, xhi_out);
        if (e != cudaSuccess) return e;
        return launch_ps_from_boxes(c, xhi_out);
    }
    cudaMemsetAsync(c->d_xhi_sum, 0, sizeof(double) * c->n_walkers * c->cfg.n_z, c->stream);
    EOR_DISPATCH(c, ionization_n, c, xhi_out)
}

cudaError_t launch_ps_from_boxes(eor_ctx* c, float* xhi_out) { EOR_DISPATCH(c, ps_from_boxes_n, c, xhi_out) }

cudaError_t launch_filtered_density(eor_ctx* c, int zi, float* out, const float* wtab) {
    EOR_DISPATCH(c, filtered_density_n, c, zi, out, wtab)
}

cudaError_t prepare_kernels(int n) {
    switch (n) {
        case 16: return prepare_n<16, 512>();
        case 32: return prepare_n<32, 512>();
        case 64: return prepare_n<64, 512>();
        case 128: {
            cudaError_t e = prepare_n<128, 512>();
            return e != cudaSuccess ? e : prepare_n<128, 1024>();
        }
        case 256: return prepare_n<256, 512>();
        default: return cudaErrorInvalidValue;
    }
}

size_t flag_words_per_pair(int n) {
    switch (n) {
        case 16: return (size_t)Pencil<16>::TILES * Pencil<16>::THREADS;
        case 32: return (size_t)Pencil<32>::TILES * Pencil<32>::THREADS;
        case 64: return (size_t)Pencil<64>::TILES * Pencil<64>::THREADS;
        case 128: return (size_t)Pencil<128>::TILES * Pencil<128>::THREADS;
        case 256: return (size_t)Pencil<256>::TILES * Pencil<256>::THREADS;
        default: return 0;
    }
}

cudaError_t launch_xhi_mean(eor_ctx* c) {
    const int n_pairs = c->n_walkers * c->cfg.n_z;
    trace_begin(c, kKFinish);
    k_xhi_mean<<<(n_pairs + 127) / 128, 128, 0, c->stream>>>(c->d_xhi_sum, n_pairs, 1.0 / (double)c->n3,
                                                              c->d_xhi_mean);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_power_spectrum(eor_ctx* c) {
    const int n_pairs = c->n_walkers * c->cfg.n_z, nb = c->cfg.n_bins;
    const double dx = c->cfg.box_mpc / c->n;
    const double vol = c->cfg.box_mpc * c->cfg.box_mpc * c->cfg.box_mpc;
    const double scale = dx * dx * dx * dx * dx * dx / (2.0 * kPi * kPi * vol);
    const int total = n_pairs * nb;
    trace_begin(c, kKFinish);
    k_finish_spectra<<<(total + 255) / 256, 256, 0, c->stream>>>(c->d_ps_sum, c->d_nmodes, c->d_ksum, n_pairs, nb,
                                                                 scale, c->d_d2, c->d_kmean, c->d_nmodes_pair);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_chi2(eor_ctx* c) {
    const eor_config& g = c->cfg;
    Chi2Args a{c->d_d2, c->d_chi2_use, c->d_nmodes, c->d_mock, c->d_mock + g.n_z * g.n_bins, c->d_chi2, c->n_walkers,
               g.n_z, g.n_bins};
    trace_begin(c, kKFinish);
    k_chi2<<<(c->n_walkers + 3) / 4, 128, 0, c->stream>>>(a);   // one warp per walker
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
