// tcgen05.cu — tensor-core (tcgen05, TMEM) kernels of libeor21.
//
// k_tc_check: one CTA computes D = A B^T (A 128 x 32, B n x 32, FP32 in global memory) with
// TF32 tcgen05 MMAs accumulating in tensor memory: the operand layout, descriptors and
// tensor-memory reads of the tensor-core contraction, checked in isolation.
#include "eor_internal.cuh"
#include "tc.cuh"

namespace eor {
namespace {

constexpr uint32_t kWaitTries = 1u << 22;

__global__ void __launch_bounds__(128) k_tc_check(const float* A, const float* B, float* D, int n, uint32_t ncols,
                                                   int* err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                       // 128 rows x 32 K, core-matrix layout (16 KB)
    unsigned char* Bs = sm + 128 * tc::kKMax * 4;  // n rows x 32 K
    uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)n * tc::kKMax * 4);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int e = t; e < 128 * tc::kKMax; e += 128)
        *reinterpret_cast<uint32_t*>(As + tc::core_offset(e / tc::kKMax, e % tc::kKMax)) = tc::to_tf32(A[e]);
    for (int e = t; e < n * tc::kKMax; e += 128)
        *reinterpret_cast<uint32_t*>(Bs + tc::core_offset(e / tc::kKMax, e % tc::kKMax)) = tc::to_tf32(B[e]);
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    if (t == 0) tc::mbar_init(bar, 1);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    if (t == 0) {
        const uint32_t idesc = tc::idesc_tf32(128, n);
        for (int s = 0; s < tc::kKMax / 8; s++) {
            const uint64_t ad = tc::smem_desc(tc::smem_addr(As) + s * 2 * tc::kLBO, tc::kLBO, tc::kSBO);
            const uint64_t bd = tc::smem_desc(tc::smem_addr(Bs) + s * 2 * tc::kLBO, tc::kLBO, tc::kSBO);
            tc::mma_tf32(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        tc::mma_commit(bar);
    }
    bool ok = tc::mbar_wait(bar, 0, kWaitTries);
    if (!ok) ok = tc::mbar_wait(bar, 0, kWaitTries);   // let an MMA in flight finish before freeing its memory
    tc::fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < n; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; i++) D[(size_t)(warp * 32 + lane) * n + c0 + i] = v[i];
        }
    } else if (lane == 0) {
        atomicOr(err, 1);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

}  // namespace
}  // namespace eor

extern "C" int eor_tensor_core_check(const float* a, const float* b, float* d, int n, int* err, void* cuda_stream) {
    using namespace eor;
    if (!a || !b || !d || !err || n < 16 || n > 256 || n % 16 != 0) {
        set_global_error("eor_tensor_core_check: n must be a multiple of 16 in 16..256 and pointers non-NULL");
        return EOR_EINVAL;
    }
    uint32_t ncols = 32;
    while (ncols < (uint32_t)n) ncols <<= 1;
    const size_t smem = (size_t)(128 + n) * tc::kKMax * 4 + 16;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaFuncSetAttribute(k_tc_check, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        k_tc_check<<<1, 128, smem, s>>>(a, b, d, n, ncols, err);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("eor_tensor_core_check: ") + cudaGetErrorString(e));
        return EOR_ECUDA;
    }
    return EOR_OK;
}

// ------------------------------------------------------------------ tensor-core contraction

namespace eor {
namespace {

constexpr int kTcThreads = 128;                    // 4 warps: one tensor-memory lane per thread and tile
constexpr int kTcTiles = 4;                        // M tiles of 128 cells
constexpr int kTcCells = 128 * kTcTiles;           // cells per CTA
constexpr int kTcN = 128;                          // (walker, radius) columns per MMA chunk
constexpr uint32_t kTileBytes = 128 * tc::kKMax * 4;   // one 128 x 32 TF32 operand tile
constexpr uint32_t kTmemCols = kTcTiles * kTcN;    // 512: the whole tensor memory

struct TcArgs {
    const float* F;             // [n_z][kb][n3] basis fields
    const float* coef;          // [walker][max_radii][kb]
    const int* cols;            // [column] walker << 8 | radius, walkers in order
    const int* ncols;           // [1] number of columns
    const PairInfo* pairs;      // [walker * n_z + zi]
    const float* delta;         // [n_z][n3]
    float* dtb;                 // [pair][n3]
    float* xhi_out;             // optional [pair][n3]
    float* xpart;               // [pair][n3 / 128] per-warp neutral-fraction sums
    int* err;
    int n_z, kb, max_radii;
    long long n3;
    float delta_c;
};

// One CTA: kTcCells cells of one redshift against every (walker, radius) column. The basis
// values of the cells (A: 4 tiles of 128 cells x 32 K) and each chunk of 128 columns'
// coefficients (B: 128 x 32 K) sit in shared memory as TF32 hi and lo parts; one thread
// issues, per tile and K step, hi*hi + hi*lo + lo*hi (3xTF32, FP32 accumulation in tensor
// memory), so delta_R(cell, column) = sum_b F_b c_b lands in tensor memory at FP32
// accuracy. Epilogue: thread t owns lane t of every tile (4 cells); per column it tests
// delta_R >= delta_crit and ORs the walker's flag; at the walker's R_cell column it forms
// x_HI and delta T_b (coalesced stores) and a warp sum of x_HI.
__global__ void __launch_bounds__(kTcThreads, 1) k_basis_ionize_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* Ahi = sm;                                   // [4][16 KB]
    unsigned char* Alo = Ahi + kTcTiles * kTileBytes;          // [4][16 KB]
    unsigned char* Bhi = Alo + kTcTiles * kTileBytes;          // [16 KB]
    unsigned char* Blo = Bhi + kTileBytes;                     // [16 KB]
    float* thr = reinterpret_cast<float*>(Blo + kTileBytes);   // [kTcN]
    int* meta = reinterpret_cast<int*>(thr + kTcN);            // [kTcN] walker << 1 | last, or -1
    uint64_t* bar = reinterpret_cast<uint64_t*>(meta + kTcN);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
    int* s_ok = reinterpret_cast<int*>(tslot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int zi = blockIdx.y, kb = a.kb;
    const long long cell0 = (long long)blockIdx.x * kTcCells;

    // basis values of the CTA's cells, split into TF32 hi + lo, K padded with zeros to 32
    for (int e = t; e < tc::kKMax * kTcCells; e += kTcThreads) {
        const int b = e / kTcCells, c = e % kTcCells;
        const float v = b < kb ? __ldg(a.F + ((size_t)zi * kb + b) * a.n3 + cell0 + c) : 0.0f;
        const uint32_t hi = tc::to_tf32(v);
        const uint32_t lo = tc::to_tf32(v - __uint_as_float(hi));
        const uint32_t off = (uint32_t)(c >> 7) * kTileBytes + tc::core_offset(c & 127, b);
        *reinterpret_cast<uint32_t*>(Ahi + off) = hi;
        *reinterpret_cast<uint32_t*>(Alo + off) = lo;
    }
    float dens[kTcTiles];
#pragma unroll
    for (int q = 0; q < kTcTiles; q++) dens[q] = __ldg(a.delta + (size_t)zi * a.n3 + cell0 + q * 128 + t);
    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    if (t == 0) {
        tc::mbar_init(bar, 1);
        *s_ok = 1;
    }
    const int ncols = *a.ncols;
    bool fl[kTcTiles] = {false, false, false, false};
    uint32_t phase = 0;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc::idesc_tf32(128, kTcN);

    for (int cbase = 0; cbase < ncols; cbase += kTcN) {
        // ---- coefficient chunk: thread t builds column cbase + t
        {
            const int c = cbase + t;
            float4 cf[tc::kKMax / 4];
            int m = -1;
            float th = INFINITY;
            if (c < ncols) {
                const int cw = a.cols[c], w = cw >> 8, j = cw & 255;
                const PairInfo& pi = a.pairs[(size_t)w * a.n_z + zi];
                const float* src = a.coef + ((size_t)w * a.max_radii + j) * kb;
#pragma unroll
                for (int q = 0; q < tc::kKMax / 4; q++)
                    cf[q] = 4 * q < kb ? __ldg(reinterpret_cast<const float4*>(src) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
                th = pi.delta_crit[j];
                m = (w << 1) | (j == pi.n_r - 1 ? 1 : 0);
            } else {
#pragma unroll
                for (int q = 0; q < tc::kKMax / 4; q++) cf[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < tc::kKMax / 4; q++) {
                const float x[4] = {cf[q].x, cf[q].y, cf[q].z, cf[q].w};
                uint32_t h[4], l[4];
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    h[i] = tc::to_tf32(x[i]);
                    l[i] = tc::to_tf32(x[i] - __uint_as_float(h[i]));
                }
                const uint32_t off = tc::core_offset(t, 4 * q);
                *reinterpret_cast<uint4*>(Bhi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                *reinterpret_cast<uint4*>(Blo + off) = make_uint4(l[0], l[1], l[2], l[3]);
            }
            thr[t] = th;
            meta[t] = m;
        }
        tc::fence_proxy_async();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // ---- D[tile] = A[tile] B^T, 3xTF32
        if (t == 0) {
            for (int q = 0; q < kTcTiles; q++) {
                const uint32_t d = tmem + (uint32_t)(q * kTcN);
                for (int s = 0; s < tc::kKMax / 8; s++) {
                    const uint32_t ko = (uint32_t)s * 2 * tc::kLBO;
                    const uint64_t ah = tc::smem_desc(tc::smem_addr(Ahi + q * kTileBytes) + ko, tc::kLBO, tc::kSBO);
                    const uint64_t al = tc::smem_desc(tc::smem_addr(Alo + q * kTileBytes) + ko, tc::kLBO, tc::kSBO);
                    const uint64_t bh = tc::smem_desc(tc::smem_addr(Bhi) + ko, tc::kLBO, tc::kSBO);
                    const uint64_t bl = tc::smem_desc(tc::smem_addr(Blo) + ko, tc::kLBO, tc::kSBO);
                    tc::mma_tf32(d, ah, bh, idesc, s > 0 ? 1u : 0u);
                    tc::mma_tf32(d, ah, bl, idesc, 1u);
                    tc::mma_tf32(d, al, bh, idesc, 1u);
                }
            }
            tc::mma_commit(bar);
        }
        bool ok = tc::mbar_wait(bar, phase, kWaitTries);
        if (!ok) ok = tc::mbar_wait(bar, phase, kWaitTries);   // an MMA in flight finishes before memory is reused
        phase ^= 1u;
        if (!ok) *s_ok = 0;
        tc::fence_after_sync();
        __syncthreads();
        if (!*s_ok) break;
        // ---- epilogue over the chunk's columns, 16 at a time
        const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c16 = 0; c16 < kTcN && cbase + c16 < ncols; c16 += 16) {
            float v[kTcTiles][16];
#pragma unroll
            for (int q = 0; q < kTcTiles; q++) tc::tmem_ld16(lane_base + (uint32_t)(q * kTcN + c16), v[q]);
#pragma unroll
            for (int i = 0; i < 16; i++) {
                const int col = c16 + i;
                const float th = thr[col];
#pragma unroll
                for (int q = 0; q < kTcTiles; q++) fl[q] |= v[q][i] >= th;
                const int m = meta[col];
                if (m >= 0 && (m & 1)) {   // R_cell of walker m >> 1: the same column for the whole CTA
                    const int w = m >> 1;
                    const PairInfo& pi = a.pairs[(size_t)w * a.n_z + zi];
                    const float zeta = pi.zeta, t0 = pi.t0, inv = pi.inv_sqrt2s2_cell;
                    const bool cell_ok = pi.cell_ok > 0.5f;
                    const size_t pair = (size_t)w * a.n_z + zi;
                    float xsum = 0.0f;
#pragma unroll
                    for (int q = 0; q < kTcTiles; q++) {
                        const float dr = v[q][i];
                        float f = 0.0f;
                        if (cell_ok) f = dr >= a.delta_c ? 1.0f : erfcf((a.delta_c - dr) * inv);
                        const float xh = fl[q] ? 0.0f : 1.0f - fminf(1.0f, zeta * f);
                        const long long cell = cell0 + q * 128 + t;
                        a.dtb[pair * a.n3 + cell] = t0 * xh * (1.0f + dens[q]);
                        if (a.xhi_out) a.xhi_out[pair * a.n3 + cell] = xh;
                        xsum += xh;
                        fl[q] = false;
                    }
                    for (int off = 16; off > 0; off >>= 1) xsum += __shfl_xor_sync(0xffffffffu, xsum, off);
                    if (lane == 0) a.xpart[pair * (size_t)(a.n3 / 128) + (size_t)blockIdx.x * 4 + warp] = xsum;
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();   // tensor memory and the B tiles are free for the next chunk
        tc::fence_after_sync();
    }
    if (t == 0 && !*s_ok) atomicOr(a.err, kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Flattened (walker, radius) columns of the walkers, in walker order, and their count.
__global__ void k_build_columns(const WalkerInfo* walkers, int n_walkers, int* cols, int* ncols) {
    if (threadIdx.x != 0) return;
    int c = 0;
    for (int w = 0; w < n_walkers; w++)
        for (int j = 0; j < walkers[w].n_r; j++) cols[c++] = (w << 8) | j;
    *ncols = c;
}

}  // namespace

size_t basis_tc_smem() {
    return 2 * kTcTiles * kTileBytes + 2 * kTileBytes + kTcN * sizeof(float) + kTcN * sizeof(int) + 32;
}

cudaError_t prepare_basis_tc(eor_ctx* c) {
    (void)c;
    return cudaFuncSetAttribute(k_basis_ionize_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)basis_tc_smem());
}

cudaError_t build_columns(eor_ctx* c, int n_walkers) {
    trace_begin(c, kKTables);
    k_build_columns<<<1, 32, 0, c->stream>>>(c->d_walkers, n_walkers, c->d_cols, c->d_ncols);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_basis_ionize_tc(eor_ctx* c, float* xhi_out) {
    TcArgs a{c->d_F, c->d_coef, c->d_cols, c->d_ncols, c->d_pairs, c->d_delta, c->d_dtb, xhi_out, c->d_xpart,
             c->d_err, c->cfg.n_z, c->kb, c->max_radii, (long long)c->n3, (float)c->cfg.delta_c};
    trace_begin(c, kKBasis);
    k_basis_ionize_tc<<<dim3((unsigned)(c->n3 / kTcCells), c->cfg.n_z), kTcThreads, basis_tc_smem(), c->stream>>>(a);
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
