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

constexpr int kTcTiles = 4;                            // M tiles of 128 cells
constexpr int kTcCells = 128 * kTcTiles;               // cells per CTA
constexpr int kTcN = 64;                               // (walker, radius) columns per chunk
constexpr uint32_t kTileBytes = 128 * tc::kKMax * 4;   // one 128 x 32 TF32 tile (16 KB)
constexpr uint32_t kABytes = 2 * kTcTiles * kTileBytes;   // hi and lo tiles of a CTA (128 KB)
constexpr uint32_t kBBytes = 2 * kTcN * tc::kKMax * 4;    // hi and lo of a 64-column chunk (16 KB)
// column meta: walker, zeta, T_0, 1/sqrt(2 s^2) at R_cell columns (64 each), end masks (4 + pad 12)
constexpr int kMetaEnds = 4 * kTcN;
constexpr uint32_t kMBytes = (4 * kTcN + 16) * 4;
constexpr uint32_t kChunkBytes = kBBytes + kMBytes;       // one chunk in global memory
constexpr uint32_t kTmemCols = 512;                       // 2 buffers x 4 tiles x 64 columns
constexpr int kTcThreads = 384;                           // warp 0 producer, warps 4-11 epilogue
constexpr int kTcEpi = 256;                               // epilogue threads
constexpr float kNever = 1.0e30f;                         // folded threshold that no delta_R reaches
constexpr float kXScale = 8388608.0f;                     // 2^23: x_HI in fixed point for exact warp sums

// Basis fields -> the CTAs' A operands: [z][cta][hi/lo][tile][128 x 32 core-matrix layout],
// K index kb holding the constant 1 (kb + 1 <= 32).
__global__ void k_format_a(const float* F, int kb, long long n3, int n_z, unsigned char* out) {
    const long long total = (long long)n_z * tc::kKMax * n3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long cell = e % n3;
        const int b = (int)((e / n3) % tc::kKMax), zi = (int)(e / (n3 * tc::kKMax));
        // basis values, then the constant 1 that carries the folded threshold, then zeros
        const float v = b < kb ? F[((size_t)zi * kb + b) * n3 + cell] : (b == kb ? 1.0f : 0.0f);
        const uint32_t hi = tc::to_tf32(v), lo = tc::to_tf32(v - __uint_as_float(hi));
        const long long cta = cell / kTcCells;
        const int c = (int)(cell % kTcCells);
        unsigned char* base = out + ((size_t)zi * (n3 / kTcCells) + cta) * kABytes + (size_t)(c >> 7) * kTileBytes +
                              tc::core_offset(c & 127, b);
        *reinterpret_cast<uint32_t*>(base) = hi;
        *reinterpret_cast<uint32_t*>(base + kTcTiles * kTileBytes) = lo;
    }
}

// Walker coefficients -> chunks of 64 columns: [z][chunk][B hi | B lo | meta]. Column
// (walker w, radius j) holds c_b(R_j) for b < kb and, at K index kb, minus its threshold, so
// that the contraction yields D = delta_R - threshold: delta_crit(R_j) (Eq. 1 flag test
// D >= 0) above R_cell, delta_c at R_cell (where f_coll needs delta_c - delta_R). An
// infinite delta_crit (no ionization possible) becomes kNever. Column slots past the last
// column carry zero coefficients and -kNever. Meta, per column: the walker at its R_cell
// column (-1 elsewhere), and there zeta, T_0 and 1/sqrt(2 s^2(R_cell)) (0 when s^2 <= 0);
// then the mask of R_cell columns of each 16 columns.
__global__ void k_format_b(const int* cols, const int* ncols, const float* coef, const PairInfo* pairs, int kb,
                           int max_radii, int n_z, int slots, float delta_c, unsigned char* out) {
    const int slot = blockIdx.x * blockDim.x + threadIdx.x, zi = blockIdx.y;
    if (slot >= slots) return;   // slots is a multiple of 64: whole warps leave together
    const int nc = *ncols;
    unsigned char* chunk = out + ((size_t)zi * (slots / kTcN) + slot / kTcN) * kChunkBytes;
    const int row = slot % kTcN;
    float thr = kNever, zeta = 0.0f, t0 = 0.0f, inv = 0.0f;
    int walker_end = -1;
    const float* src = nullptr;
    if (slot < nc) {
        const int cw = cols[slot], w = cw >> 8, j = cw & 255;
        const PairInfo& pi = pairs[(size_t)w * n_z + zi];
        src = coef + ((size_t)w * max_radii + j) * kb;
        const bool last = j == pi.n_r - 1;
        const float dcrit = pi.delta_crit[j];
        thr = last ? delta_c : (isfinite(dcrit) ? dcrit : kNever);
        if (last) {
            walker_end = w;
            zeta = pi.zeta;
            t0 = pi.t0;
            inv = pi.cell_ok > 0.5f ? pi.inv_sqrt2s2_cell : 0.0f;
        }
    }
    for (int b = 0; b < tc::kKMax; b++) {
        const float v = b < kb ? (src ? src[b] : 0.0f) : (b == kb ? -thr : 0.0f);
        const uint32_t hi = tc::to_tf32(v), lo = tc::to_tf32(v - __uint_as_float(hi));
        *reinterpret_cast<uint32_t*>(chunk + tc::core_offset(row, b)) = hi;
        *reinterpret_cast<uint32_t*>(chunk + kBBytes / 2 + tc::core_offset(row, b)) = lo;
    }
    int* meta = reinterpret_cast<int*>(chunk + kBBytes);
    float* metaf = reinterpret_cast<float*>(meta);
    meta[row] = walker_end;
    metaf[kTcN + row] = zeta;
    metaf[2 * kTcN + row] = t0;
    metaf[3 * kTcN + row] = inv;
    const unsigned ends = __ballot_sync(0xffffffffu, walker_end >= 0);
    if ((row & 15) == 0) meta[kMetaEnds + row / 16] = (int)((ends >> (threadIdx.x & 16)) & 0xFFFFu);
    if (row < 12) meta[kMetaEnds + 4 + row] = 0;
}

// Pairwise maximum tree of 16 values (depth 4).
__device__ __forceinline__ float max16(const float (&v)[16]) {
    float m8[8];
#pragma unroll
    for (int i = 0; i < 8; i++) m8[i] = fmaxf(v[i], v[i + 8]);
#pragma unroll
    for (int i = 0; i < 4; i++) m8[i] = fmaxf(m8[i], m8[i + 4]);
    return fmaxf(fmaxf(m8[0], m8[2]), fmaxf(m8[1], m8[3]));
}

struct TcArgs {
    const unsigned char* A;     // [n_z][cta][kABytes]
    const unsigned char* B;     // [n_z][chunk][kChunkBytes]
    const int* ncols;           // [1] number of columns
    const PairInfo* pairs;      // [walker * n_z + zi]
    const float* delta;         // [n_z][n3]
    float* dtb;                 // [pair][n3]
    float* xhi_out;             // optional [pair][n3]
    float* xpart;               // [pair][n3 / 64] per-warp neutral-fraction sums
    int* err;
    int n_z, chunks_per_z;
    long long n3;
    float delta_c;
};

// One CTA: 512 cells of one redshift against every (walker, radius) column, as four 128-row
// tiles. The cells' basis values (A) and each 64-column chunk of coefficients (B) arrive by
// bulk copy in the TF32 hi/lo core-matrix layout; thread 0 issues, per tile and K step,
// hi*hi + hi*lo + lo*hi (3xTF32, FP32 accumulation) into one of two tensor-memory buffers,
// so D(cell, column) = sum_b F_b c_b - threshold = delta_R - threshold. Warps 4-11 run the
// epilogue of the other buffer meanwhile, each thread two cells: the Eq. 1 flag of a
// walker is "D >= 0 at some radius above R_cell" (a max over 16 columns where no walker
// ends, bit masks of D >= 0 where one does); at the walker's R_cell column
// (D = delta_R - delta_c) it forms x_HI and delta T_b (coalesced stores) and an exact
// fixed-point warp sum of x_HI.
// Buffer hand-offs: B(c) is reloaded only after MMA(c) completed; the thresholds / meta of
// chunk c (read by the epilogue) only after the epilogue released its buffer; MMA(c + 2)
// waits for both. Every wait is bounded; on a timeout the CTA sets kErrTimeout, waits for
// its copies and MMAs in flight and frees its tensor memory.
__global__ void __launch_bounds__(kTcThreads, 1) k_basis_ionize_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                                // A hi tiles then lo tiles
    unsigned char* Bs = As + kABytes;                      // [2][kBBytes]
    unsigned char* Ms = Bs + 2 * kBBytes;                  // [2][kMBytes]
    uint64_t* bars = reinterpret_cast<uint64_t*>(Ms + 2 * kMBytes);
    uint64_t* barA = bars + 0;
    uint64_t* barB = bars + 1;       // [2] coefficient tile landed
    uint64_t* barM = bars + 3;       // [2] thresholds / meta landed
    uint64_t* barD = bars + 5;       // [2] MMAs into tensor-memory buffer done
    uint64_t* barE = bars + 7;       // [2] epilogue released the buffer
    uint64_t* barF = bars + 9;       // MMAs drained (abort path)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 10);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int zi = blockIdx.y;
    const long long cell0 = (long long)blockIdx.x * kTcCells;
    const int ncols = *a.ncols;
    const int nch = (ncols + kTcN - 1) / kTcN;

    if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
    if (t == 0) {
        tc::mbar_init(barA, 1);
        tc::mbar_init(barF, 1);
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(barB + s, 1);
            tc::mbar_init(barM + s, 1);
            tc::mbar_init(barD + s, 1);
            tc::mbar_init(barE + s, kTcEpi);
        }
        *abort = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint32_t kTries = 1u << 24;
    // producer bookkeeping: parity of the phase each copy barrier still owes, or -1
    int owedA = -1, owedB[2] = {-1, -1}, owedM[2] = {-1, -1};

    if (t == 0 && nch > 0) {
        // ---------------- producer: bulk copies and MMA issue
        const unsigned char* Ag = a.A + ((size_t)zi * (a.n3 / kTcCells) + blockIdx.x) * kABytes;
        const unsigned char* Bg = a.B + (size_t)zi * a.chunks_per_z * kChunkBytes;
        tc::mbar_expect_tx(barA, kABytes);
        tc::bulk_g2s(As, Ag, kABytes, barA);
        owedA = 0;
        for (int c = 0; c < 2 && c < nch; c++) {
            tc::mbar_expect_tx(barB + c, kBBytes);
            tc::bulk_g2s(Bs + c * kBBytes, Bg + (size_t)c * kChunkBytes, kBBytes, barB + c);
            owedB[c] = 0;
            tc::mbar_expect_tx(barM + c, kMBytes);
            tc::bulk_g2s(Ms + c * kMBytes, Bg + (size_t)c * kChunkBytes + kBBytes, kMBytes, barM + c);
            owedM[c] = 0;
        }
        bool ok = tc::mbar_wait_or_abort(barA, 0, kTries, abort);
        if (ok) owedA = -1;
        const uint32_t idesc = tc::idesc_tf32(128, kTcN);
        for (int c = 0; c < nch && ok; c++) {
            const int s = c & 1;
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            ok = tc::mbar_wait_or_abort(barB + s, par, kTries, abort);
            if (!ok) break;
            owedB[s] = -1;
            tc::fence_after_sync();
            for (int q = 0; q < kTcTiles; q++) {
                const uint32_t d = tmem + (uint32_t)(s * kTcTiles * kTcN + q * kTcN);
                for (int st = 0; st < tc::kKMax / 8; st++) {
                    const uint32_t ko = (uint32_t)st * 2 * tc::kLBO;
                    const uint64_t ah = tc::smem_desc(tc::smem_addr(As + q * kTileBytes) + ko, tc::kLBO, tc::kSBO);
                    const uint64_t al =
                        tc::smem_desc(tc::smem_addr(As + (kTcTiles + q) * kTileBytes) + ko, tc::kLBO, tc::kSBO);
                    const uint64_t bh = tc::smem_desc(tc::smem_addr(Bs + s * kBBytes) + ko, tc::kLBO, tc::kSBO);
                    const uint64_t bl =
                        tc::smem_desc(tc::smem_addr(Bs + s * kBBytes + kBBytes / 2) + ko, tc::kLBO, tc::kSBO);
                    tc::mma_tf32(d, ah, bh, idesc, st > 0 ? 1u : 0u);
                    tc::mma_tf32(d, ah, bl, idesc, 1u);
                    tc::mma_tf32(d, al, bh, idesc, 1u);
                }
            }
            tc::mma_commit(barD + s);
            if (c >= 1 && c + 1 < nch) {   // chunk c + 1 into the buffers chunk c - 1 used
                const int s1 = (c + 1) & 1;
                const uint32_t p1 = (uint32_t)((c - 1) >> 1) & 1u;
                ok = tc::mbar_wait_or_abort(barD + s1, p1, kTries, abort);   // MMA(c - 1) has read B
                if (!ok) break;
                tc::mbar_expect_tx(barB + s1, kBBytes);
                tc::bulk_g2s(Bs + s1 * kBBytes, Bg + (size_t)(c + 1) * kChunkBytes, kBBytes, barB + s1);
                owedB[s1] = (int)(((c + 1) >> 1) & 1);
                ok = tc::mbar_wait_or_abort(barE + s1, p1, kTries, abort);   // epilogue(c - 1) is done
                if (!ok) break;
                tc::mbar_expect_tx(barM + s1, kMBytes);
                tc::bulk_g2s(Ms + s1 * kMBytes, Bg + (size_t)(c + 1) * kChunkBytes + kBBytes, kMBytes, barM + s1);
                owedM[s1] = (int)(((c + 1) >> 1) & 1);
            }
        }
        if (!ok) {
            *abort = 1;
            atomicOr(a.err, kErrTimeout);
        }
    } else if (warp >= 4 && nch > 0) {
        // ---------------- epilogue warps: warp 4 + e owns tensor-memory lanes 32 (e % 4) .. + 31
        // (the quarter its warp index allows) of tiles 2 (e / 4) and 2 (e / 4) + 1
        const int e = warp - 4, lq = warp & 3, q0 = 2 * (e >> 2);
        long long cell[2];
        float dens[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            cell[u] = cell0 + (q0 + u) * 128 + lq * 32 + lane;
            dens[u] = __ldg(a.delta + (size_t)zi * a.n3 + cell[u]);
        }
        bool fl[2] = {false, false};   // the walker's Eq. 1 flag from the radii seen so far
        for (int c = 0; c < nch; c++) {
            const int s = c & 1;
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            if (!tc::mbar_wait_or_abort(barD + s, par, kTries, abort) ||
                !tc::mbar_wait_or_abort(barM + s, par, kTries, abort)) {
                if (lane == 0) atomicOr(a.err, kErrTimeout);
                *abort = 1;
                break;
            }
            tc::fence_after_sync();
            const int* meta = reinterpret_cast<const int*>(Ms + s * kMBytes);
            const float* metaf = reinterpret_cast<const float*>(meta);
            const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(s * kTcTiles * kTcN + q0 * kTcN);
            for (int g = 0; g < kTcN / 16 && c * kTcN + g * 16 < ncols; g++) {
                float v[2][16];
                tc::tmem_ld16x2(base + (uint32_t)(g * 16), base + (uint32_t)(kTcN + g * 16), v[0], v[1]);
                uint32_t ends = (uint32_t)meta[kMetaEnds + g];
                if (ends == 0u) {
#pragma unroll
                    for (int u = 0; u < 2; u++) fl[u] = fl[u] || max16(v[u]) >= 0.0f;
                    continue;
                }
                // columns of this group with D >= 0, as bits
                uint32_t pos[2] = {0u, 0u};
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    pos[0] |= v[0][i] >= 0.0f ? (1u << i) : 0u;
                    pos[1] |= v[1][i] >= 0.0f ? (1u << i) : 0u;
                }
                uint32_t start = 0;   // first column of the current walker within the group
                while (ends) {        // the same for every thread
                    const uint32_t p = (uint32_t)(__ffs(ends) - 1);
                    ends &= ends - 1u;
                    const uint32_t seg = ((1u << p) - 1u) & ~((1u << start) - 1u);   // radii above R_cell
                    const int col = g * 16 + (int)p, w = meta[col];
                    const float zeta = metaf[kTcN + col], t0 = metaf[2 * kTcN + col], inv = metaf[3 * kTcN + col];
                    float d[2];   // D = delta_R(R_cell) - delta_c
                    tc::tmem_ld1x2(base + (uint32_t)col, base + (uint32_t)(kTcN + col), d[0], d[1]);
                    const size_t pair = (size_t)w * a.n_z + zi;
                    int xq = 0;
#pragma unroll
                    for (int u = 0; u < 2; u++) {
                        float xh = 1.0f;
                        if (fl[u] || (pos[u] & seg)) {
                            xh = 0.0f;   // flagged at a larger radius (Eq. 1)
                        } else if (inv > 0.0f) {
                            const float f = d[u] >= 0.0f ? 1.0f : erfcf(-d[u] * inv);
                            xh = 1.0f - fminf(1.0f, zeta * f);
                        }
                        a.dtb[pair * a.n3 + cell[u]] = t0 * xh * (1.0f + dens[u]);
                        if (a.xhi_out) a.xhi_out[pair * a.n3 + cell[u]] = xh;
                        xq += __float2int_rn(xh * kXScale);
                        fl[u] = false;
                    }
                    xq = __reduce_add_sync(0xffffffffu, xq);   // exact: integers
                    if (lane == 0)
                        a.xpart[pair * (size_t)(a.n3 / 64) + (size_t)blockIdx.x * 8 + e] = (float)xq / kXScale;
                    start = p + 1;
                }
                const uint32_t rest = 0xFFFFu & ~((1u << start) - 1u);   // the next walker's radii
#pragma unroll
                for (int u = 0; u < 2; u++) fl[u] = (pos[u] & rest) != 0u;
            }
            tc::fence_before_sync();
            tc::mbar_arrive(barE + s);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t == 0 && nch > 0 && *abort) {
        // drain: every MMA issued so far, then every bulk copy still owed
        tc::mma_commit(barF);
        tc::mbar_wait(barF, 0, kTries);
        if (owedA >= 0) tc::mbar_wait(barA, (uint32_t)owedA, kTries);
        for (int s = 0; s < 2; s++) {
            if (owedB[s] >= 0) tc::mbar_wait(barB + s, (uint32_t)owedB[s], kTries);
            if (owedM[s] >= 0) tc::mbar_wait(barM + s, (uint32_t)owedM[s], kTries);
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) {
        __syncwarp();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
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

bool basis_tc_fits(int kb) { return kb + 1 <= tc::kKMax; }   // basis values plus the constant column

size_t basis_tc_smem() { return kABytes + 2 * kBBytes + 2 * kMBytes + 10 * sizeof(uint64_t) + 16; }
size_t basis_tc_a_bytes(long long n3, int n_z) { return (size_t)n_z * (size_t)(n3 / kTcCells) * kABytes; }
size_t basis_tc_b_bytes(int max_columns, int n_z) {
    return (size_t)n_z * (size_t)((max_columns + kTcN - 1) / kTcN) * kChunkBytes;
}

cudaError_t prepare_basis_tc(eor_ctx* c) {
    (void)c;
    return cudaFuncSetAttribute(k_basis_ionize_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)basis_tc_smem());
}

cudaError_t format_basis_tc(eor_ctx* c) {
    trace_begin(c, kKOther);
    k_format_a<<<2048, 256, 0, c->stream>>>(c->d_F, c->kb, (long long)c->n3, c->cfg.n_z, c->d_tcA);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t build_columns(eor_ctx* c, int n_walkers) {
    trace_begin(c, kKTables);
    k_build_columns<<<1, 32, 0, c->stream>>>(c->d_walkers, n_walkers, c->d_cols, c->d_ncols);
    trace_end(c);
    const int slots = (c->cfg.max_walkers * c->max_radii + kTcN - 1) / kTcN * kTcN;
    trace_begin(c, kKTables);
    k_format_b<<<dim3((slots + 127) / 128, c->cfg.n_z), 128, 0, c->stream>>>(
        c->d_cols, c->d_ncols, c->d_coef, c->d_pairs, c->kb, c->max_radii, c->cfg.n_z, slots, (float)c->cfg.delta_c,
        c->d_tcB);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_basis_ionize_tc(eor_ctx* c, float* xhi_out) {
    const int slots = (c->cfg.max_walkers * c->max_radii + kTcN - 1) / kTcN * kTcN;
    TcArgs a{c->d_tcA, c->d_tcB, c->d_ncols, c->d_pairs, c->d_delta, c->d_dtb, xhi_out, c->d_xpart, c->d_err,
             c->cfg.n_z, slots / kTcN, (long long)c->n3, (float)c->cfg.delta_c};
    trace_begin(c, kKBasis);
    k_basis_ionize_tc<<<dim3((unsigned)(c->n3 / kTcCells), c->cfg.n_z), kTcThreads, basis_tc_smem(), c->stream>>>(a);
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
