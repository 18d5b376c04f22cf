// tcgen05.cu — tensor-core (tcgen05, TMEM) kernels of libeor21.
//
// k_tc_check: one CTA computes D = A B^T (A 128 x 32, B n x 32, FP32 in global memory) with
// TF32 tcgen05 MMAs accumulating in tensor memory: the operand layout, descriptors and
// tensor-memory reads of the tensor-core contraction, checked in isolation.
#include "eor_internal.cuh"
#include "tc.cuh"

namespace eor {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s of GPU time per bounded wait

// A bounded wait ran out: set kErrTimeout and keep the first record of where,
// err[1] = role << 28 | barrier << 20 | chunk (roles 1 copy, 2 MMA, 3 epilogue; barriers
// 1 A, 2 B full, 3 B empty, 4 meta full, 5 meta empty, 6 accumulator full, 7 accumulator free).
__device__ __forceinline__ void record_timeout(int* err, int role, int bar, int chunk) {
    atomicOr(err, kErrTimeout);
    atomicCAS(err + 1, 0, (role << 28) | (bar << 20) | (chunk & 0xFFFFF));
}

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
    bool ok = tc::mbar_wait(bar, 0, kWaitNs);
    if (!ok) ok = tc::mbar_wait(bar, 0, kWaitNs);   // let an MMA in flight finish before freeing its memory
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

constexpr int kTcTiles = 2;                            // M tiles of 128 cells per CTA (their MMAs alternate)
constexpr int kTcCells = 128 * kTcTiles;               // cells per CTA
constexpr int kTcN = 128;                              // (walker, radius) columns per chunk (MMA N)
constexpr int kTcStages = 3;                           // coefficient chunks in flight
constexpr int kGroup = 32;                             // epilogue columns per tensor-memory read
constexpr uint32_t kTileBytes = 128 * tc::kKMax * 4;   // one 128 x 32 TF32 tile (16 KB)
constexpr uint32_t kABytes = 2 * kTcTiles * kTileBytes;   // hi and lo tiles of a CTA (64 KB)
constexpr uint32_t kBBytes = 2 * kTcN * tc::kKMax * 4;    // hi and lo of a chunk (32 KB)
// chunk meta: one 16-byte record per group of kGroup columns: (walker << 2 | first << 1 |
// last, or -1 for an unused group; zeta, T_0, 1/sqrt(2 s^2(R_cell)) or 0 when s^2 <= 0, or
// with a mass-dependent efficiency the inverse step of the pair's table). With a
// mass-dependent efficiency two more parts follow: per column the width delta_hi -
// delta_crit of its flag interval, and per group the partial-ionization table of the walker
// that ends there (kFTab floats), so that the epilogue reads both from shared memory.
constexpr int kGroupsPerChunk = kTcN / kGroup;
constexpr uint32_t kMRecBytes = kGroupsPerChunk * 16;
constexpr uint32_t kMTabOff = kMRecBytes + kTcN * 4;
constexpr uint32_t kMBytes = kMTabOff + kGroupsPerChunk * kFTab * 4;
constexpr uint32_t kChunkBytes = kBBytes + kMBytes;       // one chunk in global memory
constexpr int kTmemBufs = 2;                              // accumulator buffers in tensor memory
constexpr uint32_t kTmemCols = kTmemBufs * kTcTiles * kTcN;   // 2 buffers x kTcTiles x kTcN columns (512)
constexpr int kEpiSets = 1;                               // epilogue warp sets, alternating chunks
constexpr int kTcEpiSet = 2 * 128 * kTcTiles;             // threads of a set: 2 per cell
constexpr int kTcEpi = kEpiSets * kTcEpiSet;              // epilogue threads
constexpr int kTcThreads = 128 + kTcEpi;                  // warps 0-3: MMA (thread 0), copies (thread 32); then epilogue
constexpr int kTcCtasPerSm = 1;                          // one CTA holds all tensor memory of an SM
constexpr float kNever = 1.0e30f;                         // folded threshold that no delta_R reaches
constexpr float kXScale = 8388608.0f;                     // 2^23: x_HI in fixed point for exact sums
static_assert(kTmemCols <= 512, "tensor memory");
static_assert(kTmemBufs % kEpiSets == 0, "a set always meets the same buffers");
static_assert(kMBytes % 16 == 0 && kChunkBytes % 16 == 0 && kMRecBytes % 16 == 0,
              "bulk copies move multiples of 16 bytes");
static_assert(kTcEpiSet == 2 * 128 * kTcTiles, "two epilogue threads per cell: groups 0-1 and 2-3 of a chunk");
static_assert(kTcN == 128 && kGroup == 32, "k_format_b: one block per chunk, one warp per group; 4 epilogue groups");

// Basis fields -> the CTAs' A operands: [z][cta][hi/lo][tile][128 x 32 core-matrix layout]:
// the rank basis values, then at K index rank the constant 1 that carries the folded
// threshold, then zeros (rank + 1 <= 32). F is [z][kb][n3] (kb >= rank).
__global__ void k_format_a(const float* F, int kb, int rank, long long n3, int n_z, unsigned char* out) {
    const long long total = (long long)n_z * tc::kKMax * n3;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long cell = e % n3;
        const int b = (int)((e / n3) % tc::kKMax), zi = (int)(e / (n3 * tc::kKMax));
        const float v = b < rank ? F[((size_t)zi * kb + b) * n3 + cell] : (b == rank ? 1.0f : 0.0f);
        const uint32_t hi = tc::to_tf32(v), lo = tc::to_tf32(v - __uint_as_float(hi));
        const long long cta = cell / kTcCells;
        const int c = (int)(cell % kTcCells);
        unsigned char* base = out + ((size_t)zi * (n3 / kTcCells) + cta) * kABytes + (size_t)(c >> 7) * kTileBytes +
                              tc::core_offset(c & 127, b);
        *reinterpret_cast<uint32_t*>(base) = hi;
        *reinterpret_cast<uint32_t*>(base + kTcTiles * kTileBytes) = lo;
    }
}

// Walker coefficients -> chunks of kTcN columns: [z][chunk][B hi | B lo | meta], one block
// per chunk and one warp per group of kGroup columns. Column (walker w, radius j) holds
// c_b(R_j) for b < rank and, at K index rank, minus its threshold, so that the contraction
// yields D = delta_R - threshold: delta_crit(R_j) (Eq. 1 flag test D >= 0) above R_cell,
// delta_c at R_cell (where f_coll needs delta_c - delta_R). An infinite delta_crit (no
// ionization possible) becomes kNever. Padding columns carry zero coefficients and
// -kNever, so that D = -kNever there.
__global__ void __launch_bounds__(kTcN) k_format_b(const int* cols, const int* gmeta, const int* ncols,
                                                   const float* coef, const PairInfo* pairs, int kb, int rank,
                                                   int max_radii,
                                                   int n_z, int chunks_per_z, float delta_c, const float* ftab,
                                                   unsigned char* out) {
    const int pops = ftab != nullptr;
    const int row = threadIdx.x, zi = blockIdx.y, slot = blockIdx.x * kTcN + row;
    const int nc = *ncols;
    unsigned char* chunk = out + ((size_t)zi * chunks_per_z + blockIdx.x) * kChunkBytes;
    float thr = kNever, width = INFINITY;
    const float* src = nullptr;
    const int cw = slot < nc ? cols[slot] : -1;
    if (cw >= 0) {
        const int w = cw >> 8, j = cw & 255;
        const PairInfo& pi = pairs[(size_t)w * n_z + zi];
        src = coef + ((size_t)w * max_radii + j) * kb;
        const float dcrit = pi.delta_crit[j];
        thr = j == pi.n_r - 1 ? delta_c : (isfinite(dcrit) ? dcrit : kNever);
        if (j != pi.n_r - 1 && isfinite(dcrit) && isfinite(pi.delta_hi[j])) width = pi.delta_hi[j] - dcrit;
    }
    reinterpret_cast<float*>(chunk + kBBytes + kMRecBytes)[row] = width;
    if (pops) {   // the tables of the walkers that end in each group
        for (int g = 0; g < kGroupsPerChunk; g++) {
            const int gi = blockIdx.x * kGroupsPerChunk + g;
            const int info = gi < nc / kGroup ? gmeta[gi] : -1;
            float* dst = reinterpret_cast<float*>(chunk + kBBytes + kMTabOff) + g * kFTab;
            const float* src = info >= 0 && (info & 1) ? ftab + ((size_t)(info >> 2) * n_z + zi) * kFTab : nullptr;
            for (int e = row; e < kFTab; e += kTcN) dst[e] = src ? src[e] : 0.0f;
        }
    }
    for (int b = 0; b < tc::kKMax; b++) {
        const float v = b < rank ? (src ? src[b] : 0.0f) : (b == rank ? -thr : 0.0f);
        const uint32_t hi = tc::to_tf32(v), lo = tc::to_tf32(v - __uint_as_float(hi));
        *reinterpret_cast<uint32_t*>(chunk + tc::core_offset(row, b)) = hi;
        *reinterpret_cast<uint32_t*>(chunk + kBBytes / 2 + tc::core_offset(row, b)) = lo;
    }
    if ((row & (kGroup - 1)) == 0) {
        const int g = row / kGroup, gi = blockIdx.x * kGroupsPerChunk + g;
        const int info = gi < nc / kGroup ? gmeta[gi] : -1;
        float zeta = 0.0f, t0 = 0.0f, inv = 0.0f;
        if (info >= 0) {
            const PairInfo& pi = pairs[(size_t)(info >> 2) * n_z + zi];
            zeta = pi.zeta;
            t0 = pi.t0;
            inv = pops ? pi.f_inv_h : (pi.cell_ok > 0.5f ? pi.inv_sqrt2s2_cell : 0.0f);
        }
        reinterpret_cast<int4*>(chunk + kBBytes)[g] =
            make_int4(info, __float_as_int(zeta), __float_as_int(t0), __float_as_int(inv));
    }
}

// AND of v[1..31] (LOP3 tree): its sign bit is clear iff some of them has a clear sign bit.
__device__ __forceinline__ uint32_t and31(const float (&v)[32]) {
    uint32_t m[8];
#pragma unroll
    for (int i = 0; i < 8; i++)
        m[i] = (i == 0 ? 0xFFFFFFFFu : __float_as_uint(v[i])) & __float_as_uint(v[i + 8]) &
               __float_as_uint(v[i + 16]) & __float_as_uint(v[i + 24]);
    return (m[0] & m[1] & m[2]) & (m[3] & m[4] & m[5]) & (m[6] & m[7]);
}

// erfc(x) for x >= 0 from the Chebyshev fit of Numerical Recipes (Press et al. 1992, Sec. 6.2,
// "erfcc"; fractional error below 1.2e-7 everywhere): t = 1 / (1 + x/2) and
// erfc(x) = t exp(-x^2 + P(t)) with P a degree-9 polynomial. Branch-free.
__device__ __forceinline__ float erfc_cheb(float x) {
    const float t = __frcp_rn(fmaf(0.5f, x, 1.0f));
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
    return t * expf(fmaf(-x, x, p));
}

struct TcArgs {
    const unsigned char* A;     // [n_z][cta][kABytes]
    const unsigned char* B;     // [n_z][chunk][kChunkBytes]
    const int* ncols;           // [1] number of columns
    const float* delta;         // [n_z][n3]
    float* dtb;                 // [pair][n3]
    float* xhi_out;             // optional [pair][n3]
    unsigned long long* xq;     // [pair] fixed-point (2^23) sums of x_HI
    const float* ftab;          // [pair][kFTab] with a mass-dependent efficiency, else nullptr
    int* err;
    int n_z, chunks_per_z;
    int ksteps;                 // MMA K steps of 8: (rank + 1) / 8 rounded up
    long long n3;
};

// One CTA: 256 cells of one redshift (two 128-row tiles) against every (walker, radius)
// column. The cells' basis values (A) and each 128-column chunk of coefficients (B) arrive by
// bulk copy in the TF32 hi/lo core-matrix layout; thread 0 issues, per K step, product and
// tile, hi*hi + hi*lo + lo*hi (3xTF32, FP32 accumulation) into one of two tensor-memory
// buffers, so D(cell, column) = sum_b F_b c_b - threshold = delta_R - threshold. Each
// walker's columns start on a group of 32: its R_cell column first (D = delta_R - delta_c),
// then its radii from R_mfp down, then padding. Warps 4-19 run the epilogue of the other
// buffer meanwhile (kEpiSets = 1: one set takes every chunk), two threads per cell
// (groups 0-1 and 2-3 of the chunk): the Eq. 1 flag
// of a walker, "D >= 0 (sign bit clear) at some radius above R_cell", is an AND of sign bits
// over its columns; at its last group the thread forms x_HI and delta T_b (coalesced stores)
// and the warp adds its exact fixed-point x_HI sum to the pair's total.
// Roles: thread 32 issues the bulk copies, thread 0 the MMAs (it waits only for operands and
// a free accumulator buffer, so the tensor pipe stays fed), warps 4-19 the epilogue.
// Hand-offs: chunk c + 3 reuses chunk c's stage after MMA(c) (coefficients) and the
// epilogue's read of chunk c's meta; MMA(c) reuses the tensor memory of chunk c - 2 after
// its epilogue. Every wait is bounded in GPU time; on a timeout the CTA records where, sets
// kErrTimeout, waits for its copies and MMAs in flight and frees its tensor memory.
// POPS: the mass-dependent efficiency (interval flags, partial ionization from the tables
// in the chunk meta); otherwise the step function (sign-bit AND, erfc). The meta stage holds
// only the group records without POPS.
template <bool POPS>
__global__ void __launch_bounds__(kTcThreads, kTcCtasPerSm) k_basis_ionize_tc(TcArgs a) {
    constexpr uint32_t kMB = POPS ? kMBytes : kMRecBytes;  // meta bytes copied and staged per chunk
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                                // A hi tiles then lo tiles
    unsigned char* Bs = As + kABytes;                      // [kTcStages][kBBytes]
    unsigned char* Ms = Bs + kTcStages * kBBytes;          // [kTcStages][kMB]
    uint64_t* bars = reinterpret_cast<uint64_t*>(Ms + kTcStages * kMB);
    uint64_t* barA = bars;
    uint64_t* barB = bars + 1;                  // [kTcStages] coefficient tile landed
    uint64_t* barBe = barB + kTcStages;         // [kTcStages] its MMAs are done: stage free
    uint64_t* barM = barBe + kTcStages;         // [kTcStages] meta landed
    uint64_t* barMe = barM + kTcStages;         // [kTcStages] the epilogue has read it: stage free
    uint64_t* barD = barMe + kTcStages;         // [kTmemBufs] MMAs into tensor-memory buffer done
    uint64_t* barE = barD + kTmemBufs;          // [kTmemBufs] epilogue released the buffer
    uint64_t* barF = barE + kTmemBufs;          // MMAs drained (abort path)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(barF + 1);
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
        for (int s = 0; s < kTcStages; s++) {
            tc::mbar_init(barB + s, 1);
            tc::mbar_init(barBe + s, 1);
            tc::mbar_init(barM + s, 1);
            tc::mbar_init(barMe + s, kTcEpiSet);
        }
        for (int s = 0; s < kTmemBufs; s++) {
            tc::mbar_init(barD + s, 1);
            tc::mbar_init(barE + s, kTcEpiSet);
        }
        *abort = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    constexpr uint64_t kTries = kWaitNs;   // time limit of every wait below
    // copy-thread bookkeeping: parity of the phase each copy barrier still owes, or -1
    int owedA = -1, owedB[kTcStages], owedM[kTcStages];
#pragma unroll
    for (int s = 0; s < kTcStages; s++) owedB[s] = owedM[s] = -1;

    if (t == 32 && nch > 0) {
        // ---------------- copy thread: the CTA's A operands once, then chunk c into stage
        // c % kTcStages as soon as chunk c - kTcStages has left it
        const unsigned char* Ag = a.A + ((size_t)zi * (a.n3 / kTcCells) + blockIdx.x) * kABytes;
        const unsigned char* Bg = a.B + (size_t)zi * a.chunks_per_z * kChunkBytes;
        tc::mbar_expect_tx(barA, kABytes);
        tc::bulk_g2s(As, Ag, kABytes, barA);
        owedA = 0;
        bool ok = true;
        for (int c = 0; c < nch && ok; c++) {
            const int st = c % kTcStages;
            const uint32_t use = (uint32_t)(c / kTcStages);   // how many chunks used the stage before
            if (use > 0) ok = tc::mbar_wait_or_abort(barBe + st, (use - 1) & 1u, kTries, abort);
            if (!ok) { record_timeout(a.err, 1, 3, c); break; }
            tc::mbar_expect_tx(barB + st, kBBytes);
            tc::bulk_g2s(Bs + st * kBBytes, Bg + (size_t)c * kChunkBytes, kBBytes, barB + st);
            owedB[st] = (int)(use & 1u);
            if (use > 0) ok = tc::mbar_wait_or_abort(barMe + st, (use - 1) & 1u, kTries, abort);
            if (!ok) { record_timeout(a.err, 1, 5, c); break; }
            tc::mbar_expect_tx(barM + st, kMB);
            tc::bulk_g2s(Ms + st * kMB, Bg + (size_t)c * kChunkBytes + kBBytes, kMB, barM + st);
            owedM[st] = (int)(use & 1u);
        }
        if (!ok) *abort = 1;
    } else if (t == 0 && nch > 0) {
        // ---------------- MMA thread: waits only for operands and a free accumulator buffer
        bool ok = tc::mbar_wait_or_abort(barA, 0, kTries, abort);
        if (!ok) record_timeout(a.err, 2, 1, 0);
        const uint32_t idesc = tc::idesc_tf32(128, kTcN);
        for (int c = 0; c < nch && ok; c++) {
            const int st = c % kTcStages, tb = c % kTmemBufs;
            ok = tc::mbar_wait_or_abort(barB + st, (uint32_t)(c / kTcStages) & 1u, kTries, abort);
            if (!ok) { record_timeout(a.err, 2, 2, c); break; }
            if (c >= kTmemBufs)   // the epilogue of chunk c - kTmemBufs has released buffer tb
                ok = tc::mbar_wait_or_abort(barE + tb, (uint32_t)((c - kTmemBufs) / kTmemBufs) & 1u, kTries,
                                            abort);
            if (!ok) { record_timeout(a.err, 2, 7, c); break; }
            tc::fence_after_sync();
            // the tiles' accumulators alternate, so that consecutive MMAs are independent
            for (int ks = 0; ks < a.ksteps; ks++) {
                const uint32_t ko = (uint32_t)ks * 2 * tc::kLBO;
                const uint64_t bh = tc::smem_desc(tc::smem_addr(Bs + st * kBBytes) + ko, tc::kLBO, tc::kSBO);
                const uint64_t bl = tc::smem_desc(tc::smem_addr(Bs + st * kBBytes + kBBytes / 2) + ko, tc::kLBO, tc::kSBO);
                uint64_t ah[kTcTiles], al[kTcTiles];
#pragma unroll
                for (int q = 0; q < kTcTiles; q++) {
                    ah[q] = tc::smem_desc(tc::smem_addr(As + q * kTileBytes) + ko, tc::kLBO, tc::kSBO);
                    al[q] = tc::smem_desc(tc::smem_addr(As + (kTcTiles + q) * kTileBytes) + ko, tc::kLBO, tc::kSBO);
                }
#pragma unroll
                for (int q = 0; q < kTcTiles; q++)
                    tc::mma_tf32(tmem + (uint32_t)(tb * kTcTiles * kTcN + q * kTcN), ah[q], bh, idesc, ks > 0 ? 1u : 0u);
#pragma unroll
                for (int q = 0; q < kTcTiles; q++)
                    tc::mma_tf32(tmem + (uint32_t)(tb * kTcTiles * kTcN + q * kTcN), ah[q], bl, idesc, 1u);
#pragma unroll
                for (int q = 0; q < kTcTiles; q++)
                    tc::mma_tf32(tmem + (uint32_t)(tb * kTcTiles * kTcN + q * kTcN), al[q], bh, idesc, 1u);
            }
            tc::mma_commit(barD + tb);    // accumulators ready for the epilogue
            tc::mma_commit(barBe + st);   // coefficient stage free for the copy thread
        }
        if (!ok) *abort = 1;
    } else if (warp >= 4 && nch > 0) {
        // ---------------- epilogue warps: set `set` (8 kTcTiles warps) takes the chunks
        // c = set (mod kEpiSets); within it warp 4 + e owns tensor-memory lanes 32 (e % 4) ..
        // + 31 (the quarter its warp index allows) of tile (ei / 4) % kTcTiles, and groups g0
        // and g0 + 1 of its chunks: one cell, half the columns. A walker never spans the two
        // halves (multi-group walkers start on an even group).
        const int e = warp - 4, set = e / (8 * kTcTiles), ei = e % (8 * kTcTiles);
        const int lq = warp & 3, q = (ei >> 2) % kTcTiles, g0 = 2 * ((ei >> 2) / kTcTiles);
        const long long cell = cell0 + q * 128 + lq * 32 + lane;
        const float dens = __ldg(a.delta + (size_t)zi * a.n3 + cell);
        for (int c = set; c < nch; c += kEpiSets) {
            const int st = c % kTcStages, tb = c % kTmemBufs;
            const bool okD = tc::mbar_wait_or_abort(barD + tb, (uint32_t)(c / kTmemBufs) & 1u, kTries, abort);
            const bool okM = okD && tc::mbar_wait_or_abort(barM + st, (uint32_t)(c / kTcStages) & 1u, kTries, abort);
            if (!okM) {
                if (lane == 0) record_timeout(a.err, 3, okD ? 4 : 6, c);
                *abort = 1;
                break;
            }
            tc::fence_after_sync();
            const int4* gm = reinterpret_cast<const int4*>(Ms + st * kMB) + g0;
            const uint32_t base = tmem + ((uint32_t)(lq * 32) << 16) +
                                  (uint32_t)(tb * kTcTiles * kTcN + q * kTcN + g0 * kGroup);
            int4 m[2];
            float dd[2], pf[2] = {0.0f, 0.0f};
            uint32_t fa[2];
            {
                float v[2][32];
                tc::tmem_ld32x2(base, v[0], v[1]);
                m[0] = gm[0];
                m[1] = gm[1];
                const bool second = (m[1].x & 2) == 0;   // group 1 continues the walker of group 0
                if constexpr (POPS) {
                    // mass-dependent efficiency: flagged where 0 <= D <= width (the interval of
                    // delta_R between the two crossings of zeta f_coll = 1); the efficiency-
                    // weighted f_coll at R_cell from the ending walker's table in nu = -D
                    const unsigned char* meta = Ms + st * kMB;
                    const float4* wd4 = reinterpret_cast<const float4*>(meta + kMRecBytes) + g0 * (kGroup / 4);
                    const float* tb = reinterpret_cast<const float*>(meta + kMTabOff) + g0 * kFTab;
                    const float d1 = second ? v[0][0] : v[1][0];
                    const float f0 = (m[0].x >= 0 && (m[0].x & 1)) ? pop_table_f(tb, -v[0][0], __int_as_float(m[0].w)) : 0.0f;
                    const float f1 = (m[1].x >= 0 && (m[1].x & 1)) ? pop_table_f(tb + kFTab, -d1, __int_as_float(m[1].w)) : 0.0f;
                    // a column does not flag iff D < 0 or D > width: the sign bit of D | (width - D)
                    // (width - D = +inf for an infinite width); the columns' values are replaced by
                    // that word and AND-ed as for the step function
                    float w10 = 0.0f;
#pragma unroll
                    for (int q = 0; q < kGroup / 4; q++) {
                        const float4 wa = wd4[q], wb = wd4[kGroup / 4 + q];
                        const float xa[4] = {wa.x, wa.y, wa.z, wa.w}, xb[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const int i = 4 * q + k;
                            if (i == 0) {
                                w10 = xb[0];
                                continue;
                            }
                            v[0][i] = __uint_as_float(__float_as_uint(v[0][i]) | __float_as_uint(xa[k] - v[0][i]));
                            v[1][i] = __uint_as_float(__float_as_uint(v[1][i]) | __float_as_uint(xb[k] - v[1][i]));
                        }
                    }
                    tc::mbar_arrive(barMe + st);   // meta read: its stage may be refilled
                    const uint32_t x10 = __float_as_uint(v[1][0]) | __float_as_uint(w10 - v[1][0]);
                    const uint32_t a0 = and31(v[0]), a1 = and31(v[1]);
                    fa[0] = a0;
                    fa[1] = second ? a0 & a1 & x10 : a1;
                    pf[0] = f0;
                    pf[1] = f1;
                } else {
                    tc::mbar_arrive(barMe + st);   // meta read: its stage may be refilled
                    // flags: AND of sign bits over the walker's radii above R_cell (column 0 of its
                    // first group is R_cell, D = delta_R - delta_c)
                    const uint32_t a0 = and31(v[0]), a1 = and31(v[1]);
                    fa[0] = a0;
                    fa[1] = second ? a0 & a1 & __float_as_uint(v[1][0]) : a1;
                }
                dd[0] = v[0][0];
                dd[1] = second ? v[0][0] : v[1][0];
            }
            float xh[2];
#pragma unroll
            for (int u = 0; u < 2; u++) {   // two independent chains
                const float zeta = __int_as_float(m[u].y), inv = __int_as_float(m[u].w);
                if constexpr (POPS) {
                    xh[u] = 1.0f - fminf(1.0f, pf[u]);
                } else {
                    // f_coll at R_cell (1 where delta_R >= delta_c), no ionization where s^2 <= 0
                    const float f = dd[u] >= 0.0f ? 1.0f : erfc_cheb(-dd[u] * inv);
                    xh[u] = inv > 0.0f ? 1.0f - fminf(1.0f, zeta * f) : 1.0f;
                }
                xh[u] = (fa[u] >> 31) == 0u ? 0.0f : xh[u];   // flagged at a larger radius (Eq. 1)
            }
#pragma unroll
            for (int u = 0; u < 2; u++) {
                if (m[u].x < 0 || !(m[u].x & 1)) continue;   // no walker ends in this group (uniform)
                const size_t pair = (size_t)(m[u].x >> 2) * a.n_z + zi;
                a.dtb[pair * a.n3 + cell] = __int_as_float(m[u].z) * xh[u] * (1.0f + dens);
                if (a.xhi_out) a.xhi_out[pair * a.n3 + cell] = xh[u];
                const int xq = __reduce_add_sync(0xffffffffu, __float2int_rn(xh[u] * kXScale));   // exact
                if (lane == 0) atomicAdd(a.xq + pair, (unsigned long long)xq);
            }
            tc::fence_before_sync();
            tc::mbar_arrive(barE + tb);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (nch > 0 && *abort) {
        if (t == 0) {   // drain every MMA issued so far
            tc::mma_commit(barF);
            tc::mbar_wait(barF, 0, kTries);
        } else if (t == 32) {   // wait for every bulk copy that may still land
            if (owedA >= 0) tc::mbar_wait(barA, (uint32_t)owedA, kTries);
            for (int s = 0; s < kTcStages; s++) {
                if (owedB[s] >= 0) tc::mbar_wait(barB + s, (uint32_t)owedB[s], kTries);
                if (owedM[s] >= 0) tc::mbar_wait(barM + s, (uint32_t)owedM[s], kTries);
            }
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) {
        __syncwarp();
        tc::tmem_dealloc(tmem, kTmemCols);
    }
}

// Fixed-point x_HI totals -> the per-pair FP64 sums the power-spectrum stage reads.
__global__ void k_xq_finish(const unsigned long long* xq, int pairs, double* xhi_sum) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < pairs) xhi_sum[i] = (double)xq[i] / (double)kXScale;
}

// Columns of the walkers, in walker order, each walker starting on a group of kGroup columns
// (on an even group when it needs two, so that no walker spans the two halves of a chunk):
// its R_cell radius first, then its radii from R_mfp down, then padding (-1) to the end of
// its last group. cols[] holds walker << 8 | radius index; gmeta[] per group walker << 2 |
// first << 1 | last, or -1 for a group left empty; *ncols the number of columns including
// padding. Thread 0 places the walkers, then the block fills the columns.
__global__ void k_build_columns(const WalkerInfo* walkers, int n_walkers, int* goff, int* cols, int* gmeta,
                                int* ncols) {
    static_assert(kMaxRadii <= 2 * kGroup, "a walker spans at most two groups");
    if (threadIdx.x == 0) {
        int g = 0;
        for (int w = 0; w < n_walkers; w++) {
            const int ng = (walkers[w].n_r + kGroup - 1) / kGroup;
            if (ng == 2 && (g & 1)) g++;
            goff[w] = g;
            g += ng;
        }
        goff[n_walkers] = g;
        *ncols = g * kGroup;
    }
    __syncthreads();
    const int total = goff[n_walkers];
    for (int i = threadIdx.x; i < total * kGroup; i += blockDim.x) cols[i] = -1;
    for (int i = threadIdx.x; i < total; i += blockDim.x) gmeta[i] = -1;
    __syncthreads();
    for (int w = threadIdx.x / 32; w < n_walkers; w += blockDim.x / 32) {
        const int nr = walkers[w].n_r, g0 = goff[w], ng = (nr + kGroup - 1) / kGroup;
        for (int i = threadIdx.x % 32; i < ng * kGroup; i += 32) {
            const int j = i == 0 ? nr - 1 : (i < nr ? i - 1 : -1);
            cols[(size_t)g0 * kGroup + i] = j >= 0 ? (w << 8) | j : -1;
        }
        for (int i = threadIdx.x % 32; i < ng; i += 32)
            gmeta[g0 + i] = (w << 2) | (i == 0 ? 2 : 0) | (i == ng - 1 ? 1 : 0);
    }
}

// Column slots: every walker's radii rounded up to whole groups (plus the group an aligned
// two-group walker may skip), then to whole chunks.
int tc_slots(const eor_ctx* c) {
    const int groups = (c->max_radii + kGroup - 1) / kGroup;
    const int per_walker = (groups > 1 ? groups + 1 : groups) * kGroup;
    return (c->cfg.max_walkers * per_walker + kTcN - 1) / kTcN * kTcN;
}

}  // namespace

bool basis_tc_fits(int rank) { return rank + 1 <= tc::kKMax; }   // basis values plus the constant column

size_t basis_tc_smem(bool pops) {
    return kABytes + kTcStages * (kBBytes + (pops ? kMBytes : kMRecBytes)) +
           (4 * kTcStages + 2 * kTmemBufs + 2) * sizeof(uint64_t) + 16;
}
size_t basis_tc_a_bytes(long long n3, int n_z) { return (size_t)n_z * (size_t)(n3 / kTcCells) * kABytes; }
size_t basis_tc_b_bytes(const eor_ctx* c) { return (size_t)c->cfg.n_z * (size_t)(tc_slots(c) / kTcN) * kChunkBytes; }
size_t basis_tc_column_slots(const eor_ctx* c) { return (size_t)tc_slots(c); }

cudaError_t prepare_basis_tc(eor_ctx* c) {
    (void)c;
    cudaError_t e =
        cudaFuncSetAttribute(k_basis_ionize_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)basis_tc_smem(false));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_basis_ionize_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)basis_tc_smem(true));
    return e;
}

cudaError_t format_basis_tc(eor_ctx* c) {
    trace_begin(c, kKOther);
    k_format_a<<<2048, 256, 0, c->stream>>>(c->d_F, c->kb, c->basis_rank, (long long)c->n3, c->cfg.n_z, c->d_tcA);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t build_columns(eor_ctx* c, int n_walkers) {
    trace_begin(c, kKTables);
    k_build_columns<<<1, 256, 0, c->stream>>>(c->d_walkers, n_walkers, c->d_goff, c->d_cols, c->d_gmeta, c->d_ncols);
    trace_end(c);
    const int chunks = tc_slots(c) / kTcN;
    trace_begin(c, kKTables);
    k_format_b<<<dim3(chunks, c->cfg.n_z), kTcN, 0, c->stream>>>(c->d_cols, c->d_gmeta, c->d_ncols, c->d_coef,
                                                               c->d_pairs, c->kb, c->basis_rank, c->max_radii, c->cfg.n_z,
                                                               chunks,
                                                               (float)c->cfg.delta_c, pop_tables(c), c->d_tcB);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t launch_basis_ionize_tc(eor_ctx* c, float* xhi_out) {
    const int pairs = c->n_walkers * c->cfg.n_z;
    cudaError_t e = cudaMemsetAsync(c->d_xq, 0, sizeof(unsigned long long) * pairs, c->stream);
    if (e != cudaSuccess) return e;
    TcArgs a{c->d_tcA, c->d_tcB, c->d_ncols, brightness_base(c), c->d_dtb, xhi_out, c->d_xq, pop_tables(c), c->d_err,
             c->cfg.n_z, tc_slots(c) / kTcN, (c->basis_rank + 1 + 7) / 8, (long long)c->n3};
    trace_begin(c, kKBasis);
    const dim3 grid((unsigned)(c->n3 / kTcCells), c->cfg.n_z);
    if (a.ftab)
        k_basis_ionize_tc<true><<<grid, kTcThreads, basis_tc_smem(true), c->stream>>>(a);
    else
        k_basis_ionize_tc<false><<<grid, kTcThreads, basis_tc_smem(false), c->stream>>>(a);
    trace_end(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    trace_begin(c, kKFinish);
    k_xq_finish<<<(pairs + 255) / 256, 256, 0, c->stream>>>(c->d_xq, pairs, c->d_xhi_sum);
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
