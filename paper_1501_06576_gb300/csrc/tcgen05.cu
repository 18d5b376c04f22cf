// tcgen05.cu — tensor-core (tcgen05, TMEM) kernels of libeor21.
//
// k_tc_check: one CTA computes D = A B^T (A 128 x 32, B n x 32, FP32 in global memory) with
// TF32 tcgen05 MMAs accumulating in tensor memory: the operand layout, descriptors and
// tensor-memory reads of the tensor-core contraction, checked in isolation.
#include <cuda_fp16.h>

#include "eor_internal.cuh"
#include "tc.cuh"

namespace eor {
namespace {

constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s of GPU time per bounded wait

// A bounded wait ran out: set kErrTimeout and keep the first record of where,
// err[1] = role << 28 | barrier << 20 | chunk (roles 1 copy, 2 MMA, 3 epilogue; barriers
// 1 A, 2 B full, 3 B empty, 4 meta full, 5 meta empty, 6 accumulator full, 7 accumulator free).
// The fence orders the record before the abort flag that the caller raises next, so a thread
// that gives up only because it saw that flag cannot overwrite the first record.
__device__ __forceinline__ void record_timeout(int* err, int role, int bar, int chunk) {
    atomicOr(err, kErrTimeout);
    atomicCAS(err + 1, 0, (role << 28) | (bar << 20) | (chunk & 0xFFFFF));
    __threadfence();
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
    // test-only failure injection (off: withhold = -1): the epilogue withholds its release of
    // the accumulator buffer of chunk `withhold`, and the MMA thread's wait for that release
    // gives up after free_wait_ns (every other wait keeps kWaitNs)
    int withhold;
    uint64_t free_wait_ns;
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
                ok = tc::mbar_wait_or_abort(barE + tb, (uint32_t)((c - kTmemBufs) / kTmemBufs) & 1u,
                                            a.free_wait_ns, abort);
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
            if (c != a.withhold) tc::mbar_arrive(barE + tb);
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
// padding. Thread 0 places the walkers (from their group counts, gathered by the block into
// shared memory 256 at a time: one dependent global load per walker made the serial loop
// take tens of microseconds), then the block fills the columns.
__global__ void k_build_columns(const WalkerInfo* walkers, int n_walkers, int* goff, int* cols, int* gmeta,
                                int* ncols, int rcell_first) {
    static_assert(kMaxRadii <= 2 * kGroup, "a walker spans at most two groups");
    constexpr int kChunk = 256;
    __shared__ unsigned char s_ng[kChunk];
    // columns of a walker: all its radii (R_cell first) or only those above R_cell (at least
    // one group, which carries the walker's x_HI even when it has no radius above R_cell)
    auto width = [&](int nr) { return rcell_first ? nr : nr - 1; };
    auto groups = [&](int nr) { const int ng = (width(nr) + kGroup - 1) / kGroup; return ng > 0 ? ng : 1; };
    int g = 0;   // thread 0's running group count
    for (int w0 = 0; w0 < n_walkers; w0 += kChunk) {
        for (int i = threadIdx.x; i < kChunk && w0 + i < n_walkers; i += blockDim.x)
            s_ng[i] = (unsigned char)groups(walkers[w0 + i].n_r);
        __syncthreads();
        if (threadIdx.x == 0)
            for (int i = 0; i < kChunk && w0 + i < n_walkers; i++) {
                const int ng = s_ng[i];
                if (ng == 2 && (g & 1)) g++;
                goff[w0 + i] = g;
                g += ng;
            }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        goff[n_walkers] = g;
        *ncols = g * kGroup;
    }
    __syncthreads();
    const int total = goff[n_walkers];
    for (int i = threadIdx.x; i < total * kGroup; i += blockDim.x) cols[i] = -1;
    for (int i = threadIdx.x; i < total; i += blockDim.x) gmeta[i] = -1;
    __syncthreads();
    for (int w = threadIdx.x / 32; w < n_walkers; w += blockDim.x / 32) {
        const int nr = walkers[w].n_r, g0 = goff[w], ng = groups(nr);
        for (int i = threadIdx.x % 32; i < ng * kGroup; i += 32) {
            const int j = rcell_first ? (i == 0 ? nr - 1 : (i < nr ? i - 1 : -1)) : (i < nr - 1 ? i : -1);
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
    k_build_columns<<<1, 256, 0, c->stream>>>(c->d_walkers, n_walkers, c->d_goff, c->d_cols, c->d_gmeta, c->d_ncols, 1);
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
             c->cfg.n_z, tc_slots(c) / kTcN, (c->basis_rank + 1 + 7) / 8, (long long)c->n3,
             c->dbg_withhold, c->dbg_withhold >= 0 ? c->dbg_wait_ns : kWaitNs};
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

// ------------------------------------------------------------------ FP16 split contraction

namespace {

//
// The step-function efficiency's contraction as a persistent kernel on FP16 tensor-core
// operands. Each basis field is scaled by a power of two so that |F_b| 2^14 / sigma_b <= 2^14
// (sigma_b >= max |F_b| over the box), each coefficient column by a power of two t so that
// its largest entry lies in [2^13, 2^14); both sides are split x = hi + lo into two FP16
// values (hi = x rounded to FP16, lo = the remainder rounded to FP16: 22 significant bits,
// the same as the TF32 hi/lo split) and the three products hi*hi + hi*lo + lo*hi are laid
// side by side along K, so that one K = 3 (rank + 1) contraction (padded to a multiple of 16)
// gives D = t (delta_R - delta_crit(R)) with FP32 accumulation. t > 0 keeps the sign: the
// Eq. 1 flag is again "sign bit of D clear at some radius". The R_cell radius is not a
// column: delta at R_cell is the same field for every walker (delta_Rcell, one filtered
// density per box), read per cell for the partial ionization.
constexpr int kFM = 128;                        // cells per tile (MMA M)
constexpr int kFN = 256;                        // coefficient columns per chunk (MMA N)
constexpr int kFKMax = 96;                      // FP16 K slots at most (six MMA steps of 16)
constexpr int kFStagesMax = 3;                  // coefficient chunks in flight (3, or 2 when 3 do not fit)
constexpr int kFGT = 4;                         // cell tiles per group: a coefficient chunk serves kFGT tiles
constexpr int kFMetaStages = 8;                 // group records (and widths) of chunks in flight
constexpr int kFGroups = kFN / kGroup;          // walker groups per chunk
constexpr uint32_t kFRecBytes = kFGroups * 16;  // group records
constexpr uint32_t kFWidthBytes = kFN * 4;      // per column t (delta_hi - delta_crit) (mass-dependent efficiency)
constexpr uint32_t f16_meta_bytes(bool pops) { return kFRecBytes + (pops ? kFWidthBytes : 0u); }
constexpr int kFEpiWarps = 16;                  // four per tensor-memory lane quarter
#ifndef EOR_F16_EPI_SETS
#define EOR_F16_EPI_SETS 2
#endif
constexpr int kFEpiSets = EOR_F16_EPI_SETS;     // epilogue warp sets, alternating units (1 or 2)
constexpr int kFSetWarps = kFEpiWarps / kFEpiSets;   // warps of one set: one arrival each on the set's barriers
constexpr int kFRounds = kFEpiSets;             // 64-column rounds of an epilogue warp per unit
constexpr int kFThreads = 128 + 32 * kFEpiWarps;
constexpr uint32_t kFTmemCols = 2 * kFN;        // two accumulator buffers
constexpr float kFScale = 16384.0f;             // 2^14
static_assert(kFTmemCols <= 512, "tensor memory");
static_assert(kFN == 8 * kGroup && kFEpiWarps == 16 && (kFEpiSets == 1 || kFEpiSets == 2),
              "epilogue: a set's warp (q, p) reads 64 kFRounds columns of lane quarter q, 64 per round");

__host__ __device__ constexpr int f16_kslots(int rank) { return (3 * (rank + 1) + 15) / 16 * 16; }
__host__ __device__ constexpr uint32_t f16_sbo(int k) { return (uint32_t)(k / 8) * 128u; }

// sigma_b: the smallest power of two >= max |F_b| over the cells of box z (1 for a zero
// field), as the bits of a positive float in fmax_bits[z][b] (atomicMax on the bits orders
// positive floats).
__global__ void k_field_absmax(const float* F, int kb, int rank, long long n3, unsigned int* fmax_bits) {
    const int b = blockIdx.y, zi = blockIdx.z;
    if (b >= rank) return;
    const float* f = F + ((size_t)zi * kb + b) * n3;
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(f[i]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(fmax_bits + zi * 32 + b, __float_as_uint(m));
}

__global__ void k_field_scale(const unsigned int* fmax_bits, int n_z, float* fscale) {
    const int i = threadIdx.x;
    if (i >= n_z * 32) return;
    const float m = __uint_as_float(fmax_bits[i]);
    fscale[i] = m > 0.0f ? exp2f(ceilf(log2f(m))) : 1.0f;
    if (fscale[i] < m) fscale[i] *= 2.0f;   // guard the rounding of log2f
}

// FP16 hi/lo split of a value whose magnitude is at most 2^14.
__device__ __forceinline__ void split_f16(float x, __half& hi, __half& lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// A operands: [z][tile of 128 cells][128 x K FP16, core-matrix layout]. Row = cell, K slots:
// segment 0 hi(a), segment 1 hi(a), segment 2 lo(a) with a_b = F_b 2^14 / sigma_b (b < rank)
// and a_rank = 2^14 (the constant that carries the threshold), each segment rank + 1 long,
// zero after 3 (rank + 1). One thread writes one 16-byte core row (8 K slots).
__global__ void k_format_a16(const float* F, int kb, int rank, long long n3, int n_z, const float* fscale, int kslots,
                             unsigned char* out) {
    const int ls = rank + 1, kc = kslots / 8;
    const uint32_t sbo = f16_sbo(kslots);
    const size_t tile_bytes = (size_t)kFM * kslots * 2;
    const long long total = (long long)n_z * n3 * kc;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(e % kc);
        const long long cell = (e / kc) % n3;
        const int zi = (int)(e / ((long long)kc * n3));
        __align__(16) __half v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = q * 8 + i, seg = k / ls, b = k % ls;
            float a = 0.0f;
            if (seg < 3) a = b < rank ? F[((size_t)zi * kb + b) * n3 + cell] * (kFScale / fscale[zi * 32 + b])
                                      : (b == rank ? kFScale : 0.0f);
            __half hi, lo;
            split_f16(a, hi, lo);
            v[i] = seg == 2 ? lo : (seg < 3 ? hi : __float2half_rn(0.0f));
        }
        const long long tile = cell / kFM;
        const int row = (int)(cell % kFM);
        unsigned char* dst = out + ((size_t)zi * (n3 / kFM) + tile) * tile_bytes + tc::core_offset16(row, q * 8, sbo);
        *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(v);
    }
}

// Coefficient chunks: [z][chunk of 256 columns][256 x K FP16 | kFGroups group records of 16 B].
// Column (walker w, radius j > ... above R_cell) holds b_b = t c_b(R_j) sigma_b / 2^14 (b < rank)
// and b_rank = -t delta_crit(R_j) / 2^14, t a power of two that puts the largest |b| in
// [2^13, 2^14); segments: hi(b), lo(b), hi(b). An infinite delta_crit becomes kNever. Padding
// columns: b = 0 and b_rank = -2^13 (D < 0 everywhere). One block per chunk, one thread per
// column; group records as the TF32 path's (walker << 2 | first << 1 | last, zeta, T0,
// 1/sqrt(2 s^2(R_cell)) or 0).
__global__ void __launch_bounds__(kFN) k_format_b16(const int* cols, const int* gmeta, const int* ncols,
                                                    const float* coef, const PairInfo* pairs, int kb, int rank,
                                                    int max_radii, int n_z, int chunks_per_z, const float* fscale,
                                                    int kslots, int pops, unsigned char* out) {
    const int row = threadIdx.x, zi = blockIdx.y, slot = blockIdx.x * kFN + row;
    const int nc = *ncols, ls = rank + 1;
    const uint32_t sbo = f16_sbo(kslots);
    const size_t bbytes = (size_t)kFN * kslots * 2;
    unsigned char* chunk = out + ((size_t)zi * chunks_per_z + blockIdx.x) * (bbytes + f16_meta_bytes(pops != 0));
    float v[kBasisMax + 1];
    const int cw = slot < nc ? cols[slot] : -1;
    float mx = 0.0f, width = INFINITY;
    if (cw >= 0) {
        const int w = cw >> 8, j = cw & 255;
        const float* src = coef + ((size_t)w * max_radii + j) * kb;
        const PairInfo& pi = pairs[(size_t)w * n_z + zi];
        const float dcrit = pi.delta_crit[j];
        for (int b = 0; b < rank; b++) v[b] = src[b] * (fscale[zi * 32 + b] / kFScale);
        v[rank] = -(isfinite(dcrit) ? dcrit : kNever) / kFScale;
        if (isfinite(dcrit) && isfinite(pi.delta_hi[j])) width = pi.delta_hi[j] - dcrit;
    } else {
        for (int b = 0; b < rank; b++) v[b] = 0.0f;
        v[rank] = -1.0f;
    }
    for (int b = 0; b <= rank; b++) mx = fmaxf(mx, fabsf(v[b]));
    const float t = mx > 0.0f ? exp2f((float)(13 - ilogbf(mx))) : 1.0f;   // mx t in [2^13, 2^14)
    // the flag interval delta_crit <= delta_R <= delta_hi in the units of D = t (delta_R - delta_crit)
    if (pops) reinterpret_cast<float*>(chunk + bbytes + kFRecBytes)[row] = width * t;
    for (int q = 0; q < kslots / 8; q++) {
        __align__(16) __half h[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
            const int k = q * 8 + i, seg = k / ls, b = k % ls;
            __half hi = __float2half_rn(0.0f), lo = __float2half_rn(0.0f);
            if (seg < 3) split_f16(v[b] * t, hi, lo);
            h[i] = seg == 1 ? lo : hi;
        }
        *reinterpret_cast<uint4*>(chunk + tc::core_offset16(row, q * 8, sbo)) = *reinterpret_cast<const uint4*>(h);
    }
    if ((row & (kGroup - 1)) == 0) {
        const int g = row / kGroup, gi = blockIdx.x * kFGroups + g;
        const int info = gi < nc / kGroup ? gmeta[gi] : -1;
        float zeta = 0.0f, t0 = 0.0f, inv = 0.0f;
        if (info >= 0) {
            const PairInfo& pi = pairs[(size_t)(info >> 2) * n_z + zi];
            zeta = pi.zeta;
            t0 = pi.t0;
            inv = pi.cell_ok > 0.5f ? pi.inv_sqrt2s2_cell : 0.0f;
        }
        reinterpret_cast<int4*>(chunk + bbytes)[g] =
            make_int4(info, __float_as_int(zeta), __float_as_int(t0), __float_as_int(inv));
    }
}

// AND of all 32 values (LOP3 tree): its sign bit is clear iff some value has a clear sign bit.
__device__ __forceinline__ uint32_t and32(const float (&v)[32]) {
    uint32_t m[8];
#pragma unroll
    for (int i = 0; i < 8; i++)
        m[i] = __float_as_uint(v[i]) & __float_as_uint(v[i + 8]) & __float_as_uint(v[i + 16]) & __float_as_uint(v[i + 24]);
    return (m[0] & m[1] & m[2]) & (m[3] & m[4] & m[5]) & (m[6] & m[7]);
}

struct F16Args {
    const unsigned char* A;     // [n_z][tiles_per_z][a_bytes]
    const unsigned char* B;     // [n_z][chunks_per_z][b_bytes + meta_bytes]
    const int* ncols;           // [1] number of columns
    uint32_t* flags;            // [pair][n3 / 32] Eq. 1 flags above R_cell, bit = cell % 32
    int* err;
    int n_z, chunks_per_z, tiles_per_z, ksteps;
    uint32_t a_bytes, b_bytes, sbo;
    uint32_t meta_bytes;        // group records (and with POPS the columns' interval widths)
    long long n3;
    int withhold;               // test-only failure injection (see TcArgs), -1 off
    uint64_t free_wait_ns;
};

// Persistent CTA (one per SM): groups of kFGT consecutive 128-cell tiles of one box, grp =
// blockIdx.x, blockIdx.x + gridDim.x, ... (all groups of box 0 first). Work unit u = (group,
// chunk, tile of the group) in that order: a coefficient chunk is copied once per group and
// serves its kFGT tiles, whose A operands stay in kFGT slots for the group (each chunk copy
// costs its copy thread a few hundred cycles whatever its size, and the chunks of all SMs
// share L2 bandwidth, so one chunk per tile fell behind the MMAs). Roles: thread 32 copies
// chunk k's group records into ring slot k % kFMetaStages and its coefficients into stage
// k % S (k counts the CTA's chunks over its groups) once the slot / stage is free, and the
// next group's A operands into slot i as soon as this group's last MMAs on slot i are done
// (tested between and during its other waits, so that no A copy holds up a coefficient
// copy); thread 0 issues the MMAs (per unit ksteps M128 N256 K16 FP16 MMAs into
// tensor-memory buffer u % 2; it waits only for operands and a free buffer); warps 4-19 run
// the epilogue in two sets taking alternate units (set s, buffer s): a set's warp (q = lane
// quarter, p) reads 128 columns of its 32 cells in two rounds of 64, releases the buffer
// after the last read and, for the walkers of the groups it read, stores the Eq. 1 flags of
// its 32 cells as one word each (a walker's flag: the AND of the sign bits of its columns is
// clear). x_HI, delta T_b and the power spectrum follow in the pencil pass. POPS (a
// mass-dependent efficiency): a column flags where 0 <= D <= t (delta_hi - delta_crit), the
// width staged with the group records. Every wait is bounded; on a timeout the CTA records
// where (err[1]: role, barrier, unit or chunk), stops, waits for its MMAs and copies in
// flight and frees its tensor memory.
template <bool POPS, int S>
__global__ void __launch_bounds__(kFThreads, 1) k_basis_ionize_f16(F16Args a) {
    static_assert(S == 2 || S == 3, "coefficient stages");
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* As = sm;                                    // [kFGT][a_bytes]
    unsigned char* Bs = As + kFGT * a.a_bytes;                 // [S][b_bytes]
    unsigned char* Ms = Bs + S * a.b_bytes;                    // [kFMetaStages][meta_bytes]
    uint64_t* bars = reinterpret_cast<uint64_t*>(Ms + kFMetaStages * a.meta_bytes);
    uint64_t* barA = bars;                   // [kFGT] A slot landed
    uint64_t* barAe = barA + kFGT;           // [kFGT] A slot free (the group's last MMAs on it are done)
    uint64_t* barB = barAe + kFGT;           // [S] coefficient stage landed
    uint64_t* barBe = barB + kFStagesMax;    // [S] its MMAs are done
    uint64_t* barM = barBe + kFStagesMax;    // [kFMetaStages] group records landed
    uint64_t* barMe = barM + kFMetaStages;   // [kFMetaStages] the epilogue has read them (kFGT units)
    uint64_t* barD = barMe + kFMetaStages;   // [2] accumulator buffer ready
    uint64_t* barE = barD + 2;               // [2] accumulator buffer released by the epilogue
    uint64_t* barF = barE + 2;               // MMAs drained (abort path)
    uint32_t* tslot = reinterpret_cast<uint32_t*>(barF + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tslot + 1);

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int ncols = *a.ncols;
    const int nch = (ncols + kFN - 1) / kFN;
    const int groups_per_z = a.tiles_per_z / kFGT;
    const int total = a.n_z * groups_per_z;
    const int my_groups = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const bool work = nch > 0 && my_groups > 0;
    auto group_of = [&](int gi) { return (int)blockIdx.x + gi * (int)gridDim.x; };

    if (warp == 0) tc::tmem_alloc(tslot, kFTmemCols);
    if (t == 0) {
        for (int s = 0; s < kFGT; s++) {
            tc::mbar_init(barA + s, 1);
            tc::mbar_init(barAe + s, 1);
        }
        for (int s = 0; s < 2; s++) {
            tc::mbar_init(barD + s, 1);
            tc::mbar_init(barE + s, kFSetWarps);
        }
        for (int s = 0; s < S; s++) {
            tc::mbar_init(barB + s, 1);
            tc::mbar_init(barBe + s, 1);
        }
        for (int s = 0; s < kFMetaStages; s++) {
            tc::mbar_init(barM + s, 1);
            tc::mbar_init(barMe + s, kFGT * kFSetWarps);
        }
        tc::mbar_init(barF, 1);
        *abort = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    // copy-thread bookkeeping (registers): bit 2s of a mask = slot / stage s has a copy that
    // may still land, bit 2s + 1 = the parity of the phase it completes
    uint32_t owedA = 0, owedB = 0, owedM = 0;

    if (t == 32 && work) {
        // ---------------- copy thread (counters, no division in the loop)
        const size_t chunk_bytes = (size_t)a.b_bytes + a.meta_bytes;
        auto copy_a = [&](int gi, int i) {   // A operands of group gi's tile i into slot i
            const size_t tile = (size_t)group_of(gi) * kFGT + i;
            tc::mbar_expect_tx(barA + i, a.a_bytes);
            tc::bulk_g2s(As + (size_t)i * a.a_bytes, a.A + tile * a.a_bytes, a.a_bytes, barA + i);
            owedA = (owedA & ~(3u << (2 * i))) | ((1u | ((uint32_t)gi & 1u) << 1) << (2 * i));
        };
        int na_g = 1, na_i = 0;   // the next A copy: group na_g, slot na_i (after group na_g - 1 freed it)
        auto poll_a = [&]() {
            while (na_g < my_groups && tc::mbar_test(barAe + na_i, (uint32_t)(na_g - 1) & 1u)) {
                copy_a(na_g, na_i);
                if (++na_i == kFGT) {
                    na_i = 0;
                    na_g++;
                }
            }
        };
        // wait for a phase, issuing the A copies that become possible meanwhile; false on a
        // timeout or an abort
        auto wait_poll = [&](uint64_t* bar, uint32_t parity) -> bool {
            if (tc::mbar_test(bar, parity)) return true;
            const long long t0 = clock64(), limit = tc::wait_cycles(kWaitNs);
            while (true) {
                poll_a();
                if (tc::mbar_try(bar, parity)) return true;
                if (*abort) return false;
                if (clock64() - t0 > limit) return false;
            }
        };
        for (int i = 0; i < kFGT; i++) copy_a(0, i);
        bool ok = true;
        int st = 0, ms = 0, k = 0;
        uint32_t use = 0, muse = 0;   // the use-th filling of stage st, the muse-th of ring slot ms
        for (int gi = 0; gi < my_groups && ok; gi++) {
            const unsigned char* Bz = a.B + (size_t)(group_of(gi) / groups_per_z) * a.chunks_per_z * chunk_bytes;
            for (int c = 0; c < nch; c++, k++) {
                if (muse > 0 && !(ok = wait_poll(barMe + ms, (muse - 1) & 1u))) {
                    record_timeout(a.err, 1, 5, k);
                    break;
                }
                tc::mbar_expect_tx(barM + ms, a.meta_bytes);
                tc::bulk_g2s(Ms + (size_t)ms * a.meta_bytes, Bz + (size_t)c * chunk_bytes + a.b_bytes, a.meta_bytes,
                             barM + ms);
                owedM = (owedM & ~(3u << (2 * ms))) | ((1u | (muse & 1u) << 1) << (2 * ms));
                if (++ms == kFMetaStages) {
                    ms = 0;
                    muse++;
                }
                if (use > 0 && !(ok = wait_poll(barBe + st, (use - 1) & 1u))) {
                    record_timeout(a.err, 1, 3, k);
                    break;
                }
                tc::mbar_expect_tx(barB + st, a.b_bytes);
                tc::bulk_g2s(Bs + (size_t)st * a.b_bytes, Bz + (size_t)c * chunk_bytes, a.b_bytes, barB + st);
                owedB = (owedB & ~(3u << (2 * st))) | ((1u | (use & 1u) << 1) << (2 * st));
                if (++st == S) {
                    st = 0;
                    use++;
                }
                poll_a();
            }
        }
        while (ok && na_g < my_groups) {   // A copies still pending
            if (!(ok = wait_poll(barAe + na_i, (uint32_t)(na_g - 1) & 1u))) {
                record_timeout(a.err, 1, 9, na_g);
                break;
            }
            poll_a();
        }
        if (!ok) *abort = 1;
    } else if (t == 0 && work) {
        // ---------------- MMA thread. Its own instructions are kept few (descriptors built once
        // and advanced by constants): it shares its scheduler with four epilogue warps, and
        // while it runs them the tensor pipe's short queue of MMAs drains.
        const uint32_t idesc = tc::idesc_f16(kFM, kFN);
        // descriptors of K step 0 of A slot i and of B stage 0; a K step lies 256 bytes further
        // (16 in the descriptor's address field, which holds address / 16), a stage b_bytes
        uint64_t adesc[kFGT];
#pragma unroll
        for (int i = 0; i < kFGT; i++) adesc[i] = tc::smem_desc(tc::smem_addr(As + (size_t)i * a.a_bytes), tc::kLBO, a.sbo);
        const uint64_t bdesc0 = tc::smem_desc(tc::smem_addr(Bs), tc::kLBO, a.sbo);
        const uint64_t bstep = a.b_bytes >> 4;
        const int ksteps = a.ksteps;
        bool ok = true;
        int st = 0, u = 0;
        uint32_t use = 0;   // phase parity of stage st is use & 1
        uint64_t bdesc = bdesc0;
        for (int gi = 0; gi < my_groups && ok; gi++) {
            for (int c = 0; c < nch && ok; c++) {
                if (!(ok = tc::mbar_wait_or_abort(barB + st, use & 1u, kWaitNs, abort))) {
                    record_timeout(a.err, 2, 2, u);
                    break;
                }
#pragma unroll
                for (int i = 0; i < kFGT; i++, u++) {
                    if (c == 0 && !(ok = tc::mbar_wait_or_abort(barA + i, (uint32_t)gi & 1u, kWaitNs, abort))) {
                        record_timeout(a.err, 2, 1, u);
                        break;
                    }
                    const int tb = u & 1;
                    if (u >= 2 &&   // the epilogue of unit u - 2 has released buffer tb
                        !(ok = tc::mbar_wait_or_abort(barE + tb, (uint32_t)((u - 2) >> 1) & 1u, a.free_wait_ns, abort))) {
                        record_timeout(a.err, 2, 7, u);
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t d = tmem + (uint32_t)(tb * kFN);
                    tc::mma_f16(d, adesc[i], bdesc, idesc, 0u);
                    for (int ks = 1; ks < ksteps; ks++)
                        tc::mma_f16(d, adesc[i] + 16u * (uint32_t)ks, bdesc + 16u * (uint32_t)ks, idesc, 1u);
                    tc::mma_commit(barD + tb);                     // accumulators ready for the epilogue
                    if (c == nch - 1) tc::mma_commit(barAe + i);   // the group's last MMAs on slot i
                }
                if (!ok) break;
                tc::mma_commit(barBe + st);   // coefficient stage free for the copy thread
                if (++st == S) {
                    st = 0;
                    use++;
                    bdesc = bdesc0;
                } else {
                    bdesc += bstep;
                }
            }
        }
        if (!ok) *abort = 1;
    } else if (warp >= 4 && work) {
        // ---------------- epilogue warps: set `set` takes the units u with u % kFEpiSets == set;
        // its warp (q = lane quarter, p) reads columns (64 p kFRounds + 64 r) (r < kFRounds)
        const int e = warp - 4, q = warp & 3, set = e / (kFEpiWarps / kFEpiSets), p = (e % (kFEpiWarps / kFEpiSets)) >> 2;
        const long long words = a.n3 / 32;
        bool ok = true;
        int k = 0;
        for (int gi = 0; gi < my_groups && ok; gi++) {
            const int grp = group_of(gi), zi = grp / groups_per_z;
            for (int c = 0; c < nch && ok; c++, k++) {
                const int ms = k % kFMetaStages;
                for (int i = set; i < kFGT; i += kFEpiSets) {   // u % kFEpiSets == i % kFEpiSets (kFGT even)
                    const int u = kFGT * k + i, tb = u & 1;
                    const long long word = (long long)((grp * kFGT + i) % a.tiles_per_z) * (kFM / 32) + q;
                    const bool okD = tc::mbar_wait_or_abort(barD + tb, (uint32_t)(u >> 1) & 1u, kWaitNs, abort);
                    const bool okM =
                        okD && tc::mbar_wait_or_abort(barM + ms, (uint32_t)(k / kFMetaStages) & 1u, kWaitNs, abort);
                    if (!okM) {
                        if (lane == 0) record_timeout(a.err, 3, okD ? 4 : 6, u);
                        *abort = 1;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const unsigned char* meta = Ms + (size_t)ms * a.meta_bytes;
                    // both rounds' reads first, with only the sign-bit ANDs between them, so that the
                    // buffer is released as early as possible (the MMAs two units on wait for it);
                    // the ballots and stores follow the release
                    static_assert(kFRounds <= 2, "at most two rounds per unit");
                    uint32_t b00 = 0u, b01 = 0u, b10 = 0u, b11 = 0u;   // (round, 32-column group) ANDs
#pragma unroll 1
                    for (int r = 0; r < kFRounds; r++) {
                        const int col = p * 64 * kFRounds + r * 64;   // first column of this round
                        float v0[32], v1[32];
                        tc::tmem_ld32x2(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(tb * kFN + col), v0, v1);
                        if (r == kFRounds - 1) {
                            tc::fence_before_sync();
                            // accumulators read: buffer free (one arrival per warp, not per thread: the
                            // barrier takes 8 updates instead of 256)
                            __syncwarp();
                            if (lane == 0 && u != a.withhold) tc::mbar_arrive(barE + tb);
                        }
                        if constexpr (POPS) {
                            // a column does not flag iff D < 0 or D > width: the sign bit of D | (width - D)
                            // (+inf for an infinite width), then the same AND of sign bits
                            const float4* wd = reinterpret_cast<const float4*>(meta + kFRecBytes) + col / 4;
#pragma unroll
                            for (int kk = 0; kk < 8; kk++) {
                                const float4 wa = wd[kk], wb = wd[8 + kk];
                                const float xa[4] = {wa.x, wa.y, wa.z, wa.w}, xb[4] = {wb.x, wb.y, wb.z, wb.w};
#pragma unroll
                                for (int hh = 0; hh < 4; hh++) {
                                    const int ii = 4 * kk + hh;
                                    v0[ii] = __uint_as_float(__float_as_uint(v0[ii]) | __float_as_uint(xa[hh] - v0[ii]));
                                    v1[ii] = __uint_as_float(__float_as_uint(v1[ii]) | __float_as_uint(xb[hh] - v1[ii]));
                                }
                            }
                        }
                        const uint32_t x0 = and32(v0), x1 = and32(v1);
                        if (r == 0) {
                            b00 = x0;
                            b01 = x1;
                        } else {
                            b10 = x0;
                            b11 = x1;
                        }
                    }
#pragma unroll
                    for (int r = 0; r < kFRounds; r++) {
                        // Eq. 1 flags: AND of the sign bits over the walker's radii above R_cell; the
                        // second group of the pair continues the walker of the first when it is not a
                        // first group (a two-group walker starts on an even group)
                        const int col = p * 64 * kFRounds + r * 64;
                        const int4* gm = reinterpret_cast<const int4*>(meta) + col / kGroup;
                        const int m0 = gm[0].x, m1 = gm[1].x;
                        const uint32_t a0 = r == 0 ? b00 : b10, a1 = r == 0 ? b01 : b11;
                        const uint32_t w0 = __ballot_sync(0xffffffffu, (a0 >> 31) == 0u);
                        const uint32_t w1 = __ballot_sync(0xffffffffu, (((m1 & 2) == 0 ? (a0 & a1) : a1) >> 31) == 0u);
                        if (lane == 0) {
                            if (m0 >= 0 && (m0 & 1)) a.flags[((size_t)(m0 >> 2) * a.n_z + zi) * words + word] = w0;
                            if (m1 >= 0 && (m1 & 1)) a.flags[((size_t)(m1 >> 2) * a.n_z + zi) * words + word] = w1;
                        }
                    }
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(barMe + ms);   // this unit has read the chunk's records (and widths)
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (work && *abort) {
        if (t == 0) {   // drain every MMA issued so far
            tc::mma_commit(barF);
            tc::mbar_wait(barF, 0, kWaitNs);
        } else if (t == 32) {   // wait for every bulk copy that may still land
            for (int s = 0; s < kFGT; s++)
                if ((owedA >> (2 * s)) & 1u) tc::mbar_wait(barA + s, (owedA >> (2 * s + 1)) & 1u, kWaitNs);
            for (int s = 0; s < S; s++)
                if ((owedB >> (2 * s)) & 1u) tc::mbar_wait(barB + s, (owedB >> (2 * s + 1)) & 1u, kWaitNs);
            for (int s = 0; s < kFMetaStages; s++)
                if ((owedM >> (2 * s)) & 1u) tc::mbar_wait(barM + s, (owedM >> (2 * s + 1)) & 1u, kWaitNs);
        }
    }
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) {
        __syncwarp();
        tc::tmem_dealloc(tmem, kFTmemCols);
    }
}

int f16_slots(const eor_ctx* c) {
    const int groups = (c->max_radii + kGroup - 1) / kGroup;
    const int per_walker = (groups > 1 ? groups + 1 : groups) * kGroup;
    return (c->cfg.max_walkers * per_walker + kFN - 1) / kFN * kFN;
}

// Dynamic shared memory of the contraction with `stages` coefficient stages: at least 120 KB,
// so that one CTA holds an SM (and all of its tensor memory) at every basis size.
size_t f16_smem(int kslots, bool pops, int stages) {
    const size_t a = (size_t)kFM * kslots * 2, b = (size_t)kFN * kslots * 2;
    const size_t need = kFGT * a + stages * b + kFMetaStages * (size_t)f16_meta_bytes(pops) +
                        (2 * kFGT + 2 * kFStagesMax + 2 * kFMetaStages + 4 + 1) * sizeof(uint64_t) + 16;
    return need > (120u << 10) ? need : (120u << 10);
}

// Three coefficient stages where they fit in 227 KB, else two.
int f16_stages(int kslots, bool pops) { return f16_smem(kslots, pops, 3) <= (227u << 10) ? 3 : 2; }

}  // namespace

bool basis_f16_fits(int rank) { return rank >= 1 && f16_kslots(rank) <= kFKMax; }
int basis_f16_kslots(int rank) { return f16_kslots(rank); }
size_t basis_f16_a_bytes(long long n3, int n_z, int rank) { return (size_t)n_z * (size_t)n3 * f16_kslots(rank) * 2; }
size_t basis_f16_b_bytes(const eor_ctx* c) {
    return (size_t)c->cfg.n_z * (size_t)(f16_slots(c) / kFN) *
           ((size_t)kFN * c->k16 * 2 + f16_meta_bytes(c->cfg.efficiency_model != 0));
}
size_t basis_f16_column_slots(const eor_ctx* c) { return (size_t)f16_slots(c); }

cudaError_t prepare_basis_f16(eor_ctx* c) {
    if (!c->f16) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    for (int pops = 0; pops < 2 && e == cudaSuccess; pops++) {
        const int st = f16_stages(c->k16, pops != 0);
        const int bytes = (int)f16_smem(c->k16, pops != 0, st);
        auto k = pops ? (st == 3 ? k_basis_ionize_f16<true, 3> : k_basis_ionize_f16<true, 2>)
                      : (st == 3 ? k_basis_ionize_f16<false, 3> : k_basis_ionize_f16<false, 2>);
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    }
    return e;
}

// At eor_init_boxes: the power-of-two bounds of the basis fields, delta at R_cell of every box
// (the filtered density of the per-radius path, one per box) and the A operands.
cudaError_t format_basis_f16(eor_ctx* c) {
    cudaError_t e;
    const int nz = c->cfg.n_z;
    unsigned int* bits = reinterpret_cast<unsigned int*>(c->d_fscale + nz * 32);   // scratch after the scales
    if ((e = cudaMemsetAsync(bits, 0, sizeof(unsigned int) * nz * 32, c->stream)) != cudaSuccess) return e;
    trace_begin(c, kKOther);
    k_field_absmax<<<dim3(256, c->basis_rank, nz), 256, 0, c->stream>>>(c->d_F, c->kb, c->basis_rank, (long long)c->n3,
                                                                         bits);
    trace_end(c);
    trace_begin(c, kKOther);
    k_field_scale<<<1, 256, 0, c->stream>>>(bits, nz, c->d_fscale);
    trace_end(c);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double dx = c->cfg.box_mpc / c->n;
    const double r_cell = c->cfg.r_cell_rule == 1 ? dx : cbrt(3.0 / (4.0 * kPi)) * dx;
    if ((e = launch_window_table(c, r_cell, c->d_diag_wtab)) != cudaSuccess) return e;
    for (int zi = 0; zi < nz; zi++)
        if ((e = launch_filtered_density(c, zi, c->d_dcell + (size_t)zi * c->n3, c->d_diag_wtab)) != cudaSuccess)
            return e;
    trace_begin(c, kKOther);
    k_format_a16<<<4096, 256, 0, c->stream>>>(c->d_F, c->kb, c->basis_rank, (long long)c->n3, nz, c->d_fscale, c->k16,
                                              c->d_a16);
    trace_end(c);
    return cudaGetLastError();
}

cudaError_t build_columns_f16(eor_ctx* c, int n_walkers) {
    trace_begin(c, kKTables);
    k_build_columns<<<1, 256, 0, c->stream>>>(c->d_walkers, n_walkers, c->d_goff, c->d_cols, c->d_gmeta, c->d_ncols, 0);
    trace_end(c);
    const int chunks = f16_slots(c) / kFN;
    trace_begin(c, kKTables);
    k_format_b16<<<dim3(chunks, c->cfg.n_z), kFN, 0, c->stream>>>(c->d_cols, c->d_gmeta, c->d_ncols, c->d_coef,
                                                                 c->d_pairs, c->kb, c->basis_rank, c->max_radii,
                                                                 c->cfg.n_z, chunks, c->d_fscale, c->k16,
                                                                 c->cfg.efficiency_model != 0, c->d_b16);
    trace_end(c);
    return cudaGetLastError();
}

void launch_xq_finish(const unsigned long long* xq, int pairs, double* xhi_sum, cudaStream_t s) {
    k_xq_finish<<<(pairs + 255) / 256, 256, 0, s>>>(xq, pairs, xhi_sum);
}

cudaError_t launch_basis_ionize_f16(eor_ctx* c) {
    const int tiles_per_z = (int)(c->n3 / kFM);
    const int total = tiles_per_z * c->cfg.n_z;
    const bool pops = c->cfg.efficiency_model != 0;
    const int stages = f16_stages(c->k16, pops);
    F16Args a{c->d_a16, c->d_b16, c->d_ncols, c->d_fwords, c->d_err, c->cfg.n_z, f16_slots(c) / kFN, tiles_per_z,
              c->k16 / 16, (uint32_t)(kFM * c->k16 * 2), (uint32_t)(kFN * c->k16 * 2), f16_sbo(c->k16),
              f16_meta_bytes(pops), (long long)c->n3, c->dbg_withhold,
              c->dbg_withhold >= 0 ? c->dbg_wait_ns : kWaitNs};
    const int groups = total / kFGT;   // tiles per box are a multiple of kFGT (n >= 16)
    const int grid = groups < c->num_sms ? groups : c->num_sms;
    trace_begin(c, kKBasis);
    auto k = pops ? (stages == 3 ? k_basis_ionize_f16<true, 3> : k_basis_ionize_f16<true, 2>)
                  : (stages == 3 ? k_basis_ionize_f16<false, 3> : k_basis_ionize_f16<false, 2>);
    k<<<grid, kFThreads, f16_smem(c->k16, pops, stages), c->stream>>>(a);
    trace_end(c);
    return cudaGetLastError();
}

}  // namespace eor
