// noalloc.cu — eor_box_power_spectrum_noalloc: the power spectrum of one box without any
// device allocation.
//
// Some callers cannot allocate GPU memory where they need this result: applications that
// hand all device memory to their own pool or budget (a cudaMalloc outside it fails or
// breaks their accounting), and code that must not synchronize the device (cudaMalloc and
// cudaFree can). This entry point creates no context and calls no cudaMalloc, cudaFree or
// allocating library routine. Its scratch (the half spectrum of the box, the bin of every
// |m|^2, the shell sums and mode counts) is one file-scope device array of kNoAllocBytes
// that every GPU which loads the library holds until the process exits. Every call shares
// that array and overwrites it: calls that overlap on the GPU race, so issue them on one
// stream (or otherwise serialize them).
#include <math.h>

#include <mutex>

#include "eor_internal.cuh"

namespace eor {
namespace {

constexpr int kNoAllocMaxN = EOR21_NOALLOC_MAX_N;
constexpr int kMaxM2 = 3 * (kNoAllocMaxN / 2) * (kNoAllocMaxN / 2) + 1;
constexpr size_t kSpecBytes = (size_t)(kNoAllocMaxN / 2 + 1) * kNoAllocMaxN * kNoAllocMaxN * sizeof(float2);
constexpr size_t kBinsOff = kSpecBytes;                                   // signed char [kMaxM2]
constexpr size_t kSumsOff = (kBinsOff + kMaxM2 + 255) / 256 * 256;        // double [EOR21_MAX_BINS]
constexpr size_t kCountsOff = kSumsOff + EOR21_MAX_BINS * sizeof(double); // unsigned long long [EOR21_MAX_BINS]
constexpr size_t kPairOff = kCountsOff + EOR21_MAX_BINS * sizeof(unsigned long long);   // one PairInfo
constexpr size_t kNoAllocBytes = (kPairOff + sizeof(PairInfo) + 255) / 256 * 256;
static_assert(kNoAllocBytes <= EOR21_NOALLOC_SCRATCH_BYTES, "scratch size stated in eor21.h");

static __device__ __align__(256) unsigned char g_noalloc_scratch[EOR21_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
constexpr int kSizes = 4;                                  // n = 16, 32, 64, 128
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
bool g_prepared[kMaxDevices][kSizes] = {};

// Bin of every |m|^2 (FP64 decision, -1 outside [k_lo, k_hi) or k = 0).
__global__ void k_noalloc_bins(int n_m2, double kf, double k_lo, double k_hi, int n_bins, signed char* bin) {
    const int m2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (m2 >= n_m2) return;
    int b = -1;
    if (m2 > 0) {
        const double k = kf * sqrt((double)m2);
        if (k >= k_lo && k < k_hi) {
            b = (int)floor(n_bins * log(k / k_lo) / log(k_hi / k_lo));
            if (b < 0 || b >= n_bins) b = -1;
        }
    }
    bin[m2] = (signed char)b;
}

// Modes per bin over the full n^3 grid.
__global__ void k_noalloc_counts(int n, const signed char* bin, int n_bins, unsigned long long* cnt) {
    __shared__ unsigned long long s_cnt[EOR21_MAX_BINS];
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) s_cnt[b] = 0ull;
    __syncthreads();
    const long long n3 = (long long)n * n * n;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n3;
         idx += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(idx / ((long long)n * n)), iy = (int)((idx / n) % n), iz = (int)(idx % n);
        const int mx = ix < n / 2 ? ix : ix - n, my = iy < n / 2 ? iy : iy - n, mz = iz < n / 2 ? iz : iz - n;
        const int b = bin[mx * mx + my * my + mz * mz];
        if (b >= 0) atomicAdd(&s_cnt[b], 1ull);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < n_bins; b += blockDim.x) atomicAdd(&cnt[b], s_cnt[b]);
}

__global__ void k_noalloc_finish(const double* sums, const unsigned long long* cnt, int n_bins, double scale,
                                 double* d2, long long* nmodes) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_bins) return;
    const unsigned long long k = cnt[b];
    d2[b] = k > 0 ? sums[b] * scale / (double)k : nan("");
    if (nmodes) nmodes[b] = (long long)k;
}

// Device address of the scratch array on the current device (looked up once per device) and
// the shared-memory limits of the two FFT kernels at grid size n (set once per device and n).
cudaError_t scratch_for_current_device(int n, unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    const int si = n == 16 ? 0 : n == 32 ? 1 : n == 64 ? 2 : 3;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    }
    if (!g_prepared[dev][si]) {
        e = prepare_box_ps_raw(n);
        if (e != cudaSuccess) return e;
        g_prepared[dev][si] = true;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace eor

extern "C" int eor_box_power_spectrum_noalloc(int n, double box_mpc, int n_bins, double k_lo, double k_hi,
                                              const float* box, double* d2, long long* nmodes, void* cuda_stream) {
    using namespace eor;
    if (!(n == 16 || n == 32 || n == 64 || n == 128) || n > kNoAllocMaxN) {
        set_global_error("eor_box_power_spectrum_noalloc: n must be 16, 32, 64 or 128");
        return EOR_EINVAL;
    }
    if (!(box_mpc > 0.0) || !isfinite(box_mpc) || n_bins < 1 || n_bins > EOR21_MAX_BINS || !(k_lo > 0.0) ||
        !(k_hi > k_lo) || !box || !d2) {
        set_global_error("eor_box_power_spectrum_noalloc: bad size, range or NULL pointer");
        return EOR_EINVAL;
    }
    unsigned char* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(n, &scratch);
    if (e != cudaSuccess) {
        set_global_error(std::string("eor_box_power_spectrum_noalloc set-up: ") + cudaGetErrorString(e));
        return EOR_ECUDA;
    }
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    float2* spec = reinterpret_cast<float2*>(scratch);
    signed char* bins = reinterpret_cast<signed char*>(scratch + kBinsOff);
    double* sums = reinterpret_cast<double*>(scratch + kSumsOff);
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(scratch + kCountsOff);
    PairInfo* pair = reinterpret_cast<PairInfo*>(scratch + kPairOff);
    const int n_m2 = 3 * (n / 2) * (n / 2) + 1;
    const double kf = 2.0 * kPi / box_mpc;
    // the previous call's contents stay in the array: clear what is accumulated
    e = cudaMemsetAsync(scratch + kSumsOff, 0, kPairOff + sizeof(PairInfo) - kSumsOff, stream);
    if (e == cudaSuccess) {
        k_noalloc_bins<<<(n_m2 + 255) / 256, 256, 0, stream>>>(n_m2, kf, k_lo, k_hi, n_bins, bins);
        k_noalloc_counts<<<64, 256, 0, stream>>>(n, bins, n_bins, cnt);
        const float kff = (float)kf;
        e = launch_box_ps_raw(n, box, spec, bins, sums, n_bins, kff * kff * kff, pair, stream);
    }
    if (e == cudaSuccess) {
        const double dx = box_mpc / n, vol = box_mpc * box_mpc * box_mpc;
        const double scale = dx * dx * dx * dx * dx * dx / (2.0 * kPi * kPi * vol);
        k_noalloc_finish<<<1, 64, 0, stream>>>(sums, cnt, n_bins, scale, d2, nmodes);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        set_global_error(std::string("eor_box_power_spectrum_noalloc: ") + cudaGetErrorString(e));
        return EOR_ECUDA;
    }
    return EOR_OK;
}
