// fft_core.cuh — FP32 complex FFT building blocks held in registers and exchanged
// through shared memory (sm_103a). Used by the plane and pencil kernels of the
// excursion-set path; nothing here is specific to one grid size.
//
// A length-N transform is split N = R1 * R2. A team of R2 threads owns one line:
// thread i first holds x[j*R2 + i] (j < R1), runs an R1-point DFT in registers,
// multiplies by w_N^(i*k1), and writes to shared memory; after a barrier each
// thread runs R1/R2 DFTs of length R2 over i, producing X[k1 + R1*k2].
//
// Sign convention: DIR = -1 is exp(-2 pi i jk/N) (forward), DIR = +1 inverse.
// Transforms are unnormalised.
#pragma once
#include <cuda_runtime.h>

namespace eor {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// cos and sin of 2 pi m / 16, m = 0..15 (exact values of the unit circle's 16th roots).
__device__ __forceinline__ constexpr float c16(int m) {
    constexpr float t[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                             0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
    return t[m & 15];
}
__device__ __forceinline__ constexpr float s16(int m) { return c16(m - 4); }

// v * w_16^(DIR*m) with the trivial roots (multiples of pi/2, pi/4) done without multiplies.
template <int M, int DIR>
__device__ __forceinline__ float2 rot16(float2 v) {
    constexpr int m = ((M % 16) + 16) % 16;
    if constexpr (m == 0) {
        return v;
    } else if constexpr (m == 4) {          // w = DIR * i
        return DIR > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
    } else if constexpr (m == 8) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (m == 12) {         // w = -DIR * i
        return DIR > 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
    } else {
        constexpr float c = c16(m), s = DIR * s16(m);
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

template <int R>
__host__ __device__ constexpr int bitrev(int i) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) { r = (r << 1) | (i & 1); i >>= 1; }
    return r;
}

// In-register R-point DFT (R = 2, 4, 8 or 16), natural order in and out.
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "radix");
    if constexpr (R == 1) return;
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; i++) t[i] = v[bitrev<R>(i)];
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
        for (int base = 0; base < R; base += len) {
#pragma unroll
            for (int k = 0; k < len / 2; k++) {
                float2 a = t[base + k];
                float2 b = t[base + k + len / 2];
                // twiddle w_len^(DIR*k) = w_16^(DIR*k*16/len)
                switch (k * (16 / len)) {
                    case 0: break;
                    case 1: b = rot16<1, DIR>(b); break;
                    case 2: b = rot16<2, DIR>(b); break;
                    case 3: b = rot16<3, DIR>(b); break;
                    case 4: b = rot16<4, DIR>(b); break;
                    case 5: b = rot16<5, DIR>(b); break;
                    case 6: b = rot16<6, DIR>(b); break;
                    case 7: b = rot16<7, DIR>(b); break;
                }
                t[base + k] = cadd(a, b);
                t[base + k + len / 2] = csub(a, b);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < R; i++) v[i] = t[i];
}

// Radix split of each supported length: N = R1 * R2 with R1 >= R2.
template <int N> struct Split;
template <> struct Split<4>   { static constexpr int R1 = 2,  R2 = 2; };
template <> struct Split<8>   { static constexpr int R1 = 4,  R2 = 2; };
template <> struct Split<16>  { static constexpr int R1 = 4,  R2 = 4; };
template <> struct Split<32>  { static constexpr int R1 = 8,  R2 = 4; };
template <> struct Split<64>  { static constexpr int R1 = 8,  R2 = 8; };
template <> struct Split<128> { static constexpr int R1 = 16, R2 = 8; };

// Table of w_N^m = (cos 2 pi m/N, sin 2 pi m/N), m < N, filled by the whole block.
template <int N>
__device__ __forceinline__ void fill_twiddles(float2* tw) {
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        float s, c;
        sincospif(2.0f * (float)m / (float)N, &s, &c);
        tw[m] = make_float2(c, s);
    }
}

// w_N^(DIR * e) from the table (e taken modulo N).
template <int N, int DIR>
__device__ __forceinline__ float2 tw_get(const float2* tw, int e) {
    float2 w = tw[e & (N - 1)];
    return DIR > 0 ? w : make_float2(w.x, -w.y);
}

}  // namespace eor
