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

// Multiply by DIR * i.
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 v) {
    return DIR > 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
}

// Straight-line DFT codelets (natural order in and out). Written out statement by
// statement so that every value stays in a register.
template <int DIR>
__device__ __forceinline__ void dft2(float2& a0, float2& a1) {
    const float2 t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3), t3 = mul_i<DIR>(csub(a1, a3));
    a0 = cadd(t0, t2);
    a2 = csub(t0, t2);
    a1 = cadd(t1, t3);
    a3 = csub(t1, t3);
}

// 8 points: two 4-point DFTs on the even and odd samples, then twiddles w8^k and butterflies.
template <int DIR>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
    dft4<DIR>(v[0], v[2], v[4], v[6]);
    dft4<DIR>(v[1], v[3], v[5], v[7]);
    const float2 o0 = v[1], o1 = rot16<2, DIR>(v[3]), o2 = rot16<4, DIR>(v[5]), o3 = rot16<6, DIR>(v[7]);
    const float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// 16 points as 4 x 4: DFT over n1 of x[n2 + 4 n1], twiddle w16^(n2 k1), DFT over n2;
// X[k1 + 4 k2] ends in v[4 k1 + k2] and is renamed into natural order.
template <int DIR>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
    dft4<DIR>(v[0], v[4], v[8], v[12]);
    dft4<DIR>(v[1], v[5], v[9], v[13]);
    dft4<DIR>(v[2], v[6], v[10], v[14]);
    dft4<DIR>(v[3], v[7], v[11], v[15]);
    v[5] = rot16<1, DIR>(v[5]);  v[6] = rot16<2, DIR>(v[6]);  v[7] = rot16<3, DIR>(v[7]);
    v[9] = rot16<2, DIR>(v[9]);  v[10] = rot16<4, DIR>(v[10]); v[11] = rot16<6, DIR>(v[11]);
    v[13] = rot16<3, DIR>(v[13]); v[14] = rot16<6, DIR>(v[14]); v[15] = rot16<9, DIR>(v[15]);
    dft4<DIR>(v[0], v[1], v[2], v[3]);
    dft4<DIR>(v[4], v[5], v[6], v[7]);
    dft4<DIR>(v[8], v[9], v[10], v[11]);
    dft4<DIR>(v[12], v[13], v[14], v[15]);
    const float2 t1 = v[1], t2 = v[2], t3 = v[3], t6 = v[6], t7 = v[7], t11 = v[11];
    v[1] = v[4]; v[2] = v[8]; v[3] = v[12];
    v[4] = t1; v[6] = v[9]; v[7] = v[13];
    v[8] = t2; v[9] = t6; v[11] = v[14];
    v[12] = t3; v[13] = t7; v[14] = t11;
}

// In-register R-point DFT (R = 1, 2, 4, 8 or 16), natural order in and out.
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
    static_assert(R == 1 || R == 2 || R == 4 || R == 8 || R == 16, "radix");
    if constexpr (R == 2) dft2<DIR>(v[0], v[1]);
    else if constexpr (R == 4) dft4<DIR>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 8) dft8<DIR>(v);
    else if constexpr (R == 16) dft16<DIR>(v);
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
