// fft_regs.cuh -- register-resident DFT building blocks for the OLS kernels.
//
// Sec. 3.4 of the paper computes each segment's FFT inside the convolution
// kernel ("device-callable" FFTs on data held in shared memory and
// registers).  These are the in-register pieces: small DFTs of 2, 4, 8 and 16
// points on a thread's own values, with every internal rotation a
// compile-time constant.  INV selects the sign of the exponent:
//   forward  X[k] = sum_n x[n] exp(-2 pi i n k / r)
//   inverse  x[n] = sum_k X[k] exp(+2 pi i n k / r)   (unnormalised)
//
// The kernels are issue-bound: every FP32, load/store and integer
// instruction competes for one issue slot per scheduler and cycle.  Complex
// additions therefore use the packed two-lane FP32 add of sm_100+
// (__fadd2_rn: one instruction for re and im, each lane rounded exactly like
// a scalar add, so results are bitwise those of scalar code).  Where one
// operand is multiplied by +-i the lanes cross, and two scalar adds are used.
#pragma once

#include <cuda_runtime.h>

namespace ols {

#ifndef OLS_PACKED_ADD
#define OLS_PACKED_ADD 1
#endif
#if OLS_PACKED_ADD
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
#else
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
#endif

// a + r b and a - r b with r = -i (forward) or +i (inverse): lanes cross, scalar adds.
template <bool INV>
__device__ __forceinline__ float2 add_rot(float2 a, float2 b) {
    return INV ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
template <bool INV>
__device__ __forceinline__ float2 sub_rot(float2 a, float2 b) {
    return INV ? make_float2(a.x + b.y, a.y - b.x) : make_float2(a.x - b.y, a.y + b.x);
}

// a * b
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a * w (INV = false) or a * conj(w) (INV = true)
template <bool INV>
__device__ __forceinline__ float2 ctw(float2 a, float2 w) { return INV ? cmulc(a, w) : cmul(a, w); }

// a * (-i) for the forward sign, a * (+i) for the inverse sign
template <bool INV>
__device__ __forceinline__ float2 rot_quarter(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
__device__ __forceinline__ float2 cneg(float2 a) { return make_float2(-a.x, -a.y); }
// a * (wr + i wi) for compile-time constants
__device__ __forceinline__ float2 cmul_const(float2 a, float wr, float wi) {
    return make_float2(fmaf(a.x, wr, -a.y * wi), fmaf(a.x, wi, a.y * wr));
}

// cos / sin of 2 pi e / 16 for e in [0, 16), as exact-as-float constants.
__device__ __forceinline__ constexpr float c16(int e) {
    constexpr float t[16] = {1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.0f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.0f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                             0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
    return t[e & 15];
}
__device__ __forceinline__ constexpr float s16(int e) { return c16((e + 12) & 15); }  // sin(x) = cos(x - pi/2)

// a * exp(-+ 2 pi i E / 16): trivial rotations cost nothing, the rest a
// complex multiply by a compile-time constant.
template <int E, bool INV, class C>
__device__ __forceinline__ C rot16(C a) {
    constexpr int e = E & 15;
    if constexpr (e == 0) {
        return a;
    } else if constexpr (e == 8) {
        return cneg(a);
    } else if constexpr (e == 4) {
        return rot_quarter<INV>(a);
    } else if constexpr (e == 12) {
        return rot_quarter<!INV>(a);
    } else {
        constexpr float wr = c16(e);
        constexpr float wi = INV ? s16(e) : -s16(e);
        return cmul_const(a, wr, wi);
    }
}

template <bool INV, class C>
__device__ __forceinline__ void dft2(C &a0, C &a1) {
    const C t = a0;
    a0 = cadd(t, a1);
    a1 = csub(t, a1);
}

template <bool INV, class C>
__device__ __forceinline__ void dft4(C &a0, C &a1, C &a2, C &a3) {
    const C u0 = cadd(a0, a2), u1 = csub(a0, a2);
    const C v0 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(u0, v0);
    a2 = csub(u0, v0);
    a1 = add_rot<INV>(u1, d);     // u1 + r (a1 - a3)
    a3 = sub_rot<INV>(u1, d);
}

// dft4 of (a0, a1, r a2, a3), r = -i (forward) / +i (inverse): the rotation of
// a2 is folded into the first adds.
template <bool INV, class C>
__device__ __forceinline__ void dft4_r2(C &a0, C &a1, C &a2, C &a3) {
    const C u0 = add_rot<INV>(a0, a2), u1 = sub_rot<INV>(a0, a2);
    const C v0 = cadd(a1, a3), d = csub(a1, a3);
    a0 = cadd(u0, v0);
    a2 = csub(u0, v0);
    a1 = add_rot<INV>(u1, d);
    a3 = sub_rot<INV>(u1, d);
}

// 8-point DFT in place on x[0..7] (natural order in and out): 8 = 4 x 2.
// n = 2 n1 + n2, k = k1 + 4 k2:  DFT-4 over n1, rotate by W8^(n2 k1), DFT-2 over n2.
template <bool INV, class C>
__device__ __forceinline__ void dft8(C *x) {
    dft4<INV>(x[0], x[2], x[4], x[6]);   // n2 = 0 -> A[k1][0] at x[2 k1]
    dft4<INV>(x[1], x[3], x[5], x[7]);   // n2 = 1 -> A[k1][1] at x[2 k1 + 1]
    x[3] = rot16<2, INV>(x[3]);          // W8^1
    x[7] = rot16<6, INV>(x[7]);          // W8^3  (W8^2 = r on x[5] is folded below)
    C y[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        if (k1 == 2) {
            y[k1] = add_rot<INV>(x[4], x[5]);
            y[k1 + 4] = sub_rot<INV>(x[4], x[5]);
        } else {
            y[k1] = cadd(x[2 * k1], x[2 * k1 + 1]);
            y[k1 + 4] = csub(x[2 * k1], x[2 * k1 + 1]);
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = y[k];
}

// 16-point DFT in place on x[0..15] (natural order in and out): 16 = 4 x 4.
// n = 4 n1 + n2, k = k1 + 4 k2:  DFT-4 over n1, rotate by W16^(n2 k1), DFT-4 over n2.
template <bool INV, class C>
__device__ __forceinline__ void dft16(C *x) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    // x[4 k1 + n2] = A[k1][n2]
    x[5] = rot16<1, INV>(x[5]);
    x[6] = rot16<2, INV>(x[6]);
    x[7] = rot16<3, INV>(x[7]);
    x[9] = rot16<2, INV>(x[9]);
    x[11] = rot16<6, INV>(x[11]);
    x[13] = rot16<3, INV>(x[13]);
    x[14] = rot16<6, INV>(x[14]);
    x[15] = rot16<9, INV>(x[15]);
    dft4<INV>(x[0], x[1], x[2], x[3]);
    dft4<INV>(x[4], x[5], x[6], x[7]);
    dft4_r2<INV>(x[8], x[9], x[10], x[11]);    // x[10] carries W16^4 = r
    dft4<INV>(x[12], x[13], x[14], x[15]);
    // x[4 k1 + k2] = X[k1 + 4 k2]; return natural order
    C y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// R-point DFT on each of the 16/R consecutive groups of x[0..15].
template <int R, bool INV, class C>
__device__ __forceinline__ void dft_groups(C *x) {
    if constexpr (R == 16) {
        dft16<INV>(x);
    } else {
#pragma unroll
        for (int i = 0; i < 16 / R; ++i) {
            if constexpr (R == 8) dft8<INV>(x + 8 * i);
            else if constexpr (R == 4) dft4<INV>(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
            else dft2<INV>(x[2 * i], x[2 * i + 1]);
        }
    }
}

}  // namespace ols
