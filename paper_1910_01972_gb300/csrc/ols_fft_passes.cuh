// ols_fft_passes.cuh -- the in-kernel segment FFT shared by the OLS kernels.
//
// A segment of N = 2^LOG2N complex points is transformed by N/16 threads,
// 16 points each: radix-16 passes (one 16-point DFT per thread, all
// rotations compile-time constants) followed by one pass of radix 2/4/8/16 at
// stride 1, exchanging through shared memory between passes.
// * forward passes: decimation in frequency, natural-order input, spectrum
//   left in mixed-radix digit-reversed order (no reordering step: Sec. 3.3
//   notes the order is irrelevant to a point-wise product as long as both
//   operands and the inverse transform share it);
// * inverse passes: the exact reverse (decimation in time), digit-reversed
//   input, natural-order output, unnormalised.
// After the last forward pass thread t holds storage positions 16 t + j in
// register j; before the first inverse pass it needs exactly those, so
// point-wise products happen in registers.  In the layout of the first pass
// (and after the last inverse pass) thread t holds time index k T + t in
// register k, which makes every global load and store coalesced.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "fft_regs.cuh"

// Tuning knobs (compile-time; defaults are the measured best on GB300).
#ifndef OLS_PREFETCH_H
#define OLS_PREFETCH_H 1     // load filter f+1's spectrum while filter f is transformed
#endif
#ifndef OLS_H_L2ONLY
#define OLS_H_L2ONLY 0       // 1: spectra bypass L1 (__ldcg) instead of __ldg
#endif
#ifndef OLS_XBUFS
#define OLS_XBUFS 2          // exchange buffers per segment (2: one barrier per exchange)
#endif
#ifndef OLS_TW_GLOBAL
#define OLS_TW_GLOBAL 1      // twiddles read through L1 (1) or staged in shared memory (0)
#endif
#ifndef OLS_WARPS_PER_SM
#define OLS_WARPS_PER_SM 16  // resident warps per SM the register budget must allow
#endif

namespace ols {

template <int LOG2N>
struct Geo {
    static constexpr int N = 1 << LOG2N;
    static constexpr int T = N / 16;
    static constexpr int NP = (LOG2N + 3) / 4;
    static constexpr int RL = (LOG2N % 4) ? (1 << (LOG2N % 4)) : 16;
    static constexpr int SEGS = T >= 128 ? 1 : 128 / T;
    static constexpr int BLOCK = T * SEGS;
    static constexpr int MINB = (OLS_WARPS_PER_SM * 32 + BLOCK - 1) / BLOCK;
    static constexpr int PADN = N + N / 16;
    __host__ __device__ static constexpr int stride(int p) { return p == NP - 1 ? 1 : (N >> (4 * (p + 1))); }
    __host__ __device__ static constexpr int radix(int p) { return p == NP - 1 ? RL : 16; }
    __host__ __device__ static constexpr int tw_off(int p) {
        int o = 0;
        for (int i = 0; i < p; ++i) o += 15 * stride(i);
        return o;
    }
    static constexpr int TWN = tw_off(NP - 1);
    static constexpr int TWN_PAD = OLS_TW_GLOBAL ? 0 : ((TWN + 1) & ~1);   // keep buffers 16-byte aligned
    static constexpr int XBUFS = OLS_XBUFS;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)(TWN_PAD + SEGS * XBUFS * PADN);
};

// Padded shared-memory base of thread t in the layout of pass P:
// positions (t / s) * 16 s + (t % s) + k s, padded q -> q + q / 16.
template <int LOG2N, int P>
__device__ __forceinline__ int pad_base(int t) {
    constexpr int s = Geo<LOG2N>::stride(P);
    const int q = (t / s) * 16 * s + (t % s);
    return q + (q >> 4);
}
template <int LOG2N, int P>
__device__ __forceinline__ constexpr int pad_off(int k) {
    constexpr int s = Geo<LOG2N>::stride(P);
    return k * s + ((k * s) >> 4);
}

// Write x in the layout of pass PW, barrier, read it back in the layout of PR.
template <int LOG2N, int PW, int PR>
__device__ __forceinline__ void exchange(float2 *x, float2 *buf, int t) {
    if constexpr (Geo<LOG2N>::XBUFS == 1) __syncthreads();   // previous readers of buf are done
    const int bw = pad_base<LOG2N, PW>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) buf[bw + pad_off<LOG2N, PW>(k)] = x[k];
    __syncthreads();
    const int br = pad_base<LOG2N, PR>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = buf[br + pad_off<LOG2N, PR>(k)];
}

// Multiply element k of pass P's 16-point group by W_{16 s}^{(t mod s) k}
// (conjugated for the inverse).
template <int LOG2N, int P, bool INV>
__device__ __forceinline__ void twiddle(float2 *x, const float2 *tw, int t) {
    using G = Geo<LOG2N>;
    constexpr int s = G::stride(P);
    const float2 *w = tw + G::tw_off(P) + (t % s);
#pragma unroll
    for (int k = 1; k < 16; ++k) {
#if OLS_TW_GLOBAL
        const float2 wk = __ldg(w + (k - 1) * s);
#else
        const float2 wk = w[(k - 1) * s];
#endif
        x[k] = ctw<INV>(x[k], wk);
    }
}

template <int LOG2N, int P>
__device__ __forceinline__ void forward_passes(float2 *x, float2 *bufs, const float2 *tw, int t, int &xc) {
    using G = Geo<LOG2N>;
    dft_groups<G::radix(P), false>(x);
    if constexpr (P < G::NP - 1) {
        twiddle<LOG2N, P, false>(x, tw, t);
        exchange<LOG2N, P, P + 1>(x, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        forward_passes<LOG2N, P + 1>(x, bufs, tw, t, xc);
    }
}

// x holds pass P+1's layout (or pass NP-1's when P == NP-1); runs the
// inverse of passes P, P-1, ..., 0.
template <int LOG2N, int P>
__device__ __forceinline__ void inverse_passes(float2 *x, float2 *bufs, const float2 *tw, int t, int &xc) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        exchange<LOG2N, P + 1, P>(x, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        twiddle<LOG2N, P, true>(x, tw, t);
    }
    dft_groups<G::radix(P), true>(x);
    if constexpr (P > 0) inverse_passes<LOG2N, P - 1>(x, bufs, tw, t, xc);
}

__device__ __forceinline__ float4 load_spectrum(const float4 *p) {
#if OLS_H_L2ONLY
    return __ldcg(p);
#else
    return __ldg(p);
#endif
}


}  // namespace ols
