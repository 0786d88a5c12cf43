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
#include <type_traits>

#include "fft_regs.cuh"
#include "tmem.cuh"

// Tuning knobs (compile-time; defaults are the measured best on GB300).
#ifndef OLS_PREFETCH_H
#define OLS_PREFETCH_H 1     // load filter f+1's spectrum while filter f is transformed
#endif
#ifndef OLS_H_L2ONLY
#define OLS_H_L2ONLY 0       // 1: spectra bypass L1 (__ldcg), 2: not allocated in L1, instead of __ldg
#endif
#ifndef OLS_XBUFS
#define OLS_XBUFS 2          // exchange buffers per segment (2: one barrier per exchange)
#endif
#ifndef OLS_TW_GLOBAL
#define OLS_TW_GLOBAL 1      // twiddles read through L1 (1) or staged in shared memory (0)
#endif
#ifndef OLS_FWD_TW_TMEM
#define OLS_FWD_TW_TMEM 1    // fused kernels keep twiddles and the segment spectrum in TMEM (0: registers and L1)
#endif
#ifndef OLS_TW_TMEM_LATE
#define OLS_TW_TMEM_LATE 0   // 1: TMEM twiddles of an inverse pass are read after its exchange, not before
#endif
#ifndef OLS_FWD_X_TMEM
#define OLS_FWD_X_TMEM 0     // 1: the forward kernel keeps only the segment spectrum in TMEM
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
    // TMEM twiddles: 128 columns per 128 threads (a thread's lane, 32 columns per pass)
    static constexpr uint32_t TMEM_COLS = (uint32_t)(BLOCK / 128) * 128u;
    static constexpr int TMEM_MAX_CTAS = 512 / (int)TMEM_COLS;
    // segment spectrum alone in TMEM: 32 columns per 128 threads, rounded to the 32-column minimum
    static constexpr uint32_t XT_COLS = (BLOCK / 128) * 32u < 32u ? 32u : (uint32_t)(BLOCK / 128) * 32u;
    // shared memory requested with TMEM twiddles: enough that no more CTAs fit on
    // an SM (228 KB) than TMEM can serve, so allocation never waits
    static constexpr size_t SMEM_TMEM = !OLS_FWD_TW_TMEM ? SMEM
                                        : (SEGS * XBUFS * PADN * sizeof(float2) > (228u * 1024u) / (TMEM_MAX_CTAS + 1))
                                            ? SEGS * XBUFS * PADN * sizeof(float2)
                                            : (228u * 1024u) / (TMEM_MAX_CTAS + 1) + 1024u;
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

// Barrier policies of an exchange: the whole CTA (kernels whose segments
// advance in lock step), or only the NT threads of one segment (named
// barrier `id`; a warp barrier over the segment's lanes when it fits in one
// warp, so segments sharing a warp may follow different paths).
struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int NT>
struct SegmentBarrier {
    int id;
    __device__ __forceinline__ void operator()() const {
        if constexpr (NT < 32) {
            const unsigned lane = threadIdx.x & 31u;
            __syncwarp(((1u << NT) - 1u) << (lane & ~(unsigned)(NT - 1)));
        } else if constexpr (NT == 32) {
            __syncwarp();
        } else {
            asm volatile("bar.sync %0, %1;" ::"r"(id), "n"(NT) : "memory");
        }
    }
};

// Write x in the layout of pass PW, barrier, read it back in the layout of PR.
template <int LOG2N, int PW, int PR, class BAR = CtaBarrier>
__device__ __forceinline__ void exchange(float2 *x, float2 *buf, int t, const BAR &bar = BAR{}) {
    if constexpr (Geo<LOG2N>::XBUFS == 1) bar();   // previous readers of buf are done
    const int bw = pad_base<LOG2N, PW>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) buf[bw + pad_off<LOG2N, PW>(k)] = x[k];
    bar();
    const int br = pad_base<LOG2N, PR>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = buf[br + pad_off<LOG2N, PR>(k)];
}

// Twiddle sources.  Element k of pass P's 16-point group is multiplied by
// W_{16 s}^{(t mod s) k} (s = the pass's stride), conjugated for the inverse.
// Each source splits the step into fetch() (issue the loads) and apply()
// (wait and multiply), so the pass functions can put a barrier-bound
// exchange between the two and hide the load latency.
//
// TwGlobal: read through L1 from the plan's table (entry (k-1) s + n' of
// pass P at offset tw_off(P)).
// Only the first OLS_TW_LOADS powers w^1.. of a pass's twiddle are loaded
// (1, 2, 4 or 15); the others are formed as products (w^2 = w w, w^3 = w w^2,
// w^4 = w^2 w^2, w^8 = w^4 w^4, w^12 = w^4 w^8, w^k = w^(k&3) w^(k&12)), at
// most five roundings deep for a single load: the L1 data path, the binding
// resource of the fused kernel, is traded for FP32 multiplies, which have
// headroom.
#ifndef OLS_TW_LOADS
#define OLS_TW_LOADS 4
#endif
#define OLS_TW_RECUR (OLS_TW_LOADS < 15)
struct TwGlobal {
    const float2 *tw;
    struct Fetched {
        float2 w[OLS_TW_LOADS];
    };
    template <int LOG2N, int P>
    __device__ __forceinline__ void fetch(Fetched &f, int t) const {
        using G = Geo<LOG2N>;
        constexpr int s = G::stride(P);
        const float2 *w = tw + G::tw_off(P) + (t % s);
#pragma unroll
        for (int k = 1; k <= OLS_TW_LOADS; ++k) {
#if OLS_TW_GLOBAL
            f.w[k - 1] = __ldg(w + (k - 1) * s);
#else
            f.w[k - 1] = w[(k - 1) * s];
#endif
        }
    }
    template <bool INV>
    __device__ __forceinline__ void apply(float2 *x, const Fetched &f) const {
#if OLS_TW_RECUR
        float2 w[16];
#pragma unroll
        for (int k = 1; k <= OLS_TW_LOADS; ++k) w[k] = f.w[k - 1];
        if (OLS_TW_LOADS < 2) w[2] = cmul(w[1], w[1]);
        if (OLS_TW_LOADS < 3) w[3] = cmul(w[1], w[2]);
        if (OLS_TW_LOADS < 4) w[4] = cmul(w[2], w[2]);
        w[8] = cmul(w[4], w[4]);
        w[12] = cmul(w[4], w[8]);
#pragma unroll
        for (int k = 5; k < 16; ++k)
            if (k != 8 && k != 12) w[k] = cmul(w[k & 3], w[k & 12]);
#pragma unroll
        for (int k = 1; k < 16; ++k) x[k] = ctw<INV>(x[k], w[k]);
#else
#pragma unroll
        for (int k = 1; k < 16; ++k) x[k] = ctw<INV>(x[k], f.w[k - 1]);
#endif
    }
};

// TwTmem: the thread's own 15 twiddles of every pass, preloaded into its
// TMEM lane (pass P at columns 32 P .. 32 P + 29 of `base`): no L1 traffic.
struct TwTmem {
    uint32_t base;
    struct Fetched {
        float v[32];
    };
    template <int LOG2N, int P>
    __device__ __forceinline__ void fetch(Fetched &f, int) const {
        tmem::ld32(base + 32 * P, f.v);
    }
    template <bool INV>
    __device__ __forceinline__ void apply(float2 *x, const Fetched &f) const {
        tmem::wait_ld();
#pragma unroll
        for (int k = 1; k < 16; ++k) x[k] = ctw<INV>(x[k], make_float2(f.v[2 * k - 2], f.v[2 * k - 1]));
    }
};

// Fill a TwTmem for thread t from the plan's twiddle table.
template <int LOG2N, int P = 0>
__device__ __forceinline__ void tw_tmem_fill(const float2 *tw, uint32_t base, int t) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        constexpr int s = G::stride(P);
        const float2 *w = tw + G::tw_off(P) + (t % s);
        float v[32];
#pragma unroll
        for (int k = 1; k < 16; ++k) {
            const float2 wk = __ldg(w + (k - 1) * s);
            v[2 * k - 2] = wk.x;
            v[2 * k - 1] = wk.y;
        }
        v[30] = v[31] = 0.f;
        tmem::st32(base + 32 * P, v);
        tw_tmem_fill<LOG2N, P + 1>(tw, base, t);
    } else {
        tmem::wait_st();
    }
}

// One global-table twiddle step (fetch and apply back to back).
template <int LOG2N, int P, bool INV>
__device__ __forceinline__ void twiddle(float2 *x, const float2 *tw, int t) {
    const TwGlobal g{tw};
    TwGlobal::Fetched f;
    g.template fetch<LOG2N, P>(f, t);
    g.template apply<INV>(x, f);
}

template <int LOG2N, int P, class TW, class BAR = CtaBarrier>
__device__ __forceinline__ void forward_passes(float2 *x, float2 *bufs, const TW &tw, int t, int &xc,
                                               const BAR &bar = BAR{}) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        typename TW::Fetched f;
        tw.template fetch<LOG2N, P>(f, t);            // in flight during the DFT
        dft_groups<G::radix(P), false>(x);
        tw.template apply<false>(x, f);
        exchange<LOG2N, P, P + 1>(x, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t, bar);
        ++xc;
        forward_passes<LOG2N, P + 1>(x, bufs, tw, t, xc, bar);
    } else {
        dft_groups<G::radix(P), false>(x);
    }
}
template <int LOG2N, int P>
__device__ __forceinline__ void forward_passes(float2 *x, float2 *bufs, const float2 *tw, int t, int &xc) {
    forward_passes<LOG2N, P>(x, bufs, TwGlobal{tw}, t, xc);
}

// x holds pass P+1's layout (or pass NP-1's when P == NP-1); runs the
// inverse of passes P, P-1, ..., 0.
template <int LOG2N, int P, class TW, class BAR = CtaBarrier>
__device__ __forceinline__ void inverse_passes(float2 *x, float2 *bufs, const TW &tw, int t, int &xc,
                                               const BAR &bar = BAR{}) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        typename TW::Fetched f;
        // in flight during the exchange, except TMEM twiddles with OLS_TW_TMEM_LATE
        // (their 30 registers then are not live across the exchange)
        constexpr bool late = OLS_TW_TMEM_LATE && std::is_same<TW, TwTmem>::value;
        if constexpr (!late) tw.template fetch<LOG2N, P>(f, t);
        exchange<LOG2N, P + 1, P>(x, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t, bar);
        ++xc;
        if constexpr (late) tw.template fetch<LOG2N, P>(f, t);
        tw.template apply<true>(x, f);
    }
    dft_groups<G::radix(P), true>(x);
    if constexpr (P > 0) inverse_passes<LOG2N, P - 1>(x, bufs, tw, t, xc, bar);
}
template <int LOG2N, int P>
__device__ __forceinline__ void inverse_passes(float2 *x, float2 *bufs, const float2 *tw, int t, int &xc) {
    inverse_passes<LOG2N, P>(x, bufs, TwGlobal{tw}, t, xc);
}

__device__ __forceinline__ float4 load_spectrum(const float4 *p) {
#if OLS_H_L2ONLY == 2
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
#elif OLS_H_L2ONLY
    return __ldcg(p);
#else
    return __ldg(p);
#endif
}


}  // namespace ols
