// ols_pair.cu -- the fused OLS kernel processing two segments per thread in
// split form (segments of N = 2048 and 4096).
//
// Same algorithm and the same per-lane arithmetic as ols_forward.cu
// (Algorithm 2: segment FFT on chip, kept for all filters, per filter the
// point-wise product, inverse FFT, discard of the M-1 aliased samples), but
// every thread carries the same 16 positions of two consecutive segments A
// and B, stored as pairs re = (Re A, Re B), im = (Im A, Im B):
// * every complex add, rotation by +-i, constant rotation, twiddle and
//   spectrum multiply is one packed FP32x2 instruction for both segments
//   (no lane crossing, so no scalar fallbacks);
// * one 128-bit shared-memory store / load moves a position of both
//   segments in each exchange;
// * the filter spectrum and the twiddles are loaded once for both segments
//   (the twiddle table holds broadcast pairs (wr, wr, wi, wi)).
// Each lane performs the exact operation sequence of the single-segment
// kernel, so results are bitwise identical to it.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_fft_passes.cuh"
#include "ols_internal.h"
#include "tmem.cuh"

#ifndef OLS_PAIR_WARPS_PER_SM
#define OLS_PAIR_WARPS_PER_SM 8  // resident warps per SM the register budget must allow
#endif
#ifndef OLS_PAIR_XBUFS
#define OLS_PAIR_XBUFS 2         // exchange buffers (1: an extra barrier per exchange, half the shared memory)
#endif
#ifndef OLS_PAIR_X_TMEM
#define OLS_PAIR_X_TMEM 0        // 1: the segment spectra wait in TMEM between filters, not in registers
#endif

namespace ols {
namespace pairk {

template <int LOG2N>
struct PGeo {
    using G = Geo<LOG2N>;
    static_assert(G::T >= 128, "pair kernel needs one segment per 128-thread multiple");
    static constexpr int BLOCK = G::T;
    static constexpr int MINB = (OLS_PAIR_WARPS_PER_SM * 32 + BLOCK - 1) / BLOCK;
    static constexpr size_t SMEM = sizeof(float4) * OLS_PAIR_XBUFS * (size_t)G::PADN;   // exchange buffers
};

__device__ __forceinline__ float4 pack(const cpair &c) { return make_float4(c.re.x, c.re.y, c.im.x, c.im.y); }
__device__ __forceinline__ cpair unpack(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }

template <int LOG2N, int PW, int PR>
__device__ __forceinline__ void exchange(cpair *x, float4 *buf, int t) {
    if constexpr (OLS_PAIR_XBUFS == 1) __syncthreads();   // previous readers of buf are done
    const int bw = pad_base<LOG2N, PW>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) buf[bw + pad_off<LOG2N, PW>(k)] = pack(x[k]);
    __syncthreads();
    const int br = pad_base<LOG2N, PR>(t);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = unpack(buf[br + pad_off<LOG2N, PR>(k)]);
}

// Twiddles from the broadcast table: entry (k-1) s + n' of pass P (offset
// tw_off(P)) is (wr, wr, wi, wi) of W_{16 s}^{n' k}; the first OLS_TW_LOADS
// powers are loaded and the others multiplied out exactly as in TwGlobal.
struct TwPair {
    const float4 *tw;
    struct Fetched {
        float4 w[OLS_TW_LOADS];
    };
    template <int LOG2N, int P>
    __device__ __forceinline__ void fetch(Fetched &f, int t) const {
        using G = Geo<LOG2N>;
        constexpr int s = G::stride(P);
        const float4 *w = tw + G::tw_off(P) + (t % s);
#pragma unroll
        for (int k = 1; k <= OLS_TW_LOADS; ++k) f.w[k - 1] = __ldg(w + (k - 1) * s);
    }
    template <bool INV>
    __device__ __forceinline__ void apply(cpair *x, const Fetched &f) const {
        cpair w[16];
#pragma unroll
        for (int k = 1; k <= OLS_TW_LOADS; ++k) w[k] = unpack(f.w[k - 1]);
#if OLS_TW_RECUR
        if (OLS_TW_LOADS < 2) w[2] = cmul(w[1], w[1].re, w[1].im);
        if (OLS_TW_LOADS < 3) w[3] = cmul(w[1], w[2].re, w[2].im);
        if (OLS_TW_LOADS < 4) w[4] = cmul(w[2], w[2].re, w[2].im);
        w[8] = cmul(w[4], w[4].re, w[4].im);
        w[12] = cmul(w[4], w[8].re, w[8].im);
#pragma unroll
        for (int k = 5; k < 16; ++k)
            if (k != 8 && k != 12) w[k] = cmul(w[k & 3], w[k & 12].re, w[k & 12].im);
#endif
#pragma unroll
        for (int k = 1; k < 16; ++k) x[k] = INV ? cmulc(x[k], w[k].re, w[k].im) : cmul(x[k], w[k].re, w[k].im);
    }
};

template <int LOG2N, int P>
__device__ __forceinline__ void forward_passes(cpair *x, float4 *bufs, const TwPair &tw, int t, int &xc) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        TwPair::Fetched f;
        tw.template fetch<LOG2N, P>(f, t);
        dft_groups<G::radix(P), false>(x);
        tw.template apply<false>(x, f);
        exchange<LOG2N, P, P + 1>(x, bufs + (OLS_PAIR_XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        forward_passes<LOG2N, P + 1>(x, bufs, tw, t, xc);
    } else {
        dft_groups<G::radix(P), false>(x);
    }
}

template <int LOG2N, int P>
__device__ __forceinline__ void inverse_passes(cpair *x, float4 *bufs, const TwPair &tw, int t, int &xc) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        TwPair::Fetched f;
        tw.template fetch<LOG2N, P>(f, t);
        exchange<LOG2N, P + 1, P>(x, bufs + (OLS_PAIR_XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        tw.template apply<true>(x, f);
    }
    dft_groups<G::radix(P), true>(x);
    if constexpr (P > 0) inverse_passes<LOG2N, P - 1>(x, bufs, tw, t, xc);
}

}  // namespace pairk

template <int LOG2N>
__global__ void __launch_bounds__(pairk::PGeo<LOG2N>::BLOCK, pairk::PGeo<LOG2N>::MINB)
ols_pair_kernel(const float2 *__restrict__ sig, long long Ns, const float4 *__restrict__ Hk,
                const float4 *__restrict__ twp, float2 *__restrict__ y, int M, int F, long long L, long long nseg,
                long long Nout) {
    using G = Geo<LOG2N>;
    extern __shared__ float4 smem4[];
    const int t = threadIdx.x;
    const pairk::TwPair tw{twp};
    const int lo = M - 1;
    int xc = 0;
#if OLS_PAIR_X_TMEM
    // 64 TMEM columns per CTA: thread t's lane holds its 16 spectrum pairs.
    __shared__ uint32_t tbase;
    if (threadIdx.x < 32) tmem::alloc(&tbase, 64);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    const uint32_t xcol = tbase + tmem::lane_bits();
#endif
    const long long npair = (nseg + 1) / 2;
    for (long long pi = blockIdx.x; pi < npair; pi += gridDim.x) {
        const long long sa = 2 * pi, sb = 2 * pi + 1;
        const bool act_b = sb < nseg;
        const long long start_a = sa * L, start_b = sb * L;
        cpair X[16];
        {
            const long long av_a = Ns - start_a, av_b = act_b ? Ns - start_b : 0;
            const int lim_a = (int)(av_a < G::N ? av_a : G::N);
            const int lim_b = (int)(av_b < G::N ? av_b : G::N);
            const float2 *src_a = sig + start_a + t;
            const float2 *src_b = sig + (act_b ? start_b : 0) + t;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int n = k * G::T + t;
                const float2 a = n < lim_a ? __ldg(src_a + k * G::T) : make_float2(0.f, 0.f);
                const float2 b = n < lim_b ? __ldg(src_b + k * G::T) : make_float2(0.f, 0.f);
                X[k] = {make_float2(a.x, b.x), make_float2(a.y, b.y)};
            }
        }
        pairk::forward_passes<LOG2N, 0>(X, smem4, tw, t, xc);
#if OLS_PAIR_X_TMEM
        tmem::st32(xcol, reinterpret_cast<const float *>(X));
        tmem::st32(xcol + 32, reinterpret_cast<const float *>(X + 8));
        tmem::wait_st();
#endif

        const long long rem_a = Nout - start_a, rem_b = act_b ? Nout - start_b : 0;
        const int span_a = (int)(rem_a < (long long)(G::N - lo) ? rem_a : (long long)(G::N - lo));
        const int span_b = (int)(rem_b < (long long)(G::N - lo) ? rem_b : (long long)(G::N - lo));
        const long long obase_a = start_a - lo, obase_b = start_b - lo;

        float4 hn[8];
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2) hn[j2] = load_spectrum(Hk + j2 * G::T + t);
        for (int f = 0; f < F; ++f) {
            cpair x[16];
#if OLS_PAIR_X_TMEM
            tmem::ld32(xcol, reinterpret_cast<float *>(x));
            tmem::ld32(xcol + 32, reinterpret_cast<float *>(x + 8));
            tmem::wait_ld();
#else
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = X[j];
#endif
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                x[2 * j2] = cmul(x[2 * j2], make_float2(hn[j2].x, hn[j2].x), make_float2(hn[j2].y, hn[j2].y));
                x[2 * j2 + 1] = cmul(x[2 * j2 + 1], make_float2(hn[j2].z, hn[j2].z), make_float2(hn[j2].w, hn[j2].w));
            }
            if (f + 1 < F) {
                const float4 *hp = Hk + (size_t)(f + 1) * (G::N / 2) + t;
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2) hn[j2] = load_spectrum(hp + j2 * G::T);
            }
            pairk::inverse_passes<LOG2N, G::NP - 1>(x, smem4, tw, t, xc);
            float2 *dst = y + (size_t)f * (size_t)Nout;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int n = k * G::T + t;
                if ((unsigned)(n - lo) < (unsigned)span_a) dst[obase_a + n] = make_float2(x[k].re.x, x[k].im.x);
                if ((unsigned)(n - lo) < (unsigned)span_b) dst[obase_b + n] = make_float2(x[k].re.y, x[k].im.y);
            }
        }
    }
#if OLS_PAIR_X_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, 64);
#endif
}

template <int LOG2N>
static cudaError_t pair_prepare_n(ols_plan_s &p) {
    using PG = pairk::PGeo<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute(ols_pair_kernel<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PG::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_PAIR_X_TMEM)
        e = resident_blocks_tmem(ols_pair_kernel<LOG2N>, PG::BLOCK, PG::SMEM, 64, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_pair_kernel<LOG2N>, PG::BLOCK, PG::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.pair_grid_cap = per_sm * p.sm_count;
    return cudaSuccess;
}

cudaError_t pair_prepare(ols_plan_s &p) {
    switch (p.log2N) {
        case 11: return pair_prepare_n<11>(p);
        case 12: return pair_prepare_n<12>(p);
        default: return cudaErrorInvalidValue;
    }
}

template <int LOG2N>
static cudaError_t pair_launch_n(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y, int64_t L,
                                 int64_t nseg, int64_t Nout, cudaStream_t st) {
    using PG = pairk::PGeo<LOG2N>;
    const int64_t npair = (nseg + 1) / 2;
    const int grid = (int)(npair < p.pair_grid_cap ? npair : p.pair_grid_cap);
    ols_pair_kernel<LOG2N><<<grid, PG::BLOCK, PG::SMEM, st>>>(s, Ns, reinterpret_cast<const float4 *>(p.Hk),
                                                              p.tw_pair, y, p.M, p.F, L, nseg, Nout);
    return cudaGetLastError();
}

cudaError_t pair_launch(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y, int64_t L, int64_t nseg,
                        int64_t Nout, cudaStream_t st) {
    switch (p.log2N) {
        case 11: return pair_launch_n<11>(p, s, Ns, y, L, nseg, Nout, st);
        case 12: return pair_launch_n<12>(p, s, Ns, y, L, nseg, Nout, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ols
