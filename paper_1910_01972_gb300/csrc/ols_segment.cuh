// ols_segment.cuh -- one segment of Algorithm 2, shared by the plain and the
// batched fused kernels: load the segment (zero past Ns), forward FFT into
// registers (kept there for all filters; with TMEM twiddles, in the thread's
// TMEM lane instead, columns 96..127), then for every filter: point-wise
// product with its spectrum (the next filter's spectrum already in flight),
// inverse FFT, and store of the samples not aliased (n >= M-1) that fall
// inside the output.
#pragma once

#include <type_traits>

#include "ols_fft_passes.cuh"

namespace ols {

// XT: the segment spectrum waits in the thread's TMEM lane at column xcol_t
// (32 columns) instead of registers; implied by TMEM twiddles (columns 96..127).
// BAR: the barrier of the segment's exchanges (the whole CTA by default, or
// only the segment's own threads).  status: the plan's status word, for the
// bounds checks of OLS_CHECK builds (may be null).
template <int LOG2N, class TW, bool XT = is_tw_tmem<TW>::value, class BAR = CtaBarrier>
__device__ __forceinline__ void ols_segment(const float2 *__restrict__ sig, long long Ns,
                                            const float4 *__restrict__ Hk, const TW &tw,
                                            float2 *__restrict__ y, int M, int F, long long L,
                                            long long Nout, long long seg, bool active, float2 *bufs,
                                            int t, int &xc, uint32_t xcol_t = 0, const BAR &bar = BAR{},
                                            int *status = nullptr) {
    using G = Geo<LOG2N>;
    const int lo = M - 1;                      // aliased samples per segment
    const long long start = seg * L;

    // Segment load: samples start + k T + t, zero past Ns.
    float2 X[16];
    {
        const long long avail = active ? (Ns - start) : 0;
        const int lim = (int)(avail < G::N ? avail : G::N);
        const float2 *src = sig + (active ? start : 0) + t;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            X[k] = (k * G::T + t < lim && in_bounds((active ? start : 0) + k * G::T + t < Ns, status))
                       ? __ldg(src + k * G::T)
                       : make_float2(0.f, 0.f);
    }
    forward_passes<LOG2N, 0>(X, bufs, tw, t, xc, bar);
    constexpr bool x_in_tmem = XT;
    uint32_t xcol = 0;
    if constexpr (x_in_tmem) {
        if constexpr (is_tw_tmem<TW>::value) xcol = tw.base + 96;
        else xcol = xcol_t;
        tmem::st32(xcol, reinterpret_cast<const float *>(X));
        tmem::wait_st();
    }

    // Valid outputs of this segment: n in [lo, lo + span), n = k T + t.
    const long long rem = active ? (Nout - start) : 0;
    const int span = (int)(rem < (long long)(G::N - lo) ? rem : (long long)(G::N - lo));
    const long long obase = start - lo;

    // segment lengths in Geo<>::TX_NOPF run the TMEM exchange without the
    // spectrum prefetch: its 32 registers make them spill (filter banks of 32
    // filters, Ns = 2^23: N = 512 0.479 against 0.531 ms, N = 1024 0.153
    // against 0.166 ms at Ns = 2^22, N = 4096 0.664 against 0.714 ms)
    constexpr bool prefetch = OLS_PREFETCH_H && !(G::TX_NOPF && tw_xchg<TW>());
    float4 hn[8];
    const long long hn_end = (long long)F * (G::N / 2);   // float4 entries of the spectra
    if constexpr (prefetch) {
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2)
            if (in_bounds(j2 * G::T + t < hn_end, status)) hn[j2] = load_spectrum(Hk + j2 * G::T + t);
    }
    for (int f = 0; f < F; ++f) {
        float2 x[16];
        if constexpr (x_in_tmem) {
            tmem::ld32(xcol, reinterpret_cast<float *>(x));
            tmem::wait_ld();
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = X[j];
        }
        if constexpr (!prefetch) {
            const float4 *hp = Hk + (size_t)f * (G::N / 2) + t;
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2)
                if (in_bounds((long long)f * (G::N / 2) + j2 * G::T + t < hn_end, status))
                    hn[j2] = load_spectrum(hp + j2 * G::T);
        }
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2) {
            x[2 * j2] = cmul(x[2 * j2], make_float2(hn[j2].x, hn[j2].y));
            x[2 * j2 + 1] = cmul(x[2 * j2 + 1], make_float2(hn[j2].z, hn[j2].w));
        }
        if constexpr (prefetch) {
            if (f + 1 < F) {
                const float4 *hp = Hk + (size_t)(f + 1) * (G::N / 2) + t;
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2)
                    if (in_bounds((long long)(f + 1) * (G::N / 2) + j2 * G::T + t < hn_end, status))
                        hn[j2] = load_spectrum(hp + j2 * G::T);
            }
        }
        inverse_passes<LOG2N, G::NP - 1>(x, bufs, tw, t, xc, bar);
        float2 *dst = y + (size_t)f * (size_t)Nout;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int n = k * G::T + t;
            if ((unsigned)(n - lo) < (unsigned)span && in_bounds(obase + n >= 0 && obase + n < Nout, status))
                dst[obase + n] = x[k];
        }
    }
}

}  // namespace ols
