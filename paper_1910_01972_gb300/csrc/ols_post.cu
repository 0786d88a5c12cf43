// ols_post.cu -- the fused OLS kernel with post-processing of the convolved
// output inside the kernel, before anything is written (Sec. 3.2: OLS's
// "optional post-processing" step; Sec. 4.3: per-element and non-local
// post-processing; Sec. 4.4: reducing the output before it leaves the GPU).
//
// Four epilogues on the same segment body as ols_forward.cu (segment FFT
// kept in registers for all filters; per filter the point-wise product, the
// inverse FFT and the discard of aliased samples):
// * POWER   (per element)   p_f[j] = |y_f[j]|^2, written as FP32 (half the
//   output bytes of y);
// * DETECT  (per element + selection) the candidates (f, j) whose power
//   reaches a threshold, appended to a caller list through one atomic per
//   warp and store step (warp-aggregated), nothing else written;
// * DERIV   (non-local)     the numerical derivative of y along j: central
//   differences (y[j+1] - y[j-1]) / 2 inside, one-sided differences at j = 0
//   and j = Nout-1.  Each segment advances by L-2 instead of L and starts one
//   output early, so every derivative it writes has both neighbours among
//   its own unaliased samples (the "immediate neighbourhood" of Sec. 4.3);
//   the neighbours are exchanged through a shared-memory buffer of their own.
// * PEAK    (non-local + selection) the peaks of the power (Sec. 4.4's peak
//   finding): (f, j) whose power reaches the threshold, is above the power of
//   j - 1 and at least that of j + 1 (no neighbour at the two ends of the
//   stream), appended like DETECT; segments laid out like DERIV.  Candidates
//   are rare, so a warp fetches neighbour powers (warp shuffles) only when
//   one of its lanes reaches the threshold; in segments of several warps each
//   warp's first and last thread also publish their 16 powers in a small
//   shared buffer for the neighbouring warps.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_fft_passes.cuh"
#include "ols_internal.h"
#include "tmem.cuh"

namespace ols {

template <int LOG2N, int MODE>
struct PostGeo {
    using G = Geo<LOG2N>;
    // the modes that read the neighbours j - 1 and j + 1 of an output
    static constexpr bool NEIGH = MODE == POST_DERIV || MODE == POST_PEAK;
    // per segment (float2 units): the exchange buffers; DERIV's neighbourhood
    // buffer; PEAK's warp-edge powers [2][T/32][16] floats (segments of several warps)
    static constexpr int EDGE = (MODE == POST_PEAK && G::T > 32) ? (G::T / 32) * 16 : 0;
    static constexpr int SLOT = G::XBUFS * G::PADN + (MODE == POST_DERIV ? G::PADN : 0) + EDGE;
    static constexpr size_t SMEM_USED = sizeof(float2) * (size_t)(G::SEGS * SLOT);
    // requested: at least enough that no more blocks fit on an SM (228 KB)
    // than TMEM can serve, so a block's tcgen05.alloc never waits
    static constexpr size_t SMEM = !OLS_FWD_TW_TMEM ? SMEM_USED
                                   : (SMEM_USED > (228u * 1024u) / (G::TMEM_MAX_CTAS + 1))
                                       ? SMEM_USED
                                       : (228u * 1024u) / (G::TMEM_MAX_CTAS + 1) + 1024u;
    // the derivative's epilogue holds more live values: one resident block
    // fewer per SM keeps it free of register spills
    static constexpr int MINB = (MODE == POST_DERIV && G::MINB > 1) ? G::MINB - 1 : G::MINB;
};

// The peak test of one output with a candidate power pk (called by whole warps,
// only when some lane has a candidate: it stays out of the common path's
// register allocation).  Neighbours n - 1 and n + 1 of output n = k T + t are
// register k of threads t - 1 and t + 1: rotating shuffles within the W
// threads of the segment in a warp, whose wrap-around carries `up` (register
// k - 1 of thread T - 1, for thread 0) and `dn` (register k + 1 of thread 0,
// for thread T - 1); in segments of several warps, the threads at a warp's
// edge read the neighbouring warp's powers from `edge` instead.
template <int T>
__device__ __noinline__ bool peak_test(bool hit, float pk, float up, float dn, int t, int k, bool first, bool last,
                                       const float *edge) {
    constexpr int W = T < 32 ? T : 32;
    const int gl = t % W;
    float prv = __shfl_sync(0xffffffffu, up, gl == 0 ? W - 1 : gl - 1, W);
    float nxt = __shfl_sync(0xffffffffu, dn, gl == W - 1 ? 0 : gl + 1, W);
    if constexpr (T > 32) {
        const int w = t / 32, nw = T / 32;
        if (gl == 0) prv = w > 0 ? edge[(nw + w - 1) * 16 + k] : edge[(2 * nw - 1) * 16 + (k > 0 ? k - 1 : 0)];
        if (gl == W - 1) nxt = w < nw - 1 ? edge[(w + 1) * 16 + k] : edge[k < 15 ? k + 1 : 15];
    }
    if (hit && !first) hit = pk > prv;
    if (hit && !last) hit = pk >= nxt;
    return hit;
}

// Append candidate (j, f, power) for every lane with `hit`: one atomic per
// warp (warp-aggregated); records past `cap` are dropped, the count is kept.
__device__ __forceinline__ void append_candidates(bool hit, long long j, int f, float pw, ols_candidate *cand,
                                                  unsigned long long *count, long long cap, long long Nout,
                                                  int *status) {
    const unsigned lane = threadIdx.x & 31u;
    const unsigned mask = __ballot_sync(0xffffffffu, hit);
    if (mask) {
        unsigned long long base = 0;
        const unsigned leader = __ffs(mask) - 1;
        if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (hit) {
            const unsigned long long i = base + __popc(mask & ((1u << lane) - 1u));
            if (i < (unsigned long long)cap && in_bounds(j < Nout, status)) {
                ols_candidate c;
                c.j = j;
                c.f = f;
                c.power = pw;
                cand[i] = c;
            }
        }
    }
}

template <int LOG2N, int MODE>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK, (PostGeo<LOG2N, MODE>::MINB))
ols_post_kernel(const float2 *__restrict__ sig, long long Ns, const float4 *__restrict__ Hk,
                const float2 *__restrict__ twg, void *__restrict__ out, int M, int F, long long step,
                long long nseg, long long Nout, float thr, ols_candidate *__restrict__ cand,
                unsigned long long *__restrict__ count, long long cap, int *status) {
    using G = Geo<LOG2N>;
    using PG = PostGeo<LOG2N, MODE>;
    extern __shared__ float4 smem_raw[];
    __shared__ uint32_t tbase;
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *bufs = smem + slot * PG::SLOT;
    float2 *dbuf = bufs + G::XBUFS * G::PADN;        // DERIV: the output's neighbourhood; PEAK: warp edges
#if OLS_FWD_TW_TMEM
    // the forward kernel's TMEM layout: twiddles, then the segment spectrum (columns 96..127)
    if (threadIdx.x < 32) tmem::alloc(&tbase, G::TMEM_COLS);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    // the derivative runs the TMEM exchange at N = 2048 (at other N it
    // spills); power and detection keep the exchange in shared memory (with
    // it their epilogues spill: 0.525 vs 0.535 ms and 0.582 vs 0.613 ms on
    // the filter bank)
    constexpr bool xch = MODE == POST_DERIV && LOG2N == 11;
    const TwTmemT<xch> tw{tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 128u};
    tw_tmem_fill<LOG2N, xch>(twg, tw.base, t);
    const uint32_t xcol = tw.base + 96;
#else
    (void)tbase;
    const TwGlobal tw{twg};
#endif
    // circular position of a segment's first output, and its input offset
    const int n0 = PG::NEIGH ? M : M - 1;
    const long long off = PG::NEIGH ? -1 : 0;
    int xc = 0;
    const long long nblk = (nseg + G::SEGS - 1) / G::SEGS;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long seg = blk * G::SEGS + slot;
        const bool active = seg < nseg;
        const long long j0 = seg * step;                 // first output of this segment
        const long long start = j0 + off;                // first input sample (may be -1)

        // segment load: samples start + k T + t inside [0, Ns), zero elsewhere
        float2 X[16];
        {
            const long long avail = active ? (Ns - start) : 0;
            const int lim = (int)(avail < G::N ? avail : G::N);
            const int first = active ? (int)(-start > 0 ? -start : 0) : 0;   // 1 only before s[0]
            const float2 *src = sig + (active ? start : 0) + t;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int n = k * G::T + t;
                const long long i = (active ? start : 0) + n;
                X[k] = (n >= first && n < lim && in_bounds(i >= 0 && i < Ns, status)) ? __ldg(src + k * G::T)
                                                                                     : make_float2(0.f, 0.f);
            }
        }
        forward_passes<LOG2N, 0>(X, bufs, tw, t, xc);
#if OLS_FWD_TW_TMEM
        tmem::st32(xcol, reinterpret_cast<const float *>(X));
        tmem::wait_st();
#endif

        const long long rem = active ? (Nout - j0) : 0;
        const int span = (int)(rem < step ? rem : step);

        float4 hn[8];
        const long long hn_end = (long long)F * (G::N / 2);   // float4 entries of the spectra
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2)
            if (in_bounds(j2 * G::T + t < hn_end, status)) hn[j2] = load_spectrum(Hk + j2 * G::T + t);
        for (int f = 0; f < F; ++f) {
            float2 x[16];
#if OLS_FWD_TW_TMEM
            tmem::ld32(xcol, reinterpret_cast<float *>(x));
            tmem::wait_ld();
#else
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = X[j];
#endif
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                x[2 * j2] = cmul(x[2 * j2], make_float2(hn[j2].x, hn[j2].y));
                x[2 * j2 + 1] = cmul(x[2 * j2 + 1], make_float2(hn[j2].z, hn[j2].w));
            }
            if (f + 1 < F) {
                const float4 *hp = Hk + (size_t)(f + 1) * (G::N / 2) + t;
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2)
                    if (in_bounds((long long)(f + 1) * (G::N / 2) + j2 * G::T + t < hn_end, status))
                        hn[j2] = load_spectrum(hp + j2 * G::T);
            }
            inverse_passes<LOG2N, G::NP - 1>(x, bufs, tw, t, xc);

            if constexpr (MODE == POST_POWER) {
                float *dst = static_cast<float *>(out) + (size_t)f * (size_t)Nout + (j0 - n0);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    if ((unsigned)(n - n0) < (unsigned)span && in_bounds(j0 - n0 + n >= 0 && j0 - n0 + n < Nout, status))
                        dst[n] = fmaf(x[k].x, x[k].x, x[k].y * x[k].y);
                }
            } else if constexpr (MODE == POST_DETECT) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    const float p = fmaf(x[k].x, x[k].x, x[k].y * x[k].y);
                    const bool hit = (unsigned)(n - n0) < (unsigned)span && p >= thr;
                    append_candidates(hit, j0 + (n - n0), f, p, cand, count, cap, Nout, status);
                }
            } else if constexpr (MODE == POST_PEAK) {
                constexpr int W = G::T < 32 ? G::T : 32;          // threads of the segment in one warp
                const int gl = t % W;
                float pw[16];
#pragma unroll
                for (int k = 0; k < 16; ++k) pw[k] = fmaf(x[k].x, x[k].x, x[k].y * x[k].y);
                // segments of several warps: first[w][k] at edge[w * 16 + k], last[w][k] after them
                float *edge = reinterpret_cast<float *>(dbuf);
                if constexpr (PG::EDGE > 0) {
                    if (gl == 0 || gl == W - 1) {
                        float4 *e = reinterpret_cast<float4 *>(edge + ((gl == 0 ? 0 : G::T / 32) + t / 32) * 16);
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            e[q] = make_float4(pw[4 * q], pw[4 * q + 1], pw[4 * q + 2], pw[4 * q + 3]);
                    }
                    __syncthreads();
                }
                // circular positions of outputs j = 0 and j = Nout-1 (one neighbour only), if in this segment
                const int n_first = j0 == 0 ? n0 : -2;
                const int n_last = (rem <= step) ? (int)(rem - 1) + n0 : -2;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    bool hit = (unsigned)(n - n0) < (unsigned)span && pw[k] >= thr &&
                               in_bounds(n >= 1 && n + 1 < G::N, status);
                    if (__any_sync(0xffffffffu, hit))
                        hit = peak_test<G::T>(hit, pw[k], (gl == W - 1) ? pw[k > 0 ? k - 1 : 0] : pw[k],
                                              (gl == 0) ? pw[k < 15 ? k + 1 : 15] : pw[k], t, k, n == n_first,
                                              n == n_last, edge);
                    append_candidates(hit, j0 + (n - n0), f, pw[k], cand, count, cap, Nout, status);
                }
            } else {
                // write y (circular order) to the neighbourhood buffer, padded q -> q + q/16
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    dbuf[n + (n >> 4)] = x[k];
                }
                __syncthreads();
                float2 *dst = static_cast<float2 *>(out) + (size_t)f * (size_t)Nout + (j0 - n0);
                // circular positions of outputs j = 0 and j = Nout-1 (one-sided ends), if in this segment
                const int n_first = j0 == 0 ? n0 : -2;
                const int n_last = (rem <= step) ? (int)(rem - 1) + n0 : -2;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    if ((unsigned)(n - n0) < (unsigned)span &&
                        in_bounds(j0 - n0 + n >= 0 && j0 - n0 + n < Nout && n >= 1 && n + 1 < G::N, status)) {
                        const int lo = (n == n_first) ? n : n - 1;
                        const int hi = (n == n_last) ? n : n + 1;
                        const float sc = (lo == n || hi == n) ? 1.f : 0.5f;
                        const float2 a = dbuf[lo + (lo >> 4)], b = dbuf[hi + (hi >> 4)];
                        dst[n] = make_float2((b.x - a.x) * sc, (b.y - a.y) * sc);
                    }
                }
            }
        }
    }
#if OLS_FWD_TW_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, G::TMEM_COLS);
#endif
}

template <int LOG2N, int MODE>
static cudaError_t post_prepare_nm(ols_plan_s &p) {
    using G = Geo<LOG2N>;
    using PG = PostGeo<LOG2N, MODE>;
    cudaError_t e = cudaFuncSetAttribute(ols_post_kernel<LOG2N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PG::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_FWD_TW_TMEM)
        e = resident_blocks_tmem(ols_post_kernel<LOG2N, MODE>, G::BLOCK, PG::SMEM, (int)G::TMEM_COLS, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_post_kernel<LOG2N, MODE>, G::BLOCK, PG::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.post_grid_cap[MODE] = per_sm * p.sm_count;
    return cudaSuccess;
}

template <int LOG2N>
static cudaError_t post_prepare_n(ols_plan_s &p) {
    cudaError_t e = post_prepare_nm<LOG2N, POST_POWER>(p);
    if (e == cudaSuccess) e = post_prepare_nm<LOG2N, POST_DETECT>(p);
    if (e == cudaSuccess) e = post_prepare_nm<LOG2N, POST_DERIV>(p);
    if (e == cudaSuccess) e = post_prepare_nm<LOG2N, POST_PEAK>(p);
    return e;
}

cudaError_t post_prepare(ols_plan_s &p) {
    switch (p.log2N) {
        case 8: return post_prepare_n<8>(p);
        case 9: return post_prepare_n<9>(p);
        case 10: return post_prepare_n<10>(p);
        case 11: return post_prepare_n<11>(p);
        case 12: return post_prepare_n<12>(p);
        case 13: return post_prepare_n<13>(p);
        default: return cudaErrorInvalidValue;
    }
}

template <int LOG2N, int MODE>
static cudaError_t post_launch_nm(const ols_plan_s &p, const PostArgs &a, cudaStream_t st) {
    using G = Geo<LOG2N>;
    using PG = PostGeo<LOG2N, MODE>;
    const int64_t nblk = (a.nseg + G::SEGS - 1) / G::SEGS;
    const int cap = p.post_grid_cap[MODE];
    const int grid = fused_grid(LOG2N, nblk, cap);
    ols_post_kernel<LOG2N, MODE><<<grid, G::BLOCK, PG::SMEM, st>>>(
        a.s, a.Ns, reinterpret_cast<const float4 *>(p.Hk), p.tw, a.out, p.M, p.F, a.step, a.nseg, a.Nout, a.thr,
        a.cand, a.count, a.cap, p.d_status);
    return cudaGetLastError();
}

template <int LOG2N>
static cudaError_t post_launch_n(const ols_plan_s &p, const PostArgs &a, cudaStream_t st) {
    switch (a.mode) {
        case POST_POWER: return post_launch_nm<LOG2N, POST_POWER>(p, a, st);
        case POST_DETECT: return post_launch_nm<LOG2N, POST_DETECT>(p, a, st);
        case POST_DERIV: return post_launch_nm<LOG2N, POST_DERIV>(p, a, st);
        case POST_PEAK: return post_launch_nm<LOG2N, POST_PEAK>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t post_launch(const ols_plan_s &p, const PostArgs &a, cudaStream_t st) {
    switch (p.log2N) {
        case 8: return post_launch_n<8>(p, a, st);
        case 9: return post_launch_n<9>(p, a, st);
        case 10: return post_launch_n<10>(p, a, st);
        case 11: return post_launch_n<11>(p, a, st);
        case 12: return post_launch_n<12>(p, a, st);
        case 13: return post_launch_n<13>(p, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ols
