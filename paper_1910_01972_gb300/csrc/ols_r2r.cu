// ols_r2r.cu -- the fused overlap-and-save convolution of a REAL signal with
// a bank of REAL filters (the paper's R2R variant, Sec. 3.4 and Algorithm 2).
//
// The paper runs its R2R kernel on half-length complex FFTs (Stockham
// autosort, with real-to-complex and complex-to-real post-processing).  Here
// the saving of the real data is taken along the filter axis instead, which
// keeps the reorder-free complex kernel of the C2C path:
// * filters are paired, g_p = h_{2p} + i h_{2p+1} (p < ceil(F/2); the last
//   pair of an odd bank has a zero imaginary part), and the plan holds the
//   spectra of the complex sequences g_p;
// * a segment a of the real signal is transformed as a complex sequence with
//   zero imaginary part (its spectrum A is Hermitian);
// * for each pair, one inverse FFT of A G_p gives a * g_p = a * h_{2p} +
//   i (a * h_{2p+1}); both convolutions are real, so the real part is the
//   output of filter 2p and the imaginary part that of filter 2p+1
//   (linearity of Eq. 1).
// Per two output streams: one N-point complex inverse FFT, the same work as
// two N/2-point transforms plus the post-processing of the paper's form, and
// the stores and the signal read move 4-byte real samples.  The forward FFT
// of the segment is done once per segment and amortised over the pairs.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_fft_passes.cuh"
#include "ols_internal.h"
#include "tmem.cuh"

namespace ols {

// g[p][k] = (h[2p][k], h[2p+1][k]) with h[F][M] real; the missing partner of
// an odd F is zero.
__global__ void pack_real_pairs_kernel(const float *__restrict__ h, int M, int F, float2 *__restrict__ g) {
    const int Fc = (F + 1) / 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)Fc * M) return;
    const int p = (int)(i / M), k = (int)(i % M);
    const float re = h[(size_t)(2 * p) * M + k];
    const float im = (2 * p + 1 < F) ? h[(size_t)(2 * p + 1) * M + k] : 0.f;
    g[i] = make_float2(re, im);
}

cudaError_t launch_pack_real_pairs(const float *h, int M, int F, float2 *g, cudaStream_t st) {
    const long long total = (long long)((F + 1) / 2) * M;
    const int blocks = (int)((total + 255) / 256);
    pack_real_pairs_kernel<<<blocks, 256, 0, st>>>(h, M, F, g);
    return cudaGetLastError();
}

// One persistent kernel: resident blocks loop over segments (SEGS segments
// of N/16 threads per block for small N, advancing in lock step).
template <int LOG2N>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK, Geo<LOG2N>::MINB)
ols_r2r_kernel(const float *__restrict__ sig, long long Ns, const float4 *__restrict__ Hk,
               const float2 *__restrict__ twg, float *__restrict__ y, int M, int F, long long L, long long nseg,
               long long Nout, int *status) {
    using G = Geo<LOG2N>;
    extern __shared__ float4 smem_raw[];
    __shared__ uint32_t tbase;
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *bufs = smem + slot * G::XBUFS * G::PADN;
#if OLS_FWD_TW_TMEM
    // the forward kernel's TMEM layout: the thread's twiddles, then (columns
    // 96..127) the segment spectrum, in its own lane
    if (threadIdx.x < 32) tmem::alloc(&tbase, G::TMEM_COLS);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    // the TMEM exchange at N = 2048 only (at other N this kernel spills with it)
    constexpr bool xch = LOG2N == 11;
    const TwTmemT<xch> tw{tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 128u};
    tw_tmem_fill<LOG2N, xch>(twg, tw.base, t);
    const uint32_t xcol = tw.base + 96;
#else
    (void)tbase;
    const TwGlobal tw{twg};
#endif
    const int Fc = (F + 1) / 2;
    const int lo = M - 1;                      // aliased samples per segment
    int xc = 0;
    const long long nblk = (nseg + G::SEGS - 1) / G::SEGS;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long seg = blk * G::SEGS + slot;
        const bool active = seg < nseg;
        const long long start = seg * L;

        // Segment load: real samples start + k T + t (zero past Ns) as complex values.
        float2 X[16];
        {
            const long long avail = active ? (Ns - start) : 0;
            const int lim = (int)(avail < G::N ? avail : G::N);
            const float *src = sig + (active ? start : 0) + t;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                X[k] = make_float2(
                    (k * G::T + t < lim && in_bounds((active ? start : 0) + k * G::T + t < Ns, status))
                        ? __ldg(src + k * G::T)
                        : 0.f,
                    0.f);
        }
        forward_passes<LOG2N, 0>(X, bufs, tw, t, xc);
#if OLS_FWD_TW_TMEM
        tmem::st32(xcol, reinterpret_cast<const float *>(X));
        tmem::wait_st();
#endif

        const long long rem = active ? (Nout - start) : 0;
        const int span = (int)(rem < (long long)(G::N - lo) ? rem : (long long)(G::N - lo));
        const long long obase = start - lo;

        float4 hn[8];
        const long long hn_end = (long long)Fc * (G::N / 2);   // float4 entries of the paired spectra
#pragma unroll
        for (int j2 = 0; j2 < 8; ++j2)
            if (in_bounds(j2 * G::T + t < hn_end, status)) hn[j2] = load_spectrum(Hk + j2 * G::T + t);
        for (int p = 0; p < Fc; ++p) {
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
            if (p + 1 < Fc) {
                const float4 *hp = Hk + (size_t)(p + 1) * (G::N / 2) + t;
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2)
                    if (in_bounds((long long)(p + 1) * (G::N / 2) + j2 * G::T + t < hn_end, status))
                        hn[j2] = load_spectrum(hp + j2 * G::T);
            }
            inverse_passes<LOG2N, G::NP - 1>(x, bufs, tw, t, xc);
            float *dre = y + (size_t)(2 * p) * (size_t)Nout + obase;
            float *dim = dre + Nout;
            // the pair test is uniform: taken once per filter pair, so each
            // store below is a plain predicated store
            if (2 * p + 1 < F) {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    const bool ok = (unsigned)(n - lo) < (unsigned)span &&
                                    in_bounds(obase + n >= 0 && obase + n < Nout, status);
                    if (ok) dre[n] = x[k].x;
                    if (ok) dim[n] = x[k].y;
                }
            } else {
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    if ((unsigned)(n - lo) < (unsigned)span && in_bounds(obase + n >= 0 && obase + n < Nout, status))
                        dre[n] = x[k].x;
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

template <int LOG2N>
static cudaError_t r2r_prepare_n(ols_plan_s &p) {
    using G = Geo<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute(ols_r2r_kernel<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::SMEM_TMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_FWD_TW_TMEM)
        e = resident_blocks_tmem(ols_r2r_kernel<LOG2N>, G::BLOCK, G::SMEM_TMEM, (int)G::TMEM_COLS, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_r2r_kernel<LOG2N>, G::BLOCK, G::SMEM_TMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.r2r_grid_cap = per_sm * p.sm_count;
    return cudaSuccess;
}

template <int LOG2N>
static cudaError_t r2r_launch_n(const ols_plan_s &p, const float *s, int64_t Ns, float *y, int64_t L, int64_t nseg,
                                int64_t Nout, cudaStream_t st) {
    using G = Geo<LOG2N>;
    const int64_t nblk = (nseg + G::SEGS - 1) / G::SEGS;
    const int grid = fused_grid(LOG2N, nblk, p.r2r_grid_cap);
    ols_r2r_kernel<LOG2N><<<grid, G::BLOCK, G::SMEM_TMEM, st>>>(s, Ns, reinterpret_cast<const float4 *>(p.Hk), p.tw, y,
                                                           p.M, p.F, L, nseg, Nout, p.d_status);
    return cudaGetLastError();
}

cudaError_t r2r_prepare(ols_plan_s &p) {
    switch (p.log2N) {
        case 8: return r2r_prepare_n<8>(p);
        case 9: return r2r_prepare_n<9>(p);
        case 10: return r2r_prepare_n<10>(p);
        case 11: return r2r_prepare_n<11>(p);
        case 12: return r2r_prepare_n<12>(p);
        case 13: return r2r_prepare_n<13>(p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t r2r_launch(const ols_plan_s &p, const float *s, int64_t Ns, float *y, int64_t L, int64_t nseg,
                       int64_t Nout, cudaStream_t st) {
    switch (p.log2N) {
        case 8: return r2r_launch_n<8>(p, s, Ns, y, L, nseg, Nout, st);
        case 9: return r2r_launch_n<9>(p, s, Ns, y, L, nseg, Nout, st);
        case 10: return r2r_launch_n<10>(p, s, Ns, y, L, nseg, Nout, st);
        case 11: return r2r_launch_n<11>(p, s, Ns, y, L, nseg, Nout, st);
        case 12: return r2r_launch_n<12>(p, s, Ns, y, L, nseg, Nout, st);
        case 13: return r2r_launch_n<13>(p, s, Ns, y, L, nseg, Nout, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ols
