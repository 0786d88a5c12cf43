// ols_w64.cu -- the fused OLS kernel for segments of N = 2048: one warp per
// segment, 64 points per thread, one shared-memory exchange per FFT.
//
// Algorithm 2 of the paper (segment FFT kept on chip, per filter point-wise
// product, inverse FFT, discard of the M-1 aliased samples, store), laid out
// for the GB300's data paths, which the generic 16-point kernel saturates
// (two exchanges per inverse FFT plus twiddle loads keep the L1/shared-memory
// path near its peak):
// * 2048 = 32 x 64.  Forward pass 0: thread t does the DFT-32s of the two
//   interleaved groups n' = 2t, 2t+1 (elements n' + 64 k), then multiplies by
//   W_2048^(n' k); pass 1: the DFT-64 of block t (positions 64 t + j).  The
//   inverse reverses the two passes.  So one exchange per FFT, through a
//   padded per-warp shared buffer (row 66: 128-bit accesses without bank
//   conflicts in both layouts), synchronised with __syncwarp only: the warps
//   of a CTA never wait on each other.
// * The segment spectrum (64 complex per thread) and the thread's 62 twiddles
//   live in TMEM (the thread's own lane, 252 columns): reading them per filter
//   costs no registers between uses, no shared-memory bandwidth and no L1
//   traffic.  A CTA is 4 warps (the 4 TMEM lane quarters) and allocates 256
//   columns; the dynamic shared-memory request keeps at most two CTAs on an
//   SM, so the 512 columns are never oversubscribed.
// * All 32 16-byte loads of a filter's spectrum are issued together into the
//   registers that then hold the product; outputs of the two groups are
//   adjacent samples and go out as 16-byte stores when aligned.
#include <cuda_runtime.h>
#include <cstdint>

#include "fft_regs.cuh"
#include "ols_internal.h"
#include "tmem.cuh"

#ifndef OLS_W64_NEXT_SEG_PREFETCH
#define OLS_W64_NEXT_SEG_PREFETCH 1   // prefetch the warp's next segment into L2
#endif

namespace ols {
namespace w64 {

constexpr int N = 2048;
constexpr int ROW = 66;                 // padded row (complex) of the exchange buffer
constexpr int BUF = 32 * ROW;           // complex per warp
constexpr int WARPS = 4;                // segments (warps) per CTA
constexpr int THREADS = 32 * WARPS;
constexpr uint32_t NCOLS = 256;         // TMEM: spectrum [0, 128), twiddles [128, 252)
constexpr size_t SMEM_USED = sizeof(float2) * WARPS * BUF;
constexpr size_t SMEM = 80 * 1024;      // > 227 KB / 3: at most two CTAs (512 TMEM columns) per SM
static_assert(SMEM >= SMEM_USED, "exchange buffers must fit");

// x[k] *= w_a[k], x[32 + k] *= w_b[k] for k = 1..31 (conjugated for the
// inverse); twiddle i of the thread sits in TMEM columns 128 + 2i, 2i + 1:
// i < 31 -> group a, k = i + 1; i >= 31 -> group b, k = i - 30.
template <bool INV>
__device__ __forceinline__ void twiddle(float2 *x, uint32_t tm) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float w[32];
        tmem::ld32(tm + 128 + 32 * c, w);
        tmem::wait_ld();
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = 16 * c + q;
            const float2 wv = make_float2(w[2 * q], w[2 * q + 1]);
            if (i < 31) x[i + 1] = ctw<INV>(x[i + 1], wv);
            else if (i < 62) x[32 + i - 30] = ctw<INV>(x[32 + i - 30], wv);
        }
    }
}

__device__ __forceinline__ void st_shared4(float2 *p, float2 a, float2 b) {
    *reinterpret_cast<float4 *>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void ld_shared4(const float2 *p, float2 &a, float2 &b) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}

}  // namespace w64

__global__ void __launch_bounds__(w64::THREADS, 1)
ols_w64_kernel(const float2 *__restrict__ sig, long long Ns, const float4 *__restrict__ Hk,
               const float2 *__restrict__ twg, float2 *__restrict__ y, int M, int F, long long L, long long nseg,
               long long Nout) {
    using namespace w64;
    extern __shared__ float4 smem_raw[];
    __shared__ uint32_t tbase;
    const int warp = threadIdx.x >> 5, t = threadIdx.x & 31;
    float2 *buf = reinterpret_cast<float2 *>(smem_raw) + warp * BUF;

    if (warp == 0) tmem::alloc(&tbase, NCOLS);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    const uint32_t tm = tbase + tmem::lane_bits();

    // this thread's twiddles W_2048^(n' k), n' = 2t (i < 31) and 2t + 1 (i >= 31)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        float v[32];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int i = 16 * c + q;
            float2 w = make_float2(0.f, 0.f);
            if (i < 31) w = twg[i * 64 + 2 * t];
            else if (i < 62) w = twg[(i - 31) * 64 + 2 * t + 1];
            v[2 * q] = w.x;
            v[2 * q + 1] = w.y;
        }
        tmem::st32(tm + 128 + 32 * c, v);
    }
    tmem::wait_st();

    const int lo = M - 1;
    const long long seg_step = (long long)gridDim.x * WARPS;
    for (long long seg = (long long)blockIdx.x * WARPS + warp; seg < nseg; seg += seg_step) {
        const long long start = seg * L;
        float2 x[64];
        {
            const long long avail = Ns - start;
            const int lim = (int)(avail < N ? avail : N);
            const float2 *src = sig + start;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int n = 64 * k + 2 * t;
                x[k] = n < lim ? __ldg(src + n) : make_float2(0.f, 0.f);
                x[32 + k] = n + 1 < lim ? __ldg(src + n + 1) : make_float2(0.f, 0.f);
            }
        }
#if OLS_W64_NEXT_SEG_PREFETCH
        {
            const long long nx = seg + seg_step;
            if (nx < nseg) {
                const char *p = reinterpret_cast<const char *>(sig + nx * L);
                const long long bytes = (Ns - nx * L < N ? Ns - nx * L : N) * (long long)sizeof(float2);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const long long off = (long long)(t + 32 * i) * 128;
                    if (off < bytes) asm volatile("prefetch.global.L2 [%0];" ::"l"(p + off));
                }
            }
        }
#endif
        // forward: pass 0 (two DFT-32 + twiddles), exchange, pass 1 (DFT-64)
        dft32<false>(x);
        dft32<false>(x + 32);
        w64::twiddle<false>(x, tm);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 32; ++k) w64::st_shared4(buf + ROW * k + 2 * t, x[k], x[32 + k]);
        __syncwarp();
#pragma unroll
        for (int j2 = 0; j2 < 32; ++j2) w64::ld_shared4(buf + ROW * t + 2 * j2, x[2 * j2], x[2 * j2 + 1]);
        dft64<false>(x);
        // segment spectrum -> TMEM (storage position 64 t + j in columns 2j, 2j+1)
#pragma unroll
        for (int c = 0; c < 4; ++c) tmem::st32(tm + 32 * c, reinterpret_cast<const float *>(x + 16 * c));
        tmem::wait_st();

        const long long rem = Nout - start;
        const int span = (int)(rem < (long long)(N - lo) ? rem : (long long)(N - lo));
        const long long obase = start - lo;
        const bool pair_aligned = ((obase & 1) == 0) && ((Nout & 1) == 0) &&
                                  ((reinterpret_cast<uintptr_t>(y) & 15) == 0);

        for (int f = 0; f < F; ++f) {
            // spectrum of filter f: 32 x 16 B, all in flight together, then X . H in place
            const float4 *hp = Hk + (size_t)f * (N / 2) + t;
#pragma unroll
            for (int j2 = 0; j2 < 32; ++j2) {
                const float4 h = __ldg(hp + j2 * 32);
                x[2 * j2] = make_float2(h.x, h.y);
                x[2 * j2 + 1] = make_float2(h.z, h.w);
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                float X[32];
                tmem::ld32(tm + 32 * c, X);
                tmem::wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) x[16 * c + q] = cmul(make_float2(X[2 * q], X[2 * q + 1]), x[16 * c + q]);
            }
            // inverse: pass 1 (DFT-64), exchange, twiddles, pass 0 (two DFT-32)
            dft64<true>(x);
            __syncwarp();
#pragma unroll
            for (int j2 = 0; j2 < 32; ++j2) w64::st_shared4(buf + ROW * t + 2 * j2, x[2 * j2], x[2 * j2 + 1]);
            __syncwarp();
#pragma unroll
            for (int k = 0; k < 32; ++k) w64::ld_shared4(buf + ROW * k + 2 * t, x[k], x[32 + k]);
            w64::twiddle<true>(x, tm);
            dft32<true>(x);
            dft32<true>(x + 32);
            // x[k] -> time 64 k + 2 t, x[32 + k] -> 64 k + 2 t + 1
            float2 *dst = y + (size_t)f * (size_t)Nout + obase;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int n = 64 * k + 2 * t;
                const bool v0 = (unsigned)(n - lo) < (unsigned)span;
                const bool v1 = (unsigned)(n + 1 - lo) < (unsigned)span;
                if (pair_aligned && v0 && v1) {
                    *reinterpret_cast<float4 *>(dst + n) = make_float4(x[k].x, x[k].y, x[32 + k].x, x[32 + k].y);
                } else {
                    if (v0) dst[n] = x[k];
                    if (v1) dst[n + 1] = x[32 + k];
                }
            }
        }
    }
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (warp == 0) tmem::dealloc(tbase, NCOLS);
}

cudaError_t w64_prepare(ols_plan_s &p) {
    cudaError_t e = cudaFuncSetAttribute(ols_w64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)w64::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = resident_blocks_tmem(ols_w64_kernel, w64::THREADS, w64::SMEM, (int)w64::NCOLS, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.w64_grid_cap = per_sm * p.sm_count;
    return cudaSuccess;
}

cudaError_t w64_launch(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y, int64_t L, int64_t nseg,
                       int64_t Nout, cudaStream_t st) {
    const int64_t nblk = (nseg + w64::WARPS - 1) / w64::WARPS;
    const int grid = (int)(nblk < p.w64_grid_cap ? nblk : p.w64_grid_cap);
    ols_w64_kernel<<<grid, w64::THREADS, w64::SMEM, st>>>(s, Ns, reinterpret_cast<const float4 *>(p.Hk_w64),
                                                          p.tw_w64, y, p.M, p.F, L, nseg, Nout);
    return cudaGetLastError();
}

}  // namespace ols
