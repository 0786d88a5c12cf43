// ols_forward.cu -- the fused overlap-and-save convolution kernel (FP32).
//
// Algorithm 2 / Sec. 3.4 of the paper: one kernel; a thread-block owns a
// segment; the segment's forward FFT is done on chip and its spectrum kept
// on chip (Sec. 3.4 keeps it in registers), then for every filter: point-wise
// product with the filter's precomputed spectrum, inverse FFT, removal of
// the M-1 aliased samples, store (Sec. 3.2).
//
// GB300 design:
// * Each thread holds 16 complex points; a segment of N points uses N/16
//   threads.  The FFT is a sequence of radix-16 passes (one 16-point DFT per
//   thread, all rotations compile-time constants) plus one pass of radix
//   2/4/8/16 at stride 1.
// * Forward: decimation in frequency, natural-order input, digit-reversed
//   spectrum.  Inverse: the exact reverse of the passes (decimation in time),
//   digit-reversed input, natural-order output.  No reordering step (Sec. 3.4
//   notes the order is irrelevant to the point-wise product).
// * Tensor memory holds, in each thread's own lane, its pass twiddles and the
//   segment spectrum (read back once per filter), and stages the exchange
//   between the last two passes (N = 512 .. 4096), which stays inside a warp;
//   the exchange that crosses warps goes through padded shared memory, one
//   barrier per exchange (two alternating buffers).
// * The filter spectra are pre-laid-out so each thread's 16 values arrive in
//   eight coalesced 16-byte loads; the next filter's spectrum is loaded while
//   the current one is transformed (except where that spills: see Geo).
// * Global loads and stores: for each register k, consecutive threads touch
//   consecutive samples (fully coalesced); the valid-output test is one
//   unsigned compare per sample.
// * Residency computed from the SM's registers, shared memory, threads and
//   TMEM columns; blocks loop over segments (persistent grid from N = 4096,
//   one block per segment block below: see fused_grid).
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_internal.h"
#include "ols_segment.cuh"

namespace ols {

template <int LOG2N>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK, Geo<LOG2N>::MINB)
ols_forward_kernel(const float2 *__restrict__ sig, long long Ns, const float4 *__restrict__ Hk,
                   const float2 *__restrict__ twg, float2 *__restrict__ y, int M, int F,
                   long long L, long long nseg, long long Nout, int *status) {
    using G = Geo<LOG2N>;
    extern __shared__ float4 smem_raw[];
    __shared__ uint32_t tbase;
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *bufs = smem + slot * G::XBUFS * G::PADN;
#if OLS_FWD_TW_TMEM
    // twiddles in TMEM: warp 0 allocates, every thread fills its own lane
    if (threadIdx.x < 32) tmem::alloc(&tbase, G::TMEM_COLS);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    const TwTmem tw{tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 128u};
    tw_tmem_fill<LOG2N>(twg, tw.base, t);
#else
    const TwGlobal tw{twg};
#if OLS_FWD_X_TMEM
    // the segment spectrum in TMEM: 32 columns per 128 threads (a thread's lane)
    if (threadIdx.x < 32) tmem::alloc(&tbase, G::XT_COLS);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    const uint32_t xcol_t = tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 32u;
#else
    (void)tbase;
    const uint32_t xcol_t = 0;
#endif
#endif
    int xc = 0;
    const long long nblk = (nseg + G::SEGS - 1) / G::SEGS;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const long long seg = blk * G::SEGS + slot;
#if OLS_FWD_TW_TMEM
        ols_segment<LOG2N>(sig, Ns, Hk, tw, y, M, F, L, Nout, seg, seg < nseg, bufs, t, xc, 0u, CtaBarrier{}, status);
#else
        ols_segment<LOG2N, TwGlobal, OLS_FWD_X_TMEM != 0>(sig, Ns, Hk, tw, y, M, F, L, Nout, seg, seg < nseg, bufs,
                                                          t, xc, xcol_t, CtaBarrier{}, status);
#endif
    }
#if OLS_FWD_X_TMEM && !OLS_FWD_TW_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, G::XT_COLS);
#endif
#if OLS_FWD_TW_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, G::TMEM_COLS);
#endif
}

template <int LOG2N>
static cudaError_t prepare_one(ols_plan_s &p) {
    using G = Geo<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute(ols_forward_kernel<LOG2N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM_TMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_FWD_TW_TMEM || OLS_FWD_X_TMEM)
        e = resident_blocks_tmem(ols_forward_kernel<LOG2N>, G::BLOCK, G::SMEM_TMEM,
                                 OLS_FWD_TW_TMEM ? (int)G::TMEM_COLS : (int)G::XT_COLS, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_forward_kernel<LOG2N>, G::BLOCK, G::SMEM_TMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (OLS_FWD_TW_TMEM && per_sm > G::TMEM_MAX_CTAS) per_sm = G::TMEM_MAX_CTAS;
    p.fwd_grid_cap = per_sm * p.sm_count;
    return cudaSuccess;
}

template <int LOG2N>
static cudaError_t launch_one(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y, int64_t L,
                              int64_t nseg, int64_t Nout, cudaStream_t st) {
    using G = Geo<LOG2N>;
    const int64_t nblk = (nseg + G::SEGS - 1) / G::SEGS;
    const int grid = fused_grid(LOG2N, nblk, p.fwd_grid_cap);
    ols_forward_kernel<LOG2N><<<grid, G::BLOCK, G::SMEM_TMEM, st>>>(
        s, Ns, reinterpret_cast<const float4 *>(p.Hk), p.tw, y, p.M, p.F, L, nseg, Nout, p.d_status);
    return cudaGetLastError();
}

cudaError_t prepare_forward(ols_plan_s &p) {
    switch (p.log2N) {
        case 8: return prepare_one<8>(p);
        case 9: return prepare_one<9>(p);
        case 10: return prepare_one<10>(p);
        case 11: return prepare_one<11>(p);
        case 12: return prepare_one<12>(p);
        case 13: return prepare_one<13>(p);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_forward(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y, int64_t L,
                           int64_t nseg, int64_t Nout, cudaStream_t st, int *launches) {
    *launches = 1;
    switch (p.log2N) {
        case 8: return launch_one<8>(p, s, Ns, y, L, nseg, Nout, st);
        case 9: return launch_one<9>(p, s, Ns, y, L, nseg, Nout, st);
        case 10: return launch_one<10>(p, s, Ns, y, L, nseg, Nout, st);
        case 11: return launch_one<11>(p, s, Ns, y, L, nseg, Nout, st);
        case 12: return launch_one<12>(p, s, Ns, y, L, nseg, Nout, st);
        case 13: return launch_one<13>(p, s, Ns, y, L, nseg, Nout, st);
        default: *launches = 0; return cudaErrorInvalidValue;
    }
}

// Host mirror of Geo<>: the twiddle tables and spectral order are built from it.
PassPlan make_pass_plan(int log2N) {
    PassPlan pp{};
    pp.log2N = log2N;
    pp.N = 1 << log2N;
    pp.T = pp.N / 16;
    pp.np = (log2N + 3) / 4;
    const int rl = (log2N % 4) ? (1 << (log2N % 4)) : 16;
    int off = 0;
    for (int p = 0; p < pp.np; ++p) {
        pp.radix[p] = (p == pp.np - 1) ? rl : 16;
        pp.stride[p] = (p == pp.np - 1) ? 1 : (pp.N >> (4 * (p + 1)));
        pp.tw_off[p] = off;
        if (p < pp.np - 1) off += 15 * pp.stride[p];
    }
    pp.twn = off;
    return pp;
}

}  // namespace ols
