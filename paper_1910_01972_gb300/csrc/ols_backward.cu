// ols_backward.cu -- adjoint of the fused OLS convolution (FP32).
//
// The paper has no backward pass; this is the adjoint of the valid-mode
// convolution of Eq. 1, which Sec. 3.2's OLS evaluates.  With the gradient
// convention g = dL/dRe y + i dL/dIm y:
//   ds[m]   = sum_f sum_k g_f[m-M+1+k] conj(h_f[k])
//   dh_f[k] = sum_j g_f[j] conj(s[j+M-1-k])
//
// Both are computed window by window with the same FFT machinery as the
// forward kernel.  Window i covers output indices j in [iL, iL+L) (L = N-M+1,
// non-overlapping) and the signal segment a = s[iL, iL+N):
//   b_f  = g_f[iL, iL+L) zero-padded to N          B_f = FFT(b_f)
//   A    = FFT(a)   (recomputed, never stored)
//   dh_f[k] = sum_i IFFT(B_f^(i) conj(A^(i)))[(k + L) mod N]   (k < M: no wrap-around)
//   ds over [iL, iL+N) = IFFT(sum_f B_f Ht_f),  Ht_f = FFT(conj(h_f[M-1-.]))/N
// (the last is a linear convolution of support L + M - 1 = N, so no
// aliasing).  The inverse FFT is linear, so the sum over windows of dh is
// taken in the frequency domain: each CTA accumulates
// P_f = sum over its windows of B_f conj(A), and one inverse FFT per filter
// at the end gives dh.  Per window that is F + 2 FFTs (A, the F gradient
// windows, one inverse for ds) instead of the 2F + 2 of a per-window dh.
//
// Kernel shape: a CTA of BwdGeo::BLOCK threads holds BwdGeo::SLOTS windows
// (one per N/16-thread slot); a slot's FFT exchanges synchronise that slot
// only (named barrier), and once per filter the slots' products B_f conj(A)
// are summed in shared memory in slot order and added to the CTA's P_f in
// the workspace (L2-resident: grid x F x N complex).  Consecutive ds windows
// overlap by M-1 samples: each window writes its exclusive middle [M-1, L)
// directly and its first and last M-1 samples to a workspace; a second
// kernel adds the overlaps and sums the CTAs' P_f in CTA order with
// compensated FP32 summation; a third runs the F inverse FFTs.  The result
// is deterministic for a given plan and device.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_fft_passes.cuh"
#include "ols_internal.h"
#include "tmem.cuh"

#ifndef OLS_BWD_BLOCK
#define OLS_BWD_BLOCK 512        // threads per adjoint CTA (slots of N/16 threads), one CTA per SM ...
#endif
#ifndef OLS_BWD_BLOCK_1024
#define OLS_BWD_BLOCK_1024 256   // ... except for N = 1024: two CTAs of 256 per SM (measured)
#endif
#ifndef OLS_BWD_MINB_1024
#define OLS_BWD_MINB_1024 2
#endif
#ifndef OLS_BWD_L2HINTS
#define OLS_BWD_L2HINTS 1        // streamed s and g loads evict first, the per-CTA dh spectra evict last
#endif
#ifndef OLS_BWD_TW_TMEM
#define OLS_BWD_TW_TMEM OLS_FWD_TW_TMEM   // twiddles and the window's signal spectrum A in TMEM
#endif
#ifndef OLS_BWD_PREFETCH
#define OLS_BWD_PREFETCH 1       // pull the next gradient window toward L2 while this one is transformed
#endif

#ifndef OLS_BWD_XCHG
#define OLS_BWD_XCHG 0
#endif

namespace ols {

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 eviction priorities: the signal and gradient are read once and stream
// through L2 (evict first); the CTAs' dh spectra (grid x F x N complex) are
// updated once per window and should stay resident (evict last).
struct L2Hints {
    uint64_t stream, keep;
    __device__ __forceinline__ static L2Hints make() {
        L2Hints h;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(h.stream));
        asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(h.keep));
        return h;
    }
};

__device__ __forceinline__ float2 ld_stream(const float2 *p, const L2Hints &h) {
#if OLS_BWD_L2HINTS
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(p), "l"(h.stream));
    return v;
#else
    (void)h;
    return __ldg(p);
#endif
}

// *p += v without waiting for the old value (an L2 reduction).  Only one
// thread ever updates a given entry and its updates to one address are
// applied in program order, so the sum is deterministic; IEEE round to
// nearest like an FP32 add.
__device__ __forceinline__ void red_add(float4 *p, float4 v, const L2Hints &h) {
#if OLS_BWD_L2HINTS
    asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(h.keep)
                 : "memory");
#else
    (void)h;
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
#endif
}

__device__ __forceinline__ void st_keep(float4 *p, float4 v, const L2Hints &h) {
#if OLS_BWD_L2HINTS
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(h.keep)
                 : "memory");
#else
    (void)h;
    *p = v;
#endif
}

template <int LOG2N>
struct BwdGeo {
    using G = Geo<LOG2N>;
    static constexpr int TARGET = G::T == 64 ? OLS_BWD_BLOCK_1024 : OLS_BWD_BLOCK;
    static constexpr int MINB = G::T == 64 ? OLS_BWD_MINB_1024 : 1;   // CTAs per SM for the register budget
    static constexpr int SLOTS = TARGET / G::T > 1 ? TARGET / G::T : 1;
    static constexpr int BLOCK = SLOTS * G::T;
    static_assert(SLOTS <= 15 || G::T <= 32, "one named barrier per slot");
    static constexpr int HALF = G::N / 2;      // float4 entries of one spectrum
    // exchange buffers of every slot, then each slot's signal spectrum A (in
    // TMEM instead with OLS_BWD_TW_TMEM)
    static constexpr size_t XBYTES = sizeof(float2) * (size_t)SLOTS * G::XBUFS * G::PADN;
    static constexpr size_t SMEM = XBYTES + (OLS_BWD_TW_TMEM ? 0 : sizeof(float4) * (size_t)SLOTS * HALF);
    static constexpr uint32_t TMEM_COLS = (uint32_t)(BLOCK / 128) * 128u;   // a 128-column lane range per 128 threads
    static_assert(G::XBUFS == 2, "the product buffer is the exchange buffer not in use");
};

template <int LOG2N, bool WANT_DS, bool WANT_DH>
__global__ void __launch_bounds__(BwdGeo<LOG2N>::BLOCK, BwdGeo<LOG2N>::MINB)
ols_backward_kernel(const float2 *__restrict__ sig, long long Ns, const float2 *__restrict__ g,
                    long long Nout, const float4 *__restrict__ Htk, const float2 *__restrict__ twg,
                    float2 *__restrict__ ds, float2 *__restrict__ edge, float4 *__restrict__ P,
                    int M, int F, long long L, long long nseg, int *status) {
    using G = Geo<LOG2N>;
    using BG = BwdGeo<LOG2N>;
    extern __shared__ float4 smem_raw[];
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *const xbase = reinterpret_cast<float2 *>(smem_raw);
    float2 *bufs = xbase + slot * G::XBUFS * G::PADN;
    const SegmentBarrier<G::T> bar{1 + slot};
#if OLS_BWD_TW_TMEM
    // the forward kernel's TMEM layout: the thread's twiddles, then (columns
    // 96..127) the window's signal spectrum A, in its own lane
    __shared__ uint32_t tbase;
    if (threadIdx.x < 32) tmem::alloc(&tbase, BG::TMEM_COLS);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    // without the TMEM exchange: with it the N = 1024 adjoint takes 0.248 ms
    // instead of 0.239 ms (72 bytes of spills), and the N = 2048 one spills more
    constexpr bool xch = OLS_BWD_XCHG && LOG2N == 10;
    const TwTmemT<xch> tw{tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 128u};
    tw_tmem_fill<LOG2N, xch>(twg, tw.base, t);
    const uint32_t acol = tw.base + 96;
#else
    float4 *Asm = reinterpret_cast<float4 *>(reinterpret_cast<char *>(smem_raw) + BG::XBYTES) + slot * BG::HALF;
    const TwGlobal tw{twg};
#endif
    const L2Hints l2 = L2Hints::make();
    const int lo = M - 1;
    const int Li = (int)L;
    float4 *Pc = WANT_DH ? P + (size_t)blockIdx.x * F * BG::HALF : nullptr;
    int xc = 0;
    const long long nblk = (nseg + BG::SLOTS - 1) / BG::SLOTS;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const bool first = blk == blockIdx.x;
        const long long seg = blk * BG::SLOTS + slot;
        const bool active = seg < nseg;
        const long long start = active ? seg * L : 0;

        if constexpr (WANT_DH) {
            float2 A[16];
            const long long avail = active ? (Ns - start) : 0;
            const int lim = (int)(avail < G::N ? avail : G::N);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                A[k] = (k * G::T + t < lim && in_bounds(start + k * G::T + t < Ns, status))
                           ? ld_stream(sig + start + k * G::T + t, l2)
                           : make_float2(0.f, 0.f);
            forward_passes<LOG2N, 0>(A, bufs, tw, t, xc, bar);
#if OLS_BWD_TW_TMEM
            tmem::st32(acol, reinterpret_cast<const float *>(A));
            tmem::wait_st();
#else
            // kept in shared memory (the thread's own entries) rather than 32 registers
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2)
                Asm[j2 * G::T + t] = make_float4(A[2 * j2].x, A[2 * j2].y, A[2 * j2 + 1].x, A[2 * j2 + 1].y);
#endif
        }
        float2 D[16];
        if constexpr (WANT_DS) {
#pragma unroll
            for (int k = 0; k < 16; ++k) D[k] = make_float2(0.f, 0.f);
        }
        // valid gradient samples of this window: j in [start, start + gl)
        const long long grem = active ? (Nout - start) : 0;
        const int gl = (int)(grem < L ? grem : L);

        for (int f = 0; f < F; ++f) {
            float2 b[16];
            const float2 *gf = g + (size_t)f * (size_t)Nout + start + t;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                b[k] = (k * G::T + t < gl && in_bounds(start + k * G::T + t < Nout, status))
                           ? ld_stream(gf + k * G::T, l2)
                           : make_float2(0.f, 0.f);
#if OLS_BWD_PREFETCH
            // a window is at most N/16 = T lines of 128 B: one line per thread
            if (f + 1 < F) {
                if (t * 16 < gl) prefetch_l2(gf - t + Nout + t * 16);
            } else {   // the last filter: the slot's next window (signal and first gradient row)
                const long long nstart = (seg + (long long)gridDim.x * BG::SLOTS) * L + t * 16;
                if (WANT_DH && nstart < Ns) prefetch_l2(sig + nstart);
                if (nstart < Nout) prefetch_l2(g + nstart);
            }
#endif
            forward_passes<LOG2N, 0>(b, bufs, tw, t, xc, bar);
            if constexpr (WANT_DS) {
                const float4 *hp = Htk + (size_t)f * BG::HALF + t;
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2) {
                    const float4 h = in_bounds((long long)f * BG::HALF + j2 * G::T + t < (long long)F * BG::HALF,
                                               status)
                                         ? load_spectrum(hp + j2 * G::T)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                    D[2 * j2] = cadd(D[2 * j2], cmul(b[2 * j2], make_float2(h.x, h.y)));
                    D[2 * j2 + 1] = cadd(D[2 * j2 + 1], cmul(b[2 * j2 + 1], make_float2(h.z, h.w)));
                }
            }
            if constexpr (WANT_DH) {
                // B_f conj(A) at this thread's storage positions 16 t + j (entries j2 T + t)
                float4 q[8];
#if OLS_BWD_TW_TMEM
#pragma unroll
                for (int h = 0; h < 2; ++h) {               // A in two 16-column halves
                    float a[16];
                    tmem::ld16(acol + 16 * h, a);
                    tmem::wait_ld();
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int j2 = 4 * h + i;
                        const float2 q0 = cmulc(b[2 * j2], make_float2(a[4 * i], a[4 * i + 1]));
                        const float2 q1 = cmulc(b[2 * j2 + 1], make_float2(a[4 * i + 2], a[4 * i + 3]));
                        q[j2] = make_float4(q0.x, q0.y, q1.x, q1.y);
                    }
                }
#else
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2) {
                    const float4 a = Asm[j2 * G::T + t];
                    const float2 q0 = cmulc(b[2 * j2], make_float2(a.x, a.y));
                    const float2 q1 = cmulc(b[2 * j2 + 1], make_float2(a.z, a.w));
                    q[j2] = make_float4(q0.x, q0.y, q1.x, q1.y);
                }
#endif
                float4 *Pf = Pc + (size_t)f * BG::HALF;
                if constexpr (BG::SLOTS == 1) {
#pragma unroll
                    for (int j2 = 0; j2 < 8; ++j2) {
                        float4 *dst = Pf + j2 * G::T + t;
                        if (!in_bounds(j2 * G::T + t < BG::HALF, status)) continue;
                        if (first) st_keep(dst, q[j2], l2);
                        else red_add(dst, q[j2], l2);
                    }
                } else {
                    // the slots' products summed in slot order, then added to the CTA's P_f.
                    // Staged in each slot's exchange buffer that the next exchange writes
                    // (xc & 1): its last readers are past this FFT's final exchange, and
                    // its next writer comes after the second barrier below.
                    float4 *prod = reinterpret_cast<float4 *>(xbase + (xc & 1) * G::PADN);
                    constexpr int SSTRIDE = G::XBUFS * G::PADN / 2;   // float4 between slots
#pragma unroll
                    for (int j2 = 0; j2 < 8; ++j2) prod[slot * SSTRIDE + j2 * G::T + t] = q[j2];
                    __syncthreads();
                    for (int e = threadIdx.x; e < BG::HALF; e += BG::BLOCK) {
                        float4 acc = prod[e];
#pragma unroll
                        for (int s2 = 1; s2 < BG::SLOTS; ++s2) acc = f4add(acc, prod[s2 * SSTRIDE + e]);
                        if (!in_bounds(e < BG::HALF, status)) continue;
                        if (first) st_keep(Pf + e, acc, l2);
                        else red_add(Pf + e, acc, l2);
                    }
                    __syncthreads();
                }
            }
        }
        if constexpr (WANT_DS) {
            inverse_passes<LOG2N, G::NP - 1>(D, bufs, tw, t, xc, bar);
            if (active) {
                float2 *eh = edge + (size_t)seg * 2 * lo;      // head [0, lo), tail [lo, 2 lo)
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int u = k * G::T + t;
                    if (u < lo) {
                        eh[u] = D[k];
                    } else if (u >= Li) {
                        if (in_bounds(u - Li < lo, status)) eh[lo + (u - Li)] = D[k];
                    } else if (start + u < Ns) {
                        ds[start + u] = D[k];
                    }
                }
            }
        }
    }
#if OLS_BWD_TW_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, BG::TMEM_COLS);
#endif
}

// ds overlaps: ds[b L + u] = head_b[u] + tail_{b-1}[u] for b in [0, nseg],
// u < M-1.  dh spectra: Pr[e] = compensated sum of the CTAs' P[c][e] in a
// fixed order (e over F x N/2 float4 entries).
__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
    const float y = v - c;
    const float tt = s + y;
    c = (tt - s) - y;
    s = tt;
}

constexpr int kFinishLanes = 8;   // threads per dh spectrum entry in the finishing sum

__global__ void __launch_bounds__(256)
ols_backward_finish_kernel(const float2 *__restrict__ edge, float2 *__restrict__ ds, long long Ns, long long L,
                           long long nseg, int M, const float4 *__restrict__ P, int npart,
                           float4 *__restrict__ Pr, long long FH, int *status) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nred = Pr ? FH * kFinishLanes : 0;
    if (gid < nred) {
        // lane r of entry e sums the partials p = r, r + 8, ... (compensated); the
        // 8 lanes' sums are then added in lane order, also compensated
        const long long e = gid / kFinishLanes;
        const int r = (int)(gid % kFinishLanes);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll 4
        for (int p = r; p < npart; p += kFinishLanes) {
            const float4 v = __ldcs(P + (size_t)p * FH + e);
            kahan_add(s0, c0, v.x);
            kahan_add(s1, c1, v.y);
            kahan_add(s2, c2, v.z);
            kahan_add(s3, c3, v.w);
        }
        // the 8 lanes of an entry are consecutive threads of one warp (nred is a
        // multiple of 8 and warps start at multiples of 32)
        const unsigned base = threadIdx.x & 31u & ~(unsigned)(kFinishLanes - 1);
        const unsigned grp = ((1u << kFinishLanes) - 1u) << base;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f, d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
        for (int q = 0; q < kFinishLanes; ++q) {
            const int src = (int)base + q;
            kahan_add(t0, d0, __shfl_sync(grp, s0, src) - __shfl_sync(grp, c0, src));
            kahan_add(t1, d1, __shfl_sync(grp, s1, src) - __shfl_sync(grp, c1, src));
            kahan_add(t2, d2, __shfl_sync(grp, s2, src) - __shfl_sync(grp, c2, src));
            kahan_add(t3, d3, __shfl_sync(grp, s3, src) - __shfl_sync(grp, c3, src));
        }
        if (r == 0) Pr[e] = make_float4(t0, t1, t2, t3);
        return;
    }
    const long long e = gid - nred;
    const int lo = M - 1;
    if (!ds || lo == 0 || e < 0 || e >= (nseg + 1) * (long long)lo) return;
    const long long b = e / lo;
    const int u = (int)(e % lo);
    const long long m = b * L + u;
    if (m >= Ns || !in_bounds(m >= 0 && b <= nseg, status)) return;
    float2 v = make_float2(0.f, 0.f);
    if (b < nseg) v = edge[(size_t)b * 2 * lo + u];
    if (b > 0) {
        const float2 w = edge[(size_t)(b - 1) * 2 * lo + lo + u];
        v = make_float2(v.x + w.x, v.y + w.y);
    }
    ds[m] = v;
}

// dh_f[k] = IFFT(Pr_f)[(k + L) mod N] / N for k < M: one slot per filter.
template <int LOG2N>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK)
ols_backward_dh_kernel(const float4 *__restrict__ Pr, const float2 *__restrict__ twg, float2 *__restrict__ dh,
                       int M, int F, long long L) {
    using G = Geo<LOG2N>;
    extern __shared__ float4 smem_raw[];
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *bufs = reinterpret_cast<float2 *>(smem_raw) + slot * G::XBUFS * G::PADN;
    const int f = blockIdx.x * G::SEGS + slot;
    const bool active = f < F;
    float2 x[16];
    const float4 *src = Pr + (size_t)(active ? f : 0) * (G::N / 2) + t;
#pragma unroll
    for (int j2 = 0; j2 < 8; ++j2) {
        const float4 v = active ? src[j2 * G::T] : make_float4(0.f, 0.f, 0.f, 0.f);
        x[2 * j2] = make_float2(v.x, v.y);
        x[2 * j2 + 1] = make_float2(v.z, v.w);
    }
    int xc = 0;
    inverse_passes<LOG2N, G::NP - 1>(x, bufs, TwGlobal{twg}, t, xc);
    if (!active) return;
    const float invN = 1.0f / (float)G::N;
    const int Li = (int)L;
    float2 *dst = dh + (size_t)f * M;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int n = k * G::T + t;           // x[k] holds c[n]
        int kk = -1;
        if (n >= Li) kk = n - Li;
        else if (n == 0) kk = M - 1;
        if (kk >= 0) dst[kk] = make_float2(x[k].x * invN, x[k].y * invN);
    }
}

template <int LOG2N, bool DS, bool DH>
static cudaError_t prepare_bwd_one(ols_plan_s &p, int idx) {
    using BG = BwdGeo<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute(ols_backward_kernel<LOG2N, DS, DH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BG::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_BWD_TW_TMEM)
        e = resident_blocks_tmem(ols_backward_kernel<LOG2N, DS, DH>, BG::BLOCK, BG::SMEM, (int)BG::TMEM_COLS, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_backward_kernel<LOG2N, DS, DH>, BG::BLOCK,
                                                          BG::SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    p.bwd_grid_cap[idx] = per_sm * p.sm_count;
    return cudaSuccess;
}

template <int LOG2N>
static cudaError_t prepare_bwd_n(ols_plan_s &p) {
    cudaError_t e = prepare_bwd_one<LOG2N, true, true>(p, 0);
    if (e == cudaSuccess) e = prepare_bwd_one<LOG2N, true, false>(p, 1);
    if (e == cudaSuccess) e = prepare_bwd_one<LOG2N, false, true>(p, 2);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ols_backward_dh_kernel<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)Geo<LOG2N>::SMEM);
    return e;
}

cudaError_t prepare_backward(ols_plan_s &p) {
    switch (p.log2N) {
        case 8: return prepare_bwd_n<8>(p);
        case 9: return prepare_bwd_n<9>(p);
        case 10: return prepare_bwd_n<10>(p);
        case 11: return prepare_bwd_n<11>(p);
        case 12: return prepare_bwd_n<12>(p);
        case 13: return prepare_bwd_n<13>(p);
        default: return cudaErrorInvalidValue;
    }
}

int backward_segs_per_block(int log2N) {
    switch (log2N) {
        case 8: return BwdGeo<8>::SLOTS;
        case 9: return BwdGeo<9>::SLOTS;
        case 10: return BwdGeo<10>::SLOTS;
        case 11: return BwdGeo<11>::SLOTS;
        case 12: return BwdGeo<12>::SLOTS;
        case 13: return BwdGeo<13>::SLOTS;
        default: return 1;
    }
}

int backward_grid(const ols_plan_s &p, int64_t nseg, bool want_ds, bool want_dh) {
    const int idx = want_ds ? (want_dh ? 0 : 1) : 2;
    const int segs = backward_segs_per_block(p.log2N);
    const int64_t nblk = (nseg + segs - 1) / segs;
    return (int)(nblk < p.bwd_grid_cap[idx] ? nblk : p.bwd_grid_cap[idx]);
}

template <int LOG2N, bool DS, bool DH>
static void launch_bwd_one(const ols_plan_s &p, const BackwardArgs &a, cudaStream_t st) {
    using BG = BwdGeo<LOG2N>;
    ols_backward_kernel<LOG2N, DS, DH><<<a.grid, BG::BLOCK, BG::SMEM, st>>>(
        a.s, a.Ns, a.g, a.Nout, reinterpret_cast<const float4 *>(p.Htk), p.tw, a.ds, a.edge, a.P, p.M, p.F, a.L,
        a.nseg, p.d_status);
}

template <int LOG2N>
static void launch_bwd_n(const ols_plan_s &p, const BackwardArgs &a, cudaStream_t st) {
    if (a.ds && a.dh) launch_bwd_one<LOG2N, true, true>(p, a, st);
    else if (a.ds) launch_bwd_one<LOG2N, true, false>(p, a, st);
    else launch_bwd_one<LOG2N, false, true>(p, a, st);
}

template <int LOG2N>
static void launch_dh_n(const ols_plan_s &p, const BackwardArgs &a, cudaStream_t st) {
    using G = Geo<LOG2N>;
    const int grid = (p.F + G::SEGS - 1) / G::SEGS;
    ols_backward_dh_kernel<LOG2N><<<grid, G::BLOCK, G::SMEM, st>>>(a.Pr, p.tw, a.dh, p.M, p.F, a.L);
}

cudaError_t launch_backward(const ols_plan_s &p, const BackwardArgs &a, cudaStream_t st, int *launches) {
    *launches = 0;
    switch (p.log2N) {
        case 8: launch_bwd_n<8>(p, a, st); break;
        case 9: launch_bwd_n<9>(p, a, st); break;
        case 10: launch_bwd_n<10>(p, a, st); break;
        case 11: launch_bwd_n<11>(p, a, st); break;
        case 12: launch_bwd_n<12>(p, a, st); break;
        case 13: launch_bwd_n<13>(p, a, st); break;
        default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *launches = 1;
    const long long FH = a.dh ? (long long)p.F * (p.N / 2) : 0;
    const long long nfix = a.ds ? (a.nseg + 1) * (long long)(p.M - 1) : 0;
    const long long total = FH * kFinishLanes + nfix;
    if (total > 0) {
        ols_backward_finish_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            a.edge, a.ds, a.Ns, a.L, a.nseg, p.M, a.P, a.grid, a.dh ? a.Pr : nullptr, FH, p.d_status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches = 2;
    }
    if (a.dh) {
        switch (p.log2N) {
            case 8: launch_dh_n<8>(p, a, st); break;
            case 9: launch_dh_n<9>(p, a, st); break;
            case 10: launch_dh_n<10>(p, a, st); break;
            case 11: launch_dh_n<11>(p, a, st); break;
            case 12: launch_dh_n<12>(p, a, st); break;
            case 13: launch_dh_n<13>(p, a, st); break;
            default: return cudaErrorInvalidValue;
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches = 3;
    }
    return cudaSuccess;
}

}  // namespace ols
