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
//   dh_f^(i)[k] = IFFT(B_f conj(A))[(k + L) mod N]   (k < M: no wrap-around)
//   ds over [iL, iL+N) = IFFT(sum_f B_f Ht_f),  Ht_f = FFT(conj(h_f[M-1-.]))/N
// (the last is a linear convolution of support L + M - 1 = N, so no
// aliasing).  2F + 2 FFTs per window.  Consecutive ds windows overlap by
// M-1 samples: each window writes its exclusive middle [M-1, L) directly and
// its first and last M-1 samples to a workspace; a second kernel adds the
// overlaps.  dh is accumulated per (block, slot) over that slot's windows in
// a workspace and summed by the second kernel in a fixed order with
// compensated FP32 summation: the result is deterministic for a given plan
// and device.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_fft_passes.cuh"
#include "ols_internal.h"

#ifndef OLS_BWD_WARPS_PER_SM
#define OLS_BWD_WARPS_PER_SM 8   // the adjoint keeps three spectra in registers: fewer, fatter warps
#endif

namespace ols {

template <int LOG2N>
struct BwdGeo {
    static constexpr int MINB = (OLS_BWD_WARPS_PER_SM * 32 + Geo<LOG2N>::BLOCK - 1) / Geo<LOG2N>::BLOCK;
};

template <int LOG2N, bool WANT_DS, bool WANT_DH>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK, BwdGeo<LOG2N>::MINB)
ols_backward_kernel(const float2 *__restrict__ sig, long long Ns, const float2 *__restrict__ g,
                    long long Nout, const float4 *__restrict__ Htk, const float2 *__restrict__ twg,
                    float2 *__restrict__ ds, float2 *__restrict__ edge, float2 *__restrict__ dh_part,
                    int M, int F, long long L, long long nseg) {
    using G = Geo<LOG2N>;
    extern __shared__ float4 smem_raw[];
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *bufs = smem + G::TWN_PAD + slot * G::XBUFS * G::PADN;
#if OLS_TW_GLOBAL
    const float2 *tw = twg;
#else
    float2 *tw = smem;
    for (int i = threadIdx.x; i < G::TWN; i += G::BLOCK) tw[i] = twg[i];
    __syncthreads();
#endif
    const int lo = M - 1;
    const int Li = (int)L;
    const float invN = 1.0f / (float)G::N;
    float2 *dhp = WANT_DH ? dh_part + ((size_t)blockIdx.x * G::SEGS + slot) * (size_t)F * M : nullptr;
    int xc = 0;
    const long long nblk = (nseg + G::SEGS - 1) / G::SEGS;
    for (long long blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const bool first = blk == blockIdx.x;
        const long long seg = blk * G::SEGS + slot;
        const bool active = seg < nseg;
        const long long start = active ? seg * L : 0;

        float2 A[16];
        if constexpr (WANT_DH) {
            const long long avail = active ? (Ns - start) : 0;
            const int lim = (int)(avail < G::N ? avail : G::N);
#pragma unroll
            for (int k = 0; k < 16; ++k)
                A[k] = (k * G::T + t < lim) ? __ldg(sig + start + k * G::T + t) : make_float2(0.f, 0.f);
            forward_passes<LOG2N, 0>(A, bufs, tw, t, xc);
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
            for (int k = 0; k < 16; ++k) b[k] = (k * G::T + t < gl) ? __ldg(gf + k * G::T) : make_float2(0.f, 0.f);
            forward_passes<LOG2N, 0>(b, bufs, tw, t, xc);
            if constexpr (WANT_DS) {
                const float4 *hp = Htk + (size_t)f * (G::N / 2) + t;
#pragma unroll
                for (int j2 = 0; j2 < 8; ++j2) {
                    const float4 h = load_spectrum(hp + j2 * G::T);
                    const float2 p0 = cmul(b[2 * j2], make_float2(h.x, h.y));
                    const float2 p1 = cmul(b[2 * j2 + 1], make_float2(h.z, h.w));
                    D[2 * j2] = cadd(D[2 * j2], p0);
                    D[2 * j2 + 1] = cadd(D[2 * j2 + 1], p1);
                }
            }
            if constexpr (WANT_DH) {
#pragma unroll
                for (int j = 0; j < 16; ++j) b[j] = cmulc(b[j], A[j]);
                inverse_passes<LOG2N, G::NP - 1>(b, bufs, tw, t, xc);
                // b[k] holds c[n], n = k T + t;  dh_f[n - L] for n >= L, dh_f[M-1] for n = 0
                float2 *dst = dhp + (size_t)f * M;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    int kk = -1;
                    if (n >= Li) kk = n - Li;
                    else if (n == 0) kk = lo;
                    if (active && kk >= 0) {
                        const float2 v = make_float2(b[k].x * invN, b[k].y * invN);
                        dst[kk] = first ? v : cadd(dst[kk], v);
                    }
                }
            }
        }
        if constexpr (WANT_DS) {
            inverse_passes<LOG2N, G::NP - 1>(D, bufs, tw, t, xc);
            if (active) {
                float2 *eh = edge + (size_t)seg * 2 * lo;      // head [0, lo), tail [lo, 2 lo)
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int u = k * G::T + t;
                    if (u < lo) {
                        eh[u] = D[k];
                    } else if (u >= Li) {
                        eh[lo + (u - Li)] = D[k];
                    } else if (start + u < Ns) {
                        ds[start + u] = D[k];
                    }
                }
            }
        }
    }
}

// ds overlaps: ds[b L + u] = head_b[u] + tail_{b-1}[u] for b in [0, nseg],
// u < M-1.  dh: compensated sum of the per-slot partials in slot order.
__global__ void ols_backward_finish_kernel(const float2 *__restrict__ edge, float2 *__restrict__ ds, long long Ns,
                                           long long L, long long nseg, int M, const float2 *__restrict__ dh_part,
                                           int npart, float2 *__restrict__ dh, int FM) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (dh && gid < FM) {
        float sr = 0.f, si = 0.f, cr = 0.f, ci = 0.f;
        for (int p = 0; p < npart; ++p) {
            const float2 v = dh_part[(size_t)p * FM + gid];
            const float yr = v.x - cr, yi = v.y - ci;
            const float tr = sr + yr, ti = si + yi;
            cr = (tr - sr) - yr;
            ci = (ti - si) - yi;
            sr = tr;
            si = ti;
        }
        dh[gid] = make_float2(sr, si);
        return;
    }
    const long long e = gid - (dh ? FM : 0);
    const int lo = M - 1;
    if (!ds || lo == 0 || e < 0 || e >= (nseg + 1) * (long long)lo) return;
    const long long b = e / lo;
    const int u = (int)(e % lo);
    const long long m = b * L + u;
    if (m >= Ns) return;
    float2 v = make_float2(0.f, 0.f);
    if (b < nseg) v = edge[(size_t)b * 2 * lo + u];
    if (b > 0) {
        const float2 w = edge[(size_t)(b - 1) * 2 * lo + lo + u];
        v = make_float2(v.x + w.x, v.y + w.y);
    }
    ds[m] = v;
}

template <int LOG2N, bool DS, bool DH>
static cudaError_t prepare_bwd_one(ols_plan_s &p, int idx) {
    using G = Geo<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute(ols_backward_kernel<LOG2N, DS, DH>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_backward_kernel<LOG2N, DS, DH>, G::BLOCK,
                                                      G::SMEM);
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
        case 8: return Geo<8>::SEGS;
        case 9: return Geo<9>::SEGS;
        case 10: return Geo<10>::SEGS;
        case 11: return Geo<11>::SEGS;
        case 12: return Geo<12>::SEGS;
        case 13: return Geo<13>::SEGS;
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
    using G = Geo<LOG2N>;
    ols_backward_kernel<LOG2N, DS, DH><<<a.grid, G::BLOCK, G::SMEM, st>>>(
        a.s, a.Ns, a.g, a.Nout, reinterpret_cast<const float4 *>(p.Htk), p.tw, a.ds, a.edge, a.dh_part, p.M,
        p.F, a.L, a.nseg);
}

template <int LOG2N>
static void launch_bwd_n(const ols_plan_s &p, const BackwardArgs &a, cudaStream_t st) {
    if (a.ds && a.dh) launch_bwd_one<LOG2N, true, true>(p, a, st);
    else if (a.ds) launch_bwd_one<LOG2N, true, false>(p, a, st);
    else launch_bwd_one<LOG2N, false, true>(p, a, st);
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
    const int FM = a.dh ? p.F * p.M : 0;
    const long long nfix = a.ds ? (a.nseg + 1) * (long long)(p.M - 1) : 0;
    const long long total = FM + nfix;
    if (total > 0) {
        ols_backward_finish_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
            a.edge, a.ds, a.Ns, a.L, a.nseg, p.M, a.dh_part, a.npart, a.dh, FM);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        *launches = 2;
    }
    return cudaSuccess;
}

}  // namespace ols
