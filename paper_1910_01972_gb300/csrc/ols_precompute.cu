// ols_precompute.cu -- plan-time FP64 kernels: the twiddle table W_N^m and
// the filter spectra (Algorithms 1 and 2, "forward FFT of the filters",
// done once before the convolution kernel; Fig. 1's first step).
//
// FP64 is used only here, off the convolution path: every exponent is
// reduced exactly in integers ((nu * k) mod N) before the table lookup, so
// each spectrum value is a correctly accumulated FP64 sum rounded once to
// FP32.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_internal.h"

namespace ols {

__global__ void tw64_kernel(double2 *tw64, int N) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= N) return;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)N, &sn, &cs);   // argument exact: N is a power of two
    tw64[m] = make_double2(cs, -sn);                     // exp(-2 pi i m / N)
}

// H[f][nu] = (1/N) sum_{k<M} h_f[k] W_N^{nu k}, written at storage position
// q (nu = nu_tab[q]) in the kernel's register layout: thread t = q / 16 holds
// register j = q % 16, and registers (2i, 2i+1) of all threads of a segment
// are interleaved so one 16-byte load fetches a pair.
// With adjoint != 0 the transformed filter is conj(h_f[M-1-k]) (the adjoint
// of the convolution correlates with h).
__global__ void spectra_kernel(const float2 *__restrict__ h, int M, int F, int log2N,
                               const int32_t *__restrict__ nu_tab, const double2 *__restrict__ tw64,
                               float2 *__restrict__ Hk, int adjoint) {
    const int N = 1 << log2N;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)F * N) return;
    const int f = (int)(gid >> log2N);
    const int q = (int)(gid & (N - 1));
    const long long nu = nu_tab[q];
    const float2 *hf = h + (size_t)f * M;
    double ar = 0.0, ai = 0.0;
    for (int k = 0; k < M; ++k) {
        const double2 w = tw64[(nu * k) & (N - 1)];
        float2 hk = hf[adjoint ? (M - 1 - k) : k];
        if (adjoint) hk.y = -hk.y;
        ar = fma((double)hk.x, w.x, fma(-(double)hk.y, w.y, ar));
        ai = fma((double)hk.x, w.y, fma((double)hk.y, w.x, ai));
    }
    const double inv = 1.0 / (double)N;
    const int T = N / 16, t = q >> 4, j = q & 15;
    const size_t idx = (size_t)f * N + (size_t)(j >> 1) * (2 * T) + 2 * t + (j & 1);
    Hk[idx] = make_float2((float)(ar * inv), (float)(ai * inv));
}

// Natural-order copy of the plan's spectra: H[f][nu_tab[q]] = Hk[f][layout(q)].
__global__ void spectra_natural_kernel(const float2 *__restrict__ Hk, int F, int log2N,
                                       const int32_t *__restrict__ nu_tab, float2 *__restrict__ H) {
    const int N = 1 << log2N;
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (long long)F * N) return;
    const int f = (int)(gid >> log2N);
    const int q = (int)(gid & (N - 1));
    const int T = N / 16, t = q >> 4, j = q & 15;
    const size_t idx = (size_t)f * N + (size_t)(j >> 1) * (2 * T) + 2 * t + (j & 1);
    H[(size_t)f * N + nu_tab[q]] = Hk[idx];
}

cudaError_t launch_tw64(double2 *tw64, int N, cudaStream_t st) {
    tw64_kernel<<<(N + 255) / 256, 256, 0, st>>>(tw64, N);
    return cudaGetLastError();
}

cudaError_t launch_spectra(const float2 *h, int M, int F, int log2N, const int32_t *nu,
                           const double2 *tw64, float2 *Hk, int adjoint, cudaStream_t st) {
    const long long total = (long long)F << log2N;
    spectra_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(h, M, F, log2N, nu, tw64, Hk, adjoint);
    return cudaGetLastError();
}

cudaError_t launch_spectra_natural(const float2 *Hk, int F, int log2N, const int32_t *nu, float2 *H,
                                   cudaStream_t st) {
    const long long total = (long long)F << log2N;
    spectra_natural_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Hk, F, log2N, nu, H);
    return cudaGetLastError();
}

}  // namespace ols
