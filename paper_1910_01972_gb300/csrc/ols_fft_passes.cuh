// ols_fft_passes.cuh -- the in-kernel segment FFT shared by the OLS kernels.
//
// A segment of N = 2^LOG2N complex points is transformed by N/16 threads,
// 16 points each: radix-16 passes (one 16-point DFT per thread, all
// rotations compile-time constants) followed by one pass of radix 2/4/8/16 at
// stride 1, exchanging between passes through shared memory or, for the last
// exchange of kernels with TMEM twiddles (N = 512 .. 4096), through TMEM.
// * forward passes: decimation in frequency, natural-order input, spectrum
//   left in mixed-radix digit-reversed order (no reordering step: Sec. 3.4
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
#ifndef OLS_TMEM_XCHG
#define OLS_TMEM_XCHG 1      // N = 512..4096: the exchange between the last two passes goes through TMEM (0: shared memory)
#endif
#ifndef OLS_TX_MASK
#define OLS_TX_MASK 0xF      // segment lengths with the TMEM exchange: bit i for N = 2^(9 + i)
#endif
#ifndef OLS_TX_NOPF_MASK
#define OLS_TX_NOPF_MASK 0xB // ... and among them those run without the spectrum prefetch (512, 1024, 4096)
#endif
#ifndef OLS_WARPS_PER_SM
#define OLS_WARPS_PER_SM 16  // resident warps per SM the register budget must allow
#endif
#ifndef OLS_CHECK
#define OLS_CHECK 0          // 1: debug build, every global access of the main kernels bounds-checked
#endif

namespace ols {

// Bits of a plan's device status word.
constexpr int kStatusWaitExpired = 1;   // a bounded device wait gave up
constexpr int kStatusOutOfBounds = 2;   // (OLS_CHECK builds) an index failed its bounds check

// In a build with OLS_CHECK=1: `ok`, and a false check is recorded in the
// status word (the caller then skips the access) -- a bounds checker that
// needs no external tool and never traps.  In a normal build: true, and the
// check compiles away.
__device__ __forceinline__ bool in_bounds(bool ok, int *status) {
#if OLS_CHECK
    if (!ok && status) atomicOr(status, kStatusOutOfBounds);
    return ok;
#else
    (void)ok;
    (void)status;
    return true;
#endif
}

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
    // the exchange between the last two passes goes through TMEM (kernels
    // with TMEM twiddles; columns 64..95 of the thread's block are free)
    static constexpr bool TX = OLS_TMEM_XCHG && OLS_FWD_TW_TMEM && LOG2N >= 9 && LOG2N <= 12 &&
                               ((OLS_TX_MASK >> (LOG2N - 9)) & 1);
    static constexpr bool TX_NOPF = TX && ((OLS_TX_NOPF_MASK >> (LOG2N - 9)) & 1);
    // ... with pass NP-2's lanes relabelled (N = 2048)
    static constexpr bool TX_RELABEL = TX;
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

// Whether segment length 2^LOG2N is in a mask of segment lengths (bit i for
// N = 2^(9 + i)), the form of the per-kernel TMEM-exchange choices.
template <int LOG2N>
__host__ __device__ constexpr bool in_tx_mask(unsigned mask) {
    return LOG2N >= 9 && LOG2N <= 12 && ((mask >> (LOG2N - 9)) & 1u);
}

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

// ---------------------------------------------------------------------------
// The TMEM exchange (Geo<>::TX, N = 512 .. 4096, three passes).  Between the
// last two passes only lane and register bits of a position trade places and
// the warp bits stay, so that exchange never leaves a warp.  The 16-lane
// tcgen05 shapes (tmem.cuh) map a thread's registers to other lanes, so a
// store in one shape and a load in another trade thread bits for column
// bits: one or two such round trips replace the shared-memory exchange and
// its barrier.  Pass 1's lanes are relabelled where that makes the trade
// possible; its shared-memory exchange with pass 0 then uses the per-N
// layout below (conflict-free for both layouts, 16 distinct 8-byte bank
// pairs per half warp), and its twiddle index follows the relabelling.
//
// N = 2048 (Geo<11>::TX): positions carry 11 bits p0..p10; pass 0 (radix 16
// over p7..p10): thread t = p0..p6, register k = p7..p10; pass 1 (radix 16
// over p3..p6): register k = p3..p6, thread lanes (bits 0..4) = (p8, p0, p1,
// p2, p7), warp = p9, p10; pass 2 (radix 8 over p0..p2): thread = p4..p10,
// register = p0..p3 (the layout of the spectrum).  Shared exchange of passes
// 0 and 1: position q at q ^ (p8 << 3) (no padding).
__device__ __forceinline__ int tx11_addr0(int t, int k) { return ((k & 2) ? (t ^ 8) : t) + 128 * k; }
__device__ __forceinline__ int tx11_addr1(int t, int k) {
    const int base = ((t >> 1) & 7) + 128 * ((t >> 4) & 1) + 256 * (t & 1) + 512 * (t >> 5);
    return base + 8 * ((k & 1) ^ (t & 1)) + 16 * (k >> 1);
}

// N = 4096 (Geo<12>::TX): pass 0 thread = p0..p7, register = p8..p11; pass 1
// (radix 16 over p4..p7) lanes (p0, p1, p8, p2, p3), warp p9..p11; pass 2
// thread = p4..p11.  Shared exchange of passes 0 and 1: position q at
// q + 8 (q >> 8): 16 distinct bank pairs per half warp in both layouts.
__device__ __forceinline__ int tx12_addr0(int t, int k) { return t + 264 * k; }
__device__ __forceinline__ int tx12_addr1(int t, int k) {
    return (t & 3) + 4 * ((t >> 3) & 1) + 8 * ((t >> 4) & 1) + 264 * ((t >> 2) & 1) + 528 * (t >> 5) + 16 * k;
}
// N = 512 (Geo<9>::TX): pass 0 thread = p0..p4, register = p5..p8; pass 1
// (radix 16 over p1..p4) lanes (p5, p0, p6, p7, p8); pass 2 thread = p4..p8.
// Shared exchange: position q at q + 2 (q >> 5).
__device__ __forceinline__ int tx9_addr0(int t, int k) { return t + 34 * k; }
__device__ __forceinline__ int tx9_addr1(int t, int k) {
    return ((t >> 1) & 1) + 34 * ((t & 1) + 2 * ((t >> 2) & 1) + 4 * ((t >> 3) & 1) + 8 * ((t >> 4) & 1)) + 2 * k;
}
// N = 1024 (Geo<10>::TX): pass 0 thread = p0..p5, register = p6..p9; pass 1
// (radix 16 over p2..p5) lanes (p6, p7, p8, p0, p1), warp p9; pass 2 (radix 4
// over p0, p1) thread = p4..p9.  Shared exchange: position q at q + 2 (q >> 6).
__device__ __forceinline__ int tx10_addr0(int t, int k) { return t + 66 * k; }
__device__ __forceinline__ int tx10_addr1(int t, int k) {
    return ((t >> 3) & 3) + 66 * ((t & 7) + 8 * (t >> 5)) + 4 * k;
}
template <int LOG2N, int P>
__device__ __forceinline__ int tx_addr(int t, int k) {
    if constexpr (LOG2N == 10) return P == 0 ? tx10_addr0(t, k) : tx10_addr1(t, k);
    else if constexpr (LOG2N == 11) return P == 0 ? tx11_addr0(t, k) : tx11_addr1(t, k);
    else if constexpr (LOG2N == 12) return P == 0 ? tx12_addr0(t, k) : tx12_addr1(t, k);
    else return P == 0 ? tx9_addr0(t, k) : tx9_addr1(t, k);
}
// The shared-memory exchange of passes 0 and 1 when pass 1 is relabelled.
template <int LOG2N, int PW, int PR, class BAR>
__device__ __forceinline__ void exchange_tx(float2 *x, float2 *buf, int t, const BAR &bar) {
    if constexpr (Geo<LOG2N>::XBUFS == 1) bar();
#pragma unroll
    for (int k = 0; k < 16; ++k) buf[tx_addr<LOG2N, PW>(t, k)] = x[k];
    bar();
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = buf[tx_addr<LOG2N, PR>(t, k)];
}

// A warp's TMEM stores are complete (wait::st) before any lane loads them
// back (the barrier measured free: 0.536 ms with it, 0.540 ms without).
__device__ __forceinline__ void tx_sync() { __syncwarp(); }

// Pass 1 -> pass 2 inside the warp, through 32 TMEM columns at xb (lane
// field = the warp's quarter), as two round trips:
//  1. 16x32bx2 stores, half offset 4 (lane = (p8, p0, p1, p2, p3), column =
//     (re/im, p6, p7, p4, p5)); 16x256b loads: thread lanes (p6, p7, p8, p0,
//     p1), registers z[p3][4 (p4 + 2 p5) + 2 p2 + re/im];
//  2. a 32x32b store (column = (re/im, p4, p5, p2, p3)); 16x256b loads:
//     thread lanes (p4..p8), x[p0 + 2 p1 + 4 p2 + 8 p3] from
//     w[p1][4 (p2 + 2 p3) + 2 p0 + re/im].
__device__ __forceinline__ void tx11_forward(float2 *x, uint32_t xb) {
#pragma unroll
    for (int k = 0; k < 8; ++k)      // k = p3 + 2 p4 + 4 p5; registers (x[k], x[k + 8]) differ in p6
        tmem::st16x32bx2_x4<4>(xb + ((uint32_t)(k & 1) << 20) + 8u * ((k >> 1) & 1) + 16u * (k >> 2), x[k].x,
                               x[k].y, x[k + 8].x, x[k + 8].y);
    tmem::wait_st();
    tx_sync();
    float z[2][16];
    tmem::ld16x256b_x4(xb, z[0]);
    tmem::ld16x256b_x4(xb + (16u << 16), z[1]);
    tmem::wait_ld();
    float v[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {   // m = re/im + 2 (p2 + 2 p3 + 4 p4 + 8 p5)
        const int e = m & 1, p2 = (m >> 1) & 1, p3 = (m >> 2) & 1, p4 = (m >> 3) & 1, p5 = (m >> 4) & 1;
        v[2 * (p4 + 2 * p5 + 4 * p2 + 8 * p3) + e] = z[p3][4 * (p4 + 2 * p5) + 2 * p2 + e];
    }
    tmem::st32(xb, v);
    tmem::wait_st();
    tx_sync();
    float w[2][16];
    tmem::ld16x256b_x4(xb, w[0]);
    tmem::ld16x256b_x4(xb + (16u << 16), w[1]);
    tmem::wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {   // k = p0 + 2 p1 + 4 p2 + 8 p3
        const int p0 = k & 1, p1 = (k >> 1) & 1, p2 = (k >> 2) & 1, p3 = k >> 3;
        x[k] = make_float2(w[p1][4 * (p2 + 2 * p3) + 2 * p0], w[p1][4 * (p2 + 2 * p3) + 2 * p0 + 1]);
    }
}
// The reverse: pass 2 -> pass 1 (the same round trips backwards).
__device__ __forceinline__ void tx11_inverse(float2 *x, uint32_t xb) {
    float w[2][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int p0 = k & 1, p1 = (k >> 1) & 1, p2 = (k >> 2) & 1, p3 = k >> 3;
        w[p1][4 * (p2 + 2 * p3) + 2 * p0] = x[k].x;
        w[p1][4 * (p2 + 2 * p3) + 2 * p0 + 1] = x[k].y;
    }
    tmem::st16x256b_x4(xb, w[0]);
    tmem::st16x256b_x4(xb + (16u << 16), w[1]);
    tmem::wait_st();
    tx_sync();
    float v[32];
    tmem::ld32(xb, v);
    tmem::wait_ld();
    float z[2][16];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int e = m & 1, p2 = (m >> 1) & 1, p3 = (m >> 2) & 1, p4 = (m >> 3) & 1, p5 = (m >> 4) & 1;
        z[p3][4 * (p4 + 2 * p5) + 2 * p2 + e] = v[2 * (p4 + 2 * p5 + 4 * p2 + 8 * p3) + e];
    }
    tmem::st16x256b_x4(xb, z[0]);
    tmem::st16x256b_x4(xb + (16u << 16), z[1]);
    tmem::wait_st();
    tx_sync();
#pragma unroll
    for (int k = 0; k < 8; ++k)
        tmem::ld16x32bx2_x4<4>(xb + ((uint32_t)(k & 1) << 20) + 8u * ((k >> 1) & 1) + 16u * (k >> 2), x[k].x,
                               x[k].y, x[k + 8].x, x[k + 8].y);
    tmem::wait_ld();
}

// N = 4096, pass 1 -> pass 2 (registers p4 + 2 p5 + 4 p6 + 8 p7), two round
// trips:
//  1. 16x256b stores (lane = (p8, p2, p3, p6, p4), column = (p7, p0, p1,
//     re/im, p5)); 16x64b loads: thread lanes (p6, p7, p8, p2, p3), registers
//     z[p4][p0 + 2 p1 + 4 re/im + 8 p5];
//  2. a 32x32b store (column = (re/im, p4, p5, p0, p1)); 16x256b loads: thread
//     lanes (p4..p8), x[p0 + 2 p1 + 4 p2 + 8 p3] from w[p3][4 (p0 + 2 p1) + 2 p2
//     + re/im].
__device__ __forceinline__ void tx12_forward(float2 *x, uint32_t xb) {
#pragma unroll
    for (int p4 = 0; p4 < 2; ++p4) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {   // i = p7 + 2 p6 + 4 (re/im + 2 p5)
            const int p7 = i & 1, p6 = (i >> 1) & 1, e = (i >> 2) & 1, p5 = i >> 3;
            const float2 u = x[p4 + 2 * p5 + 4 * p6 + 8 * p7];
            v[i] = e ? u.y : u.x;
        }
        tmem::st16x256b_x4(xb + ((uint32_t)p4 << 20), v);
    }
    tmem::wait_st();
    tx_sync();
    float z[2][16];
    tmem::ld16x64b_x16(xb, z[0]);
    tmem::ld16x64b_x16(xb + (16u << 16), z[1]);
    tmem::wait_ld();
    float v[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {   // m = re/im + 2 p4 + 4 p5 + 8 p0 + 16 p1 (the column)
        const int e = m & 1, p4 = (m >> 1) & 1, p5 = (m >> 2) & 1, p0 = (m >> 3) & 1, p1 = m >> 4;
        v[m] = z[p4][p0 + 2 * p1 + 4 * e + 8 * p5];
    }
    tmem::st32(xb, v);
    tmem::wait_st();
    tx_sync();
    float w[2][16];
    tmem::ld16x256b_x4(xb, w[0]);
    tmem::ld16x256b_x4(xb + (16u << 16), w[1]);
    tmem::wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {   // k = p0 + 2 p1 + 4 p2 + 8 p3
        const int p01 = k & 3, p2 = (k >> 2) & 1, p3 = k >> 3;
        x[k] = make_float2(w[p3][4 * p01 + 2 * p2], w[p3][4 * p01 + 2 * p2 + 1]);
    }
}
__device__ __forceinline__ void tx12_inverse(float2 *x, uint32_t xb) {
    float w[2][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int p01 = k & 3, p2 = (k >> 2) & 1, p3 = k >> 3;
        w[p3][4 * p01 + 2 * p2] = x[k].x;
        w[p3][4 * p01 + 2 * p2 + 1] = x[k].y;
    }
    tmem::st16x256b_x4(xb, w[0]);
    tmem::st16x256b_x4(xb + (16u << 16), w[1]);
    tmem::wait_st();
    tx_sync();
    float v[32];
    tmem::ld32(xb, v);
    tmem::wait_ld();
    float z[2][16];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        const int e = m & 1, p4 = (m >> 1) & 1, p5 = (m >> 2) & 1, p0 = (m >> 3) & 1, p1 = m >> 4;
        z[p4][p0 + 2 * p1 + 4 * e + 8 * p5] = v[m];
    }
    tmem::st16x64b_x16(xb, z[0]);
    tmem::st16x64b_x16(xb + (16u << 16), z[1]);
    tmem::wait_st();
    tx_sync();
    float u[2][16];
    tmem::ld16x256b_x4(xb, u[0]);
    tmem::ld16x256b_x4(xb + (16u << 16), u[1]);
    tmem::wait_ld();
#pragma unroll
    for (int p4 = 0; p4 < 2; ++p4)
#pragma unroll
        for (int m = 0; m < 8; ++m) {   // re at i = p7 + 2 p6 + 8 p5, im at i + 4
            const int p7 = m & 1, p6 = (m >> 1) & 1, p5 = m >> 2, i = p7 + 2 * p6 + 8 * p5;
            x[p4 + 2 * p5 + 4 * p6 + 8 * p7] = make_float2(u[p4][i], u[p4][i + 4]);
        }
}

// N = 512, pass 1 -> pass 2 (registers p1 + 2 p2 + 4 p3 + 8 p4), one round
// trip: 16x256b stores (lane = (p6, p7, p8, p1, p2), column = (p4, p5, p0,
// re/im, p3)); 16x128b loads: thread lanes (p4..p8), x[p0 + 2 p1 + 4 p2 + 8 p3]
// from w[p2][2 (p0 + 2 re/im + 4 p3) + p1].
__device__ __forceinline__ void tx9_forward(float2 *x, uint32_t xb) {
#pragma unroll
    for (int p2 = 0; p2 < 2; ++p2) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {   // i = p4 + 2 p1 + 4 (re/im + 2 p3)
            const int p4 = i & 1, p1 = (i >> 1) & 1, e = (i >> 2) & 1, p3 = i >> 3;
            const float2 u = x[p1 + 2 * p2 + 4 * p3 + 8 * p4];
            v[i] = e ? u.y : u.x;
        }
        tmem::st16x256b_x4(xb + ((uint32_t)p2 << 20), v);
    }
    tmem::wait_st();
    tx_sync();
    float w[2][16];
    tmem::ld16x128b_x8(xb, w[0]);
    tmem::ld16x128b_x8(xb + (16u << 16), w[1]);
    tmem::wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {   // k = p0 + 2 p1 + 4 p2 + 8 p3
        const int p0 = k & 1, p1 = (k >> 1) & 1, p2 = (k >> 2) & 1, p3 = k >> 3;
        x[k] = make_float2(w[p2][2 * (p0 + 4 * p3) + p1], w[p2][2 * (p0 + 2 + 4 * p3) + p1]);
    }
}
__device__ __forceinline__ void tx9_inverse(float2 *x, uint32_t xb) {
    float w[2][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int p0 = k & 1, p1 = (k >> 1) & 1, p2 = (k >> 2) & 1, p3 = k >> 3;
        w[p2][2 * (p0 + 4 * p3) + p1] = x[k].x;
        w[p2][2 * (p0 + 2 + 4 * p3) + p1] = x[k].y;
    }
    tmem::st16x128b_x8(xb, w[0]);
    tmem::st16x128b_x8(xb + (16u << 16), w[1]);
    tmem::wait_st();
    tx_sync();
    float v[2][16];
    tmem::ld16x256b_x4(xb, v[0]);
    tmem::ld16x256b_x4(xb + (16u << 16), v[1]);
    tmem::wait_ld();
#pragma unroll
    for (int p2 = 0; p2 < 2; ++p2)
#pragma unroll
        for (int m = 0; m < 8; ++m) {   // re at i = p4 + 2 p1 + 8 p3, im at i + 4
            const int p4 = m & 1, p1 = (m >> 1) & 1, p3 = m >> 2, i = p4 + 2 * p1 + 8 * p3;
            x[p1 + 2 * p2 + 4 * p3 + 8 * p4] = make_float2(v[p2][i], v[p2][i + 4]);
        }
}

// N = 1024, pass 1 (lanes (p6, p7, p8, p0, p1), registers p2 + 2 p3 + 4 p4 +
// 8 p5) -> pass 2 in one round trip that keeps re and im of a point in
// adjacent registers on both sides (no register moves; a form with the plain
// pass-1 layout, 16x256b store and 16x64b load, split them: 0.501 vs 0.493
// ms): a 32x32b store (column = (re/im, p4, p5,
// p2, p3)), 16x256b loads: x[p0 + 2 p1 + 4 p2 + 8 p3] from w[p1][4 (p2 + 2 p3) +
// 2 p0 + re/im].
__device__ __forceinline__ void tx10_forward(float2 *x, uint32_t xb) {
    float v[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) {   // m = re/im + 2 p4 + 4 p5 + 8 p2 + 16 p3 (the column)
        const int e = m & 1, p4 = (m >> 1) & 1, p5 = (m >> 2) & 1, p2 = (m >> 3) & 1, p3 = m >> 4;
        const float2 u = x[p2 + 2 * p3 + 4 * p4 + 8 * p5];
        v[m] = e ? u.y : u.x;
    }
    tmem::st32(xb, v);
    tmem::wait_st();
    tx_sync();
    float w[2][16];
    tmem::ld16x256b_x4(xb, w[0]);
    tmem::ld16x256b_x4(xb + (16u << 16), w[1]);
    tmem::wait_ld();
#pragma unroll
    for (int k = 0; k < 16; ++k) {   // k = p0 + 2 p1 + 4 p2 + 8 p3
        const int p0 = k & 1, p1 = (k >> 1) & 1, p23 = k >> 2;
        x[k] = make_float2(w[p1][4 * p23 + 2 * p0], w[p1][4 * p23 + 2 * p0 + 1]);
    }
}
__device__ __forceinline__ void tx10_inverse(float2 *x, uint32_t xb) {
    float w[2][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        const int p0 = k & 1, p1 = (k >> 1) & 1, p23 = k >> 2;
        w[p1][4 * p23 + 2 * p0] = x[k].x;
        w[p1][4 * p23 + 2 * p0 + 1] = x[k].y;
    }
    tmem::st16x256b_x4(xb, w[0]);
    tmem::st16x256b_x4(xb + (16u << 16), w[1]);
    tmem::wait_st();
    tx_sync();
    float v[32];
    tmem::ld32(xb, v);
    tmem::wait_ld();
#pragma unroll
    for (int m = 0; m < 32; m += 2) {
        const int p4 = (m >> 1) & 1, p5 = (m >> 2) & 1, p2 = (m >> 3) & 1, p3 = m >> 4;
        x[p2 + 2 * p3 + 4 * p4 + 8 * p5] = make_float2(v[m], v[m + 1]);
    }
}

template <int LOG2N>
__device__ __forceinline__ void tx_forward(float2 *x, uint32_t xb) {
    if constexpr (LOG2N == 12) tx12_forward(x, xb);
    else if constexpr (LOG2N == 11) tx11_forward(x, xb);
    else if constexpr (LOG2N == 10) tx10_forward(x, xb);
    else tx9_forward(x, xb);
}
template <int LOG2N>
__device__ __forceinline__ void tx_inverse(float2 *x, uint32_t xb) {
    if constexpr (LOG2N == 12) tx12_inverse(x, xb);
    else if constexpr (LOG2N == 11) tx11_inverse(x, xb);
    else if constexpr (LOG2N == 10) tx10_inverse(x, xb);
    else tx9_inverse(x, xb);
}

// Index n' = position mod s of pass P's twiddle W_{16 s}^{n' k} for thread t
// (XCH: the kernel uses the TMEM exchange, which relabels pass NP-2).
template <int LOG2N, int P, bool XCH>
__device__ __forceinline__ int tw_index(int t) {
    using G = Geo<LOG2N>;
    if constexpr (XCH && G::TX_RELABEL && P == G::NP - 2) {   // the relabelled lanes holding p0 .. p(s-1)
        if constexpr (LOG2N == 11) return (t >> 1) & 7;
        else if constexpr (LOG2N == 12) return (t & 3) + 4 * ((t >> 3) & 1) + 8 * ((t >> 4) & 1);
        else if constexpr (LOG2N == 10) return (t >> 3) & 3;
        else return (t >> 1) & 1;
    }
    else return t % G::stride(P);
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

// TwTmemT: the thread's own 15 twiddles of every pass, preloaded into its
// TMEM lane (pass P at columns 32 P .. 32 P + 29 of `base`): no L1 traffic.
// XCH: the segment FFT also uses the TMEM exchange where Geo<>::TX allows it
// (kernels whose epilogue needs the registers opt out).
template <bool XCH = true>
struct TwTmemT {
    static constexpr bool xchg = XCH;
    uint32_t base;
    // columns 64..95: the staging area of the TMEM exchange
    __device__ __forceinline__ uint32_t xbase() const { return base + 64; }
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

using TwTmem = TwTmemT<true>;
template <class TW>
struct is_tw_tmem : std::false_type {};
template <bool X>
struct is_tw_tmem<TwTmemT<X>> : std::true_type {};
template <class TW>
__device__ __forceinline__ constexpr bool tw_xchg() {
    if constexpr (is_tw_tmem<TW>::value) return TW::xchg;
    else return false;
}

// Fill a TwTmemT<XCH> for thread t from the plan's twiddle table.
template <int LOG2N, bool XCH = true, int P = 0>
__device__ __forceinline__ void tw_tmem_fill(const float2 *tw, uint32_t base, int t) {
    using G = Geo<LOG2N>;
    if constexpr (P < G::NP - 1) {
        constexpr int s = G::stride(P);
        const float2 *w = tw + G::tw_off(P) + tw_index<LOG2N, P, XCH>(t);
        float v[32];
#pragma unroll
        for (int k = 1; k < 16; ++k) {
            const float2 wk = __ldg(w + (k - 1) * s);
            v[2 * k - 2] = wk.x;
            v[2 * k - 1] = wk.y;
        }
        v[30] = v[31] = 0.f;
        tmem::st32(base + 32 * P, v);
        tw_tmem_fill<LOG2N, XCH, P + 1>(tw, base, t);
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
        constexpr bool tx = G::TX && tw_xchg<TW>();
        if constexpr (tx && P == G::NP - 2) {
            tx_forward<LOG2N>(x, tw.xbase());
        } else {
            float2 *buf = bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0);
            if constexpr (tx && G::TX_RELABEL && P + 1 == G::NP - 2) exchange_tx<LOG2N, P, P + 1>(x, buf, t, bar);
            else exchange<LOG2N, P, P + 1>(x, buf, t, bar);
            ++xc;
        }
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
        // or before the TMEM exchange (their 30 registers then are not live
        // across the exchange: with them the kernel spills)
        constexpr bool tx = G::TX && tw_xchg<TW>();
        constexpr bool late = (OLS_TW_TMEM_LATE || (tx && P == G::NP - 2)) && is_tw_tmem<TW>::value;
        if constexpr (!late) tw.template fetch<LOG2N, P>(f, t);
        if constexpr (tx && P == G::NP - 2) {
            tx_inverse<LOG2N>(x, tw.xbase());
        } else {
            float2 *buf = bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0);
            if constexpr (tx && G::TX_RELABEL && P + 1 == G::NP - 2) exchange_tx<LOG2N, P + 1, P>(x, buf, t, bar);
            else exchange<LOG2N, P + 1, P>(x, buf, t, bar);
            ++xc;
        }
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
