// ols_tc.cu -- fused OLS with every radix-16 FFT stage on the tensor cores
// (tcgen05), in split 16-bit precision with FP32 accumulation.
//
// Same algorithm as ols_forward.cu (Algorithm 2: segment FFT kept on chip,
// per filter point-wise product, inverse FFT, discard of the M-1 aliased
// samples), but each 16-point DFT of a pass is a matrix product on the
// tensor cores instead of register arithmetic:
// * A thread's 16 complex values form one row of A = [Re x_0..15 | Im x_0..15]
//   (K = 32).  They are split x = x_hi + x_lo into two 16-bit numbers (FP16 or
//   BF16) and stored with tcgen05.st into the thread's own TMEM lane
//   (128 threads = 128 lanes = one M = 128 tile).
// * The DFT-16 is the real 32x32 matrix B = [[C, S], [-S, C]] (C = cos, S = the
//   imaginary part of the twiddle), also split B = B_hi + B_lo, held in
//   shared memory in the no-swizzle K-major core-matrix layout.
// * D = A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term is below the
//   16-bit split's resolution), six tcgen05.mma of K = 16 per tile, FP32
//   accumulation in TMEM.  Each 128-thread tile synchronises on a named
//   barrier of its own; its first thread issues the tile's MMAs and commits
//   them to the tile's mbarrier; the tile's threads wait (bounded) and read
//   their rows back with tcgen05.ld.
// * Two filters are in flight (TMEM groups a and b of each tile), skewed by
//   half a pass: the MMAs of one group run while the other group's threads
//   read back, exchange, twiddle and split.
// * Twiddles, the point-wise product and the exchanges between passes stay
//   in FP32 registers and shared memory, as in the FP32 kernel.  A remainder
//   pass of radix 2/4/8 (N not a power of 16) stays in FP32 registers.
// * Range: forward passes are unscaled (|input| <= 1.42 grows to <= 362
//   before the last forward pass); inverse passes after the first are scaled
//   by 1/4 (exact), and the filter spectra by 4^(passes-1), which keeps every
//   16-bit operand below 65504 for inputs with |s| <= 1.42 and unit-L2 filters.
// Waits on the mbarriers are bounded: on expiry the kernel records an error in
// the plan's status word and stops at the end of the filter pair; each tile's
// issuing thread then waits (bounded again) for the commits it issued and did
// not see complete, and the CTA releases its TMEM and returns.  The in-loop limit is a launch
// argument (the plan's), and so is a test switch that points the in-loop
// waits at a second mbarrier nothing ever arrives on, so that a test can make
// a wait run out without any fault; the drain before the TMEM release always
// watches the real mbarrier with the long limit.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "ols_internal.h"
#include "ols_fft_passes.cuh"

namespace ols {

namespace tc {

constexpr int kCols = 128;           // TMEM columns per 128-row tile: two groups of A_hi 16, A_lo 16, D 32
constexpr int kBytesB = 32 * 32 * 2; // one 32x32 16-bit matrix
constexpr long long kWaitLimit = 1ll << 20;   // polls; also the drain limit before tcgen05.dealloc

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-bit split of an FP32 pair into packed hi and lo words.
template <bool BF16>
__device__ __forceinline__ void split2(float a, float b, uint32_t &hi, uint32_t &lo) {
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                 "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *d) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3]), "=f"(d[4]), "=f"(d[5]), "=f"(d[6]), "=f"(d[7]),
                   "=f"(d[8]), "=f"(d[9]), "=f"(d[10]), "=f"(d[11]), "=f"(d[12]), "=f"(d[13]), "=f"(d[14]),
                   "=f"(d[15]), "=f"(d[16]), "=f"(d[17]), "=f"(d[18]), "=f"(d[19]), "=f"(d[20]), "=f"(d[21]),
                   "=f"(d[22]), "=f"(d[23]), "=f"(d[24]), "=f"(d[25]), "=f"(d[26]), "=f"(d[27]), "=f"(d[28]),
                   "=f"(d[29]), "=f"(d[30]), "=f"(d[31])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of
// 8 rows x 16 bytes; LBO = byte step between core matrices along K (512),
// SBO = byte step along N (128); descriptor version 1.
__device__ __forceinline__ uint64_t b_desc(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(512 >> 4) << 16;
    d |= (uint64_t)(128 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: D FP32, A and B FP16 (0) or BF16 (1),
// both K-major, N = 32, M = 128.
template <bool BF16>
__device__ __forceinline__ constexpr uint32_t idesc() {
    return (1u << 4) | ((BF16 ? 1u : 0u) << 7) | ((BF16 ? 1u : 0u) << 10) | ((32u >> 3) << 17) |
           ((128u >> 4) << 24);
}

// Per-thread view of its tile (128 rows = 128 threads = the TMEM lanes of
// warps 4 tile .. 4 tile + 3).  Two groups of operands per tile, a and b (two
// filters in flight): group g's A rows (hi: 16 columns, lo: 16) at column
// 64 g of the tile, its D (32 FP32 columns) at 64 g + 32.  The tile's first
// thread issues the tile's MMAs and commits them to the group's mbarrier.
struct Ctx {
    uint32_t lane_base;    // TMEM address of this thread's lane in its tile (column 0 of the tile)
    uint32_t tile_base;    // TMEM address of the tile (lane 0, column 0) for the MMAs
    uint32_t mbar[2];      // this tile's mbarriers, groups a and b
    uint32_t wbar[2];      // what in-loop waits watch: mbar, or (test switch) one nothing arrives on
    uint32_t phase[2];     // parity expected next; frozen once a wait has run out
    uint32_t b_smem;       // shared address of the four B matrices (fwd hi, fwd lo, inv hi, inv lo)
    long long wait_limit;  // polls per in-loop wait
    int *status;           // plan status word (error flag)
    int tile;
    bool leader;           // issues this tile's MMAs
    bool pending[2];       // leader: a commit issued and not yet seen complete
    bool failed;           // this thread saw a wait run out
    bool stop;             // some thread of the CTA did (agreed once per filter pair): leave the loops
};

// Group g's A rows from split words: hi[w] / lo[w] pack (Re x_2w, Re x_2w+1)
// for w < 8 and (Im x_2(w-8), Im x_2(w-8)+1) for w >= 8.
__device__ __forceinline__ void store_words(const uint32_t *hi, const uint32_t *lo, const Ctx &c, int g) {
    const uint32_t a = c.lane_base + 64u * (uint32_t)g;
    tmem_st16(a, hi);
    tmem_st16(a + 16, lo);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// Group g's A rows from FP32 values (x scaled by `scale` first), split here.
template <bool BF16>
__device__ __forceinline__ void store_rows(const float2 *x, float scale, const Ctx &c, int g) {
    uint32_t hi[16], lo[16];
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        split2<BF16>(x[2 * w].x * scale, x[2 * w + 1].x * scale, hi[w], lo[w]);
        split2<BF16>(x[2 * w].y * scale, x[2 * w + 1].y * scale, hi[8 + w], lo[8 + w]);
    }
    store_words(hi, lo, c, g);
}

// Every thread of the tile has stored its rows; the leader issues the tile's
// six MMAs (D = A_hi B_hi + A_hi B_lo + A_lo B_hi, K = 32 as two halves) and
// commits them to group g's mbarrier.  Collective over the tile.
template <bool INV, bool BF16>
__device__ __forceinline__ void issue(Ctx &c, int g) {
    asm volatile("bar.sync %0, 128;" ::"r"(1 + c.tile) : "memory");
    if (c.leader && !c.failed) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t bh = c.b_smem + (INV ? 2 : 0) * kBytesB, bl = bh + kBytesB;
        const uint32_t base = c.tile_base + 64u * (uint32_t)g;
        const uint32_t d = base + 32;
#pragma unroll
        for (int term = 0; term < 3; ++term) {
            const uint32_t a = base + (term == 2 ? 16 : 0);          // A_hi, A_hi, A_lo
            const uint32_t b = term == 1 ? bl : bh;                    // B_hi, B_lo, B_hi
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const uint32_t acc = (term | kk) != 0;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
                             "r"(a + kk * 8), "l"(b_desc(b + kk * 1024)), "r"(idesc<BF16>()), "r"(acc)
                             : "memory");
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(c.mbar[g])
                     : "memory");
        c.pending[g] = true;
    }
}

// Bounded poll of mbarrier `bar` for parity `phase`; true once it completed.
__device__ __forceinline__ bool poll(uint32_t bar, uint32_t phase, long long limit) {
    uint32_t done = 0;
    for (long long it = 0; it < limit && !done; ++it) {
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done)
                     : "r"(bar), "r"(phase)
                     : "memory");
    }
    return done != 0;
}

// Wait (bounded) for group g's MMAs and read this thread's row of D into x.
// A thread whose wait runs out records it, keeps the group's parity (so the
// leader's drain before the TMEM release watches the commit it gave up on)
// and skips its later waits; its results are then undefined and not stored.
__device__ __forceinline__ void wait_load(float2 *x, Ctx &c, int g) {
    if (!c.failed) {
        if (poll(c.wbar[g], c.phase[g], c.wait_limit)) {
            c.phase[g] ^= 1u;
            c.pending[g] = false;
        } else {
            c.failed = true;
            atomicOr(c.status, 1);
        }
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float d[32];
    tmem_ld32(c.lane_base + 64u * (uint32_t)g + 32, d);
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = make_float2(d[j], d[16 + j]);
}

// Rows of A from samples already stored split: hs[k] / ls[k] hold
// (Re, Im) of point k as two 16-bit numbers; A wants (Re x_2w, Re x_2w+1).
__device__ __forceinline__ void rows_from_planes(const uint32_t *hs, const uint32_t *ls, uint32_t *hi, uint32_t *lo) {
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        hi[w] = __byte_perm(hs[2 * w], hs[2 * w + 1], 0x5410);       // low halves: Re
        hi[8 + w] = __byte_perm(hs[2 * w], hs[2 * w + 1], 0x7632);   // high halves: Im
        lo[w] = __byte_perm(ls[2 * w], ls[2 * w + 1], 0x5410);
        lo[8 + w] = __byte_perm(ls[2 * w], ls[2 * w + 1], 0x7632);
    }
}

// Forward passes P.. of the segment (once per segment, group a, no overlap).
// With PRE (pre-split input) the first pass takes its A rows as given
// (rows_hi / rows_lo) instead of splitting x.
template <int LOG2N, int P, bool BF16, bool PRE = false>
__device__ __forceinline__ void tc_forward_passes(float2 *x, float2 *bufs, const float2 *tw, int t, int &xc, Ctx &c,
                                                  const uint32_t *rows_hi = nullptr, const uint32_t *rows_lo = nullptr) {
    using G = Geo<LOG2N>;
    static_assert(G::radix(0) == 16, "the first forward pass is radix 16 for every supported N");
    if constexpr (G::radix(P) == 16) {
        if constexpr (P == 0 && PRE) store_words(rows_hi, rows_lo, c, 0);
        else store_rows<BF16>(x, 1.0f, c, 0);
        issue<false, BF16>(c, 0);
        wait_load(x, c, 0);
    } else {
        dft_groups<G::radix(P), false>(x);
    }
    if constexpr (P < G::NP - 1) {
        twiddle<LOG2N, P, false>(x, tw, t);
        exchange<LOG2N, P, P + 1>(x, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        tc_forward_passes<LOG2N, P + 1, BF16>(x, bufs, tw, t, xc, c);
    }
}

// Inverse passes P, P-1, ..., 0 of two filters in flight (group a: xa, group
// b: xb), skewed by half a pass: the MMAs of a's pass P run while b finishes
// pass P+1 and prepares pass P (wait, exchange, twiddle, split), and those of
// b's pass P while a finishes pass P and prepares pass P-1.  Inverse passes
// after the first are scaled by 1/4 (exact; the spectra carry the gain).
template <int LOG2N, int P, bool BF16>
__device__ __forceinline__ void tc_inverse_pair(float2 *xa, float2 *xb, float2 *bufs, const float2 *tw, int t,
                                                int &xc, Ctx &c) {
    using G = Geo<LOG2N>;
    constexpr bool TCP = G::radix(P) == 16;                                  // pass P on the tensor cores
    constexpr bool B_IN_FLIGHT = P + 1 <= G::NP - 1 && G::radix(P + 1) == 16; // b's pass P+1 not read back yet
    constexpr float scale = P == G::NP - 1 ? 1.0f : 0.25f;
    // a: enter pass P
    if constexpr (P < G::NP - 1) {
        exchange<LOG2N, P + 1, P>(xa, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        twiddle<LOG2N, P, true>(xa, tw, t);
    }
    if constexpr (TCP) {
        store_rows<BF16>(xa, scale, c, 0);
        issue<true, BF16>(c, 0);
    } else {
        dft_groups<G::radix(P), true>(xa);
    }
    // b: finish pass P+1, enter pass P
    if constexpr (B_IN_FLIGHT) wait_load(xb, c, 1);
    if constexpr (P < G::NP - 1) {
        exchange<LOG2N, P + 1, P>(xb, bufs + (G::XBUFS == 2 ? (xc & 1) * G::PADN : 0), t);
        ++xc;
        twiddle<LOG2N, P, true>(xb, tw, t);
    }
    if constexpr (TCP) {
        store_rows<BF16>(xb, scale, c, 1);
        issue<true, BF16>(c, 1);
    } else {
        dft_groups<G::radix(P), true>(xb);
    }
    // a: finish pass P
    if constexpr (TCP) wait_load(xa, c, 0);
    if constexpr (P > 0) {
        tc_inverse_pair<LOG2N, P - 1, BF16>(xa, xb, bufs, tw, t, xc, c);
    } else {
        static_assert(TCP, "pass 0 is radix 16");
        wait_load(xb, c, 1);                         // b: finish pass 0
    }
}

// Inverse passes after the first are scaled by 1/4: the spectra get 4^(k),
// k = number of scaled radix-16 passes.
template <int LOG2N>
__host__ __device__ constexpr float spectrum_gain() {
    float g = 1.0f;
    for (int p = 0; p < Geo<LOG2N>::NP - 1; ++p)
        if (Geo<LOG2N>::radix(p) == 16) g *= 4.0f;
    return g;
}

}  // namespace tc

// PRE: the signal comes as two planes of 16-bit (Re, Im) pairs, hi and lo
// (sig_hi / sig_lo, one 32-bit word per sample), instead of FP32 (sig).
template <int LOG2N, bool BF16, bool PRE>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK, Geo<LOG2N>::MINB)
ols_tc_kernel(const float2 *__restrict__ sig, const uint32_t *__restrict__ sig_hi, const uint32_t *__restrict__ sig_lo,
              long long Ns, const float4 *__restrict__ Hk,
              const float2 *__restrict__ twg, const uint16_t *__restrict__ bmat, float2 *__restrict__ y, int M, int F,
              long long L, long long nseg, long long Nout, int *status, long long wait_limit,
              int wait_never) {
    using G = Geo<LOG2N>;
    constexpr int NT = G::BLOCK / 128;           // M = 128 tiles per CTA
    constexpr uint32_t NCOLS = NT * tc::kCols;
    static_assert(G::BLOCK % 128 == 0, "the tensor-core form needs 128-thread multiples");
    extern __shared__ float4 smem_raw[];
    __shared__ __align__(8) uint64_t mbar[NT][2];   // per tile, groups a and b
    __shared__ __align__(8) uint64_t mbar_never;   // test switch: no thread or MMA ever arrives here
    __shared__ uint32_t tbase;
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
    uint16_t *bsm = reinterpret_cast<uint16_t *>(smem);                     // 4 x 2 KB, 1 KB aligned
    float2 *bufs0 = smem + (4 * tc::kBytesB) / sizeof(float2);
    const int slot = threadIdx.x / G::T;
    const int t = threadIdx.x % G::T;
    float2 *bufs = bufs0 + slot * G::XBUFS * G::PADN;
    const float2 *tw = twg;

    for (int i = threadIdx.x; i < 4 * tc::kBytesB / 2; i += G::BLOCK) bsm[i] = bmat[i];
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT; ++i)
            for (int g = 0; g < 2; ++g)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&mbar[i][g])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&mbar_never)));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tbase)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    tc::Ctx c;
    c.tile = threadIdx.x / 128;
    c.tile_base = tbase + (uint32_t)c.tile * tc::kCols;
    c.lane_base = c.tile_base + ((uint32_t)(((threadIdx.x / 32) % 4) * 32) << 16);
    for (int g = 0; g < 2; ++g) {
        c.mbar[g] = tc::smem_u32(&mbar[c.tile][g]);
        c.wbar[g] = wait_never ? tc::smem_u32(&mbar_never) : c.mbar[g];
        c.phase[g] = 0;
        c.pending[g] = false;
    }
    c.b_smem = tc::smem_u32(bsm);
    c.wait_limit = wait_limit;
    c.status = status;
    c.leader = threadIdx.x % 128 == 0;
    c.failed = false;
    c.stop = false;

    const int lo = M - 1;
    const float gain = tc::spectrum_gain<LOG2N>();
    int xc = 0;
    const long long nblk = (nseg + G::SEGS - 1) / G::SEGS;
    for (long long blk = blockIdx.x; blk < nblk && !c.stop; blk += gridDim.x) {
        const long long seg = blk * G::SEGS + slot;
        const bool active = seg < nseg;
        const long long start = seg * L;
        float2 X[16];
        const long long avail = active ? (Ns - start) : 0;
        const int lim = (int)(avail < G::N ? avail : G::N);
        if constexpr (PRE) {
            uint32_t hs[16], ls[16], rh[16], rl[16];
            const uint32_t *sh = sig_hi + (active ? start : 0) + t, *sl = sig_lo + (active ? start : 0) + t;
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const bool in = k * G::T + t < lim && in_bounds((active ? start : 0) + k * G::T + t < Ns, status);
                hs[k] = in ? __ldg(sh + k * G::T) : 0u;
                ls[k] = in ? __ldg(sl + k * G::T) : 0u;
            }
            tc::rows_from_planes(hs, ls, rh, rl);
            tc::tc_forward_passes<LOG2N, 0, BF16, true>(X, bufs, tw, t, xc, c, rh, rl);
        } else {
            const float2 *src = sig + (active ? start : 0) + t;
#pragma unroll
            for (int k = 0; k < 16; ++k)
                X[k] = (k * G::T + t < lim && in_bounds((active ? start : 0) + k * G::T + t < Ns, status))
                           ? __ldg(src + k * G::T)
                           : make_float2(0.f, 0.f);
            tc::tc_forward_passes<LOG2N, 0, BF16>(X, bufs, tw, t, xc, c);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) X[k] = make_float2(X[k].x * gain, X[k].y * gain);
        const long long rem = active ? (Nout - start) : 0;
        const int span = (int)(rem < (long long)(G::N - lo) ? rem : (long long)(G::N - lo));
        const long long obase = start - lo;
        // filters in pairs (two in flight); an odd bank's last filter runs as
        // both groups and only group a's result is stored
        for (int f = 0; f < F && !c.stop; f += 2) {
            const int fb = f + 1 < F ? f + 1 : f;
            float2 xa[16], xb[16];
            const float4 *ha = Hk + (size_t)f * (G::N / 2) + t, *hb = Hk + (size_t)fb * (G::N / 2) + t;
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                const float4 h = load_spectrum(ha + j2 * G::T);
                xa[2 * j2] = cmul(X[2 * j2], make_float2(h.x, h.y));
                xa[2 * j2 + 1] = cmul(X[2 * j2 + 1], make_float2(h.z, h.w));
            }
#pragma unroll
            for (int j2 = 0; j2 < 8; ++j2) {
                const float4 h = load_spectrum(hb + j2 * G::T);
                xb[2 * j2] = cmul(X[2 * j2], make_float2(h.x, h.y));
                xb[2 * j2 + 1] = cmul(X[2 * j2 + 1], make_float2(h.z, h.w));
            }
            tc::tc_inverse_pair<LOG2N, G::NP - 1, BF16>(xa, xb, bufs, tw, t, xc, c);
            if (!c.failed) {
                float2 *da = y + (size_t)f * (size_t)Nout, *db = y + (size_t)fb * (size_t)Nout;
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int n = k * G::T + t;
                    if ((unsigned)(n - lo) < (unsigned)span && in_bounds(obase + n >= 0 && obase + n < Nout, status)) {
                        da[obase + n] = xa[k];
                        if (fb != f) db[obase + n] = xb[k];
                    }
                }
            }
            c.stop = __syncthreads_or(c.failed) != 0;   // the CTA's agreement, once per filter pair
        }
    }
    // release TMEM: a tile's leader first waits (bounded, long limit) for every
    // commit it issued and did not see complete -- after a wait ran out, at most
    // one per group, at the parity the group's phase kept
    if (c.leader) {
        for (int g = 0; g < 2; ++g)
            if (c.pending[g]) tc::poll(c.mbar[g], c.phase[g], tc::kWaitLimit);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (threadIdx.x < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(NCOLS));
}

template <int LOG2N>
struct TcGeo {
    static constexpr size_t SMEM = 4 * tc::kBytesB + sizeof(float2) * (size_t)(Geo<LOG2N>::SEGS * Geo<LOG2N>::XBUFS *
                                                                               Geo<LOG2N>::PADN);
};

template <int LOG2N, bool BF16, bool PRE>
static cudaError_t tc_prepare_kernel(int sm_count, int *grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(ols_tc_kernel<LOG2N, BF16, PRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TcGeo<LOG2N>::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    const int cols = (Geo<LOG2N>::BLOCK / 128) * tc::kCols;   // TMEM holds every resident CTA's columns
    e = resident_blocks_tmem(ols_tc_kernel<LOG2N, BF16, PRE>, Geo<LOG2N>::BLOCK, TcGeo<LOG2N>::SMEM, cols, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid_cap = per_sm * sm_count;
    return cudaSuccess;
}

template <int LOG2N, bool BF16>
static cudaError_t tc_prepare_one(ols_plan_s &p) {
    cudaError_t e = tc_prepare_kernel<LOG2N, BF16, false>(p.sm_count, &p.tc_grid_cap);
    if (e == cudaSuccess) e = tc_prepare_kernel<LOG2N, BF16, true>(p.sm_count, &p.tc_split_grid_cap);
    return e;
}

cudaError_t tc_prepare(ols_plan_s &p, bool bf16) {
    switch (p.log2N) {
        case 8: return bf16 ? tc_prepare_one<8, true>(p) : tc_prepare_one<8, false>(p);
        case 9: return bf16 ? tc_prepare_one<9, true>(p) : tc_prepare_one<9, false>(p);
        case 10: return bf16 ? tc_prepare_one<10, true>(p) : tc_prepare_one<10, false>(p);
        case 11: return bf16 ? tc_prepare_one<11, true>(p) : tc_prepare_one<11, false>(p);
        case 12: return bf16 ? tc_prepare_one<12, true>(p) : tc_prepare_one<12, false>(p);
        case 13: return bf16 ? tc_prepare_one<13, true>(p) : tc_prepare_one<13, false>(p);
        default: return cudaErrorInvalidValue;
    }
}

template <int LOG2N, bool BF16, bool PRE>
static cudaError_t tc_launch_one(const ols_plan_s &p, const TcSignal &sg, int64_t Ns, float2 *y, int64_t L,
                                 int64_t nseg, int64_t Nout, cudaStream_t st) {
    using G = Geo<LOG2N>;
    const int64_t nblk = (nseg + G::SEGS - 1) / G::SEGS;
    const int cap = PRE ? p.tc_split_grid_cap : p.tc_grid_cap;
    const int grid = (int)(nblk < cap ? nblk : cap);
    ols_tc_kernel<LOG2N, BF16, PRE><<<grid, G::BLOCK, TcGeo<LOG2N>::SMEM, st>>>(
        sg.s, sg.hi, sg.lo, Ns, reinterpret_cast<const float4 *>(p.Hk), p.tw, p.tc_bmat, y, p.M, p.F, L, nseg, Nout,
        p.d_status, p.tc_wait_limit, p.tc_wait_never ? 1 : 0);
    return cudaGetLastError();
}

template <int LOG2N>
static cudaError_t tc_launch_n(const ols_plan_s &p, const TcSignal &sg, int64_t Ns, float2 *y, int64_t L,
                               int64_t nseg, int64_t Nout, cudaStream_t st) {
    const bool bf16 = (p.flags & OLS_FLAG_TC_BF16SPLIT) != 0;
    const bool pre = sg.hi != nullptr;
    if (bf16) return pre ? tc_launch_one<LOG2N, true, true>(p, sg, Ns, y, L, nseg, Nout, st)
                         : tc_launch_one<LOG2N, true, false>(p, sg, Ns, y, L, nseg, Nout, st);
    return pre ? tc_launch_one<LOG2N, false, true>(p, sg, Ns, y, L, nseg, Nout, st)
               : tc_launch_one<LOG2N, false, false>(p, sg, Ns, y, L, nseg, Nout, st);
}

cudaError_t tc_launch(const ols_plan_s &p, const TcSignal &sg, int64_t Ns, float2 *y, int64_t L, int64_t nseg,
                      int64_t Nout, cudaStream_t st) {
    switch (p.log2N) {
        case 8: return tc_launch_n<8>(p, sg, Ns, y, L, nseg, Nout, st);
        case 9: return tc_launch_n<9>(p, sg, Ns, y, L, nseg, Nout, st);
        case 10: return tc_launch_n<10>(p, sg, Ns, y, L, nseg, Nout, st);
        case 11: return tc_launch_n<11>(p, sg, Ns, y, L, nseg, Nout, st);
        case 12: return tc_launch_n<12>(p, sg, Ns, y, L, nseg, Nout, st);
        case 13: return tc_launch_n<13>(p, sg, Ns, y, L, nseg, Nout, st);
        default: return cudaErrorInvalidValue;
    }
}

// The stored split form of a signal: hi = rn16(x), lo = rn16(x - hi) for the
// real and the imaginary part of every sample, written as 16-bit (Re, Im)
// pairs, one plane each -- the same rounding the kernel applies when it
// splits FP32 values itself.
template <bool BF16>
__global__ void split_signal_kernel(const float2 *__restrict__ s, long long Ns, uint32_t *__restrict__ hi,
                                    uint32_t *__restrict__ lo) {
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < Ns; n += (long long)gridDim.x * blockDim.x) {
        const float2 v = s[n];
        uint32_t h, l;
        tc::split2<BF16>(v.x, v.y, h, l);
        hi[n] = h;
        lo[n] = l;
    }
}

cudaError_t launch_split_signal(const float2 *s, int64_t Ns, bool bf16, uint32_t *hi, uint32_t *lo, int sm_count,
                                cudaStream_t st) {
    const long long want = (Ns + 255) / 256;
    const int grid = (int)(want < 8ll * sm_count ? (want > 0 ? want : 1) : 8ll * sm_count);
    if (bf16) split_signal_kernel<true><<<grid, 256, 0, st>>>(s, Ns, hi, lo);
    else split_signal_kernel<false><<<grid, 256, 0, st>>>(s, Ns, hi, lo);
    return cudaGetLastError();
}

}  // namespace ols
