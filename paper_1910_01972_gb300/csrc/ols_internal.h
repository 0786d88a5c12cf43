// ols_internal.h -- plan object and kernel launchers shared by the library's
// translation units (not part of the public ABI, see include/ols.h).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "ols.h"

namespace ols {

constexpr int kMinLog2N = 8;   // N = 256
constexpr int kMaxLog2N = 13;  // N = 8192

// Forward passes of the in-register/shared-memory FFT for N = 2^log2N:
// radix-16 passes first (strides N/16, N/256, ...), then one pass of the
// remaining radix (2, 4, 8 or 16) at stride 1.  Kept in one place so host
// tables and device index math agree.
struct PassPlan {
    int log2N;
    int N;
    int T;       // threads per segment (N / 16): each thread holds 16 points
    int np;      // number of passes
    int radix[4];
    int stride[4];
    int tw_off[4];
    int twn;     // twiddle entries of passes 0 .. np-2
};
PassPlan make_pass_plan(int log2N);

// Frequency index held at each storage position of the forward FFT output.
void spectral_order(int log2N, int32_t *nu);

// Model-based segment length (no measurement): minimises (N / L)(log2 N + c).
int64_t choose_segment_length(int32_t M);

// Every device allocation of the library goes through dev_alloc.  Host-side
// fault injection for tests: with OLS_FAIL_ALLOC=k (k >= 1) in the
// environment, the k-th allocation made under one outermost AllocScope (one
// call of ols_plan, ols_batch_plan or ols_convolve_host) fails as if the
// device were out of memory; unset or 0, nothing is injected.
cudaError_t dev_alloc_raw(void **p, size_t bytes);
template <class T>
cudaError_t dev_alloc(T **p, size_t bytes) {
    return dev_alloc_raw(reinterpret_cast<void **>(p), bytes);
}
struct AllocScope {      // nests: only the outermost scope restarts the count
    AllocScope();
    ~AllocScope();
};

// Grid of the fused forward and real-to-real kernels.  Up to N = 2048: one
// CTA per block of segments, left to the hardware scheduler, which starts a
// CTA wherever one finishes and so balances the last wave (the persistent
// grid gives every CTA a fixed share of segments: measured 1% slower on the
// 2^23-sample bank at N = 2048, 4% at N = 1024, 0.9% for the real form).
// From N = 4096 the persistent grid, whose CTAs set up their twiddles and
// tensor memory once (0.7% faster there).  Either way the shared memory each
// CTA requests bounds residency to what tensor memory can serve.
inline int fused_grid(int log2N, int64_t nblk, int persistent_cap) {
    int64_t g = (log2N <= 11) ? nblk : (nblk < persistent_cap ? nblk : persistent_cap);
    if (g > 0x7fffffff) g = 0x7fffffff;   // grid.x limit; the kernels loop over the rest
    return (int)g;
}

struct Staging {            // device buffers of ols_convolve_host
    float2 *in[2] = {nullptr, nullptr};
    float2 *out[2] = {nullptr, nullptr};
    int64_t in_cap = 0, out_cap = 0;   // elements per buffer
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev_user = nullptr, ev_done[2] = {nullptr, nullptr};
    bool timing = false;               // per-stage events (ols_host_timing)
    std::vector<cudaEvent_t> tev;      // 4 per chunk: start, after H2D, after the kernel, after D2H
    int64_t timed_chunks = 0;          // chunks of the last timed call (0: none yet)
};

// Resident blocks per SM of a kernel that allocates `tmem_cols` TMEM columns
// per block, from the SM's limits themselves (registers per sub-partition,
// shared memory, threads, blocks, the 512 TMEM columns): the runtime's
// occupancy query answers 1 for any kernel that allocates tensor memory,
// which would leave half or more of the SMs' warp slots empty.
template <class KERNEL>
cudaError_t resident_blocks_tmem(KERNEL kernel, int block, size_t dyn_smem, int tmem_cols, int *per_sm) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    int dev = 0, smem_sm = 0, regs_sm = 0, thr_sm = 0, blk_sm = 0, reserved = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    if (e != cudaSuccess) return e;
    const int warps = (block + 31) / 32;
    const int warp_regs = ((a.numRegs * 32 + 255) / 256) * 256;      // allocated per warp in 256-register units
    const int per_part = warp_regs > 0 ? (regs_sm / 4) / warp_regs : 64; // warps one sub-partition holds
    const int by_regs = per_part / ((warps + 3) / 4);                     // a block spreads over 4 sub-partitions
    const size_t blk_smem = ((dyn_smem + a.sharedSizeBytes + (size_t)reserved + 127) / 128) * 128;
    const int by_smem = blk_smem ? (int)((size_t)smem_sm / blk_smem) : blk_sm;
    const int by_thr = thr_sm / block;
    const int by_tmem = tmem_cols > 0 ? 512 / tmem_cols : blk_sm;
    int n = by_regs;
    if (by_smem < n) n = by_smem;
    if (by_thr < n) n = by_thr;
    if (blk_sm < n) n = blk_sm;
    if (by_tmem < n) n = by_tmem;
    *per_sm = n;
    return cudaSuccess;
}

}  // namespace ols

struct ols_plan_s {
    int device = 0;
    int sm_count = 0;
    int64_t N = 0;
    int log2N = 0;
    int32_t M = 0, F = 0;
    uint32_t flags = 0;
    bool filters_ready = false;
    ols::PassPlan pp{};
    float2 *Hk = nullptr;        // [F][N] spectra in kernel layout (FP32)
    float2 *Htk = nullptr;       // [F][N] spectra of conj(h_f[M-1-k]) (adjoint), kernel layout
    float2 *tw = nullptr;        // forward twiddles (FP32), pp.twn entries
    double2 *tw64 = nullptr;     // W_N^m, m in [0, N) (FP64)
    int32_t *nu = nullptr;       // spectral order (device copy)
    int fwd_grid_cap = 0;        // resident blocks of the forward kernel
    int bwd_grid_cap[3] = {0, 0, 0};  // backward kernel: (ds,dh), (ds), (dh)
    int last_launches = 0;
    int tc_grid_cap = 0;         // resident blocks of the tensor-core kernel
    int tc_split_grid_cap = 0;   // the same for its pre-split-input form
    long long tc_wait_limit = 0; // polls per in-loop mbarrier wait of the tensor-core kernel
    bool tc_wait_never = false;  // test switch: in-loop waits watch an mbarrier nothing arrives on
    int post_grid_cap[4] = {0, 0, 0, 0};  // post-processing kernels (power, detect, derivative, peaks)
    // real-to-real plans (OLS_FLAG_R2R)
    float2 *hpack = nullptr;     // [ceil(F/2)][M] paired real filters h_{2p} + i h_{2p+1}
    int r2r_grid_cap = 0;
    uint16_t *tc_bmat = nullptr; // split DFT-16 matrices (fwd hi, fwd lo, inv hi, inv lo), core-matrix layout
    int *d_status = nullptr;     // device status word (bounded-wait failures)
    ols::Staging stage;
};

namespace ols {

struct BackwardArgs {
    const float2 *s;
    int64_t Ns;
    const float2 *g;
    int64_t Nout, L, nseg;
    float2 *ds, *dh;
    float2 *edge;             // workspace: ds overlap edges (nseg x 2 x (M-1))
    float4 *P, *Pr;           // workspace: per-CTA dh spectra (grid x F x N/2), their sum (F x N/2)
    int grid;
};

// One problem of a batch, as the batched kernel reads it.
struct BatchProblemDev {
    const float4 *Hk;     // spectra in kernel layout
    long long Ns, Nout, L, nseg;
    int M, F;
    int index;            // position in the caller's pointer arrays
    int log2N;            // segment length of this problem
    int *status;          // the problem's plan status word (bounds checks of OLS_CHECK builds)
};

// Twiddle tables of every segment length, by log2 N (single-launch batches).
struct TwTables {
    const float2 *tw[kMaxLog2N + 1];
};

// The whole batch in one persistent launch: blocks of `block` threads (the
// longest segment's N/16, at least 128); a tile is block * 16 / N consecutive
// segments of one problem (one per N/16-thread slot), and an item (problem,
// first tile, tiles) a run of consecutive tiles taken with one ticket.
constexpr int kBatchOneBlock = 512;   // largest block (N = 8192 needs 512 threads)
cudaError_t batched_one_prepare(int block, int sm_count, int *grid_cap);
cudaError_t batched_one_launch(int block, int grid, const BatchProblemDev *probs, const int4 *items, long long nitems,
                               const float2 *const *s_ptrs, float2 *const *y_ptrs, unsigned long long *ticket,
                               const TwTables &tw, cudaStream_t st);

// One persistent launch: every problem of the batch with segment length 2^log2N.
struct BatchGroup {
    int log2N = 0;
    int grid = 0;
    long long nitems = 0;
    const BatchProblemDev *probs = nullptr;   // device
    const int2 *items = nullptr;              // device: (problem in group, tile)
    unsigned long long *ticket = nullptr;     // device counter, zeroed before each launch
    const float2 *tw = nullptr;               // twiddles of this N (from one of the problems' plans)
};

// Fused OLS with post-processing of the output (ols_post.cu).
enum PostMode { POST_POWER = 0, POST_DETECT = 1, POST_DERIV = 2, POST_PEAK = 3 };
struct PostArgs {
    int mode;
    const float2 *s;
    int64_t Ns, Nout, step, nseg;   // step: outputs per segment (L, or L-2 for the derivative)
    void *out;                      // POWER: float [F][Nout]; DERIV: float2 [F][Nout]
    float thr;                      // DETECT
    ols_candidate *cand;
    unsigned long long *count;
    int64_t cap;
};
cudaError_t post_prepare(ols_plan_s &p);
cudaError_t post_launch(const ols_plan_s &p, const PostArgs &a, cudaStream_t st);

// Real-to-real form (ols_r2r.cu): filters paired as h_{2p} + i h_{2p+1}.
cudaError_t launch_pack_real_pairs(const float *h, int M, int F, float2 *g, cudaStream_t st);
cudaError_t r2r_prepare(ols_plan_s &p);
cudaError_t r2r_launch(const ols_plan_s &p, const float *s, int64_t Ns, float *y, int64_t L, int64_t nseg,
                       int64_t Nout, cudaStream_t st);

// Tensor-core split-precision form (ols_tc.cu).  The signal is either FP32
// (s) or already split into 16-bit hi / lo planes of (Re, Im) pairs.
struct TcSignal {
    const float2 *s = nullptr;
    const uint32_t *hi = nullptr, *lo = nullptr;
};
cudaError_t tc_prepare(ols_plan_s &p, bool bf16);
cudaError_t tc_launch(const ols_plan_s &p, const TcSignal &sg, int64_t Ns, float2 *y, int64_t L, int64_t nseg,
                      int64_t Nout, cudaStream_t st);
cudaError_t launch_split_signal(const float2 *s, int64_t Ns, bool bf16, uint32_t *hi, uint32_t *lo, int sm_count,
                                cudaStream_t st);

cudaError_t batched_prepare(int log2N, int sm_count, int *grid_cap, int *segs);
cudaError_t batched_launch(const BatchGroup &g, const float2 *const *s_ptrs, float2 *const *y_ptrs,
                           cudaStream_t st);

// Forward fused OLS (Algorithm 2).  Returns a cudaError_t.
cudaError_t launch_forward(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y,
                           int64_t L, int64_t nseg, int64_t Nout, cudaStream_t st, int *launches);
// Occupancy / attribute set-up of the forward kernel for p.log2N.
cudaError_t prepare_forward(ols_plan_s &p);
// Argument checks shared by ols_convolve_backward and its allocation-free variant.
int backward_validate(ols_plan_t plan, const float *s, int64_t Ns, const float *g, const float *ds,
                      const float *dh);
// Adjoint (ds, dh) of the fused OLS: the window kernel plus the finishing
// kernel; `launches` receives the number of kernels enqueued.
cudaError_t prepare_backward(ols_plan_s &p);
cudaError_t launch_backward(const ols_plan_s &p, const BackwardArgs &a, cudaStream_t st, int *launches);
int backward_grid(const ols_plan_s &p, int64_t nseg, bool want_ds, bool want_dh);
int backward_segs_per_block(int log2N);
// FP64 precompute kernels.  adjoint != 0 transforms conj(h_f[M-1-k]) instead of h_f[k].
cudaError_t launch_tw64(double2 *tw64, int N, cudaStream_t st);
// Spectra in the 16-points-per-thread register layout of the kernels.
cudaError_t launch_spectra(const float2 *h, int M, int F, int log2N, const int32_t *nu,
                           const double2 *tw64, float2 *Hk, int adjoint, cudaStream_t st);
cudaError_t launch_spectra_natural(const float2 *Hk, int F, int log2N, const int32_t *nu,
                                   float2 *H, cudaStream_t st);

}  // namespace ols
