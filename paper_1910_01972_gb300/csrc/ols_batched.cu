// ols_batched.cu -- many OLS problems of uneven size in persistent launches.
//
// A batch holds B independent problems (signal b of Ns_b samples, F_b
// filters of M_b taps, segment length N_b).  Problems that share N form a
// group; each group is one persistent launch of the fused kernel whose
// resident blocks pull work items -- a tile of Geo<>::SEGS consecutive
// segments of one problem -- from an atomic ticket until the group's item
// list is exhausted.  Items are ordered by decreasing filter count (the
// most expensive first) so the dynamic schedule ends with short items.  Each
// segment is processed exactly as by the plain kernel (ols_segment), so a
// batched result equals the single-problem result bit for bit.
#include <cuda_runtime.h>
#include <cstdint>

#include "ols_internal.h"
#include "ols_segment.cuh"

// Segment lengths whose batch items use the TMEM exchange (bit i: N = 2^(9 + i)):
// N = 2048 only.  The single-launch kernel holds every segment length's body,
// so it runs at the register budget of the hungriest one: with the exchange
// also at N = 1024 the batch took 9.10 instead of 8.87 ms, at 512 and 4096
// 10.6-11.1 ms.
#ifndef OLS_BATCH_TX_MASK
#define OLS_BATCH_TX_MASK 0x4
#endif
// ... and for the kernels of the per-segment-length mode (one segment length
// each): N = 2048 only as well (at every length: 8.90 against 8.86 ms)
#ifndef OLS_BATCH_PERN_TX_MASK
#define OLS_BATCH_PERN_TX_MASK 0x4
#endif

namespace ols {

template <int LOG2N>
__global__ void __launch_bounds__(Geo<LOG2N>::BLOCK, Geo<LOG2N>::MINB)
ols_batched_kernel(const BatchProblemDev *__restrict__ probs, const int2 *__restrict__ items, long long nitems,
                   const float2 *const *__restrict__ s_ptrs, float2 *const *__restrict__ y_ptrs,
                   unsigned long long *__restrict__ ticket, const float2 *__restrict__ twg) {
    using G = Geo<LOG2N>;
    extern __shared__ float4 smem_raw[];
    __shared__ long long item_sh;
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
    // the TMEM exchange at the segment lengths of OLS_BATCH_PERN_TX_MASK
    constexpr bool xch = in_tx_mask<LOG2N>(OLS_BATCH_PERN_TX_MASK);
    const TwTmemT<xch> tw{tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 128u};
    tw_tmem_fill<LOG2N, xch>(twg, tw.base, t);
#else
    (void)tbase;
    const TwGlobal tw{twg};
#endif
    int xc = 0;
    for (;;) {
        __syncthreads();                       // previous item_sh readers are done
        if (threadIdx.x == 0) item_sh = (long long)atomicAdd(ticket, 1ull);
        __syncthreads();
        const long long item = item_sh;
        if (item >= nitems) break;
        const int2 it = items[item];           // (problem, tile)
        const BatchProblemDev P = probs[it.x];
        const long long nseg = P.nseg;
        const long long seg = (long long)it.y * G::SEGS + slot;
        ols_segment<LOG2N>(s_ptrs[P.index], P.Ns, P.Hk, tw, y_ptrs[P.index], P.M, P.F, P.L, P.Nout, seg,
                           seg < nseg, bufs, t, xc, 0u, CtaBarrier{}, P.status);
    }
#if OLS_FWD_TW_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, G::TMEM_COLS);
#endif
}

template <int LOG2N>
static cudaError_t batched_prepare_n(int sm_count, int *grid_cap, int *segs) {
    using G = Geo<LOG2N>;
    cudaError_t e = cudaFuncSetAttribute(ols_batched_kernel<LOG2N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)G::SMEM_TMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_FWD_TW_TMEM)
        e = resident_blocks_tmem(ols_batched_kernel<LOG2N>, G::BLOCK, G::SMEM_TMEM, (int)G::TMEM_COLS, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_batched_kernel<LOG2N>, G::BLOCK, G::SMEM_TMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (OLS_FWD_TW_TMEM && per_sm > G::TMEM_MAX_CTAS) per_sm = G::TMEM_MAX_CTAS;
    *grid_cap = per_sm * sm_count;
    *segs = G::SEGS;
    return cudaSuccess;
}

cudaError_t batched_prepare(int log2N, int sm_count, int *grid_cap, int *segs) {
    switch (log2N) {
        case 8: return batched_prepare_n<8>(sm_count, grid_cap, segs);
        case 9: return batched_prepare_n<9>(sm_count, grid_cap, segs);
        case 10: return batched_prepare_n<10>(sm_count, grid_cap, segs);
        case 11: return batched_prepare_n<11>(sm_count, grid_cap, segs);
        case 12: return batched_prepare_n<12>(sm_count, grid_cap, segs);
        case 13: return batched_prepare_n<13>(sm_count, grid_cap, segs);
        default: return cudaErrorInvalidValue;
    }
}

template <int LOG2N>
static void batched_launch_n(const BatchGroup &g, const float2 *const *s_ptrs, float2 *const *y_ptrs,
                             cudaStream_t st) {
    using G = Geo<LOG2N>;
    ols_batched_kernel<LOG2N><<<g.grid, G::BLOCK, G::SMEM_TMEM, st>>>(g.probs, g.items, g.nitems, s_ptrs, y_ptrs,
                                                                 g.ticket, g.tw);
}

cudaError_t batched_launch(const BatchGroup &g, const float2 *const *s_ptrs, float2 *const *y_ptrs,
                           cudaStream_t st) {
    switch (g.log2N) {
        case 8: batched_launch_n<8>(g, s_ptrs, y_ptrs, st); break;
        case 9: batched_launch_n<9>(g, s_ptrs, y_ptrs, st); break;
        case 10: batched_launch_n<10>(g, s_ptrs, y_ptrs, st); break;
        case 11: batched_launch_n<11>(g, s_ptrs, y_ptrs, st); break;
        case 12: batched_launch_n<12>(g, s_ptrs, y_ptrs, st); break;
        case 13: batched_launch_n<13>(g, s_ptrs, y_ptrs, st); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The whole batch in ONE persistent launch.  Blocks of 512 threads pull items
// from one ticket; a tile is SL = 512 / (N/16) consecutive segments of one
// problem (one per slot of N/16 threads), so every segment length fills the
// block and needs the same shared memory (two padded exchange buffers per
// slot: 139 KB).  The slots of an item run independently: each exchanges
// under its own named barrier (a warp barrier when a slot is within a warp);
// the block synchronises only to take the next item.  An item is a run of
// consecutive tiles of one problem (its length, the tile schedule, is picked
// per (M, F) by the autotuner): the block takes one ticket and loads its
// twiddles once for the whole run.  Each segment is
// processed exactly as by the plain kernel, so results are bitwise those of
// per-problem calls.
template <int BB, int LOG2N>
__device__ __forceinline__ void batch_one_tile(const BatchProblemDev &P, int tile, bool fill,
                                               const float2 *const *s_ptrs, float2 *const *y_ptrs, const float2 *tw,
                                               float2 *smem, int &xc, uint32_t tbase) {
    using G = Geo<LOG2N>;
    if constexpr (G::T <= BB) {
        constexpr int SL = BB / G::T;
        static_assert(SL <= 15 || G::T <= 32, "one named barrier per slot");
        const int slot = threadIdx.x / G::T;
        const int t = threadIdx.x % G::T;
        float2 *bufs = smem + slot * 2 * G::PADN;
        const long long seg = (long long)tile * SL + slot;
        const SegmentBarrier<G::T> bar{1 + slot};
#if OLS_FWD_TW_TMEM
        // the same TMEM layout as the plain kernel (twiddles of this N, then the
        // segment spectrum), so results stay bitwise those of per-problem calls
        // (the TMEM exchange at the segment lengths of OLS_BATCH_TX_MASK); the
        // twiddles are written on an item's first tile only
        constexpr bool xch = in_tx_mask<LOG2N>(OLS_BATCH_TX_MASK);
        using TWT = TwTmemT<xch>;
        const TWT twt{tbase + tmem::lane_bits() + (uint32_t)(threadIdx.x / 128) * 128u};
        if (fill) tw_tmem_fill<LOG2N, xch>(tw, twt.base, t);
        ols_segment<LOG2N, TWT, true, SegmentBarrier<G::T>>(s_ptrs[P.index], P.Ns, P.Hk, twt, y_ptrs[P.index],
                                                               P.M, P.F, P.L, P.Nout, seg, seg < P.nseg, bufs, t, xc,
                                                               0u, bar, P.status);
#else
        (void)tbase;
        (void)fill;
        ols_segment<LOG2N, TwGlobal, false, SegmentBarrier<G::T>>(s_ptrs[P.index], P.Ns, P.Hk, TwGlobal{tw},
                                                                  y_ptrs[P.index], P.M, P.F, P.L, P.Nout, seg,
                                                                  seg < P.nseg, bufs, t, xc, 0u, bar, P.status);
#endif
    }
}

template <int BB>
__global__ void __launch_bounds__(BB, kBatchOneBlock / BB)
ols_batched_one_kernel(const BatchProblemDev *__restrict__ probs, const int4 *__restrict__ items, long long nitems,
                       const float2 *const *__restrict__ s_ptrs, float2 *const *__restrict__ y_ptrs,
                       unsigned long long *__restrict__ ticket, TwTables tw) {
    extern __shared__ float4 smem_raw[];
    __shared__ long long item_sh;
    __shared__ uint32_t tbase;
    float2 *smem = reinterpret_cast<float2 *>(smem_raw);
#if OLS_FWD_TW_TMEM
    constexpr uint32_t kCols = (uint32_t)(BB / 128) * 128u;   // a 128-column lane range per 128 threads
    if (threadIdx.x < 32) tmem::alloc(&tbase, kCols);
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
#else
    tbase = 0;
#endif
    int xc = 0;
    // One tile per iteration.  An item's tiles run one after another (a slot
    // takes segment `slot` of each tile without synchronising with the other
    // slots); the block synchronises only to take the next item.  Only the
    // item index and the tiles left stay live across tiles: the item and its
    // problem are read again for every tile (cache hits), which keeps the
    // tile body at the register budget of one-tile items.
    long long item = 0;
    int r = 0, left = 0;
    for (;;) {
        if (left == 0) {
            __syncthreads();                   // every slot is done with the previous item
            if (threadIdx.x == 0) item_sh = (long long)atomicAdd(ticket, 1ull);
            __syncthreads();
            item = item_sh;
            if (item >= nitems) break;
            left = items[item].z;
            r = 0;
            xc = 0;                            // buffers restart with every item
        }
        const int4 it = items[item];           // (problem, first tile, tiles)
        const BatchProblemDev P = probs[it.x];
        const int tile = it.y + r;
        switch (P.log2N) {
            case 8: batch_one_tile<BB, 8>(P, tile, r == 0, s_ptrs, y_ptrs, tw.tw[8], smem, xc, tbase); break;
            case 9: batch_one_tile<BB, 9>(P, tile, r == 0, s_ptrs, y_ptrs, tw.tw[9], smem, xc, tbase); break;
            case 10: batch_one_tile<BB, 10>(P, tile, r == 0, s_ptrs, y_ptrs, tw.tw[10], smem, xc, tbase); break;
            case 11: batch_one_tile<BB, 11>(P, tile, r == 0, s_ptrs, y_ptrs, tw.tw[11], smem, xc, tbase); break;
            case 12: batch_one_tile<BB, 12>(P, tile, r == 0, s_ptrs, y_ptrs, tw.tw[12], smem, xc, tbase); break;
            case 13: batch_one_tile<BB, 13>(P, tile, r == 0, s_ptrs, y_ptrs, tw.tw[13], smem, xc, tbase); break;
            default: break;
        }
        ++r;
        --left;
    }
#if OLS_FWD_TW_TMEM
    tmem::fence_before_sync();
    __syncthreads();
    tmem::fence_after_sync();
    if (threadIdx.x < 32) tmem::dealloc(tbase, kCols);
#endif
}

// two padded exchange buffers per slot; the same for every N
template <int BB>
constexpr size_t batch_one_smem() { return sizeof(float2) * 2 * (size_t)(BB * 16 + BB); }

template <int BB>
static cudaError_t batched_one_prepare_b(int sm_count, int *grid_cap) {
    cudaError_t e = cudaFuncSetAttribute(ols_batched_one_kernel<BB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)batch_one_smem<BB>());
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (OLS_FWD_TW_TMEM)
        e = resident_blocks_tmem(ols_batched_one_kernel<BB>, BB, batch_one_smem<BB>(), (BB / 128) * 128, &per_sm);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ols_batched_one_kernel<BB>, BB,
                                                          batch_one_smem<BB>());
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    *grid_cap = per_sm * sm_count;
    return cudaSuccess;
}

cudaError_t batched_one_prepare(int block, int sm_count, int *grid_cap) {
    if (block == 128) return batched_one_prepare_b<128>(sm_count, grid_cap);
    if (block == 256) return batched_one_prepare_b<256>(sm_count, grid_cap);
    if (block == 512) return batched_one_prepare_b<512>(sm_count, grid_cap);
    return cudaErrorInvalidValue;
}

cudaError_t batched_one_launch(int block, int grid, const BatchProblemDev *probs, const int4 *items, long long nitems,
                               const float2 *const *s_ptrs, float2 *const *y_ptrs, unsigned long long *ticket,
                               const TwTables &tw, cudaStream_t st) {
    if (block == 128)
        ols_batched_one_kernel<128><<<grid, 128, batch_one_smem<128>(), st>>>(probs, items, nitems, s_ptrs, y_ptrs,
                                                                            ticket, tw);
    else if (block == 256)
        ols_batched_one_kernel<256><<<grid, 256, batch_one_smem<256>(), st>>>(probs, items, nitems, s_ptrs, y_ptrs,
                                                                            ticket, tw);
    else if (block == 512)
        ols_batched_one_kernel<512><<<grid, 512, batch_one_smem<512>(), st>>>(probs, items, nitems, s_ptrs, y_ptrs,
                                                                            ticket, tw);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace ols
