// ols_batch_api.cu -- C ABI of the batched form and the segment-length
// autotuner (include/ols.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "ols.h"
#include "ols_internal.h"

#ifndef OLS_BATCH_SMALL_BLOCKS
#define OLS_BATCH_SMALL_BLOCKS 1  // single launch: the smallest block holding the longest segment (else 512)
#endif

struct ols_batch_s {
    int device = 0;
    int sm_count = 0;
    int B = 0;
    std::vector<ols_plan_t> plans;            // one plain plan per problem (spectra, twiddles)
    std::vector<int64_t> Ns, Nout, N, L, nseg;
    std::vector<int32_t> M, F;
    std::vector<ols::BatchGroup> groups;
    ols::BatchProblemDev *d_probs = nullptr;
    int2 *d_items = nullptr;                  // per-segment-length mode: (problem, tile)
    int4 *d_items4 = nullptr;                 // single launch: (problem, first tile, tiles)
    std::vector<int32_t> tiles;               // single launch: tiles per item of each problem
    std::vector<int64_t> items_of;            // ... and the number of items of each problem
    unsigned long long *d_tickets = nullptr;
    bool filters_ready = false;
    int last_launches = 0;
    bool single = false;                      // the whole batch in one persistent launch
    int one_block = 0;                        // its block size
    ols::TwTables tw_all{};                   // single launch: twiddles of every segment length
};

namespace {

using namespace ols;

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return OLS_OK;
    if (e == cudaErrorMemoryAllocation) return OLS_ERR_ALLOC;
    return OLS_ERR_CUDA;
}

int log2_of(int64_t N) {
    if (N <= 0 || (N & (N - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < N) ++l;
    return l;
}

// ---------------------------------------------------------------- autotuner
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int64_t> g_tune_cache;
bool g_tune_file_loaded = false;

void load_tune_file_locked() {
    if (g_tune_file_loaded) return;
    g_tune_file_loaded = true;
    const char *path = std::getenv("OLS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *fh = std::fopen(path, "r");
    if (!fh) return;
    int m, f;
    long long n;
    while (std::fscanf(fh, "%d %d %lld", &m, &f, &n) == 3) {
        const int l = log2_of(n);
        if (m >= 1 && f >= 1 && l >= kMinLog2N && l <= kMaxLog2N && m <= n) g_tune_cache[{m, f}] = n;
    }
    std::fclose(fh);
}

void store_tune_file_locked(int M, int F, int64_t N) {
    const char *path = std::getenv("OLS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *fh = std::fopen(path, "a");
    if (!fh) return;
    std::fprintf(fh, "%d %d %lld\n", M, F, (long long)N);
    std::fclose(fh);
}

// Device time per output sample of the fused kernel for (N, M, F), on a
// zero signal of about two waves of segments (timing does not depend on the
// values), into *t.  Returns an ols_status (an allocation failure stays
// OLS_ERR_ALLOC).
int measure_per_output(int64_t N, int32_t M, int32_t F, double *t) {
    ols_plan_t p = nullptr;
    int rc = ols_plan(&p, N, M, F, OLS_FLAG_FP32);
    if (rc != OLS_OK) return rc;
    double result = -1.0;
    float2 *h = nullptr, *s = nullptr, *y = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int64_t L = N - M + 1;
    int64_t nseg = 2ll * p->fwd_grid_cap * 8;
    const int64_t max_out = (256ll << 20) / (8ll * F);          // <= 256 MB of output
    if (nseg * L > max_out) nseg = std::max<int64_t>(1, max_out / L);
    const int64_t Nout = nseg * L, Ns = Nout + M - 1;
    cudaError_t e = dev_alloc(&h, sizeof(float2) * (size_t)F * M);
    if (e == cudaSuccess) e = dev_alloc(&s, sizeof(float2) * (size_t)Ns);
    if (e == cudaSuccess) e = dev_alloc(&y, sizeof(float2) * (size_t)F * Nout);
    if (e == cudaSuccess) e = cudaMemset(h, 0, sizeof(float2) * (size_t)F * M);
    if (e == cudaSuccess) e = cudaMemset(s, 0, sizeof(float2) * (size_t)Ns);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && ols_set_filters(p, reinterpret_cast<float *>(h), nullptr) == OLS_OK) {
        bool ok = true;
        for (int w = 0; w < 2 && ok; ++w)
            ok = ols_convolve(p, reinterpret_cast<float *>(s), Ns, reinterpret_cast<float *>(y), nullptr) == OLS_OK;
        float best = 1e30f;
        for (int r = 0; r < 3 && ok; ++r) {
            cudaEventRecord(e0, nullptr);
            ok = ols_convolve(p, reinterpret_cast<float *>(s), Ns, reinterpret_cast<float *>(y), nullptr) == OLS_OK;
            cudaEventRecord(e1, nullptr);
            if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                best = std::min(best, ms);
            } else {
                ok = false;
            }
        }
        if (ok) result = (double)best * 1e-3 / (double)(F * Nout);
    }
    rc = e != cudaSuccess ? status_of(e) : (result < 0 ? OLS_ERR_CUDA : OLS_OK);
    *t = result;
    cudaDeviceSynchronize();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (h) cudaFree(h);
    if (s) cudaFree(s);
    if (y) cudaFree(y);
    ols_plan_destroy(p);
    return rc;
}

// ------------------------------------------------------ tile-schedule tuner
// An item of the single-launch batch is a run of consecutive tiles of one
// problem taken with one ticket; its length trades the per-item cost (the
// ticket, a block barrier, the twiddle fill) against the granularity of the
// dynamic schedule.  Candidates are 1, 2, 4 and 8 tiles per item.
constexpr int kTileChoices[4] = {1, 2, 4, 8};
std::map<std::tuple<int, int, int64_t, int>, int32_t> g_tiles_cache;   // (M, F, N, block) -> tiles

// Model: an item should carry at least ~32 transforms per slot (F + 1 per
// segment), so that the per-item cost stays within a few per cent.
int32_t tiles_model(int32_t F) {
    const int32_t want = (32 + F) / (F + 1);
    int32_t r = 1;
    while (r < want && r < 8) r *= 2;
    return r;
}

// Device time per output of the single-launch kernel for one problem of
// (M, F, N) in blocks of `block` threads, for each candidate run length, on
// a zero signal of about three waves of the longest items (at most ~1 GB of
// output); the shortest run within 1% of the fastest wins.  Returns an
// ols_status (an allocation failure stays OLS_ERR_ALLOC) and the choice.
int measure_tiles(int32_t M, int32_t F, int64_t N, int block, int sm_count, int32_t *best) {
    const int l = log2_of(N);
    if (block < N / 16) return OLS_ERR_UNSUPPORTED;
    int cap = 0;
    cudaError_t e0p = batched_one_prepare(block, sm_count, &cap);
    if (e0p != cudaSuccess) return status_of(e0p);
    ols_plan_t p = nullptr;
    int prc = ols_plan(&p, N, M, F, OLS_FLAG_FP32);
    if (prc != OLS_OK) return prc;
    const int64_t SL = (int64_t)block * 16 / N, L = N - M + 1;
    int64_t nseg = 3ll * cap * 8 * SL;
    const int64_t max_out = (int64_t(1) << 30) / (8ll * F);
    if (nseg * L > max_out) nseg = std::max<int64_t>(SL, max_out / L);
    const int64_t Nout = nseg * L, Ns = Nout + M - 1, ntiles = (nseg + SL - 1) / SL;
    float2 *h = nullptr, *s = nullptr, *y = nullptr;
    BatchProblemDev *dp = nullptr;
    int4 *di = nullptr;
    unsigned long long *tk = nullptr;
    void **ptrs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = OLS_ERR_CUDA;
    cudaError_t e = dev_alloc(&h, sizeof(float2) * (size_t)F * M);
    if (e == cudaSuccess) e = dev_alloc(&s, sizeof(float2) * (size_t)Ns);
    if (e == cudaSuccess) e = dev_alloc(&y, sizeof(float2) * (size_t)F * Nout);
    if (e == cudaSuccess) e = dev_alloc(&dp, sizeof(BatchProblemDev));
    if (e == cudaSuccess) e = dev_alloc(&di, sizeof(int4) * (size_t)ntiles);
    if (e == cudaSuccess) e = dev_alloc(&tk, sizeof(unsigned long long));
    if (e == cudaSuccess) e = dev_alloc(&ptrs, 2 * sizeof(void *));
    if (e == cudaSuccess) e = cudaMemset(h, 0, sizeof(float2) * (size_t)F * M);
    if (e == cudaSuccess) e = cudaMemset(s, 0, sizeof(float2) * (size_t)Ns);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess && ols_set_filters(p, reinterpret_cast<float *>(h), nullptr) != OLS_OK) e = cudaErrorUnknown;
    BatchProblemDev d{};
    d.Hk = reinterpret_cast<const float4 *>(p->Hk);
    d.Ns = Ns;
    d.Nout = Nout;
    d.L = L;
    d.nseg = nseg;
    d.M = M;
    d.F = F;
    d.index = 0;
    d.log2N = l;
    d.status = p->d_status;
    void *hp[2] = {s, y};
    if (e == cudaSuccess) e = cudaMemcpy(dp, &d, sizeof(d), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ptrs, hp, sizeof(hp), cudaMemcpyHostToDevice);
    TwTables tw{};
    tw.tw[l] = p->tw;
    double t_best = 1e300, t_of[4] = {0, 0, 0, 0};
    for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
        const int R = kTileChoices[c];
        std::vector<int4> items;
        for (int64_t t0 = 0; t0 < ntiles; t0 += R)
            items.push_back(make_int4(0, (int)t0, (int)std::min<int64_t>(R, ntiles - t0), 0));
        e = cudaMemcpy(di, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
        const int grid = (int)std::min<int64_t>((int64_t)items.size(), cap);
        float best_ms = 1e30f;
        for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
            e = cudaMemset(tk, 0, sizeof(unsigned long long));
            if (e == cudaSuccess) e = cudaEventRecord(e0, nullptr);
            if (e == cudaSuccess)
                e = batched_one_launch(block, grid, dp, di, (long long)items.size(),
                                       reinterpret_cast<const float2 *const *>(ptrs),
                                       reinterpret_cast<float2 *const *>(ptrs + 1), tk, tw, nullptr);
            if (e == cudaSuccess) e = cudaEventRecord(e1, nullptr);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && rep > 0) best_ms = std::min(best_ms, ms);   // rep 0 warms up
        }
        t_of[c] = (double)best_ms / (double)(F * Nout);
        t_best = std::min(t_best, t_of[c]);
    }
    if (e == cudaSuccess) {
        for (int c = 0; c < 4; ++c)
            if (t_of[c] <= 1.01 * t_best) {
                *best = kTileChoices[c];
                rc = OLS_OK;
                break;
            }
    } else {
        rc = status_of(e);
    }
    cudaDeviceSynchronize();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (void *q : {(void *)h, (void *)s, (void *)y, (void *)dp, (void *)di, (void *)tk, (void *)ptrs})
        if (q) cudaFree(q);
    ols_plan_destroy(p);
    return rc;
}

int tune_tiles(int32_t M, int32_t F, int64_t N, int block, int sm_count, uint32_t flags, int32_t *tiles) {
    if (flags & OLS_TUNE_MODEL) {
        *tiles = tiles_model(F);
        return OLS_OK;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    const auto key = std::make_tuple((int)M, (int)F, N, block);
    auto it = g_tiles_cache.find(key);
    if (it != g_tiles_cache.end()) {
        *tiles = it->second;
        return OLS_OK;
    }
    int32_t r = 0;
    const int rc = measure_tiles(M, F, N, block, sm_count, &r);
    if (rc != OLS_OK) return rc;
    g_tiles_cache[key] = r;
    *tiles = r;
    return OLS_OK;
}

void free_batch(ols_batch_s *b) {
    if (!b) return;
    for (ols_plan_t p : b->plans)
        if (p) ols_plan_destroy(p);
    if (b->d_probs) cudaFree(b->d_probs);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_items4) cudaFree(b->d_items4);
    if (b->d_tickets) cudaFree(b->d_tickets);
    delete b;
}

}  // namespace

extern "C" {

int ols_autotune(int32_t M, int32_t F, uint32_t flags, int64_t *N) {
    if (!N || M < 1 || F < 1) return OLS_ERR_INVALID;
    if (M > (1 << kMaxLog2N)) return OLS_ERR_UNSUPPORTED;
    if (flags & OLS_TUNE_MODEL) {
        *N = ols::choose_segment_length(M);
        return OLS_OK;
    }
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_tune_file_locked();
    auto it = g_tune_cache.find({M, F});
    if (it != g_tune_cache.end()) {
        *N = it->second;
        return OLS_OK;
    }
    double best = 1e300;
    int64_t bestN = 0;
    for (int l = kMinLog2N; l <= kMaxLog2N; ++l) {
        const int64_t n = int64_t(1) << l;
        if (M > n) continue;
        if ((n - M + 1) * 16 < n && n != (int64_t(1) << kMaxLog2N)) continue;   // < 1/16 of each FFT kept
        double t = -1.0;
        const int rc = measure_per_output(n, M, F, &t);
        if (rc != OLS_OK) return rc;
        if (t < best) {
            best = t;
            bestN = n;
        }
    }
    if (bestN == 0) return OLS_ERR_UNSUPPORTED;
    g_tune_cache[{M, F}] = bestN;
    store_tune_file_locked(M, F, bestN);
    *N = bestN;
    return OLS_OK;
}

int ols_batch_plan(ols_batch_t *out, int32_t B, const int64_t *Ns, const int32_t *M, const int32_t *F,
                   const int64_t *N, uint32_t flags) {
    return ols_batch_plan_tiles(out, B, Ns, M, F, N, nullptr, flags);
}

int ols_autotune_tiles(int32_t M, int32_t F, int64_t N, int32_t block, uint32_t flags, int32_t *tiles) {
    if (!tiles || M < 1 || F < 1) return OLS_ERR_INVALID;
    const int l = log2_of(N);
    if (l < kMinLog2N || l > kMaxLog2N || M > N) return OLS_ERR_UNSUPPORTED;
    if ((block != 128 && block != 256 && block != 512) || block < N / 16) return OLS_ERR_UNSUPPORTED;
    AllocScope scope;
    int dev = 0, sms = 0;
    if (!(flags & OLS_TUNE_MODEL)) {
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess)
            return OLS_ERR_CUDA;
    }
    return tune_tiles(M, F, N, block, sms, flags, tiles);
}

int ols_batch_plan_tiles(ols_batch_t *out, int32_t B, const int64_t *Ns, const int32_t *M, const int32_t *F,
                         const int64_t *N, const int32_t *tiles, uint32_t flags) {
    AllocScope scope;
    if (!out) return OLS_ERR_INVALID;
    *out = nullptr;
    if (B < 1 || !Ns || !M || !F) return OLS_ERR_INVALID;
    for (int b = 0; b < B; ++b)
        if (M[b] < 1 || F[b] < 1 || Ns[b] < M[b] || (tiles && tiles[b] < 0)) return OLS_ERR_INVALID;
    ols_batch_s *bt = new (std::nothrow) ols_batch_s();
    if (!bt) return OLS_ERR_ALLOC;
    bt->B = B;
    cudaError_t e = cudaGetDevice(&bt->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bt->sm_count, cudaDevAttrMultiProcessorCount, bt->device);
    if (e != cudaSuccess) {
        free_batch(bt);
        return status_of(e);
    }
    bt->plans.assign(B, nullptr);
    bt->Ns.assign(Ns, Ns + B);
    bt->M.assign(M, M + B);
    bt->F.assign(F, F + B);
    bt->N.resize(B);
    bt->Nout.resize(B);
    bt->L.resize(B);
    bt->nseg.resize(B);
    for (int b = 0; b < B; ++b) {
        int64_t n = N ? N[b] : 0;
        if (n == 0) {
            int rc = ols_autotune(M[b], F[b], flags, &n);
            if (rc != OLS_OK) {
                free_batch(bt);
                return rc;
            }
        }
        int rc = ols_plan(&bt->plans[b], n, M[b], F[b], OLS_FLAG_FP32);
        if (rc == OLS_OK) rc = ols_geometry(n, M[b], Ns[b], &bt->L[b], &bt->nseg[b], &bt->Nout[b]);
        if (rc != OLS_OK) {
            free_batch(bt);
            return rc;
        }
        bt->N[b] = n;
    }
    if (!(flags & OLS_BATCH_PER_N)) {
        // One persistent launch for every problem: tiles of (block x 16)/N
        // segments (one per slot of N/16 threads), items of one or more tiles.
        int cap = 0;
        int64_t maxN = 0;
        for (int b = 0; b < B; ++b) maxN = std::max<int64_t>(maxN, bt->N[b]);
        // the smallest block that holds a segment of the longest N (16 points per thread)
        bt->one_block = (int)std::min<int64_t>(512, std::max<int64_t>(128, maxN / 16));
        if (!OLS_BATCH_SMALL_BLOCKS) bt->one_block = 512;
        e = batched_one_prepare(bt->one_block, bt->sm_count, &cap);
        if (e != cudaSuccess) {
            free_batch(bt);
            return status_of(e);
        }
        bt->single = true;
        std::vector<BatchProblemDev> probs(B);
        for (int b = 0; b < B; ++b) {
            const int l = log2_of(bt->N[b]);
            BatchProblemDev &d = probs[b];
            d.Hk = reinterpret_cast<const float4 *>(bt->plans[b]->Hk);
            d.Ns = bt->Ns[b];
            d.Nout = bt->Nout[b];
            d.L = bt->L[b];
            d.nseg = bt->nseg[b];
            d.M = bt->M[b];
            d.F = bt->F[b];
            d.index = b;
            d.log2N = l;
            d.status = bt->plans[b]->d_status;
            bt->tw_all.tw[l] = bt->plans[b]->tw;
        }
        // tile schedule: tiles per item of each problem, given or tuned per
        // (M, F, N) for this block size; then, while the batch would have
        // fewer than 4 items per resident block, runs are halved (the
        // dynamic schedule needs items to balance the tail)
        bt->tiles.assign(B, 1);
        std::vector<int64_t> ntl(B);
        for (int b = 0; b < B; ++b) {
            const int64_t sl = (int64_t)bt->one_block * 16 / bt->N[b];
            ntl[b] = (bt->nseg[b] + sl - 1) / sl;
            int32_t r = tiles ? tiles[b] : 0;
            if (r == 0) {
                int rc = tune_tiles(bt->M[b], bt->F[b], bt->N[b], bt->one_block, bt->sm_count, flags, &r);
                if (rc != OLS_OK) {
                    free_batch(bt);
                    return rc;
                }
                bt->tiles[b] = -r;          // marks a tuned choice (may be halved below)
            } else {
                bt->tiles[b] = r;
            }
        }
        auto count_items = [&]() {
            int64_t n = 0;
            for (int b = 0; b < B; ++b) n += (ntl[b] + std::abs(bt->tiles[b]) - 1) / std::abs(bt->tiles[b]);
            return n;
        };
        for (bool shrunk = true; shrunk && count_items() < 4ll * cap;) {
            shrunk = false;
            for (int b = 0; b < B; ++b)
                if (bt->tiles[b] < -1) {
                    bt->tiles[b] /= 2;
                    shrunk = true;
                }
        }
        for (int b = 0; b < B; ++b) bt->tiles[b] = std::abs(bt->tiles[b]);
        // items, the most expensive first: a tile's work grows with F log2 N
        // (block x 16 points per tile whatever N), an item's with its tiles
        std::vector<int4> items;
        bt->items_of.assign(B, 0);
        for (int b = 0; b < B; ++b)
            for (int64_t t0 = 0; t0 < ntl[b]; t0 += bt->tiles[b]) {
                items.push_back(make_int4(b, (int)t0, (int)std::min<int64_t>(bt->tiles[b], ntl[b] - t0), 0));
                ++bt->items_of[b];
            }
        auto cost = [&](const int4 &it) {
            return (long long)it.z * bt->F[it.x] * log2_of(bt->N[it.x]);
        };
        std::stable_sort(items.begin(), items.end(), [&](const int4 &a, const int4 &c) { return cost(a) > cost(c); });
        BatchGroup g;
        g.log2N = 0;
        g.nitems = (long long)items.size();
        g.grid = (int)std::min<long long>(g.nitems, cap);
        e = dev_alloc(&bt->d_probs, sizeof(BatchProblemDev) * probs.size());
        if (e == cudaSuccess) e = dev_alloc(&bt->d_items4, sizeof(int4) * std::max<size_t>(1, items.size()));
        if (e == cudaSuccess) e = dev_alloc(&bt->d_tickets, sizeof(unsigned long long));
        if (e == cudaSuccess)
            e = cudaMemcpy(bt->d_probs, probs.data(), sizeof(BatchProblemDev) * probs.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpy(bt->d_items4, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_batch(bt);
            return status_of(e);
        }
        g.probs = bt->d_probs;
        g.ticket = bt->d_tickets;
        bt->groups.push_back(g);
        *out = bt;
        return OLS_OK;
    }
    // per segment length: one persistent launch per group; problems in a group by decreasing F
    std::vector<int> order(B);
    for (int b = 0; b < B; ++b) order[b] = b;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        if (bt->N[a] != bt->N[c]) return bt->N[a] < bt->N[c];
        return bt->F[a] > bt->F[c];
    });
    std::vector<BatchProblemDev> probs;
    std::vector<int2> items;
    std::vector<std::pair<size_t, size_t>> ranges;   // per group: probs begin, items begin
    for (size_t i = 0; i < order.size();) {
        const int l = log2_of(bt->N[order[i]]);
        BatchGroup g;
        g.log2N = l;
        int cap = 0, segs = 1;
        e = batched_prepare(l, bt->sm_count, &cap, &segs);
        if (e != cudaSuccess) {
            free_batch(bt);
            return status_of(e);
        }
        const size_t p0 = probs.size(), i0 = items.size();
        size_t j = i;
        for (; j < order.size() && bt->N[order[j]] == bt->N[order[i]]; ++j) {
            const int b = order[j];
            BatchProblemDev d{};
            d.Hk = reinterpret_cast<const float4 *>(bt->plans[b]->Hk);
            d.Ns = bt->Ns[b];
            d.Nout = bt->Nout[b];
            d.L = bt->L[b];
            d.nseg = bt->nseg[b];
            d.M = bt->M[b];
            d.F = bt->F[b];
            d.index = b;
            d.log2N = l;
            d.status = bt->plans[b]->d_status;
            const int pi = (int)(probs.size() - p0);
            probs.push_back(d);
            const int64_t tiles = (bt->nseg[b] + segs - 1) / segs;
            for (int64_t tl = 0; tl < tiles; ++tl) items.push_back(make_int2(pi, (int)tl));
        }
        g.nitems = (long long)(items.size() - i0);
        g.grid = (int)std::min<long long>(g.nitems, cap);
        g.tw = bt->plans[order[i]]->tw;
        bt->groups.push_back(g);
        ranges.push_back({p0, i0});
        i = j;
    }
    const size_t ng = bt->groups.size();
    e = dev_alloc(&bt->d_probs, sizeof(BatchProblemDev) * probs.size());
    if (e == cudaSuccess) e = dev_alloc(&bt->d_items, sizeof(int2) * std::max<size_t>(1, items.size()));
    if (e == cudaSuccess) e = dev_alloc(&bt->d_tickets, sizeof(unsigned long long) * ng);
    if (e == cudaSuccess)
        e = cudaMemcpy(bt->d_probs, probs.data(), sizeof(BatchProblemDev) * probs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpy(bt->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        free_batch(bt);
        return status_of(e);
    }
    for (size_t gi = 0; gi < ng; ++gi) {
        bt->groups[gi].probs = bt->d_probs + ranges[gi].first;
        bt->groups[gi].items = bt->d_items + ranges[gi].second;
        bt->groups[gi].ticket = bt->d_tickets + gi;
    }
    *out = bt;
    return OLS_OK;
}

int ols_batch_destroy(ols_batch_t batch) {
    if (!batch) return OLS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(batch);
    return status_of(e);
}

int ols_batch_query(ols_batch_t batch, int32_t b, int64_t *N, int64_t *Nout, int32_t *ngroups) {
    if (!batch || b < 0 || b >= batch->B) return OLS_ERR_INVALID;
    if (N) *N = batch->N[b];
    if (Nout) *Nout = batch->Nout[b];
    if (ngroups) *ngroups = (int32_t)batch->groups.size();
    return OLS_OK;
}

int ols_batch_set_filters(ols_batch_t batch, const float *const *h, void *stream) {
    if (!batch || !h) return OLS_ERR_INVALID;
    for (int b = 0; b < batch->B; ++b) {
        const int rc = ols_set_filters(batch->plans[b], h[b], stream);
        if (rc != OLS_OK) return rc;
    }
    batch->filters_ready = true;
    return OLS_OK;
}

int ols_convolve_batched(ols_batch_t batch, const void *s_ptrs, const void *y_ptrs, void *stream) {
    if (!batch || !s_ptrs || !y_ptrs) return OLS_ERR_INVALID;
    if (((uintptr_t)s_ptrs & 7u) || ((uintptr_t)y_ptrs & 7u)) return OLS_ERR_INVALID;
    if (!batch->filters_ready) return OLS_ERR_NOT_READY;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(batch->d_tickets, 0, sizeof(unsigned long long) * batch->groups.size(), st);
    int launches = 0;
    if (batch->single) {
        const BatchGroup &g = batch->groups[0];
        if (e == cudaSuccess)
            e = batched_one_launch(batch->one_block, g.grid, g.probs, batch->d_items4, g.nitems,
                                   static_cast<const float2 *const *>(s_ptrs),
                                   static_cast<float2 *const *>(y_ptrs), g.ticket, batch->tw_all, st);
        batch->last_launches = e == cudaSuccess ? 1 : 0;
        return status_of(e);
    }
    for (size_t gi = 0; gi < batch->groups.size() && e == cudaSuccess; ++gi) {
        e = batched_launch(batch->groups[gi], static_cast<const float2 *const *>(s_ptrs),
                           static_cast<float2 *const *>(y_ptrs), st);
        if (e == cudaSuccess) ++launches;
    }
    batch->last_launches = launches;
    return status_of(e);
}

int ols_batch_last_launch_count(ols_batch_t batch) { return batch ? batch->last_launches : -1; }

int ols_batch_status(ols_batch_t batch, int *status, int reset) {
    if (!batch || !status) return OLS_ERR_INVALID;
    int acc = 0;
    for (ols_plan_t p : batch->plans) {
        int v = 0;
        const int rc = ols_plan_status(p, &v, reset);
        if (rc != OLS_OK) return rc;
        acc |= v;
    }
    *status = acc;
    return OLS_OK;
}

int ols_batch_schedule(ols_batch_t batch, int32_t b, int32_t *tiles, int64_t *items) {
    if (!batch || b < 0 || b >= batch->B) return OLS_ERR_INVALID;
    if (!batch->single) return OLS_ERR_UNSUPPORTED;
    if (tiles) *tiles = batch->tiles[b];
    if (items) *items = batch->items_of[b];
    return OLS_OK;
}

}  // extern "C"
