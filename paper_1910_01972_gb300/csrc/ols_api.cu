// ols_api.cu -- the C ABI of include/ols.h: argument checks, plans, tables,
// and the host-buffer pipeline.  All arithmetic of the convolution runs in
// the kernels of ols_forward.cu and ols_precompute.cu.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ols.h"
#include "ols_internal.h"

namespace ols {

// Frequency index at each storage position of the forward FFT output.  The
// forward passes are decimation in frequency: pass p splits the current
// block of size B into r_p interleaved sub-blocks of stride s_p = B / r_p and
// stores output k1 of its DFT in sub-block k1.  Position q therefore
// decomposes into digits (k1 of pass 0 = q / s_0, ...), and the frequency is
// those digits read in reverse significance: nu = k1_0 + r_0 (k1_1 + r_1 (...)).
void spectral_order(int log2N, int32_t *nu) {
    const PassPlan pp = make_pass_plan(log2N);
    for (int q0 = 0; q0 < pp.N; ++q0) {
        int q = q0, size = pp.N, mult = 1, v = 0;
        for (int p = 0; p < pp.np; ++p) {
            const int s = size / pp.radix[p];
            v += (q / s) * mult;
            q %= s;
            mult *= pp.radix[p];
            size = s;
        }
        nu[q0] = v;
    }
}

static std::vector<float2> forward_twiddles(const PassPlan &pp) {
    // pass p < np-1: entry (k-1) s + n' = W_{16 s}^{n' k}, k in [1, 16), n' in [0, s)
    std::vector<float2> tw((size_t)pp.twn);
    for (int p = 0; p + 1 < pp.np; ++p) {
        const int s = pp.stride[p], B = 16 * s;
        for (int k = 1; k < 16; ++k)
            for (int n = 0; n < s; ++n) {
                const long long e = ((long long)n * k) % B;
                const double a = -2.0 * M_PI * (double)e / (double)B;
                tw[(size_t)pp.tw_off[p] + (size_t)(k - 1) * s + n] =
                    make_float2((float)std::cos(a), (float)std::sin(a));
            }
    }
    return tw;
}

// The DFT-16 as the real 32x32 matrix B[k][n] of D = A B with
// A = [Re x | Im x], D = [Re y | Im y]: B = [[C, S], [-S, C]], C = cos(2 pi pq/16),
// S = Im W^{pq} (-sin forward, +sin inverse); split B = B_hi + B_lo in 16-bit
// (FP16 or BF16) and stored in the tensor-core shared-memory layout (no
// swizzle, K-major core matrices of 8 rows x 16 bytes: element (k, n) at byte
// (k/8) 512 + (n/8) 128 + (n%8) 16 + (k%8) 2).  Order: fwd hi, fwd lo, inv hi, inv lo.
static std::vector<uint16_t> tc_dft16_tables(bool bf16) {
    std::vector<uint16_t> out(4 * 1024);
    for (int inv = 0; inv < 2; ++inv)
        for (int k = 0; k < 32; ++k)
            for (int n = 0; n < 32; ++n) {
                const int p = k % 16, q = n % 16;
                const double th = 2.0 * M_PI * (double)((p * q) % 16) / 16.0;
                const double c = std::cos(th), s = (inv ? 1.0 : -1.0) * std::sin(th);
                double v;
                if (k < 16) v = n < 16 ? c : s;
                else v = n < 16 ? -s : c;
                uint16_t hi, lo;
                if (bf16) {
                    const __nv_bfloat16 h = __double2bfloat16(v);
                    const __nv_bfloat16 l = __double2bfloat16(v - (double)__bfloat162float(h));
                    hi = *reinterpret_cast<const uint16_t *>(&h);
                    lo = *reinterpret_cast<const uint16_t *>(&l);
                } else {
                    const __half h = __double2half(v);
                    const __half l = __double2half(v - (double)__half2float(h));
                    hi = *reinterpret_cast<const uint16_t *>(&h);
                    lo = *reinterpret_cast<const uint16_t *>(&l);
                }
                const int e = ((k / 8) * 512 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2) / 2;
                out[(size_t)(2 * inv) * 1024 + e] = hi;
                out[(size_t)(2 * inv + 1) * 1024 + e] = lo;
            }
    return out;
}

static thread_local int t_alloc_depth = 0;
static thread_local int t_alloc_seq = 0;

AllocScope::AllocScope() {
    if (t_alloc_depth++ == 0) t_alloc_seq = 0;
}
AllocScope::~AllocScope() { --t_alloc_depth; }

cudaError_t dev_alloc_raw(void **p, size_t bytes) {
    ++t_alloc_seq;
    const char *v = std::getenv("OLS_FAIL_ALLOC");
    if (v && std::atoi(v) > 0 && std::atoi(v) == t_alloc_seq) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

static int log2_exact(int64_t N) {
    if (N <= 0 || (N & (N - 1))) return -1;
    int l = 0;
    while ((int64_t(1) << l) < N) ++l;
    return l;
}

static bool aligned8(const void *p) { return ((uintptr_t)p & 7u) == 0; }
static bool aligned4(const void *p) { return ((uintptr_t)p & 3u) == 0; }

// The fused convolution in the plan's arithmetic (FP32 or tensor-core split).
static cudaError_t launch_any(const ols_plan_s &p, const float2 *s, int64_t Ns, float2 *y, int64_t L, int64_t nseg,
                              int64_t Nout, cudaStream_t st, int *launches) {
    if (p.flags == OLS_FLAG_FP32) return launch_forward(p, s, Ns, y, L, nseg, Nout, st, launches);
    *launches = 1;
    TcSignal sg;
    sg.s = s;
    return tc_launch(p, sg, Ns, y, L, nseg, Nout, st);
}

static int status_of(cudaError_t e) {
    if (e == cudaSuccess) return OLS_OK;
    if (e == cudaErrorMemoryAllocation) return OLS_ERR_ALLOC;
    return OLS_ERR_CUDA;
}

// Segment-length rule (Sec. 3.2 and Sec. 5): a longer segment wastes a
// smaller fraction M-1 of each FFT but costs log2(N) per point; pick the N
// minimising the work per valid output, (N / L) (log2 N + c).
int64_t choose_segment_length(int32_t M) {
    double best = 1e300;
    int64_t bestN = 0;
    for (int l = kMinLog2N; l <= kMaxLog2N; ++l) {
        const int64_t N = int64_t(1) << l;
        if (M > N) continue;
        const double L = (double)(N - M + 1);
        const double cost = (double)N / L * ((double)l + 2.0);
        if (cost < best) {
            best = cost;
            bestN = N;
        }
    }
    return bestN;
}

static void free_staging(Staging &s) {
    for (int i = 0; i < 2; ++i) {
        if (s.in[i]) cudaFree(s.in[i]);
        if (s.out[i]) cudaFree(s.out[i]);
        if (s.st[i]) cudaStreamDestroy(s.st[i]);
        if (s.ev_done[i]) cudaEventDestroy(s.ev_done[i]);
        s.in[i] = s.out[i] = nullptr;
        s.st[i] = nullptr;
        s.ev_done[i] = nullptr;
    }
    if (s.ev_user) cudaEventDestroy(s.ev_user);
    s.ev_user = nullptr;
    for (cudaEvent_t ev : s.tev) cudaEventDestroy(ev);
    s.tev.clear();
    s.timed_chunks = 0;
    s.in_cap = s.out_cap = 0;
}

static void free_plan(ols_plan_s *p) {
    if (!p) return;
    if (p->Hk) cudaFree(p->Hk);
    if (p->Htk) cudaFree(p->Htk);
    if (p->tw) cudaFree(p->tw);
    if (p->tw64) cudaFree(p->tw64);
    if (p->nu) cudaFree(p->nu);
    if (p->tc_bmat) cudaFree(p->tc_bmat);
    if (p->hpack) cudaFree(p->hpack);
    if (p->d_status) cudaFree(p->d_status);
    free_staging(p->stage);
    delete p;
}

}  // namespace ols

using namespace ols;

extern "C" {

const char *ols_status_string(int status) {
    switch (status) {
        case OLS_OK: return "OLS_OK";
        case OLS_ERR_INVALID: return "OLS_ERR_INVALID: invalid argument";
        case OLS_ERR_UNSUPPORTED: return "OLS_ERR_UNSUPPORTED: unsupported size or flag";
        case OLS_ERR_ALLOC: return "OLS_ERR_ALLOC: allocation failed";
        case OLS_ERR_CUDA: return "OLS_ERR_CUDA: CUDA runtime error";
        case OLS_ERR_NOT_READY: return "OLS_ERR_NOT_READY: filters not set";
        case OLS_ERR_TIMEOUT: return "OLS_ERR_TIMEOUT: bounded device wait gave up";
        case OLS_ERR_WORKSPACE: return "OLS_ERR_WORKSPACE: workspace missing or too small";
        case OLS_ERR_TOO_LARGE: return "OLS_ERR_TOO_LARGE: problem exceeds the built-in scratch size";
        default: return "OLS_ERR_UNKNOWN";
    }
}

int ols_version(void) { return 101; }   // 1.1: split-storage input, batch tile schedules and status, host stage timing, peaks

int ols_geometry(int64_t N, int32_t M, int64_t Ns, int64_t *L, int64_t *nseg, int64_t *Nout) {
    if (M < 1 || Ns < M) return OLS_ERR_INVALID;
    const int l = log2_exact(N);
    if (l < kMinLog2N || l > kMaxLog2N || M > N) return OLS_ERR_UNSUPPORTED;
    const int64_t Lv = N - M + 1;
    const int64_t no = Ns - M + 1;
    if (L) *L = Lv;
    if (Nout) *Nout = no;
    if (nseg) *nseg = (no + Lv - 1) / Lv;
    return OLS_OK;
}

int ols_spectrum_order(int64_t N, int32_t *nu) {
    if (!nu) return OLS_ERR_INVALID;
    const int l = log2_exact(N);
    if (l < kMinLog2N || l > kMaxLog2N) return OLS_ERR_UNSUPPORTED;
    spectral_order(l, nu);
    return OLS_OK;
}

int ols_plan(ols_plan_t *out, int64_t N, int32_t M, int32_t F, uint32_t flags) {
    AllocScope scope;
    if (!out) return OLS_ERR_INVALID;
    *out = nullptr;
    if (M < 1 || F < 1) return OLS_ERR_INVALID;
    if (flags != OLS_FLAG_FP32 && flags != OLS_FLAG_TC_FP16SPLIT && flags != OLS_FLAG_TC_BF16SPLIT &&
        flags != OLS_FLAG_R2R)
        return OLS_ERR_UNSUPPORTED;
    if (N == 0) N = choose_segment_length(M);
    const int l = log2_exact(N);
    if (l < kMinLog2N || l > kMaxLog2N || M > N) return OLS_ERR_UNSUPPORTED;

    ols_plan_s *p = new (std::nothrow) ols_plan_s();
    if (!p) return OLS_ERR_ALLOC;
    p->N = N;
    p->log2N = l;
    p->M = M;
    p->F = F;
    p->flags = flags;
    p->pp = make_pass_plan(l);
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device);
    const bool r2r = flags == OLS_FLAG_R2R;
    const int32_t Fc = r2r ? (F + 1) / 2 : F;       // complex spectra held: paired filters for R2R
    if (e == cudaSuccess) e = dev_alloc(&p->Hk, sizeof(float2) * (size_t)Fc * (size_t)N);
    if (e == cudaSuccess && !r2r) e = dev_alloc(&p->Htk, sizeof(float2) * (size_t)F * (size_t)N);
    if (e == cudaSuccess && r2r) e = dev_alloc(&p->hpack, sizeof(float2) * (size_t)Fc * (size_t)M);
    if (e == cudaSuccess && r2r) e = r2r_prepare(*p);
    if (e == cudaSuccess) e = dev_alloc(&p->tw, sizeof(float2) * (size_t)(p->pp.twn > 0 ? p->pp.twn : 1));
    if (e == cudaSuccess) e = dev_alloc(&p->tw64, sizeof(double2) * (size_t)N);
    if (e == cudaSuccess) e = dev_alloc(&p->nu, sizeof(int32_t) * (size_t)N);
    if (e == cudaSuccess) e = dev_alloc(&p->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
    // In-loop waits of the tensor-core kernel (read at plan creation):
    // OLS_TC_WAIT_LIMIT (polls) overrides the default limit, and
    // OLS_TC_WAIT_NEVER=1 points them at an mbarrier nothing arrives on, so a
    // test can make a wait run out without any fault.
    p->tc_wait_limit = 1ll << 20;
    if (const char *wl = std::getenv("OLS_TC_WAIT_LIMIT")) {
        const long long v = std::atoll(wl);
        if (v > 0) p->tc_wait_limit = v;
    }
    if (const char *wn = std::getenv("OLS_TC_WAIT_NEVER")) p->tc_wait_never = wn[0] == '1';
    if (e == cudaSuccess && flags != OLS_FLAG_FP32 && flags != OLS_FLAG_R2R) {
        const std::vector<uint16_t> b = tc_dft16_tables(flags == OLS_FLAG_TC_BF16SPLIT);
        e = dev_alloc(&p->tc_bmat, sizeof(uint16_t) * b.size());
        if (e == cudaSuccess) e = cudaMemcpy(p->tc_bmat, b.data(), sizeof(uint16_t) * b.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = tc_prepare(*p, flags == OLS_FLAG_TC_BF16SPLIT);
    }
    if (e == cudaSuccess) {
        std::vector<float2> tw = forward_twiddles(p->pp);
        std::vector<int32_t> nu((size_t)N);
        spectral_order(l, nu.data());
        if (!tw.empty()) e = cudaMemcpy(p->tw, tw.data(), sizeof(float2) * tw.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(p->nu, nu.data(), sizeof(int32_t) * nu.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = launch_tw64(p->tw64, (int)N, 0);
    if (e == cudaSuccess) e = prepare_forward(*p);
    if (e == cudaSuccess && flags == OLS_FLAG_FP32) e = post_prepare(*p);
    if (e == cudaSuccess) e = prepare_backward(*p);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        free_plan(p);
        return status_of(e);
    }
    *out = p;
    return OLS_OK;
}

int ols_plan_destroy(ols_plan_t plan) {
    if (!plan) return OLS_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(plan);
    return status_of(e);
}

int ols_plan_query(ols_plan_t plan, int64_t Ns, int64_t *N, int32_t *M, int32_t *F, int64_t *L,
                   int64_t *nseg, int64_t *Nout) {
    if (!plan) return OLS_ERR_INVALID;
    if (N) *N = plan->N;
    if (M) *M = plan->M;
    if (F) *F = plan->F;
    if (Ns == 0) {
        if (L) *L = plan->N - plan->M + 1;
        if (nseg) *nseg = 0;
        if (Nout) *Nout = 0;
        return OLS_OK;
    }
    return ols_geometry(plan->N, plan->M, Ns, L, nseg, Nout);
}

int ols_set_filters(ols_plan_t plan, const float *h, void *stream) {
    if (!plan || !h || !aligned8(h)) return OLS_ERR_INVALID;
    if (plan->flags == OLS_FLAG_R2R) return OLS_ERR_UNSUPPORTED;
    const float2 *hh = reinterpret_cast<const float2 *>(h);
    cudaError_t e = launch_spectra(hh, plan->M, plan->F, plan->log2N, plan->nu, plan->tw64, plan->Hk, 0,
                                   (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = launch_spectra(hh, plan->M, plan->F, plan->log2N, plan->nu, plan->tw64, plan->Htk, 1,
                           (cudaStream_t)stream);
    if (e != cudaSuccess) return status_of(e);
    plan->filters_ready = true;
    return OLS_OK;
}

int ols_get_spectra(ols_plan_t plan, float *H, void *stream) {
    if (!plan || !H || !aligned8(H)) return OLS_ERR_INVALID;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    const int Fc = plan->flags == OLS_FLAG_R2R ? (plan->F + 1) / 2 : plan->F;
    return status_of(launch_spectra_natural(plan->Hk, Fc, plan->log2N, plan->nu,
                                            reinterpret_cast<float2 *>(H), (cudaStream_t)stream));
}

int ols_convolve(ols_plan_t plan, const float *s, int64_t Ns, float *y, void *stream) {
    if (!plan || !s || !y || !aligned8(s) || !aligned8(y)) return OLS_ERR_INVALID;
    if (plan->flags == OLS_FLAG_R2R) return OLS_ERR_UNSUPPORTED;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    int launches = 0;
    cudaError_t e = launch_any(*plan, reinterpret_cast<const float2 *>(s), Ns, reinterpret_cast<float2 *>(y), L,
                               nseg, Nout, (cudaStream_t)stream, &launches);
    plan->last_launches = launches;
    return status_of(e);
}

int ols_split_signal(ols_plan_t plan, const float *s, int64_t Ns, void *s_hi, void *s_lo, void *stream) {
    if (!plan || !s || !s_hi || !s_lo || !aligned8(s) || !aligned4(s_hi) || !aligned4(s_lo) || Ns < 0)
        return OLS_ERR_INVALID;
    if (plan->flags != OLS_FLAG_TC_FP16SPLIT && plan->flags != OLS_FLAG_TC_BF16SPLIT) return OLS_ERR_UNSUPPORTED;
    if (Ns == 0) return OLS_OK;
    cudaError_t e = launch_split_signal(reinterpret_cast<const float2 *>(s), Ns,
                                        plan->flags == OLS_FLAG_TC_BF16SPLIT, static_cast<uint32_t *>(s_hi),
                                        static_cast<uint32_t *>(s_lo), plan->sm_count, (cudaStream_t)stream);
    return status_of(e);
}

int ols_convolve_split(ols_plan_t plan, const void *s_hi, const void *s_lo, int64_t Ns, float *y, void *stream) {
    if (!plan || !s_hi || !s_lo || !y || !aligned4(s_hi) || !aligned4(s_lo) || !aligned8(y)) return OLS_ERR_INVALID;
    if (plan->flags != OLS_FLAG_TC_FP16SPLIT && plan->flags != OLS_FLAG_TC_BF16SPLIT) return OLS_ERR_UNSUPPORTED;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    TcSignal sg;
    sg.hi = static_cast<const uint32_t *>(s_hi);
    sg.lo = static_cast<const uint32_t *>(s_lo);
    cudaError_t e = tc_launch(*plan, sg, Ns, reinterpret_cast<float2 *>(y), L, nseg, Nout, (cudaStream_t)stream);
    plan->last_launches = 1;
    return status_of(e);
}

int ols_set_filters_real(ols_plan_t plan, const float *h, void *stream) {
    if (!plan || !h || !aligned4(h)) return OLS_ERR_INVALID;
    if (plan->flags != OLS_FLAG_R2R) return OLS_ERR_UNSUPPORTED;
    const int Fc = (plan->F + 1) / 2;
    cudaError_t e = launch_pack_real_pairs(h, plan->M, plan->F, plan->hpack, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = launch_spectra(plan->hpack, plan->M, Fc, plan->log2N, plan->nu, plan->tw64, plan->Hk, 0,
                           (cudaStream_t)stream);
    if (e != cudaSuccess) return status_of(e);
    plan->filters_ready = true;
    return OLS_OK;
}

int ols_convolve_real(ols_plan_t plan, const float *s, int64_t Ns, float *y, void *stream) {
    if (!plan || !s || !y || !aligned4(s) || !aligned4(y)) return OLS_ERR_INVALID;
    if (plan->flags != OLS_FLAG_R2R) return OLS_ERR_UNSUPPORTED;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    cudaError_t e = r2r_launch(*plan, s, Ns, y, L, nseg, Nout, (cudaStream_t)stream);
    plan->last_launches = 1;
    return status_of(e);
}

// Argument checks shared by the post-processing entry points.
static int post_common(ols_plan_t plan, const float *s, int64_t Ns, PostArgs *a) {
    if (!plan || !s || !aligned8(s)) return OLS_ERR_INVALID;
    if (plan->flags != OLS_FLAG_FP32) return OLS_ERR_UNSUPPORTED;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    *a = PostArgs{};
    a->s = reinterpret_cast<const float2 *>(s);
    a->Ns = Ns;
    a->Nout = Nout;
    a->step = L;
    a->nseg = nseg;
    return OLS_OK;
}

int ols_convolve_power(ols_plan_t plan, const float *s, int64_t Ns, float *p, void *stream) {
    if (!p || !aligned4(p)) return OLS_ERR_INVALID;
    PostArgs a;
    int rc = post_common(plan, s, Ns, &a);
    if (rc != OLS_OK) return rc;
    a.mode = POST_POWER;
    a.out = p;
    cudaError_t e = post_launch(*plan, a, (cudaStream_t)stream);
    plan->last_launches = 1;
    return status_of(e);
}

int ols_convolve_detect(ols_plan_t plan, const float *s, int64_t Ns, float threshold, ols_candidate *cand,
                        int64_t capacity, unsigned long long *count, void *stream) {
    if (!count || ((uintptr_t)count & 7u) || capacity < 0 || (capacity > 0 && (!cand || !aligned8(cand))))
        return OLS_ERR_INVALID;
    PostArgs a;
    int rc = post_common(plan, s, Ns, &a);
    if (rc != OLS_OK) return rc;
    a.mode = POST_DETECT;
    a.thr = threshold;
    a.cand = cand;
    a.count = count;
    a.cap = capacity;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), (cudaStream_t)stream);
    if (e == cudaSuccess) e = post_launch(*plan, a, (cudaStream_t)stream);
    plan->last_launches = 1;
    return status_of(e);
}

int ols_convolve_peaks(ols_plan_t plan, const float *s, int64_t Ns, float threshold, ols_candidate *cand,
                       int64_t capacity, unsigned long long *count, void *stream) {
    if (!count || ((uintptr_t)count & 7u) || capacity < 0 || (capacity > 0 && (!cand || !aligned8(cand))))
        return OLS_ERR_INVALID;
    PostArgs a;
    int rc = post_common(plan, s, Ns, &a);
    if (rc != OLS_OK) return rc;
    if (a.step < 3) return OLS_ERR_UNSUPPORTED;     // segments laid out like the derivative's
    a.mode = POST_PEAK;
    a.step -= 2;
    a.nseg = (a.Nout + a.step - 1) / a.step;
    a.thr = threshold;
    a.cand = cand;
    a.count = count;
    a.cap = capacity;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), (cudaStream_t)stream);
    if (e == cudaSuccess) e = post_launch(*plan, a, (cudaStream_t)stream);
    plan->last_launches = 1;
    return status_of(e);
}

int ols_convolve_derivative(ols_plan_t plan, const float *s, int64_t Ns, float *d, void *stream) {
    if (!d || !aligned8(d)) return OLS_ERR_INVALID;
    PostArgs a;
    int rc = post_common(plan, s, Ns, &a);
    if (rc != OLS_OK) return rc;
    if (a.Nout < 2) return OLS_ERR_INVALID;
    if (a.step < 3) return OLS_ERR_UNSUPPORTED;     // each segment needs L - 2 >= 1 outputs
    a.mode = POST_DERIV;
    a.step -= 2;
    a.nseg = (a.Nout + a.step - 1) / a.step;
    a.out = d;
    cudaError_t e = post_launch(*plan, a, (cudaStream_t)stream);
    plan->last_launches = 1;
    return status_of(e);
}

int ols_convolve_host(ols_plan_t plan, const float *s_host, int64_t Ns, float *y_host, void *stream) {
    AllocScope scope;
    if (!plan || !s_host || !y_host || !aligned8(s_host) || !aligned8(y_host)) return OLS_ERR_INVALID;
    if (plan->flags == OLS_FLAG_R2R) return OLS_ERR_UNSUPPORTED;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    const int64_t M = plan->M, F = plan->F;
    // Whole segments per chunk: aim at ~64 MB of output per chunk.
    const int64_t target = (int64_t)64 << 20;
    int64_t cseg = target / (int64_t)(sizeof(float2) * F * L);
    if (cseg < 1) cseg = 1;
    if (cseg > nseg) cseg = nseg;
    const int64_t cout = cseg * L;           // outputs per full chunk
    const int64_t cin = cout + M - 1;        // inputs per full chunk
    Staging &st = plan->stage;
    cudaError_t e = cudaSuccess;
    if (!st.st[0]) {
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaStreamCreateWithFlags(&st.st[i], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.ev_done[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.ev_user, cudaEventDisableTiming);
        if (e != cudaSuccess) return status_of(e);
    }
    if (st.in_cap < cin || st.out_cap < F * cout) {
        for (int i = 0; i < 2; ++i) {
            if (st.in[i]) cudaFree(st.in[i]);
            if (st.out[i]) cudaFree(st.out[i]);
            st.in[i] = st.out[i] = nullptr;
        }
        st.in_cap = st.out_cap = 0;
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = dev_alloc(&st.in[i], sizeof(float2) * (size_t)cin);
            if (e == cudaSuccess) e = dev_alloc(&st.out[i], sizeof(float2) * (size_t)(F * cout));
        }
        if (e != cudaSuccess) {
            for (int i = 0; i < 2; ++i) {
                if (st.in[i]) cudaFree(st.in[i]);
                if (st.out[i]) cudaFree(st.out[i]);
                st.in[i] = st.out[i] = nullptr;
            }
            return status_of(e);
        }
        st.in_cap = cin;
        st.out_cap = F * cout;
    }
    // Order after the caller's prior work on `stream` (e.g. ols_set_filters).
    e = cudaEventRecord(st.ev_user, (cudaStream_t)stream);
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(st.st[i], st.ev_user, 0);
    const float2 *sh = reinterpret_cast<const float2 *>(s_host);
    float2 *yh = reinterpret_cast<float2 *>(y_host);
    int launches = 0;
    const int64_t nchunk = (nseg + cseg - 1) / cseg;
    // stage timing: four events per chunk, created once and kept with the staging
    st.timed_chunks = 0;
    const bool timed = st.timing;
    while (timed && e == cudaSuccess && (int64_t)st.tev.size() < 4 * nchunk) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreate(&ev);
        if (e == cudaSuccess) st.tev.push_back(ev);
    }
    auto mark = [&](int64_t c, int k, cudaStream_t cs) {
        if (timed && e == cudaSuccess) e = cudaEventRecord(st.tev[(size_t)(4 * c + k)], cs);
    };
    for (int64_t c = 0; c < nchunk && e == cudaSuccess; ++c) {
        const int b = (int)(c & 1);
        cudaStream_t cs = st.st[b];
        const int64_t o0 = c * cout;                                   // first output of the chunk
        const int64_t nout_c = (Nout - o0) < cout ? (Nout - o0) : cout;
        const int64_t nin_c = nout_c + M - 1;                          // s[o0, o0 + nin_c)
        mark(c, 0, cs);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(st.in[b], sh + o0, sizeof(float2) * (size_t)nin_c, cudaMemcpyHostToDevice, cs);
        mark(c, 1, cs);
        int64_t Lc, nsegc, Noutc;
        if (e == cudaSuccess) {
            ols_geometry(plan->N, plan->M, nin_c, &Lc, &nsegc, &Noutc);
            int l = 0;
            e = launch_any(*plan, st.in[b], nin_c, st.out[b], Lc, nsegc, Noutc, cs, &l);
            launches += l;
        }
        mark(c, 2, cs);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(yh + o0, sizeof(float2) * (size_t)Nout, st.out[b], sizeof(float2) * (size_t)nout_c,
                                  sizeof(float2) * (size_t)nout_c, (size_t)F, cudaMemcpyDeviceToHost, cs);
        mark(c, 3, cs);
    }
    for (int i = 0; i < 2; ++i) {
        cudaError_t e2 = cudaStreamSynchronize(st.st[i]);
        if (e == cudaSuccess) e = e2;
    }
    if (timed && e == cudaSuccess) st.timed_chunks = nchunk;
    plan->last_launches = launches;
    return status_of(e);
}

int ols_host_timing(ols_plan_t plan, int on) {
    if (!plan) return OLS_ERR_INVALID;
    plan->stage.timing = on != 0;
    plan->stage.timed_chunks = 0;
    return OLS_OK;
}

int ols_host_stage_ms(ols_plan_t plan, double *ms) {
    if (!plan || !ms) return OLS_ERR_INVALID;
    const Staging &st = plan->stage;
    if (!st.timing || st.timed_chunks < 1) return OLS_ERR_NOT_READY;
    double sum[3] = {0.0, 0.0, 0.0}, span = 0.0;
    for (int64_t c = 0; c < st.timed_chunks; ++c) {
        for (int k = 0; k < 3; ++k) {
            float t = 0.f;
            const cudaError_t e = cudaEventElapsedTime(&t, st.tev[(size_t)(4 * c + k)], st.tev[(size_t)(4 * c + k + 1)]);
            if (e != cudaSuccess) return status_of(e);
            sum[k] += t;
        }
        float t = 0.f;
        const cudaError_t e = cudaEventElapsedTime(&t, st.tev[0], st.tev[(size_t)(4 * c + 3)]);
        if (e != cudaSuccess) return status_of(e);
        if (t > span) span = t;
    }
    for (int k = 0; k < 3; ++k) ms[k] = sum[k];
    ms[3] = span;
    ms[4] = (double)st.timed_chunks;
    return OLS_OK;
}

// Workspace of the adjoint: overlap edges of ds (nseg x 2 x (M-1) complex),
// then the per-CTA dh spectra (grid x F x N complex) and their sum (F x N
// complex), each part 256-byte aligned.
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static void backward_layout(const ols_plan_s &p, int64_t nseg, bool want_ds, bool want_dh, size_t *edge_bytes,
                            size_t *part_bytes, size_t *sum_bytes, int *grid) {
    *grid = backward_grid(p, nseg, want_ds, want_dh);
    *edge_bytes = want_ds ? align256(sizeof(float2) * (size_t)nseg * 2 * (size_t)(p.M - 1)) : 0;
    const size_t spec = sizeof(float2) * (size_t)p.F * (size_t)p.N;
    *part_bytes = want_dh ? align256(spec * (size_t)(*grid)) : 0;
    *sum_bytes = want_dh ? align256(spec) : 0;
}

int ols_backward_workspace(ols_plan_t plan, int64_t Ns, int want_ds, int want_dh, size_t *bytes) {
    if (!plan || !bytes) return OLS_ERR_INVALID;
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    size_t eb, pb, rb;
    int grid;
    backward_layout(*plan, nseg, want_ds != 0, want_dh != 0, &eb, &pb, &rb, &grid);
    *bytes = eb + pb + rb;
    return OLS_OK;
}

}  // extern "C"

namespace ols {

// Argument checks of the adjoint, in the order both adjoint entry points
// report them (pointers, plan state, flags, sizes).
int backward_validate(ols_plan_t plan, const float *s, int64_t Ns, const float *g, const float *ds,
                      const float *dh) {
    if (!plan || !g || !aligned8(g) || (!ds && !dh)) return OLS_ERR_INVALID;
    if ((ds && !aligned8(ds)) || (dh && !aligned8(dh))) return OLS_ERR_INVALID;
    if (dh && (!s || !aligned8(s))) return OLS_ERR_INVALID;
    if (!plan->filters_ready) return OLS_ERR_NOT_READY;
    if (plan->flags != OLS_FLAG_FP32) return OLS_ERR_UNSUPPORTED;     // the adjoint is FP32 only
    int64_t L, nseg, Nout;
    int rc = ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    if (rc != OLS_OK) return rc;
    if (ds && plan->M - 1 > L) return OLS_ERR_UNSUPPORTED;   // ds overlaps must span two windows at most
    return OLS_OK;
}

}  // namespace ols

extern "C" {

int ols_convolve_backward(ols_plan_t plan, const float *s, int64_t Ns, const float *g, float *ds, float *dh,
                          void *workspace, size_t workspace_bytes, void *stream) {
    int rc = backward_validate(plan, s, Ns, g, ds, dh);
    if (rc != OLS_OK) return rc;
    int64_t L, nseg, Nout;
    ols_geometry(plan->N, plan->M, Ns, &L, &nseg, &Nout);
    size_t eb, pb, rb;
    BackwardArgs a{};
    backward_layout(*plan, nseg, ds != nullptr, dh != nullptr, &eb, &pb, &rb, &a.grid);
    if (eb + pb + rb > 0 && (!workspace || workspace_bytes < eb + pb + rb || ((uintptr_t)workspace & 255u)))
        return OLS_ERR_WORKSPACE;
    a.s = reinterpret_cast<const float2 *>(s);
    a.Ns = Ns;
    a.g = reinterpret_cast<const float2 *>(g);
    a.Nout = Nout;
    a.L = L;
    a.nseg = nseg;
    a.ds = reinterpret_cast<float2 *>(ds);
    a.dh = reinterpret_cast<float2 *>(dh);
    a.edge = eb ? reinterpret_cast<float2 *>(workspace) : nullptr;
    a.P = pb ? reinterpret_cast<float4 *>(static_cast<char *>(workspace) + eb) : nullptr;
    a.Pr = rb ? reinterpret_cast<float4 *>(static_cast<char *>(workspace) + eb + pb) : nullptr;
    int launches = 0;
    cudaError_t e = launch_backward(*plan, a, (cudaStream_t)stream, &launches);
    plan->last_launches = launches;
    return status_of(e);
}

int ols_last_launch_count(ols_plan_t plan) { return plan ? plan->last_launches : -1; }

int ols_plan_status(ols_plan_t plan, int *status, int reset) {
    if (!plan || !status) return OLS_ERR_INVALID;
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && reset) e = cudaMemset(plan->d_status, 0, sizeof(int));
    if (e != cudaSuccess) return status_of(e);
    *status = v;
    return OLS_OK;
}

}  // extern "C"
