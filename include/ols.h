/*
 * ols.h -- C ABI of the GB300 overlap-and-save (OLS) convolution library.
 *
 * The operation (paper: "GPU Fast Convolution via the Overlap-and-Save Method
 * in Shared Memory", arXiv:1910.01972):
 *
 *   Eq. 1 (Sec. 1)  y[n] = sum_{k=0}^{M-1} s[n-k] h[k]
 *
 * evaluated for a bank of F filters by overlap-and-save (Sec. 3.2): the
 * signal is cut into segments of N samples that overlap by M-1; each segment
 * is Fourier transformed, multiplied point-wise by every filter's spectrum,
 * inverse transformed, and its M-1 circularly aliased samples are dropped
 * (Sec. 3.2, Fig. 1, Algorithm 2).  The result is the "valid" part of Eq. 1:
 *
 *   y_f[j] = sum_{k=0}^{M-1} s[j+M-1-k] h_f[k],   0 <= j < Nout = Ns-M+1.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex values are interleaved FP32 pairs (re, im): a complex array of n
 *   elements is 2n floats.  Every array is contiguous and row-major.
 * - Pointers are DEVICE pointers owned by the caller unless a name ends in
 *   _host; the library never frees caller memory.  Complex arrays must be
 *   8-byte aligned.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Compute entry points only enqueue work: they do not
 *   synchronise the host and do not allocate, so they can be captured in a
 *   CUDA graph.  The plan must be used on the device that was current when
 *   it was created.
 * - Every entry point returns an ols_status and never aborts or prints.
 *   Arguments are checked before any work is enqueued; on an error nothing is
 *   enqueued.  Asynchronous kernel faults surface at the caller's next
 *   synchronisation, as with any CUDA call.
 * - Sizes: N (segment / FFT length) is a power of two in [256, 8192]; the
 *   paper's kernels stop at 4096 (Sec. 2), the larger shared memory of the
 *   target allows 8192.  1 <= M <= N, F >= 1, Ns >= M.
 * - Environment (read when a plan is created, or per call where stated):
 *   OLS_AUTOTUNE_CACHE (file of measured segment lengths, see ols_autotune);
 *   OLS_TC_WAIT_LIMIT (polls of each in-loop mbarrier wait of the
 *   tensor-core forms; default 2^20; a wait that runs out sets the plan's
 *   status word, see ols_plan_status); OLS_TC_WAIT_NEVER=1 (test switch:
 *   those waits watch an mbarrier nothing arrives on, so they run out and the
 *   kernel takes its failure path; its output is then undefined);
 *   OLS_FAIL_ALLOC=k (host-side fault
 *   injection: the k-th device allocation of one ols_plan, ols_batch_plan or
 *   ols_convolve_host call fails and the call returns OLS_ERR_ALLOC, with
 *   everything it allocated before released; read at each allocation).
 */
#ifndef OLS_H
#define OLS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OLS_API __attribute__((visibility("default")))
#else
#define OLS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OLS_OK = 0,
    OLS_ERR_INVALID = 1,      /* null / misaligned pointer, size out of range */
    OLS_ERR_UNSUPPORTED = 2,  /* N not a power of two in [256, 8192], M > N, bad flag */
    OLS_ERR_ALLOC = 3,        /* device or host allocation failed */
    OLS_ERR_CUDA = 4,         /* a CUDA runtime call failed (including: no device) */
    OLS_ERR_NOT_READY = 5,    /* filters were not set on the plan */
    OLS_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    OLS_ERR_WORKSPACE = 7,    /* caller workspace missing or too small */
    OLS_ERR_TOO_LARGE = 8     /* problem needs more than a fixed built-in limit */
} ols_status;

typedef struct ols_plan_s *ols_plan_t;
typedef struct ols_batch_s *ols_batch_t;

/* Plan flags (arithmetic of the convolution). */
#define OLS_FLAG_FP32 0u
/* Every radix-16 FFT stage as a tensor-core (tcgen05) matrix product on
 * 16-bit split operands x = x_hi + x_lo and DFT matrices W = W_hi + W_lo,
 * D = x_hi W_hi + x_hi W_lo + x_lo W_hi with FP32 accumulation; twiddles,
 * the point-wise product and the exchanges stay FP32.  FP16 split: ~22
 * significant bits per operand; BF16 split: ~16 bits.  Input range: the
 * FP16 form assumes |s| <= 1.42 and unit-L2 filters (larger inputs should be
 * scaled by a power of two; outside that range 16-bit operands can
 * overflow).  Forward convolution only (ols_convolve, ols_convolve_host). */
#define OLS_FLAG_TC_FP16SPLIT 1u
#define OLS_FLAG_TC_BF16SPLIT 2u
/* Real-to-real convolution (Sec. 3.4's R2R variant and Algorithm 2 with
 * real input): real signal, F real filters, real outputs, FP32.  Such a plan
 * serves only ols_set_filters_real / ols_convolve_real (and the host-side
 * queries); the complex entry points return OLS_ERR_UNSUPPORTED for it. */
#define OLS_FLAG_R2R 4u

/* Human-readable name of a status code (static storage; never NULL). */
OLS_API const char *ols_status_string(int status);

/* Library ABI version (major*100 + minor): 101.  1.1 added the split-storage
 * input of the tensor-core forms, batch tile schedules and status, stage
 * timing of the host-buffer path and peak finding; every 1.0 call is
 * unchanged. */
OLS_API int ols_version(void);

/*
 * Segment bookkeeping of Sec. 3.2 -- pure host arithmetic, needs no GPU.
 * L = N - M + 1 valid samples per segment (M-1 aliased samples dropped);
 * Nout = Ns - M + 1 outputs per filter; nseg = ceil(Nout / L) segments,
 * segment i reading s[i*L, i*L + N) (zero past Ns) and writing
 * y[f][i*L, min(i*L + L, Nout)).  Any output pointer may be NULL.
 * Errors: OLS_ERR_INVALID if M < 1 or Ns < M; OLS_ERR_UNSUPPORTED if N is not
 * a supported power of two or M > N.
 */
OLS_API int ols_geometry(int64_t N, int32_t M, int64_t Ns, int64_t *L, int64_t *nseg, int64_t *Nout);

/*
 * The library's internal spectral order -- pure host, needs no GPU.
 * Sec. 3.4 notes that the point-wise product does not care about the order
 * of the spectrum as long as signal and filter share it and the inverse
 * transform consumes it, so the forward FFT skips the reordering step.  This
 * returns, for each storage position q in [0, N), the frequency index
 * nu[q] held there (a permutation of [0, N)).  nu: host array of N int32.
 */
OLS_API int ols_spectrum_order(int64_t N, int32_t *nu);

/*
 * Create a plan for segment length N, filter length M and F filters
 * (Sec. 3.2; N = 0 lets the library pick N from M, F and the segment-length
 * rule of Sec. 5: each N is best for a range of M).  Allocates the plan's
 * device tables (filter spectra F*N complex, twiddles) on the current
 * device.  flags: OLS_FLAG_FP32, OLS_FLAG_TC_FP16SPLIT, OLS_FLAG_TC_BF16SPLIT
 * or OLS_FLAG_R2R (real data; ceil(F/2) complex spectra).
 * Errors: INVALID (out == NULL, M < 1, F < 1), UNSUPPORTED (N, M > N, flags),
 * CUDA / ALLOC from the device.  *out is NULL on error.
 */
OLS_API int ols_plan(ols_plan_t *out, int64_t N, int32_t M, int32_t F, uint32_t flags);

/* Release a plan and its device tables (synchronises the device first).
 * NULL is accepted and ignored. */
OLS_API int ols_plan_destroy(ols_plan_t plan);

/* Plan parameters and the segment bookkeeping for a signal of Ns samples
 * (Ns may be 0 to query only N, M, F).  Any output pointer may be NULL. */
OLS_API int ols_plan_query(ols_plan_t plan, int64_t Ns, int64_t *N, int32_t *M, int32_t *F,
                   int64_t *L, int64_t *nseg, int64_t *Nout);

/*
 * Filter-spectrum precompute (Algorithm 1 and 2: "forward FFT of the
 * filters", done once before the convolution kernel runs; Fig. 1's first
 * step).  h: device [F][M] complex.  Each filter is zero-padded to N and
 * transformed in FP64 (exact index reduction of every twiddle exponent), the
 * 1/N of the inverse transform is folded in, and the result is rounded to
 * FP32 and stored in the plan in the kernel's internal spectral order and
 * register layout.  Enqueued on `stream`; h may be freed once that work is
 * done.  Errors: INVALID (plan or h NULL / misaligned), CUDA.
 */
OLS_API int ols_set_filters(ols_plan_t plan, const float *h, void *stream);

/*
 * Read back the plan's filter spectra in natural frequency order, FP32:
 * H[f][nu] = (1/N) sum_k h_f[k] exp(-2 pi i nu k / N).  H: device [F][N]
 * complex.  For tests and tooling.  Errors: INVALID, NOT_READY, CUDA.
 */
OLS_API int ols_get_spectra(ols_plan_t plan, float *H, void *stream);

/*
 * The fused OLS convolution (Algorithm 2, Sec. 3.4): one kernel; each
 * segment of s is read from HBM once, forward-transformed in registers and
 * shared memory, and for every filter multiplied by its spectrum, inverse
 * transformed, stripped of its M-1 aliased samples and written once.
 * s: device [Ns] complex.  y: device [F][Ns-M+1] complex (row f holds
 * filter f's output).  s and y must not overlap.
 * Errors: INVALID (NULL / misaligned pointer, Ns < M), NOT_READY (no
 * filters), CUDA (launch failure).
 */
OLS_API int ols_convolve(ols_plan_t plan, const float *s, int64_t Ns, float *y, void *stream);

/*
 * Tensor-core plans (OLS_FLAG_TC_FP16SPLIT / _BF16SPLIT) on a signal STORED
 * split: every sample x = (x_hi + x_lo), each part a pair of 16-bit numbers
 * (Re, Im) in the plan's 16-bit type (FP16 or BF16).  The paper has no
 * split storage; it is the input form of the split-precision convolution
 * (the tensor-core MMAs take 16-bit operands, Sec. 3.4's FFT stages as
 * matrix products), 8 bytes per sample like FP32.
 * s_hi, s_lo: device [Ns] planes of 32-bit words, each word one sample's
 * (Re, Im) pair, Re in the low half (4-byte aligned).  y: device
 * [F][Ns-M+1] complex FP32.  The first forward FFT stage takes the planes
 * as its tensor-core operands directly; the result equals ols_convolve on
 * the FP32 signal x_hi + x_lo when the planes come from ols_split_signal
 * (bit for bit).  Errors: INVALID (NULL / misaligned pointer, Ns < M),
 * UNSUPPORTED (not a tensor-core plan), NOT_READY, CUDA.
 */
OLS_API int ols_convolve_split(ols_plan_t plan, const void *s_hi, const void *s_lo, int64_t Ns, float *y,
                               void *stream);

/*
 * The split storage of an FP32 signal for ols_convolve_split: for the real
 * and imaginary part x of every sample, x_hi = round16(x), x_lo =
 * round16(x - x_hi) (round to nearest even; the 16-bit type of the plan).
 * s: device [Ns] complex FP32 (8-byte aligned); s_hi, s_lo: device [Ns]
 * planes as above.  Errors: INVALID, UNSUPPORTED (not a tensor-core plan),
 * CUDA.
 */
OLS_API int ols_split_signal(ols_plan_t plan, const float *s, int64_t Ns, void *s_hi, void *s_lo, void *stream);

/*
 * Filter spectra of a real-to-real plan (flags OLS_FLAG_R2R).  h: device
 * [F][M] real FP32 (4-byte aligned).  The filters are taken in pairs as the
 * complex sequences g_p = h_{2p} + i h_{2p+1}, p < ceil(F/2) (the partner of
 * the last filter of an odd bank is zero), and each g_p is zero-padded and
 * transformed as in ols_set_filters (FP64, 1/N folded in, rounded to FP32,
 * kernel order).  ols_get_spectra then returns these ceil(F/2) spectra.
 * Errors: INVALID (plan or h NULL / misaligned), UNSUPPORTED (not an R2R
 * plan), CUDA.
 */
OLS_API int ols_set_filters_real(ols_plan_t plan, const float *h, void *stream);

/*
 * Real-to-real fused OLS convolution (Sec. 3.4's R2R variant; Eq. 1 on real
 * data, valid part):  y_f[j] = sum_k s[j+M-1-k] h_f[k],  j < Ns-M+1.
 * s: device [Ns] real FP32; y: device [F][Ns-M+1] real FP32 (row f = filter
 * f); both 4-byte aligned, not overlapping.  One kernel: each segment of s is
 * read once and transformed once (as a complex sequence with zero imaginary
 * part); for each filter pair p one inverse FFT of the product with the
 * spectrum of g_p gives s*h_{2p} in its real part and s*h_{2p+1} in its
 * imaginary part (both convolutions are real), so each inverse FFT serves two
 * output streams.  The paper's R2R kernel instead uses half-length
 * transforms with real/complex post-processing; the outputs are the same.
 * Errors: INVALID (NULL / misaligned pointer, Ns < M), UNSUPPORTED (not an
 * R2R plan), NOT_READY (no filters), CUDA (launch failure).
 */
OLS_API int ols_convolve_real(ols_plan_t plan, const float *s, int64_t Ns, float *y, void *stream);

/* ---------------------------------------------------------------------
 * Post-processing fused into the convolution kernel (Sec. 3.2 lists an
 * optional post-processing step after the discard; Sec. 4.3 distinguishes
 * per-element post-processing such as the power spectrum from non-local
 * post-processing such as the numerical derivative, which needs each
 * output's neighbours; Sec. 4.4 notes that reducing the output, e.g. by
 * candidate selection, is what keeps the device-to-host transfer small).
 * FP32 complex plans (OLS_FLAG_FP32) only; each is one kernel launch and the
 * convolved y itself is never written.
 * --------------------------------------------------------------------- */

/*
 * Power of the convolved output: p[f][j] = |y_f[j]|^2 (FP32), y as in
 * ols_convolve.  s: device [Ns] complex; p: device [F][Ns-M+1] float,
 * 4-byte aligned.  Errors: INVALID (pointers, Ns < M), UNSUPPORTED (not an
 * FP32 complex plan), NOT_READY, CUDA.
 */
OLS_API int ols_convolve_power(ols_plan_t plan, const float *s, int64_t Ns, float *p, void *stream);

/* One detection: output index j of filter f whose power |y_f[j]|^2 reached
 * the threshold. */
typedef struct {
    int64_t j;
    int32_t f;
    float power;
} ols_candidate;

/*
 * Candidate selection on the power of the convolved output: every (f, j)
 * with |y_f[j]|^2 >= threshold is appended to cand (device array of
 * `capacity` records) in no particular order; *count (device, 8-byte
 * aligned) receives the total number found, which may exceed capacity (the
 * records beyond it are dropped).  The call zeroes *count itself (a memset
 * on `stream`, before the kernel).  Errors: INVALID (pointers, Ns < M,
 * capacity < 0), UNSUPPORTED (not an FP32 complex plan), NOT_READY, CUDA.
 */
OLS_API int ols_convolve_detect(ols_plan_t plan, const float *s, int64_t Ns, float threshold,
                                ols_candidate *cand, int64_t capacity, unsigned long long *count,
                                void *stream);

/*
 * Peak finding on the power of the convolved output (the further reduction
 * before the output leaves the GPU that Sec. 4.4 names; the paper gives no
 * rule): every (f, j) with
 *   p_f[j] >= threshold,  p_f[j] > p_f[j-1] (j > 0),  p_f[j] >= p_f[j+1] (j < Nout-1),
 * p = |y|^2, so a run of equal powers gives one peak, at its left end.
 * Records, capacity and count as ols_convolve_detect (no particular order;
 * *count zeroed by the call; may exceed capacity).  Each segment advances by
 * L-2 outputs like the derivative's, so the neighbours of every output it
 * reports are its own unaliased samples, exchanged in shared memory.  The
 * comparisons are taken in FP32 on the kernel's powers.
 * Errors: INVALID (pointers, Ns < M, capacity < 0), UNSUPPORTED (not an FP32
 * complex plan, or N - M + 1 < 3), NOT_READY, CUDA.
 */
OLS_API int ols_convolve_peaks(ols_plan_t plan, const float *s, int64_t Ns, float threshold,
                               ols_candidate *cand, int64_t capacity, unsigned long long *count,
                               void *stream);

/*
 * Numerical derivative of the convolved output along j (the paper's
 * non-local post-processing example, Sec. 4.3; the paper gives no formula,
 * this is the central difference with one-sided ends):
 *   d_f[j] = (y_f[j+1] - y_f[j-1]) / 2   for 0 < j < Nout-1,
 *   d_f[0] = y_f[1] - y_f[0],   d_f[Nout-1] = y_f[Nout-1] - y_f[Nout-2].
 * Each segment advances by L-2 outputs instead of L so that every derivative
 * it writes has both neighbours among its own unaliased outputs.
 * s: device [Ns] complex; d: device [F][Ns-M+1] complex.
 * Errors: INVALID (pointers, Ns - M + 1 < 2), UNSUPPORTED (not an FP32
 * complex plan, or N - M + 1 < 3), NOT_READY, CUDA.
 */
OLS_API int ols_convolve_derivative(ols_plan_t plan, const float *s, int64_t Ns, float *d, void *stream);

/*
 * The same convolution with HOST buffers (what a user outside the device
 * calls, Sec. 4.4 discusses the PCI-e cost): s_host [Ns] complex, y_host
 * [F][Ns-M+1] complex.  The signal is cut into chunks of whole segments;
 * each chunk's input (with its M-1 halo) is copied host->device, convolved
 * and copied device->host on a pipeline of streams so transfers overlap the
 * kernels.  Pinned (page-locked) host memory is needed for the overlap;
 * pageable memory works but serialises.  Allocates device staging buffers on
 * first use and when a larger chunk is needed; returns after y_host is
 * complete (synchronises `stream`'s work it enqueued).
 * Errors: INVALID, NOT_READY, ALLOC, CUDA.
 */
OLS_API int ols_convolve_host(ols_plan_t plan, const float *s_host, int64_t Ns, float *y_host,
                      void *stream);

/*
 * Stage timing of ols_convolve_host (off by default): with on != 0 every
 * later ols_convolve_host call on this plan records CUDA events around each
 * chunk's host->device copy, kernel and device->host copy (four per chunk,
 * created on first use and kept with the staging buffers).
 * Errors: INVALID.
 */
OLS_API int ols_host_timing(ols_plan_t plan, int on);

/*
 * The last timed ols_convolve_host call, in device milliseconds: ms[0] the
 * host->device copies, ms[1] the kernels, ms[2] the device->host copies,
 * each summed over the chunks (a stage's time includes any wait for a copy
 * engine or the SMs, so with two streams the sums can exceed the span);
 * ms[3] the span from the first chunk's start to the last chunk's end;
 * ms[4] the number of chunks.  ms: host array of 5 doubles.
 * Errors: INVALID, NOT_READY (timing off, or no call since it was turned on),
 * CUDA.
 */
OLS_API int ols_host_stage_ms(ols_plan_t plan, double *ms);

/*
 * Workspace (bytes) that ols_convolve_backward needs for a signal of Ns
 * samples, given which gradients are wanted (want_ds, want_dh: 0 or 1).
 * May be 0.  Errors: INVALID, UNSUPPORTED (as ols_geometry).
 */
OLS_API int ols_backward_workspace(ols_plan_t plan, int64_t Ns, int want_ds, int want_dh, size_t *bytes);

/*
 * Adjoint of ols_convolve (the paper has no backward pass; this is derived
 * from Eq. 1 by linearity, for training systems).  Gradient convention
 * g = dL/dRe y + i dL/dIm y, g: device [F][Ns-M+1] complex.  Outputs:
 *   ds[m]   = sum_f sum_k g_f[m-M+1+k] conj(h_f[k])          device [Ns] complex, or NULL
 *   dh_f[k] = sum_j g_f[j] conj(s[j+M-1-k])                  device [F][M] complex, or NULL
 * (at least one of them non-NULL; s may be NULL when dh is NULL).  Computed
 * window by window in the frequency domain with the segment spectrum of s
 * recomputed: F+2 on-chip FFTs per window (the signal segment, the F
 * gradient windows, one inverse for ds); dh is summed over windows as a
 * spectrum per CTA, then two small kernels add the ds overlaps, sum the
 * CTAs' spectra in a fixed order (compensated) and run one inverse FFT per
 * filter: deterministic for a given plan and device.  Outputs are overwritten, not
 * accumulated.  workspace: device buffer of at least ols_backward_workspace()
 * bytes, 256-byte aligned, owned by the caller; its contents on entry do not
 * matter.  Errors: INVALID (pointers), NOT_READY, UNSUPPORTED (ds wanted with
 * M-1 > N-M+1: choose N >= 2(M-1)), WORKSPACE (missing, small or misaligned),
 * CUDA.
 */
OLS_API int ols_convolve_backward(ols_plan_t plan, const float *s, int64_t Ns, const float *g, float *ds,
                                  float *dh, void *workspace, size_t workspace_bytes, void *stream);

/* ---------------------------------------------------------------------
 * Segment-length autotuner and the batched form.
 * Sec. 5 of the paper observes that each segment length is the fastest for
 * a range of filter lengths only (a longer segment wastes a smaller
 * fraction M-1 of each FFT but costs more per point); the autotuner measures
 * that trade-off on the device instead of fixing N.
 * --------------------------------------------------------------------- */

/* Autotuner flag: use the cost model (N/L)(log2 N + c) instead of timing. */
#define OLS_TUNE_MODEL (1u << 8)
/* Batch flag: one persistent launch per distinct segment length instead of
 * one launch for the whole batch. */
#define OLS_BATCH_PER_N (1u << 9)

/*
 * Pick the segment length N in {256, ..., 8192} (N >= M) for M taps and F
 * filters: with flags = 0 the fused kernel is timed on the current device for
 * every candidate on a zero signal of about two waves of segments (allocates
 * up to ~256 MB of temporary device memory, synchronises the device) and the
 * fastest per output sample wins; results are cached per (M, F) for the
 * process and, if the environment variable OLS_AUTOTUNE_CACHE names a file,
 * read from and appended to it ("M F N" lines).  With OLS_TUNE_MODEL, no
 * measurement.  Errors: INVALID, UNSUPPORTED (M > 8192), ALLOC, CUDA.
 */
OLS_API int ols_autotune(int32_t M, int32_t F, uint32_t flags, int64_t *N);

/*
 * A batch of B independent problems of uneven size: signal b has Ns[b]
 * samples, F[b] filters of M[b] taps, segment length N[b] (N == NULL or
 * N[b] == 0: ols_autotune(M[b], F[b], flags)).  Host arrays of B entries.
 * The whole batch is ONE persistent launch: its resident blocks (N/16
 * threads for the longest N, at least 128) pull work items (runs of segment
 * tiles of one problem, see ols_batch_plan_tiles) from an atomic ticket, the
 * most expensive first; a tile is (block size x 16)/N segments of one
 * problem, each on a slot of N/16 threads with barriers of its own.  With
 * OLS_BATCH_PER_N in flags, problems sharing a segment length form one
 * persistent launch each instead.  Every segment is computed exactly as by
 * ols_convolve on the same N, so results are identical to per-problem calls.
 * Allocates per-problem spectra and the work tables.
 * Errors: INVALID (B < 1, NULL arrays, an Ns < M, M < 1, F < 1), UNSUPPORTED,
 * ALLOC, CUDA.
 */
OLS_API int ols_batch_plan(ols_batch_t *out, int32_t B, const int64_t *Ns, const int32_t *M, const int32_t *F,
                           const int64_t *N, uint32_t flags);

/*
 * ols_batch_plan with the tile schedule of the single launch: an item is a
 * run of tiles[b] consecutive tiles of problem b, taken with one ticket (the
 * block loads the problem's twiddles once per item).  tiles == NULL or
 * tiles[b] == 0: picked per (M, F, N) by ols_autotune_tiles with this
 * batch's block size; a tuned run is halved while the batch has fewer than
 * four items per resident block (the dynamic schedule needs items to balance
 * its tail).  Items are taken most expensive first (tiles x F log2 N).
 * Ignored with OLS_BATCH_PER_N (items of one tile).  Results do not depend
 * on the schedule.  Errors: as ols_batch_plan; INVALID also for tiles[b] < 0.
 */
OLS_API int ols_batch_plan_tiles(ols_batch_t *out, int32_t B, const int64_t *Ns, const int32_t *M,
                                 const int32_t *F, const int64_t *N, const int32_t *tiles, uint32_t flags);

/*
 * Tile schedule for one problem of (M, F, N) in a single-launch batch of
 * `block` threads (128, 256 or 512, at least N/16): the run length, in
 * tiles per item, from {1, 2, 4, 8}.  With flags = 0 the single-launch
 * kernel is timed on the current device for every candidate on a zero
 * signal of about three waves of the longest items (up to ~1 GB of
 * temporary device memory; synchronises the device) and the shortest run
 * within 1% of the fastest per output wins; cached per (M, F, N, block) for
 * the process.  With OLS_TUNE_MODEL: the shortest power of two giving an
 * item ~32 transforms per slot (F + 1 per segment), at most 8.
 * Errors: INVALID, UNSUPPORTED (N, M > N, block), ALLOC, CUDA.
 */
OLS_API int ols_autotune_tiles(int32_t M, int32_t F, int64_t N, int32_t block, uint32_t flags, int32_t *tiles);

/* The schedule of problem b in a single-launch batch: tiles per item and
 * number of items.  Either pointer may be NULL.  Errors: INVALID,
 * UNSUPPORTED (an OLS_BATCH_PER_N batch). */
OLS_API int ols_batch_schedule(ols_batch_t batch, int32_t b, int32_t *tiles, int64_t *items);
OLS_API int ols_batch_destroy(ols_batch_t batch);

/* Segment length and output length of problem b, and the number of
 * persistent launches per call (1, or the distinct segment lengths with
 * OLS_BATCH_PER_N).  Any output
 * pointer may be NULL.  Errors: INVALID. */
OLS_API int ols_batch_query(ols_batch_t batch, int32_t b, int64_t *N, int64_t *Nout, int32_t *ngroups);

/* Filter spectra of every problem (as ols_set_filters): h is a HOST array of
 * B device pointers, h[b] -> [F[b]][M[b]] complex.  Errors: INVALID, CUDA. */
OLS_API int ols_batch_set_filters(ols_batch_t batch, const float *const *h, void *stream);

/*
 * Convolve every problem: s_ptrs and y_ptrs are DEVICE arrays of B device
 * pointers (s_ptrs[b] -> [Ns[b]] complex, y_ptrs[b] -> [F[b]][Ns[b]-M[b]+1]
 * complex), read by the kernels, so the call enqueues only a memset of the
 * ticket(s) and the launch (one, or one per segment length with
 * OLS_BATCH_PER_N): it can be captured in a CUDA graph and replayed with new
 * data behind the same pointers.
 * Errors: INVALID, NOT_READY, CUDA.
 */
OLS_API int ols_convolve_batched(ols_batch_t batch, const void *s_ptrs, const void *y_ptrs, void *stream);

/* Kernel launches enqueued by the last ols_convolve_batched. */
OLS_API int ols_batch_last_launch_count(ols_batch_t batch);

/*
 * Read the plan's device status word (synchronises the device): 0, or the
 * OR of these bits since the last reset (that call's output is then
 * incomplete):
 *   1  a kernel's bounded wait on the tensor cores gave up;
 *   2  (only in a library built with OLS_CHECK=1, a debug build) a global
 *      memory access of a kernel (forward, real-to-real, post-processing,
 *      tensor-core, adjoint, batched) failed its bounds check against its
 *      buffer and was skipped.
 * reset != 0 clears it.  Errors: INVALID, CUDA.
 */
OLS_API int ols_plan_status(ols_plan_t plan, int *status, int reset);

/* The OR of ols_plan_status over every problem of a batch (the batched
 * kernels report into each problem's own plan status word); reset != 0
 * clears them all.  Errors: INVALID, CUDA. */
OLS_API int ols_batch_status(ols_batch_t batch, int *status, int reset);

/* Size in bytes of the scratch array built into the library for
 * ols_convolve_backward_noalloc. */
#define OLS_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * ols_convolve_backward without a caller workspace and without allocating
 * (the paper has no counterpart: this serves callers that cannot allocate
 * device memory -- real-time pipelines that forbid allocation once running,
 * since cudaMalloc can block and synchronise the device, and hosts that own
 * every device allocation themselves).  Same arguments, results and errors
 * as ols_convolve_backward minus the workspace; the scratch is a fixed
 * device array of OLS_NOALLOC_SCRATCH_BYTES inside the library, which every
 * GPU that loads the library holds until the process exits.
 * - The argument checks of ols_convolve_backward run first, in its order;
 *   then problems whose ols_backward_workspace() exceeds that size are
 *   rejected with OLS_ERR_TOO_LARGE before any work is enqueued.
 * - The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress, with the plan's device current); make that first
 *   call before any stream capture.  The address is kept for the life of the
 *   process: it belongs to the device's primary context, so do not call this
 *   entry point again after destroying that context (cudaDeviceReset).  The
 *   plan's device must be current (else OLS_ERR_INVALID).  No cudaMalloc,
 *   cudaFree or other allocating routine is called.
 * - Every call on a device shares the one array, which keeps the last call's
 *   contents (nothing in it needs to start at zero).  Calls that overlap on
 *   the GPU -- other streams, other threads, other plans -- race on it:
 *   serialise them.
 */
OLS_API int ols_convolve_backward_noalloc(ols_plan_t plan, const float *s, int64_t Ns, const float *g, float *ds,
                                          float *dh, void *stream);

/* Number of kernel launches the last compute call on this plan enqueued
 * (ols_convolve, ols_convolve_host, ols_convolve_backward), for launch
 * accounting in benchmarks. */
OLS_API int ols_last_launch_count(ols_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* OLS_H */
