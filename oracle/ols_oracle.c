/*
 * ols_oracle.c -- FP64 CPU oracle for overlap-and-save (OLS) convolution.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * statement of what the GPU path must compute.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it.  It shares no code,
 * header, table or helper with the CUDA sources.
 *
 * What it computes
 * ----------------
 * Eq. 1 of the paper (Sec. 1) defines discrete convolution of a signal s of
 * length Ns with a filter h of length M:  y[n] = sum_{k=0}^{M-1} s[n-k] h[k].
 * OLS (Sec. 3.2, "Overlap-and-save method") keeps only the samples that are
 * free of circular aliasing, M-1 of them being discarded per segment, and it
 * states that the result does not depend on the segment length.  Therefore
 * the exact result of OLS is the "valid" part of Eq. 1:
 *
 *     y_f[j] = sum_{k=0}^{M-1} s[j + M - 1 - k] * h_f[k],   0 <= j < Nout,
 *     Nout   = Ns - M + 1,
 *
 * for every filter f of the bank (Algorithm 2 loops over the filters).  The
 * oracle is that sum written out, in complex FP64, accumulated in increasing
 * k, on the FP32 inputs widened to FP64.  No FFT, no blocking, no reordering.
 *
 * The adjoint (reverse-mode derivative) follows from Eq. 1 by linearity,
 * using the convention grad = dL/dRe + i dL/dIm:
 *
 *     ds[m]    = sum_f sum_{k : 0 <= m-M+1+k < Nout} g_f[m-M+1+k] * conj(h_f[k])
 *     dh_f[k]  = sum_{j=0}^{Nout-1} g_f[j] * conj(s[j+M-1-k])
 *
 * where g_f[j] = dL/dRe y_f[j] + i dL/dIm y_f[j].
 *
 * The paper's second variant (Sec. 3.4, the R2R SM-OLS) convolves a real
 * signal with real filters; its exact result is the same valid part of Eq. 1
 * on real data, computed here separately in real FP64 (ols_oracle_conv_real).
 *
 * Layouts: every complex array is interleaved (re, im) pairs.  s[Ns] and
 * h[F][M] are FP32 (as the GPU consumes them); g[F][Nout] and every output
 * are FP64.  Parallelism: OpenMP over independent output elements only; each
 * output is one sequential sum, so results do not depend on the thread count.
 */
#include <stdint.h>
#include <stddef.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int ols_oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void ols_oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* One output of Eq. 1 (valid part): y_f[j]. */
static void conv_one(const float *s, int32_t M, const float *hf, int64_t j,
                     double *out_re, double *out_im)
{
    double acc_re = 0.0, acc_im = 0.0;
    for (int32_t k = 0; k < M; ++k) {
        const int64_t n = j + (int64_t)M - 1 - k;     /* s index of tap k */
        const double sr = (double)s[2 * n], si = (double)s[2 * n + 1];
        const double hr = (double)hf[2 * k], hi = (double)hf[2 * k + 1];
        acc_re += sr * hr - si * hi;
        acc_im += sr * hi + si * hr;
    }
    *out_re = acc_re;
    *out_im = acc_im;
}

/*
 * Full valid-mode convolution for a bank of F filters (Eq. 1, Sec. 3.2).
 * s: [Ns] complex (FP32), h: [F][M] complex (FP32), y: [F][Ns-M+1] complex
 * (FP64).  Returns 0, or -1 on invalid sizes (Ns < M, M < 1, F < 1).
 */
int ols_oracle_conv(int64_t Ns, const float *s, int32_t M, int32_t F,
                    const float *h, double *y)
{
    if (M < 1 || F < 1 || Ns < M) return -1;
    const int64_t Nout = Ns - M + 1;
    const int64_t total = (int64_t)F * Nout;
    int64_t idx;
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < total; ++idx) {
        const int64_t f = idx / Nout, j = idx % Nout;
        conv_one(s, M, h + 2 * (size_t)f * M, j, &y[2 * idx], &y[2 * idx + 1]);
    }
    return 0;
}

/*
 * Selected outputs of the same convolution: out[i] = y_{fi[i]}[ji[i]].
 * Used to check full-size GPU results at sampled positions.  Returns 0, or -1
 * when a size or an index is out of range.
 */
int ols_oracle_conv_at(int64_t Ns, const float *s, int32_t M, int32_t F,
                       const float *h, int64_t n, const int64_t *fi,
                       const int64_t *ji, double *out)
{
    if (M < 1 || F < 1 || Ns < M) return -1;
    const int64_t Nout = Ns - M + 1;
    for (int64_t i = 0; i < n; ++i)
        if (fi[i] < 0 || fi[i] >= F || ji[i] < 0 || ji[i] >= Nout) return -1;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i)
        conv_one(s, M, h + 2 * (size_t)fi[i] * M, ji[i], &out[2 * i], &out[2 * i + 1]);
    return 0;
}

/*
 * Adjoint of the valid-mode convolution (derived from Eq. 1 by linearity).
 * g: [F][Nout] complex (FP64).  ds: [Ns] complex (FP64) or NULL.
 * dh: [F][M] complex (FP64) or NULL.  Returns 0, or -1 on invalid sizes.
 */
int ols_oracle_adjoint(int64_t Ns, const float *s, int32_t M, int32_t F,
                       const float *h, const double *g, double *ds, double *dh)
{
    if (M < 1 || F < 1 || Ns < M) return -1;
    const int64_t Nout = Ns - M + 1;
    if (ds) {
        int64_t m;
#pragma omp parallel for schedule(static)
        for (m = 0; m < Ns; ++m) {
            double acc_re = 0.0, acc_im = 0.0;
            for (int32_t f = 0; f < F; ++f) {
                const float *hf = h + 2 * (size_t)f * M;
                const double *gf = g + 2 * (size_t)f * Nout;
                for (int32_t k = 0; k < M; ++k) {
                    const int64_t j = m - (int64_t)M + 1 + k;   /* output fed by s[m] through tap k */
                    if (j < 0 || j >= Nout) continue;
                    const double gr = gf[2 * j], gi = gf[2 * j + 1];
                    const double hr = (double)hf[2 * k], hi = (double)hf[2 * k + 1];
                    /* g * conj(h) */
                    acc_re += gr * hr + gi * hi;
                    acc_im += gi * hr - gr * hi;
                }
            }
            ds[2 * m] = acc_re;
            ds[2 * m + 1] = acc_im;
        }
    }
    if (dh) {
        const int64_t total = (int64_t)F * M;
        int64_t idx;
#pragma omp parallel for schedule(static)
        for (idx = 0; idx < total; ++idx) {
            const int64_t f = idx / M, k = idx % M;
            const double *gf = g + 2 * (size_t)f * Nout;
            double acc_re = 0.0, acc_im = 0.0;
            for (int64_t j = 0; j < Nout; ++j) {
                const int64_t n = j + M - 1 - k;
                const double gr = gf[2 * j], gi = gf[2 * j + 1];
                const double sr = (double)s[2 * n], si = (double)s[2 * n + 1];
                /* g * conj(s) */
                acc_re += gr * sr + gi * si;
                acc_im += gi * sr - gr * si;
            }
            dh[2 * idx] = acc_re;
            dh[2 * idx + 1] = acc_im;
        }
    }
    return 0;
}

/* One output of Eq. 1 (valid part) on real data: y_f[j]. */
static double conv_one_real(const float *s, int32_t M, const float *hf, int64_t j)
{
    double acc = 0.0;
    for (int32_t k = 0; k < M; ++k)
        acc += (double)s[j + (int64_t)M - 1 - k] * (double)hf[k];
    return acc;
}

/*
 * Real-to-real valid-mode convolution for a bank of F filters (Eq. 1 on real
 * data, the R2R form of Sec. 3.4).  s: [Ns] real (FP32), h: [F][M] real
 * (FP32), y: [F][Ns-M+1] real (FP64).  Returns 0, or -1 on invalid sizes.
 */
int ols_oracle_conv_real(int64_t Ns, const float *s, int32_t M, int32_t F,
                         const float *h, double *y)
{
    if (M < 1 || F < 1 || Ns < M) return -1;
    const int64_t Nout = Ns - M + 1;
    const int64_t total = (int64_t)F * Nout;
    int64_t idx;
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < total; ++idx)
        y[idx] = conv_one_real(s, M, h + (size_t)(idx / Nout) * M, idx % Nout);
    return 0;
}

/* Selected outputs of the real convolution: out[i] = y_{fi[i]}[ji[i]]. */
int ols_oracle_conv_real_at(int64_t Ns, const float *s, int32_t M, int32_t F,
                            const float *h, int64_t n, const int64_t *fi,
                            const int64_t *ji, double *out)
{
    if (M < 1 || F < 1 || Ns < M) return -1;
    const int64_t Nout = Ns - M + 1;
    for (int64_t i = 0; i < n; ++i)
        if (fi[i] < 0 || fi[i] >= F || ji[i] < 0 || ji[i] >= Nout) return -1;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i)
        out[i] = conv_one_real(s, M, h + (size_t)fi[i] * M, ji[i]);
    return 0;
}

/*
 * Post-processing of the convolved output (Sec. 3.2's optional
 * post-processing step; Sec. 4.3: per-element post-processing such as the
 * power spectrum, and non-local post-processing such as the numerical
 * derivative of the convolved signal, whose formula the paper does not give).
 * Reading taken for the derivative: the central difference with one-sided
 * differences at the two ends of each output stream,
 *     d_f[j] = (y_f[j+1] - y_f[j-1]) / 2        0 < j < Nout-1
 *     d_f[0] = y_f[1] - y_f[0],   d_f[Nout-1] = y_f[Nout-1] - y_f[Nout-2],
 * defined for Nout >= 2.  The power is p_f[j] = |y_f[j]|^2.  Both are
 * computed here from the FP64 outputs of conv_one.
 */

/* Derivative of filter f's output at j (Nout >= 2). */
static void deriv_one(const float *s, int32_t M, const float *hf, int64_t Nout, int64_t j,
                      double *out_re, double *out_im)
{
    const int64_t lo = (j == 0) ? j : j - 1;
    const int64_t hi = (j == Nout - 1) ? j : j + 1;
    const double scale = (hi - lo == 2) ? 0.5 : 1.0;
    double ar, ai, br, bi;
    conv_one(s, M, hf, lo, &ar, &ai);
    conv_one(s, M, hf, hi, &br, &bi);
    *out_re = (br - ar) * scale;
    *out_im = (bi - ai) * scale;
}

/*
 * p: [F][Ns-M+1] real (FP64) power of every output.  Returns 0, or -1 on
 * invalid sizes.
 */
int ols_oracle_power(int64_t Ns, const float *s, int32_t M, int32_t F, const float *h, double *p)
{
    if (M < 1 || F < 1 || Ns < M) return -1;
    const int64_t Nout = Ns - M + 1;
    const int64_t total = (int64_t)F * Nout;
    int64_t idx;
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < total; ++idx) {
        const int64_t f = idx / Nout, j = idx % Nout;
        double yr, yi;
        conv_one(s, M, h + 2 * (size_t)f * M, j, &yr, &yi);
        p[idx] = yr * yr + yi * yi;
    }
    return 0;
}

/*
 * d: [F][Ns-M+1] complex (FP64) derivative of every output stream.  Returns
 * 0, or -1 on invalid sizes (including Nout < 2).
 */
int ols_oracle_derivative(int64_t Ns, const float *s, int32_t M, int32_t F, const float *h, double *d)
{
    if (M < 1 || F < 1 || Ns < M + 1) return -1;
    const int64_t Nout = Ns - M + 1;
    const int64_t total = (int64_t)F * Nout;
    int64_t idx;
#pragma omp parallel for schedule(static)
    for (idx = 0; idx < total; ++idx) {
        const int64_t f = idx / Nout, j = idx % Nout;
        deriv_one(s, M, h + 2 * (size_t)f * M, Nout, j, &d[2 * idx], &d[2 * idx + 1]);
    }
    return 0;
}

/*
 * Peak finding on the power (the further reduction of the output that
 * Sec. 4.4 names, "peak finding or candidate selection"; the paper gives no
 * rule).  Reading taken: (f, j) is a peak when its power reaches the
 * threshold and is a local maximum of its stream, strictly above its left
 * neighbour and at least its right one, so that a run of equal powers gives
 * one peak, at its left end:
 *     p_f[j] >= threshold,  p_f[j] > p_f[j-1] (if j > 0),
 *     p_f[j] >= p_f[j+1] (if j < Nout-1).
 * mask[f][j] = 1 for a peak, else 0, for p: [F][Nout].  Returns 0, or -1 on
 * invalid sizes.
 */
int ols_oracle_peak_mask(int32_t F, int64_t Nout, const double *p, double threshold, unsigned char *mask)
{
    if (F < 1 || Nout < 1) return -1;
    for (int32_t f = 0; f < F; ++f) {
        const double *pf = p + (size_t)f * Nout;
        unsigned char *mf = mask + (size_t)f * Nout;
        for (int64_t j = 0; j < Nout; ++j) {
            int peak = pf[j] >= threshold;
            if (j > 0 && !(pf[j] > pf[j - 1])) peak = 0;
            if (j < Nout - 1 && !(pf[j] >= pf[j + 1])) peak = 0;
            mf[j] = (unsigned char)peak;
        }
    }
    return 0;
}

/* Selected derivatives: out[i] = d_{fi[i]}[ji[i]].  Returns 0, or -1. */
int ols_oracle_derivative_at(int64_t Ns, const float *s, int32_t M, int32_t F, const float *h, int64_t n,
                             const int64_t *fi, const int64_t *ji, double *out)
{
    if (M < 1 || F < 1 || Ns < M + 1) return -1;
    const int64_t Nout = Ns - M + 1;
    for (int64_t i = 0; i < n; ++i)
        if (fi[i] < 0 || fi[i] >= F || ji[i] < 0 || ji[i] >= Nout) return -1;
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < n; ++i)
        deriv_one(s, M, h + 2 * (size_t)fi[i] * M, Nout, ji[i], &out[2 * i], &out[2 * i + 1]);
    return 0;
}
