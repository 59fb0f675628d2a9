/*
 * hos_oracle.c -- plain FP64 CPU statement of the smoothed sample bispectrum
 * and trispectrum computed the indirect way (sample cumulant -> lag window ->
 * Fourier transform), of the exact gradients of both, and of the
 * paper's direct method (Algorithm DBS: part DFTs, raw triple products, box
 * smoothing, average over parts).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may call, link or
 * load this file; only the tests, the package smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA path.
 *
 * Every routine is the definition written out as loops, in the order the
 * method states it, with no blocking or reordering of any sum.  Where the
 * paper is silent the reading is stated at the routine:
 *   - moments and time averages: Problem Statement (k-th moment, cumulants
 *     c1, c2 "and so on", ensemble averages replaced by time averages);
 *   - bispectrum / trispectrum as the Fourier transform of c3 / c4: Problem
 *     Statement;
 *   - partition into K parts, per-part mean removal, average over parts:
 *     Algorithm DBS steps 1, 2 and 6;
 *   - DFT sign e^{-j 2 pi u k / M}: Algorithm DBS step 3.
 * Readings (paper silent): biased 1/n estimator with samples outside the
 * series taken as zero; c4 by the zero-mean moment-to-cumulant identity;
 * Parzen lag window; (2 pi)^{-(k-1)} spectral normalisation; DFT grid
 * k = 0..N-1, unshifted.
 *
 * Lag arrays use the full symmetric range [-L, L] on every axis, stored
 * row-major with index (w + L).  Complex outputs are interleaved (re, im).
 *
 * Parity pins for every routine live in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HOS_ORACLE_PI 3.14159265358979323846

enum { ORACLE_WIN_PARZEN = 0, ORACLE_WIN_PARZEN_SYM = 1, ORACLE_WIN_RECT = 2 };

/* ------------------------------------------------------------------ */
/* Algorithm DBS steps 1-2: partition into parts of seg samples (seg <= 0:
 * one part, K = 1) and subtract each part's mean.  A trailing part shorter
 * than seg is its own part.  remove_mean = 0 copies x unchanged.          */
void hos_oracle_demean(const double* x, int64_t n, int64_t seg, int remove_mean, double* y)
{
    if (seg <= 0 || seg > n) seg = n;
    for (int64_t s0 = 0; s0 < n; s0 += seg) {
        int64_t s1 = s0 + seg < n ? s0 + seg : n;
        double mu = 0.0;
        if (remove_mean) {
            double sum = 0.0;
            for (int64_t i = s0; i < s1; ++i) sum += x[i];
            mu = sum / (double)(s1 - s0);
        }
        for (int64_t i = s0; i < s1; ++i) y[i] = x[i] - mu;
    }
}

/* ------------------------------------------------------------------ */
/* Parzen lag window d(w), u = |w| / L:
 *   1 - 6u^2 + 6u^3  for u <= 1/2,   2(1-u)^3 for 1/2 < u <= 1,   0 beyond. */
double hos_oracle_parzen(int64_t w, int64_t L)
{
    double u = fabs((double)w) / (double)L;
    if (u <= 0.5) return 1.0 - 6.0 * u * u + 6.0 * u * u * u;
    if (u <= 1.0) return 2.0 * (1.0 - u) * (1.0 - u) * (1.0 - u);
    return 0.0;
}

static double rect_w(int64_t w, int64_t L) { return (w >= -(L - 1) && w <= L - 1) ? 1.0 : 0.0; }

/* Lag window on the lag square.  PARZEN: d(w1) d(w2).  PARZEN_SYM:
 * d(w1) d(w2) d(w1 - w2), which keeps the six-fold symmetry of c3.
 * RECT: 1 inside |w1|, |w2| <= L-1, else 0.                           */
double hos_oracle_window2(int64_t w1, int64_t w2, int64_t L, int kind)
{
    if (kind == ORACLE_WIN_PARZEN) return hos_oracle_parzen(w1, L) * hos_oracle_parzen(w2, L);
    if (kind == ORACLE_WIN_PARZEN_SYM)
        return hos_oracle_parzen(w1, L) * hos_oracle_parzen(w2, L) * hos_oracle_parzen(w1 - w2, L);
    return rect_w(w1, L) * rect_w(w2, L);
}

/* Lag window on the lag cube.  PARZEN: d(w1) d(w2) d(w3).  RECT as above. */
double hos_oracle_window3(int64_t w1, int64_t w2, int64_t w3, int64_t L, int kind)
{
    if (kind == ORACLE_WIN_PARZEN)
        return hos_oracle_parzen(w1, L) * hos_oracle_parzen(w2, L) * hos_oracle_parzen(w3, L);
    return rect_w(w1, L) * rect_w(w2, L) * rect_w(w3, L);
}

/* ------------------------------------------------------------------ */
/* Second-order sample cumulant of a zero-mean series (Problem Statement,
 * c2(w) = m2(w) - m1^2 with m1 = 0 after mean removal), time average with
 * divisor n: c2(t) = (1/n) sum_i y(i) y(i+t), i and i+t inside [0, n).
 * Output c2[t + T] for t in [-T, T].                                      */
void hos_oracle_c2(const double* y, int64_t n, int64_t T, double* c2)
{
    for (int64_t t = -T; t <= T; ++t) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t j = i + t;
            if (j < 0 || j >= n) continue;
            s += y[i] * y[j];
        }
        c2[t + T] = s / (double)n;
    }
}

/* Third-order sample cumulant (= third moment of a zero-mean series):
 * c3(w1,w2) = (1/n) sum_i y(i) y(i+w1) y(i+w2), over every i for which all
 * three samples lie in [0, n).  Output c3[(w1+L)(2L+1) + (w2+L)].
 * The loop over w1 is split across threads; each sum keeps its order.     */
void hos_oracle_c3(const double* y, int64_t n, int64_t L, double* c3)
{
    const int64_t W = 2 * L + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w1 = -L; w1 <= L; ++w1) {
        for (int64_t w2 = -L; w2 <= L; ++w2) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                int64_t j = i + w1, k = i + w2;
                if (j < 0 || j >= n || k < 0 || k >= n) continue;
                s += y[i] * y[j] * y[k];
            }
            c3[(w1 + L) * W + (w2 + L)] = s / (double)n;
        }
    }
}

/* c3 at an explicit list of lag pairs (lags[2p], lags[2p+1]); same sum.  */
void hos_oracle_c3_at(const double* y, int64_t n, const int64_t* lags, int64_t npairs, double* out)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t w1 = lags[2 * p], w2 = lags[2 * p + 1];
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            int64_t j = i + w1, k = i + w2;
            if (j < 0 || j >= n || k < 0 || k >= n) continue;
            s += y[i] * y[j] * y[k];
        }
        out[p] = s / (double)n;
    }
}

/* Rows w1 in [w1_lo, w1_hi] of c3 (all w2 in [-L, L]); used to time a
 * bounded slice of a large workload.  Same sum as hos_oracle_c3.          */
void hos_oracle_c3_rows(const double* y, int64_t n, int64_t L, int64_t w1_lo, int64_t w1_hi, double* out)
{
    const int64_t W = 2 * L + 1;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (int64_t w1 = w1_lo; w1 <= w1_hi; ++w1) {
        for (int64_t w2 = -L; w2 <= L; ++w2) {
            double s = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                int64_t j = i + w1, k = i + w2;
                if (j < 0 || j >= n || k < 0 || k >= n) continue;
                s += y[i] * y[j] * y[k];
            }
            out[(w1 - w1_lo) * W + (w2 + L)] = s / (double)n;
        }
    }
}

/* Fourth-order sample moment m4(w1,w2,w3) = (1/n) sum_i y(i) y(i+w1)
 * y(i+w2) y(i+w3) over i with all four samples inside [0, n).
 * Output m4[((w1+L)(2L+1) + (w2+L))(2L+1) + (w3+L)].                       */
void hos_oracle_m4(const double* y, int64_t n, int64_t L, double* m4)
{
    const int64_t W = 2 * L + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t w1 = -L; w1 <= L; ++w1)
        for (int64_t w2 = -L; w2 <= L; ++w2)
            for (int64_t w3 = -L; w3 <= L; ++w3) {
                double s = 0.0;
                for (int64_t i = 0; i < n; ++i) {
                    int64_t a = i + w1, b = i + w2, c = i + w3;
                    if (a < 0 || a >= n || b < 0 || b >= n || c < 0 || c >= n) continue;
                    s += y[i] * y[a] * y[b] * y[c];
                }
                m4[((w1 + L) * W + (w2 + L)) * W + (w3 + L)] = s / (double)n;
            }
}

/* Fourth-order sample cumulant of a zero-mean series.  The paper defines
 * cumulants through c2 and then says "and so on"; the reading used is the
 * moment-to-cumulant identity for zero-mean variables:
 *   c4(w1,w2,w3) = m4(w1,w2,w3) - c2(w1) c2(w3-w2) - c2(w2) c2(w3-w1)
 *                  - c2(w3) c2(w2-w1),
 * with m4 and c2 the sample moments above (same 1/n time averages).        */
void hos_oracle_c4(const double* y, int64_t n, int64_t L, double* c4)
{
    const int64_t W = 2 * L + 1, T = 2 * L;
    double* c2 = (double*)malloc(sizeof(double) * (size_t)(2 * T + 1));
    hos_oracle_c2(y, n, T, c2);
    hos_oracle_m4(y, n, L, c4);
    for (int64_t w1 = -L; w1 <= L; ++w1)
        for (int64_t w2 = -L; w2 <= L; ++w2)
            for (int64_t w3 = -L; w3 <= L; ++w3) {
                double corr = c2[w1 + T] * c2[w3 - w2 + T] + c2[w2 + T] * c2[w3 - w1 + T] +
                              c2[w3 + T] * c2[w2 - w1 + T];
                c4[((w1 + L) * W + (w2 + L)) * W + (w3 + L)] -= corr;
            }
    free(c2);
}

/* ------------------------------------------------------------------ */
/* Fourier transform onto the N-point grid (Algorithm DBS step 3 sign):
 *   out(k1,k2) = scale * sum_{w1,w2 in [-L,L]} f(w1,w2) e^{sign i 2 pi (k1 w1 + k2 w2) / N}
 * for k = 0..N-1.  Written as the double sum taken one axis at a time
 * (inner sum over w2 first).  The phase is reduced exactly in integers
 * before the cosine and sine are taken.                                    */
static void phase(int64_t k, int64_t w, int64_t N, double sign, double* c, double* s)
{
    int64_t r = (k * w) % N;
    if (r < 0) r += N;
    double a = 2.0 * HOS_ORACLE_PI * (double)r / (double)N;
    *c = cos(a);
    *s = sign * sin(a);
}

void hos_oracle_dft2(const double* f, int64_t L, int64_t N, double sign, double scale, double* out)
{
    const int64_t W = 2 * L + 1;
    double* t = (double*)calloc((size_t)(W * N * 2), sizeof(double)); /* t[w1][k2] complex */
    for (int64_t a = 0; a < W; ++a)
        for (int64_t k2 = 0; k2 < N; ++k2) {
            double re = 0.0, im = 0.0;
            for (int64_t b = 0; b < W; ++b) {
                double c, s;
                phase(k2, b - L, N, sign, &c, &s);
                re += f[a * W + b] * c;
                im += f[a * W + b] * s;
            }
            t[(a * N + k2) * 2] = re;
            t[(a * N + k2) * 2 + 1] = im;
        }
    for (int64_t k1 = 0; k1 < N; ++k1)
        for (int64_t k2 = 0; k2 < N; ++k2) {
            double re = 0.0, im = 0.0;
            for (int64_t a = 0; a < W; ++a) {
                double c, s;
                phase(k1, a - L, N, sign, &c, &s);
                double tr = t[(a * N + k2) * 2], ti = t[(a * N + k2) * 2 + 1];
                re += tr * c - ti * s;
                im += tr * s + ti * c;
            }
            out[(k1 * N + k2) * 2] = scale * re;
            out[(k1 * N + k2) * 2 + 1] = scale * im;
        }
    free(t);
}

/* Same for the lag cube: sum over w3, then w2, then w1.                    */
void hos_oracle_dft3(const double* f, int64_t L, int64_t N, double sign, double scale, double* out)
{
    const int64_t W = 2 * L + 1;
    double* t1 = (double*)calloc((size_t)(W * W * N * 2), sizeof(double)); /* [w1][w2][k3] */
    double* t2 = (double*)calloc((size_t)(W * N * N * 2), sizeof(double)); /* [w1][k2][k3] */
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b)
            for (int64_t k3 = 0; k3 < N; ++k3) {
                double re = 0.0, im = 0.0;
                for (int64_t c3 = 0; c3 < W; ++c3) {
                    double c, s;
                    phase(k3, c3 - L, N, sign, &c, &s);
                    double v = f[(a * W + b) * W + c3];
                    re += v * c;
                    im += v * s;
                }
                t1[((a * W + b) * N + k3) * 2] = re;
                t1[((a * W + b) * N + k3) * 2 + 1] = im;
            }
    for (int64_t a = 0; a < W; ++a)
        for (int64_t k2 = 0; k2 < N; ++k2)
            for (int64_t k3 = 0; k3 < N; ++k3) {
                double re = 0.0, im = 0.0;
                for (int64_t b = 0; b < W; ++b) {
                    double c, s;
                    phase(k2, b - L, N, sign, &c, &s);
                    double tr = t1[((a * W + b) * N + k3) * 2], ti = t1[((a * W + b) * N + k3) * 2 + 1];
                    re += tr * c - ti * s;
                    im += tr * s + ti * c;
                }
                t2[((a * N + k2) * N + k3) * 2] = re;
                t2[((a * N + k2) * N + k3) * 2 + 1] = im;
            }
    for (int64_t k1 = 0; k1 < N; ++k1)
        for (int64_t k2 = 0; k2 < N; ++k2)
            for (int64_t k3 = 0; k3 < N; ++k3) {
                double re = 0.0, im = 0.0;
                for (int64_t a = 0; a < W; ++a) {
                    double c, s;
                    phase(k1, a - L, N, sign, &c, &s);
                    double tr = t2[((a * N + k2) * N + k3) * 2], ti = t2[((a * N + k2) * N + k3) * 2 + 1];
                    re += tr * c - ti * s;
                    im += tr * s + ti * c;
                }
                out[((k1 * N + k2) * N + k3) * 2] = scale * re;
                out[((k1 * N + k2) * N + k3) * 2 + 1] = scale * im;
            }
    free(t1);
    free(t2);
}

/* ------------------------------------------------------------------ */
/* Number of parts of Algorithm DBS step 1 and their bounds.                */
static int64_t n_parts(int64_t n, int64_t seg) { return (seg <= 0 || seg >= n) ? 1 : (n + seg - 1) / seg; }

/* Smoothed sample bispectrum, indirect method:
 *   per part (DBS steps 1-2): y = x - mean; c3 of the part (its own 1/m);
 *   average of the parts' c3 (DBS step 6, taken before the linear transform);
 *   lag window W(w1,w2); B(k1,k2) = (2 pi)^-2 sum_w W c3 e^{-i 2 pi k.w / N}.
 * Output B complex interleaved [k1][k2], N x N.                             */
void hos_oracle_bispectrum(const double* x, int64_t n, int64_t L, int64_t N, int window, int remove_mean,
                           int64_t seg, double* B)
{
    const int64_t W = 2 * L + 1;
    const int64_t K = n_parts(n, seg);
    const int64_t m = (K == 1) ? n : seg;
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* c3 = (double*)calloc((size_t)(W * W), sizeof(double));
    double* acc = (double*)calloc((size_t)(W * W), sizeof(double));
    hos_oracle_demean(x, n, K == 1 ? n : seg, remove_mean, y);
    for (int64_t p = 0; p < K; ++p) {
        int64_t s0 = p * m, s1 = s0 + m < n ? s0 + m : n;
        hos_oracle_c3(y + s0, s1 - s0, L, c3);
        for (int64_t q = 0; q < W * W; ++q) acc[q] += c3[q];
    }
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b)
            acc[a * W + b] = acc[a * W + b] / (double)K * hos_oracle_window2(a - L, b - L, L, window);
    double scale = 1.0 / ((2.0 * HOS_ORACLE_PI) * (2.0 * HOS_ORACLE_PI));
    hos_oracle_dft2(acc, L, N, -1.0, scale, B);
    free(y);
    free(c3);
    free(acc);
}

/* Smoothed sample trispectrum, indirect method: c4 per part, averaged,
 * windowed, T(k1,k2,k3) = (2 pi)^-3 sum_w W c4 e^{-i 2 pi k.w / N}.          */
void hos_oracle_trispectrum(const double* x, int64_t n, int64_t L, int64_t N, int window, int remove_mean,
                            int64_t seg, double* T)
{
    const int64_t W = 2 * L + 1, W3 = W * W * W;
    const int64_t K = n_parts(n, seg);
    const int64_t m = (K == 1) ? n : seg;
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* c4 = (double*)calloc((size_t)W3, sizeof(double));
    double* acc = (double*)calloc((size_t)W3, sizeof(double));
    hos_oracle_demean(x, n, K == 1 ? n : seg, remove_mean, y);
    for (int64_t p = 0; p < K; ++p) {
        int64_t s0 = p * m, s1 = s0 + m < n ? s0 + m : n;
        hos_oracle_c4(y + s0, s1 - s0, L, c4);
        for (int64_t q = 0; q < W3; ++q) acc[q] += c4[q];
    }
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b)
            for (int64_t c = 0; c < W; ++c)
                acc[(a * W + b) * W + c] =
                    acc[(a * W + b) * W + c] / (double)K * hos_oracle_window3(a - L, b - L, c - L, L, window);
    double s = 2.0 * HOS_ORACLE_PI;
    hos_oracle_dft3(acc, L, N, -1.0, 1.0 / (s * s * s), T);
    free(y);
    free(c4);
    free(acc);
}

/* ------------------------------------------------------------------ */
/* Overlapping parts (the multi-segment averaging of Algorithm DBS steps 1,
 * 2 and 6 with parts that overlap): parts of m samples starting every
 * m - overlap samples, K = floor((n - m) / (m - overlap)) + 1 of them;
 * samples past the last whole part are not used; n <= m gives one part,
 * the whole series.  Each part minus its own mean (when remove_mean), its
 * cumulant with its own 1/m, the parts' cumulants averaged, then windowed
 * and transformed as in hos_oracle_bispectrum / hos_oracle_trispectrum.     */
static void overlap_parts(int64_t n, int64_t m, int64_t overlap, int64_t* K, int64_t* len, int64_t* step)
{
    if (m <= 0 || n <= m) {
        *K = 1;
        *len = n;
        *step = n;
        return;
    }
    *step = m - overlap;
    *K = (n - m) / *step + 1;
    *len = m;
}

/* accumulate the average over the parts of c3 (order 3) or c4 (order 4) */
static void overlap_cumulant(const double* x, int64_t n, int64_t L, int order, int remove_mean, int64_t m,
                             int64_t overlap, double* acc)
{
    const int64_t W = 2 * L + 1, WW = order == 3 ? W * W : W * W * W;
    int64_t K, len, step;
    overlap_parts(n, m, overlap, &K, &len, &step);
    double* y = (double*)malloc(sizeof(double) * (size_t)len);
    double* c = (double*)malloc(sizeof(double) * (size_t)WW);
    for (int64_t q = 0; q < WW; ++q) acc[q] = 0.0;
    for (int64_t p = 0; p < K; ++p) {
        hos_oracle_demean(x + p * step, len, len, remove_mean, y);
        if (order == 3) hos_oracle_c3(y, len, L, c);
        else hos_oracle_c4(y, len, L, c);
        for (int64_t q = 0; q < WW; ++q) acc[q] += c[q];
    }
    for (int64_t q = 0; q < WW; ++q) acc[q] /= (double)K;
    free(y);
    free(c);
}

void hos_oracle_bispectrum_overlap(const double* x, int64_t n, int64_t L, int64_t N, int window, int remove_mean,
                                   int64_t seg, int64_t overlap, double* B)
{
    const int64_t W = 2 * L + 1;
    double* acc = (double*)malloc(sizeof(double) * (size_t)(W * W));
    overlap_cumulant(x, n, L, 3, remove_mean, seg, overlap, acc);
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b) acc[a * W + b] *= hos_oracle_window2(a - L, b - L, L, window);
    const double s = 2.0 * HOS_ORACLE_PI;
    hos_oracle_dft2(acc, L, N, -1.0, 1.0 / (s * s), B);
    free(acc);
}

void hos_oracle_trispectrum_overlap(const double* x, int64_t n, int64_t L, int64_t N, int window, int remove_mean,
                                    int64_t seg, int64_t overlap, double* T)
{
    const int64_t W = 2 * L + 1;
    double* acc = (double*)malloc(sizeof(double) * (size_t)(W * W * W));
    overlap_cumulant(x, n, L, 4, remove_mean, seg, overlap, acc);
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b)
            for (int64_t c = 0; c < W; ++c)
                acc[(a * W + b) * W + c] *= hos_oracle_window3(a - L, b - L, c - L, L, window);
    const double s = 2.0 * HOS_ORACLE_PI;
    hos_oracle_dft3(acc, L, N, -1.0, 1.0 / (s * s * s), T);
    free(acc);
}

/* The averaged cumulant alone (no window, no transform), over [-L, L]^2 or
 * [-L, L]^3, for checking hos_cumulant3 / hos_cumulant4.                    */
void hos_oracle_cumulant_overlap(const double* x, int64_t n, int64_t L, int order, int remove_mean, int64_t seg,
                                 int64_t overlap, double* out)
{
    overlap_cumulant(x, n, L, order, remove_mean, seg, overlap, out);
}

/* ------------------------------------------------------------------ */
/* Gradient of a real loss l(B) through the bispectrum (one part, K = 1).
 * G holds dl/dRe B + i dl/dIm B on the N x N grid (complex interleaved).
 * The chain rule is taken step by step, in reverse order of the forward:
 *   1. through the transform and window:
 *        dl/dc3(w) = W(w) (2 pi)^-2 Re sum_k G(k) e^{+i 2 pi k.w / N};
 *   2. through the triple-product loop of hos_oracle_c3: every term
 *      y(i) y(j) y(k) / n with j = i+w1, k = i+w2 sends its partial
 *      derivative to each of its three samples;
 *   3. through the mean removal y = x - mean(x): dx = dy - mean(dy).       */
void hos_oracle_bispectrum_grad(const double* x, int64_t n, int64_t L, int64_t N, int window, int remove_mean,
                                const double* G, double* dx)
{
    const int64_t W = 2 * L + 1;
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* dc = (double*)malloc(sizeof(double) * (size_t)(W * W));
    double* dy = (double*)calloc((size_t)n, sizeof(double));
    hos_oracle_demean(x, n, n, remove_mean, y);
    const double scale = 1.0 / ((2.0 * HOS_ORACLE_PI) * (2.0 * HOS_ORACLE_PI));
    for (int64_t w1 = -L; w1 <= L; ++w1)
        for (int64_t w2 = -L; w2 <= L; ++w2) {
            double re = 0.0;
            for (int64_t k1 = 0; k1 < N; ++k1)
                for (int64_t k2 = 0; k2 < N; ++k2) {
                    int64_t r = (k1 * w1 + k2 * w2) % N;
                    if (r < 0) r += N;
                    double a = 2.0 * HOS_ORACLE_PI * (double)r / (double)N;
                    const double* g = G + (k1 * N + k2) * 2;
                    re += g[0] * cos(a) - g[1] * sin(a);
                }
            dc[(w1 + L) * W + (w2 + L)] = hos_oracle_window2(w1, w2, L, window) * scale * re;
        }
    for (int64_t w1 = -L; w1 <= L; ++w1)
        for (int64_t w2 = -L; w2 <= L; ++w2) {
            double gw = dc[(w1 + L) * W + (w2 + L)] / (double)n;
            if (gw == 0.0) continue;
            for (int64_t i = 0; i < n; ++i) {
                int64_t j = i + w1, k = i + w2;
                if (j < 0 || j >= n || k < 0 || k >= n) continue;
                dy[i] += gw * y[j] * y[k];
                dy[j] += gw * y[i] * y[k];
                dy[k] += gw * y[i] * y[j];
            }
        }
    double mu = 0.0;
    if (remove_mean) {
        for (int64_t i = 0; i < n; ++i) mu += dy[i];
        mu /= (double)n;
    }
    for (int64_t i = 0; i < n; ++i) dx[i] = dy[i] - mu;
    free(y);
    free(dc);
    free(dy);
}

/* ------------------------------------------------------------------ */
/* Step 1 of the gradient alone, for large grids: dl/dc3(w) on [-L, L]^2,
 *   W(w) (2 pi)^-2 Re sum_k G(k) e^{+i 2 pi k.w / N},
 * with the double sum over k taken one axis at a time (inner sum over k2).  */
void hos_oracle_grad_lag(const double* G, int64_t L, int64_t N, int window, double* dc)
{
    const int64_t W = 2 * L + 1;
    double* t = (double*)calloc((size_t)(N * W * 2), sizeof(double)); /* t[k1][w2] complex */
    for (int64_t k1 = 0; k1 < N; ++k1)
        for (int64_t b = 0; b < W; ++b) {
            double re = 0.0, im = 0.0;
            for (int64_t k2 = 0; k2 < N; ++k2) {
                double c, s;
                phase(k2, b - L, N, +1.0, &c, &s);
                const double gr = G[(k1 * N + k2) * 2], gi = G[(k1 * N + k2) * 2 + 1];
                re += gr * c - gi * s;
                im += gr * s + gi * c;
            }
            t[(k1 * W + b) * 2] = re;
            t[(k1 * W + b) * 2 + 1] = im;
        }
    const double scale = 1.0 / ((2.0 * HOS_ORACLE_PI) * (2.0 * HOS_ORACLE_PI));
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b) {
            double re = 0.0;
            for (int64_t k1 = 0; k1 < N; ++k1) {
                double c, s;
                phase(k1, a - L, N, +1.0, &c, &s);
                re += t[(k1 * W + b) * 2] * c - t[(k1 * W + b) * 2 + 1] * s;
            }
            dc[a * W + b] = hos_oracle_window2(a - L, b - L, L, window) * scale * re;
        }
    free(t);
}

/* Step 2 of the gradient at chosen samples j (no mean removal):
 *   dy(j) = (1/n) sum_w dc(w) [ y(j+w1) y(j+w2) + y(j-w1) y(j-w1+w2) + y(j-w2) y(j-w2+w1) ],
 * the three places sample j can occupy in a triple product of the c3 loop
 * (samples outside [0, n) are zero).                                        */
void hos_oracle_dy_at(const double* y, int64_t n, int64_t L, const double* dc, const int64_t* js, int64_t count,
                      double* out)
{
    const int64_t W = 2 * L + 1;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t q = 0; q < count; ++q) {
        const int64_t j = js[q];
        double acc = 0.0;
        for (int64_t w1 = -L; w1 <= L; ++w1)
            for (int64_t w2 = -L; w2 <= L; ++w2) {
                const double g = dc[(w1 + L) * W + (w2 + L)];
                if (g == 0.0) continue;
#define YV(k) (((k) >= 0 && (k) < n) ? y[(k)] : 0.0)
                double term = YV(j + w1) * YV(j + w2);
                term += YV(j - w1) * YV(j - w1 + w2);
                term += YV(j - w2) * YV(j - w2 + w1);
#undef YV
                acc += g * term;
            }
        out[q] = acc / (double)n;
    }
}

/* ------------------------------------------------------------------ */
/* Gradient of a real loss l(T) through the trispectrum (one part, K = 1).
 * Step 1 alone: dl/dc4(w) on [-L, L]^3 for G = dl/dRe T + i dl/dIm T on the
 * N^3 grid,
 *   W(w) (2 pi)^-3 Re sum_k G(k) e^{+i 2 pi k.w / N},
 * the triple sum over k taken one axis at a time (k3, then k2, then k1).    */
void hos_oracle_grad_lag4(const double* G, int64_t L, int64_t N, int window, double* dc)
{
    const int64_t W = 2 * L + 1;
    /* t3[k1][k2][w3], t2[k1][w2][w3]: complex */
    double* t3 = (double*)calloc((size_t)(N * N * W * 2), sizeof(double));
    double* t2 = (double*)calloc((size_t)(N * W * W * 2), sizeof(double));
    for (int64_t k1 = 0; k1 < N; ++k1)
        for (int64_t k2 = 0; k2 < N; ++k2)
            for (int64_t c = 0; c < W; ++c) {
                double re = 0.0, im = 0.0;
                for (int64_t k3 = 0; k3 < N; ++k3) {
                    double cs, sn;
                    phase(k3, c - L, N, +1.0, &cs, &sn);
                    const double* g = G + ((k1 * N + k2) * N + k3) * 2;
                    re += g[0] * cs - g[1] * sn;
                    im += g[0] * sn + g[1] * cs;
                }
                t3[((k1 * N + k2) * W + c) * 2] = re;
                t3[((k1 * N + k2) * W + c) * 2 + 1] = im;
            }
    for (int64_t k1 = 0; k1 < N; ++k1)
        for (int64_t b = 0; b < W; ++b)
            for (int64_t c = 0; c < W; ++c) {
                double re = 0.0, im = 0.0;
                for (int64_t k2 = 0; k2 < N; ++k2) {
                    double cs, sn;
                    phase(k2, b - L, N, +1.0, &cs, &sn);
                    const double* t = t3 + ((k1 * N + k2) * W + c) * 2;
                    re += t[0] * cs - t[1] * sn;
                    im += t[0] * sn + t[1] * cs;
                }
                t2[((k1 * W + b) * W + c) * 2] = re;
                t2[((k1 * W + b) * W + c) * 2 + 1] = im;
            }
    const double s = 2.0 * HOS_ORACLE_PI, scale = 1.0 / (s * s * s);
    for (int64_t a = 0; a < W; ++a)
        for (int64_t b = 0; b < W; ++b)
            for (int64_t c = 0; c < W; ++c) {
                double re = 0.0;
                for (int64_t k1 = 0; k1 < N; ++k1) {
                    double cs, sn;
                    phase(k1, a - L, N, +1.0, &cs, &sn);
                    const double* t = t2 + ((k1 * W + b) * W + c) * 2;
                    re += t[0] * cs - t[1] * sn;
                }
                dc[(a * W + b) * W + c] = hos_oracle_window3(a - L, b - L, c - L, L, window) * scale * re;
            }
    free(t3);
    free(t2);
}

/* Step 2 of the gradient: dl/dc2(t), t in [-2L, 2L], from dl/dc4 and c2
 * through the three product terms of hos_oracle_c4; each term
 * c2(a) c2(b) sends dc4 * c2(b) to c2(a) and dc4 * c2(a) to c2(b).
 * dc2 has 4L + 1 entries, index t + 2L.                                     */
void hos_oracle_grad_c2(const double* dc4, const double* c2, int64_t L, double* dc2)
{
    const int64_t W = 2 * L + 1, T = 2 * L;
    for (int64_t t = 0; t < 2 * T + 1; ++t) dc2[t] = 0.0;
    for (int64_t w1 = -L; w1 <= L; ++w1)
        for (int64_t w2 = -L; w2 <= L; ++w2)
            for (int64_t w3 = -L; w3 <= L; ++w3) {
                const double g = dc4[((w1 + L) * W + (w2 + L)) * W + (w3 + L)];
                if (g == 0.0) continue;
                const int64_t a[3] = {w1, w2, w3}, b[3] = {w3 - w2, w3 - w1, w2 - w1};
                for (int q = 0; q < 3; ++q) {
                    dc2[a[q] + T] -= g * c2[b[q] + T];
                    dc2[b[q] + T] -= g * c2[a[q] + T];
                }
            }
}

/* Gradient of a real loss l(T) through the trispectrum (one part, K = 1),
 * G = dl/dRe T + i dl/dIm T on the N^3 grid.  The chain rule in reverse
 * order of the forward:
 *   1. dl/dc4 through the transform and window (hos_oracle_grad_lag4);
 *   2. through c4 = m4 - (three c2 c2 terms): dl/dm4 = dl/dc4, and dl/dc2
 *      from hos_oracle_grad_c2;
 *   3. through the m4 loop: every term y(i) y(a) y(b) y(c) / n sends its
 *      partial derivative to each of its four samples;
 *   4. through the c2 loop: every term y(i) y(i+t) / n sends its partial to
 *      both samples;
 *   5. through the mean removal: dx = dy - mean(dy).                        */
void hos_oracle_trispectrum_grad(const double* x, int64_t n, int64_t L, int64_t N, int window, int remove_mean,
                                 const double* G, double* dx)
{
    const int64_t W = 2 * L + 1, T = 2 * L;
    double* y = (double*)malloc(sizeof(double) * (size_t)n);
    double* dc4 = (double*)malloc(sizeof(double) * (size_t)(W * W * W));
    double* c2 = (double*)malloc(sizeof(double) * (size_t)(2 * T + 1));
    double* dc2 = (double*)malloc(sizeof(double) * (size_t)(2 * T + 1));
    double* dy = (double*)calloc((size_t)n, sizeof(double));
    hos_oracle_demean(x, n, n, remove_mean, y);
    hos_oracle_grad_lag4(G, L, N, window, dc4);
    hos_oracle_c2(y, n, T, c2);
    hos_oracle_grad_c2(dc4, c2, L, dc2);
    for (int64_t w1 = -L; w1 <= L; ++w1)
        for (int64_t w2 = -L; w2 <= L; ++w2)
            for (int64_t w3 = -L; w3 <= L; ++w3) {
                const double g = dc4[((w1 + L) * W + (w2 + L)) * W + (w3 + L)] / (double)n;
                if (g == 0.0) continue;
                for (int64_t i = 0; i < n; ++i) {
                    const int64_t a = i + w1, b = i + w2, c = i + w3;
                    if (a < 0 || a >= n || b < 0 || b >= n || c < 0 || c >= n) continue;
                    dy[i] += g * y[a] * y[b] * y[c];
                    dy[a] += g * y[i] * y[b] * y[c];
                    dy[b] += g * y[i] * y[a] * y[c];
                    dy[c] += g * y[i] * y[a] * y[b];
                }
            }
    for (int64_t t = -T; t <= T; ++t) {
        const double g = dc2[t + T] / (double)n;
        if (g == 0.0) continue;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t a = i + t;
            if (a < 0 || a >= n) continue;
            dy[i] += g * y[a];
            dy[a] += g * y[i];
        }
    }
    double mu = 0.0;
    if (remove_mean) {
        for (int64_t i = 0; i < n; ++i) mu += dy[i];
        mu /= (double)n;
    }
    for (int64_t i = 0; i < n; ++i) dx[i] = dy[i] - mu;
    free(y);
    free(dc4);
    free(c2);
    free(dc2);
    free(dy);
}

/* Steps 2-4 of the trispectrum gradient at chosen samples j (no mean
 * removal), for series too long for the full loops:
 *   dy(j) = (1/n) sum_w dc4(w) [ y(j+w1) y(j+w2) y(j+w3)
 *            + y(j-w1) y(j-w1+w2) y(j-w1+w3) + y(j-w2) y(j-w2+w1) y(j-w2+w3)
 *            + y(j-w3) y(j-w3+w1) y(j-w3+w2) ]
 *         + (1/n) sum_t dc2(t) [ y(j+t) + y(j-t) ],
 * the four places sample j can occupy in a product of the m4 loop and the
 * two in a product of the c2 loop (samples outside [0, n) are zero).
 * dc2 is hos_oracle_grad_c2 of dc4 and the series' c2.                      */
void hos_oracle_dy4_at(const double* y, int64_t n, int64_t L, const double* dc4, const double* dc2,
                       const int64_t* js, int64_t count, double* out)
{
    const int64_t W = 2 * L + 1, T = 2 * L;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < count; ++q) {
        const int64_t j = js[q];
        double acc = 0.0;
#define YV(k) (((k) >= 0 && (k) < n) ? y[(k)] : 0.0)
        for (int64_t w1 = -L; w1 <= L; ++w1)
            for (int64_t w2 = -L; w2 <= L; ++w2)
                for (int64_t w3 = -L; w3 <= L; ++w3) {
                    const double g = dc4[((w1 + L) * W + (w2 + L)) * W + (w3 + L)];
                    if (g == 0.0) continue;
                    double term = YV(j + w1) * YV(j + w2) * YV(j + w3);
                    term += YV(j - w1) * YV(j - w1 + w2) * YV(j - w1 + w3);
                    term += YV(j - w2) * YV(j - w2 + w1) * YV(j - w2 + w3);
                    term += YV(j - w3) * YV(j - w3 + w1) * YV(j - w3 + w2);
                    acc += g * term;
                }
        for (int64_t t = -T; t <= T; ++t) acc += dc2[t + T] * (YV(j + t) + YV(j - t));
#undef YV
        out[q] = acc / (double)n;
    }
}

/* ------------------------------------------------------------------ */
/* The direct method, Algorithm DBS steps 1-6, as the paper states it:
 *   1. parts of M samples starting every M - overlap samples (overlap = 0:
 *      the paper's partition, K = floor(n / M)); K = floor((n - M) /
 *      (M - overlap)) + 1, trailing samples past the last part not used;
 *   2. each part minus its own mean (when remove_mean);
 *   3. F_i(k) = sum_u X_i(u) e^{-j 2 pi u k / M}, k = 0..M-1, summed directly;
 *   4. raw C3_i(k1,k2) = (1/M) F_i(k1) F_i(k2) F_i*(k1+k2) -- reading: the
 *      conjugate on the third factor (the product with F(k1+k2) itself is
 *      not the bispectrum); indices mod M, F being M-periodic, so the raw
 *      estimate is defined on the whole M x M grid;
 *   5. M3 x M3 box smoothing, (1/M3^2) sum_{n1,n2 = lo}^{lo+M3-1}
 *      C3_i(k1+n1, k2+n2), lo = -floor(M3/2) (the paper's -M3/2 .. M3/2-1
 *      for even M3), indices mod M;
 *   6. average over the K parts.
 * Step 5 is the plain double sum per output point (the paper's "Naive"
 * smoothing), not window sums.  out: M*M complex, row-major [k1][k2].       */
void hos_oracle_bispectrum_direct(const double* x, int64_t n, int64_t M, int64_t M3, int64_t overlap,
                                  int remove_mean, double* out)
{
    const int64_t step = M - overlap;
    const int64_t K = n >= M ? (n - M) / step + 1 : 0;
    const int64_t lo = -(M3 / 2);
    double* y = (double*)malloc((size_t)M * sizeof(double));
    double* F = (double*)malloc((size_t)M * 2 * sizeof(double));
    double* raw = (double*)malloc((size_t)(M * M * 2) * sizeof(double));
    memset(out, 0, (size_t)(M * M * 2) * sizeof(double));
    for (int64_t part = 0; part < K; ++part) {
        const double* xp = x + part * step;
        double mean = 0.0;
        if (remove_mean) {
            for (int64_t u = 0; u < M; ++u) mean += xp[u];
            mean /= (double)M;
        }
        for (int64_t u = 0; u < M; ++u) y[u] = xp[u] - mean;
        for (int64_t k = 0; k < M; ++k) { /* step 3 */
            double re = 0.0, im = 0.0;
            for (int64_t u = 0; u < M; ++u) {
                double c, s;
                phase(u, k, M, -1.0, &c, &s);
                re += y[u] * c;
                im += y[u] * s;
            }
            F[2 * k] = re;
            F[2 * k + 1] = im;
        }
        for (int64_t k1 = 0; k1 < M; ++k1) /* step 4 */
            for (int64_t k2 = 0; k2 < M; ++k2) {
                const int64_t k3 = (k1 + k2) % M;
                const double ar = F[2 * k1], ai = F[2 * k1 + 1];
                const double br = F[2 * k2], bi = F[2 * k2 + 1];
                const double cr = F[2 * k3], ci = -F[2 * k3 + 1]; /* conjugate */
                const double pr = ar * br - ai * bi, pi = ar * bi + ai * br;
                raw[(k1 * M + k2) * 2] = (pr * cr - pi * ci) / (double)M;
                raw[(k1 * M + k2) * 2 + 1] = (pr * ci + pi * cr) / (double)M;
            }
#pragma omp parallel for schedule(static)
        for (int64_t k1 = 0; k1 < M; ++k1) /* step 5, accumulated into step 6 */
            for (int64_t k2 = 0; k2 < M; ++k2) {
                double sr = 0.0, si = 0.0;
                for (int64_t n1 = lo; n1 < lo + M3; ++n1)
                    for (int64_t n2 = lo; n2 < lo + M3; ++n2) {
                        int64_t a = (k1 + n1) % M, b = (k2 + n2) % M;
                        if (a < 0) a += M;
                        if (b < 0) b += M;
                        sr += raw[(a * M + b) * 2];
                        si += raw[(a * M + b) * 2 + 1];
                    }
                out[(k1 * M + k2) * 2] += sr / (double)(M3 * M3) / (double)K;
                out[(k1 * M + k2) * 2 + 1] += si / (double)(M3 * M3) / (double)K;
            }
    }
    free(y);
    free(F);
    free(raw);
}
