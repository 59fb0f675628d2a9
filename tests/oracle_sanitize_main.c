/*
 * Drives every routine of oracle/hos_oracle.c over small and edge-case
 * shapes (a series of one sample, lags longer than the series, odd grids,
 * overlapping parts, the direct method's overlap), so that a build of the
 * oracle with AddressSanitizer and UndefinedBehaviorSanitizer checks every
 * array access the routines make.  Exit status 0 when every call returns
 * and every output is finite.  Test support only (tests/test_oracle_sanitizers.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

void hos_oracle_demean(const double*, int64_t, int64_t, int, double*);
double hos_oracle_parzen(int64_t, int64_t);
double hos_oracle_window2(int64_t, int64_t, int64_t, int);
double hos_oracle_window3(int64_t, int64_t, int64_t, int64_t, int);
void hos_oracle_c2(const double*, int64_t, int64_t, double*);
void hos_oracle_c3(const double*, int64_t, int64_t, double*);
void hos_oracle_c3_at(const double*, int64_t, const int64_t*, int64_t, double*);
void hos_oracle_c3_rows(const double*, int64_t, int64_t, int64_t, int64_t, double*);
void hos_oracle_m4(const double*, int64_t, int64_t, double*);
void hos_oracle_c4(const double*, int64_t, int64_t, double*);
void hos_oracle_dft2(const double*, int64_t, int64_t, double, double, double*);
void hos_oracle_dft3(const double*, int64_t, int64_t, double, double, double*);
void hos_oracle_bispectrum(const double*, int64_t, int64_t, int64_t, int, int, int64_t, double*);
void hos_oracle_trispectrum(const double*, int64_t, int64_t, int64_t, int, int, int64_t, double*);
void hos_oracle_bispectrum_overlap(const double*, int64_t, int64_t, int64_t, int, int, int64_t, int64_t, double*);
void hos_oracle_trispectrum_overlap(const double*, int64_t, int64_t, int64_t, int, int, int64_t, int64_t, double*);
void hos_oracle_cumulant_overlap(const double*, int64_t, int64_t, int, int, int64_t, int64_t, double*);
void hos_oracle_bispectrum_grad(const double*, int64_t, int64_t, int64_t, int, int, const double*, double*);
void hos_oracle_grad_lag(const double*, int64_t, int64_t, int, double*);
void hos_oracle_dy_at(const double*, int64_t, int64_t, const double*, const int64_t*, int64_t, double*);
void hos_oracle_grad_lag4(const double*, int64_t, int64_t, int, double*);
void hos_oracle_grad_c2(const double*, const double*, int64_t, double*);
void hos_oracle_trispectrum_grad(const double*, int64_t, int64_t, int64_t, int, int, const double*, double*);
void hos_oracle_dy4_at(const double*, int64_t, int64_t, const double*, const double*, const int64_t*, int64_t,
                       double*);
void hos_oracle_bispectrum_direct(const double*, int64_t, int64_t, int64_t, int64_t, int, double*);

static int bad = 0;

static double* vec(int64_t n, unsigned seed) {  /* exactly n doubles, so any overrun is caught */
    double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    unsigned s = seed * 2654435761u + 12345u;
    for (int64_t i = 0; i < n; ++i) {
        s = s * 1103515245u + 12345u;
        v[i] = ((double)(s >> 8) / 16777216.0) - 0.5;
    }
    return v;
}

static void check(const char* what, const double* v, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(v[i])) {
            fprintf(stderr, "%s: non-finite output at %lld\n", what, (long long)i);
            bad = 1;
            return;
        }
}

int main(void) {
    const int64_t shapes[][3] = {{1, 1, 2}, {2, 3, 6}, {7, 2, 5}, {23, 5, 10}, {40, 4, 9}};
    for (int k = 0; k < 5; ++k) {
        const int64_t n = shapes[k][0], L = shapes[k][1], N = shapes[k][2];
        const int64_t W = 2 * L + 1, T = 2 * L;
        double* x = vec(n, 11 + k);
        double* y = vec(n, 0);
        hos_oracle_demean(x, n, 0, 1, y);
        hos_oracle_demean(x, n, 3, 1, y);
        check("demean", y, n);
        double* c2 = vec(2 * T + 1, 0);
        hos_oracle_c2(y, n, T, c2);
        check("c2", c2, 2 * T + 1);
        double* c3 = vec(W * W, 0);
        hos_oracle_c3(y, n, L, c3);
        check("c3", c3, W * W);
        int64_t lags[4] = {-L, L, 0, L};
        double at[2];
        hos_oracle_c3_at(y, n, lags, 2, at);
        double* rows = vec(2 * W, 0);
        hos_oracle_c3_rows(y, n, L, -L, -L + 1, rows);
        check("c3_rows", rows, 2 * W);
        double* c4 = vec(W * W * W, 0);
        hos_oracle_m4(y, n, L, c4);
        hos_oracle_c4(y, n, L, c4);
        check("c4", c4, W * W * W);
        double* B = vec(N * N * 2, 0);
        double* Tg = vec(N * N * N * 2, 0);
        hos_oracle_dft2(c3, L, N, -1.0, 1.0, B);
        hos_oracle_dft3(c4, L, N, -1.0, 1.0, Tg);
        for (int win = 0; win <= 2; ++win) {
            hos_oracle_bispectrum(x, n, L, N, win, 1, 0, B);
            check("bispectrum", B, N * N * 2);
            if (win != 1) {
                hos_oracle_trispectrum(x, n, L, N, win, 0, 3, Tg);
                check("trispectrum", Tg, N * N * N * 2);
            }
        }
        hos_oracle_bispectrum_overlap(x, n, L, N, 0, 1, 4, 2, B);
        hos_oracle_trispectrum_overlap(x, n, L, N, 0, 1, 4, 3, Tg);
        hos_oracle_cumulant_overlap(x, n, L, 3, 1, 4, 1, c3);
        hos_oracle_cumulant_overlap(x, n, L, 4, 0, 4, 1, c4);
        double* G2 = vec(N * N * 2, 21 + k);
        double* G3 = vec(N * N * N * 2, 31 + k);
        double* dx = vec(n, 0);
        hos_oracle_bispectrum_grad(x, n, L, N, 0, 1, G2, dx);
        check("bispectrum_grad", dx, n);
        hos_oracle_grad_lag(G2, L, N, 2, c3);
        int64_t js[3] = {0, n - 1, n / 2};
        double dy[3];
        hos_oracle_dy_at(y, n, L, c3, js, 3, dy);
        check("dy_at", dy, 3);
        hos_oracle_trispectrum_grad(x, n, L, N, 2, 1, G3, dx);
        check("trispectrum_grad", dx, n);
        hos_oracle_grad_lag4(G3, L, N, 0, c4);
        double* dc2 = vec(2 * T + 1, 0);
        hos_oracle_grad_c2(c4, c2, L, dc2);
        hos_oracle_dy4_at(y, n, L, c4, dc2, js, 3, dy);
        check("dy4_at", dy, 3);
        (void)hos_oracle_parzen(L, L);
        (void)hos_oracle_window2(-L, L, L, 1);
        (void)hos_oracle_window3(-L, 0, L, L, 2);
        free(x); free(y); free(c2); free(c3); free(rows); free(c4); free(B); free(Tg);
        free(G2); free(G3); free(dx); free(dc2);
    }
    /* the direct method: parts of M = 8 with and without overlap, box sizes 1..M */
    {
        double* x = vec(29, 41);
        double* out = vec(8 * 8 * 2, 0);
        for (int64_t M3 = 1; M3 <= 8; M3 += 3) {
            hos_oracle_bispectrum_direct(x, 29, 8, M3, 0, 1, out);
            hos_oracle_bispectrum_direct(x, 29, 8, M3, 5, 0, out);
            check("direct", out, 8 * 8 * 2);
        }
        free(x);
        free(out);
    }
    return bad;
}
