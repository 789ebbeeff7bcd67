/*
 * Memory- and undefined-behaviour check of the FP64 oracle (test
 * infrastructure only): tests/test_oracle_sanitizers.py compiles this driver
 * together with fft_oracle.c under AddressSanitizer and
 * UndefinedBehaviorSanitizer and runs it.  Every entry point of the oracle
 * is driven over small and degenerate shapes (sides of 1, lines with
 * strides, partial stages, threaded lines, the direct DFT); each radix-2
 * result is compared with the direct DFT of Section 2 eq. 1 on the same
 * input, so a sanitizer report or a wrong value both end the run with a
 * non-zero exit status.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

void oracle_bitrev_table(int L, long *rev);
int oracle_fft_line(double *z, long n, long stride, int sign, int nstages);
int oracle_fft_lines(double *z, long n, long count, long elem_stride, long line_stride,
                     int sign, int nstages);
void oracle_scale(double *z, long count, double f);
int oracle_fft2d(double *z, long rows, long cols, int sign, int row_stages, int col_stages,
                 int do_scale, int nthreads);
void oracle_gaussian_lowpass(double *z, long rows, long cols, double sr, double sc);
int oracle_dft_line(const double *x, long in_stride, double *X, long out_stride, long n,
                    int sign);
int oracle_dft2d(const double *x, double *X, long rows, long cols, int sign);
int oracle_dct_line(const double *x, long in_stride, double *X, long out_stride, long n,
                    int inverse);
int oracle_dct2d(double *z, long rows, long cols, int inverse);
double oracle_dct2d_at(const double *x, long rows, long cols, long k, long l);

static int failures = 0;

/* deterministic inputs: a small linear congruential sequence in [-1, 1) */
static unsigned long long lcg_state = 12345;
static double next_value(void)
{
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(lcg_state >> 11) / 9007199254740992.0 * 2.0 - 1.0;
}

static double *random_image(long n_complex)
{
    double *z = malloc((size_t)n_complex * 2 * sizeof(double));
    for (long i = 0; i < 2 * n_complex; i++)
        z[i] = next_value();
    return z;
}

static double rel_l2(const double *a, const double *b, long n_complex)
{
    double num = 0.0, den = 0.0;
    for (long i = 0; i < 2 * n_complex; i++) {
        num += (a[i] - b[i]) * (a[i] - b[i]);
        den += b[i] * b[i];
    }
    return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

static void check(int cond, const char *what, long a, long b)
{
    if (!cond) {
        fprintf(stderr, "FAILED: %s (%ld, %ld)\n", what, a, b);
        failures++;
    }
}

int main(void)
{
    /* bit-reversal tables: a permutation of 0 .. 2^L - 1 */
    for (int L = 0; L <= 10; L++) {
        const long n = 1L << L;
        long *rev = malloc((size_t)n * sizeof(long));
        char *seen = calloc((size_t)n, 1);
        oracle_bitrev_table(L, rev);
        for (long i = 0; i < n; i++) {
            check(rev[i] >= 0 && rev[i] < n && !seen[rev[i]], "bitrev permutation", L, i);
            if (rev[i] >= 0 && rev[i] < n)
                seen[rev[i]] = 1;
        }
        free(rev);
        free(seen);
    }

    /* one line with a stride, against the direct DFT */
    for (long n = 1, L = 0; n <= 256; n *= 2, L++) {
        for (long stride = 1; stride <= 3; stride++) {
            double *z = random_image(n * stride);
            double *x = malloc((size_t)n * 2 * sizeof(double));
            double *X = malloc((size_t)n * 2 * sizeof(double));
            for (long m = 0; m < n; m++) {
                x[2 * m] = z[2 * m * stride];
                x[2 * m + 1] = z[2 * m * stride + 1];
            }
            check(oracle_fft_line(z, n, stride, -1, (int)L) == 0, "fft_line status", n, stride);
            check(oracle_dft_line(x, 1, X, 1, n, -1) == 0, "dft_line status", n, stride);
            double *got = malloc((size_t)n * 2 * sizeof(double));
            for (long m = 0; m < n; m++) {
                got[2 * m] = z[2 * m * stride];
                got[2 * m + 1] = z[2 * m * stride + 1];
            }
            check(rel_l2(got, X, n) < 1e-12, "fft_line vs dft_line", n, stride);
            free(z);
            free(x);
            free(X);
            free(got);
        }
    }

    /* 2D: every shape with sides 1 .. 32, one and four threads, forward and
     * inverse, against the direct 2D DFT */
    for (long rows = 1; rows <= 32; rows *= 2) {
        for (long cols = 1; cols <= 32; cols *= 2) {
            for (int threads = 1; threads <= 4; threads += 3) {
                for (int sign = -1; sign <= 1; sign += 2) {
                    const long n = rows * cols;
                    double *x = random_image(n);
                    double *z = malloc((size_t)n * 2 * sizeof(double));
                    double *X = malloc((size_t)n * 2 * sizeof(double));
                    memcpy(z, x, (size_t)n * 2 * sizeof(double));
                    check(oracle_fft2d(z, rows, cols, sign, -1, -1, 0, threads) == 0,
                          "fft2d status", rows, cols);
                    check(oracle_dft2d(x, X, rows, cols, sign) == 0, "dft2d status", rows, cols);
                    check(rel_l2(z, X, n) < 1e-12, "fft2d vs dft2d", rows, cols);
                    free(x);
                    free(z);
                    free(X);
                }
            }
        }
    }

    /* partial stages, the inverse scale and many lines in one call */
    {
        const long rows = 64, cols = 32, n = rows * cols;
        double *z = random_image(n);
        for (int rs = 0; rs <= 5; rs++)
            check(oracle_fft2d(z, rows, cols, -1, rs, 6 - rs, 0, 2) == 0, "partial stages", rs,
                  6 - rs);
        check(oracle_fft2d(z, rows, cols, 1, -1, -1, 1, 3) == 0, "inverse with scale", rows, cols);
        check(oracle_fft_lines(z, cols, rows, 1, cols, -1, 5) == 0, "fft_lines", rows, cols);
        oracle_scale(z, n, 0.5);
        oracle_gaussian_lowpass(z, rows, cols, rows / 8.0, cols / 8.0);
        free(z);
    }

    /* discrete cosine transform: round trip, and single outputs against the
     * separated 2D transform, sides 1 .. 16 */
    for (long rows = 1; rows <= 16; rows *= 2) {
        for (long cols = 1; cols <= 16; cols *= 2) {
            const long n = rows * cols;
            double *x = malloc((size_t)n * sizeof(double));
            double *z = malloc((size_t)n * sizeof(double));
            for (long i = 0; i < n; i++)
                x[i] = next_value();
            memcpy(z, x, (size_t)n * sizeof(double));
            check(oracle_dct2d(z, rows, cols, 0) == 0, "dct2d status", rows, cols);
            for (long k = 0; k < rows; k++)
                for (long l = 0; l < cols; l++) {
                    const double a = oracle_dct2d_at(x, rows, cols, k, l);
                    check(fabs(a - z[k * cols + l]) <= 1e-12 * (1.0 + fabs(a)), "dct2d_at", k, l);
                }
            check(oracle_dct2d(z, rows, cols, 1) == 0, "idct2d status", rows, cols);
            double err = 0.0;
            for (long i = 0; i < n; i++)
                err = fmax(err, fabs(z[i] - x[i]));
            check(err <= 1e-12, "dct round trip", rows, cols);
            double line[16], out[16];
            check(oracle_dct_line(x, 1, out, 1, cols, 0) == 0 &&
                      oracle_dct_line(out, 1, line, 1, cols, 1) == 0,
                  "dct_line status", cols, 0);
            free(x);
            free(z);
        }
    }

    /* argument errors are reported, not acted on */
    {
        double z[8] = {0};
        check(oracle_fft2d(z, 3, 2, -1, -1, -1, 0, 1) != 0, "non power of two rejected", 3, 2);
        check(oracle_fft_line(z, 0, 1, -1, -1) != 0, "empty line rejected", 0, 1);
        check(oracle_dft2d(z, z, 0, 2, -1) != 0, "empty dft rejected", 0, 2);
    }

    if (failures) {
        fprintf(stderr, "%d check(s) failed\n", failures);
        return 1;
    }
    printf("sanitizer driver: all checks passed\n");
    return 0;
}
