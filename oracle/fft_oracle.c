/*
 * FP64 CPU oracle for the 2D radix-2 decimation-in-time FFT of an image.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA library: it is a plain, slow, obviously-correct restatement of
 * the paper "Research on the fast Fourier transform of image based on GPU"
 * (Shen, Song, Wu, Geng, Wang), written in the paper's order and notation.
 *
 * Data layout: complex numbers are interleaved doubles (re, im), i.e. the
 * memory layout of numpy complex128.  Strides are counted in complex
 * elements.
 *
 * Sign convention (the paper never defines the sign of W_N, Section 2 eq. 1):
 *   W_N = exp(sign * 2*pi*i / N), sign = -1 forward, +1 inverse.
 * Inverse normalisation (the paper only says the inverse is "easily
 * implemented", Section 5): forward unscaled, inverse multiplied by
 * 1/(rows*cols) after both axes.
 *
 * Parity status: every entry point below is pinned by the "not gpu" tests
 * (direct DFT brute force, closed forms, invariants, an independent library
 * FFT and partial-stage decimation identities).
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_OOM 2

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

/* log2 of a power of two n >= 1, or -1 if n is not a power of two. */
static int ilog2_pow2(long n)
{
    int L = 0;
    if (n < 1)
        return -1;
    while ((1L << L) < n)
        L++;
    return ((1L << L) == n) ? L : -1;
}

/*
 * Section 3.2 ("descending" module): the scramble index table.  rev[i] is i
 * with its L low bits written in reverse order.  The paper precomputes these
 * indexes once per N into an auxiliary texture; the oracle keeps the same
 * explicit table.
 */
void oracle_bitrev_table(int L, long *rev)
{
    long n = 1L << L;
    for (long i = 0; i < n; i++) {
        long r = 0;
        for (int b = 0; b < L; b++)
            if (i & (1L << b))
                r |= 1L << (L - 1 - b);
        rev[i] = r;
    }
}

/*
 * Rotation factor W_M^j = exp(sign*2*pi*i*j/M) (eq. 1 notation).  Values at
 * multiples of a quarter turn are written exactly, so that transforms whose
 * only twiddles are 1 and -i are exact on integer input.
 */
static void oracle_twiddle(long j, long M, int sign, double *wr, double *wi)
{
    j %= M;
    if (j < 0)
        j += M;
    if ((4 * j) % M == 0) {
        long q = (4 * j) / M;
        static const double cq[4] = {1.0, 0.0, -1.0, 0.0};
        static const double sq[4] = {0.0, 1.0, 0.0, -1.0};
        *wr = cq[q];
        *wi = sign * sq[q];
        return;
    }
    double ang = 2.0 * ORACLE_PI * (double)j / (double)M;
    *wr = cos(ang);
    *wi = sign * sin(ang);
}

/*
 * One line of n = 2^L points, first element at z, element stride `stride`.
 *
 *  1. Scramble (Section 3.2): y[p] = x[rev(p)], a gather through the explicit
 *     index table, so that the stages can run in place.
 *  2. Butterfly stages s = 1..nstages (Section 2 eqs. 2-3, Section 3.1 eq. 4):
 *     in every block of 2^s consecutive positions, for j < 2^(s-1),
 *        X(j)           = Xe(j) + W_{2^s}^j * Xo(j)
 *        X(j + 2^(s-1)) = Xe(j) - W_{2^s}^j * Xo(j)
 *     where Xe is the first half of the block (the DFT of the even-indexed
 *     subsequence) and Xo the second half (the DFT of the odd-indexed one).
 *
 * With nstages = L this is the full DFT of eq. 1 in natural output order.
 * With nstages < L the line is left after that many stages (a debug view
 * used to check partial execution); nstages = 0 is the scramble alone.
 */
int oracle_fft_line(double *z, long n, long stride, int sign, int nstages)
{
    int L = ilog2_pow2(n);
    if (L < 0 || nstages < 0 || nstages > L || (sign != 1 && sign != -1))
        return ORACLE_ERR_ARG;
    long *rev = (long *)malloc(sizeof(long) * (size_t)n);
    double *y = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!rev || !y) {
        free(rev);
        free(y);
        return ORACLE_ERR_OOM;
    }
    oracle_bitrev_table(L, rev);

    /* scramble: gather the line in bit-reversed order */
    for (long p = 0; p < n; p++) {
        y[2 * p] = z[2 * rev[p] * stride];
        y[2 * p + 1] = z[2 * rev[p] * stride + 1];
    }

    /* butterfly stages */
    for (int s = 1; s <= nstages; s++) {
        long span = 1L << s;       /* 2^s: size of the DFTs built at stage s */
        long half = span >> 1;     /* 2^(s-1): size of Xe and Xo           */
        for (long blk = 0; blk < n; blk += span) {
            for (long j = 0; j < half; j++) {
                double wr, wi;
                oracle_twiddle(j, span, sign, &wr, &wi);
                double *e = &y[2 * (blk + j)];
                double *o = &y[2 * (blk + j + half)];
                double tr = wr * o[0] - wi * o[1];
                double ti = wr * o[1] + wi * o[0];
                double er = e[0], ei = e[1];
                e[0] = er + tr;
                e[1] = ei + ti;
                o[0] = er - tr;
                o[1] = ei - ti;
            }
        }
    }

    for (long p = 0; p < n; p++) {
        z[2 * p * stride] = y[2 * p];
        z[2 * p * stride + 1] = y[2 * p + 1];
    }
    free(rev);
    free(y);
    return ORACLE_OK;
}

/* `count` lines of n points; line l starts at z + l*line_stride. */
int oracle_fft_lines(double *z, long n, long count, long elem_stride,
                     long line_stride, int sign, int nstages)
{
    for (long l = 0; l < count; l++) {
        int rc = oracle_fft_line(z + 2 * l * line_stride, n, elem_stride,
                                 sign, nstages);
        if (rc != ORACLE_OK)
            return rc;
    }
    return ORACLE_OK;
}

/* Multiply `count` complex values by a real factor. */
void oracle_scale(double *z, long count, double f)
{
    for (long i = 0; i < 2 * count; i++)
        z[i] *= f;
}

/*
 * Run `count` lines over `nthreads` POSIX threads: each thread takes a
 * contiguous chunk of lines and runs the same single-line code on it.  Lines
 * are independent (Section 2), so the split changes no arithmetic.
 */
struct oracle_lines_job {
    double *z;
    long n, count, elem_stride, line_stride;
    int sign, nstages, rc;
};

static void *oracle_lines_worker(void *arg)
{
    struct oracle_lines_job *j = (struct oracle_lines_job *)arg;
    j->rc = oracle_fft_lines(j->z, j->n, j->count, j->elem_stride,
                             j->line_stride, j->sign, j->nstages);
    return NULL;
}

static int oracle_lines_threaded(double *z, long n, long count, long elem_stride,
                                 long line_stride, int sign, int nstages,
                                 int nthreads)
{
    if (nthreads > count)
        nthreads = (int)count;
    if (nthreads <= 1)
        return oracle_fft_lines(z, n, count, elem_stride, line_stride, sign,
                                nstages);
    struct oracle_lines_job *jobs = (struct oracle_lines_job *)calloc(
        (size_t)nthreads, sizeof(struct oracle_lines_job));
    pthread_t *tid = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    int *started = (int *)calloc((size_t)nthreads, sizeof(int));
    if (!jobs || !tid || !started) {
        free(jobs);
        free(tid);
        free(started);
        return ORACLE_ERR_OOM;
    }
    long first = 0;
    for (int t = 0; t < nthreads; t++) {
        long cnt = count / nthreads + (t < count % nthreads ? 1 : 0);
        jobs[t].z = z + 2 * first * line_stride;
        jobs[t].n = n;
        jobs[t].count = cnt;
        jobs[t].elem_stride = elem_stride;
        jobs[t].line_stride = line_stride;
        jobs[t].sign = sign;
        jobs[t].nstages = nstages;
        jobs[t].rc = ORACLE_OK;
        first += cnt;
        if (pthread_create(&tid[t], NULL, oracle_lines_worker, &jobs[t]) == 0)
            started[t] = 1;
        else
            oracle_lines_worker(&jobs[t]); /* no thread: run it here */
    }
    int rc = ORACLE_OK;
    for (int t = 0; t < nthreads; t++) {
        if (started[t])
            pthread_join(tid[t], NULL);
        if (rc == ORACLE_OK && jobs[t].rc != ORACLE_OK)
            rc = jobs[t].rc;
    }
    free(jobs);
    free(tid);
    free(started);
    return rc;
}

/*
 * 2D transform of a rows x cols row-major image (Section 2: the 2D DFT is
 * separable; the paper allows either order, this oracle does rows first,
 * then columns, each axis scrambled along itself before its stages).
 * row_stages / col_stages < 0 mean "all stages".  For the inverse
 * (sign = +1) with do_scale != 0 the result is multiplied by 1/(rows*cols).
 * nthreads >= 1 host threads share the lines of each axis.
 */
int oracle_fft2d(double *z, long rows, long cols, int sign, int row_stages,
                 int col_stages, int do_scale, int nthreads)
{
    int Lr = ilog2_pow2(rows), Lc = ilog2_pow2(cols);
    if (Lr < 0 || Lc < 0)
        return ORACLE_ERR_ARG;
    if (row_stages < 0)
        row_stages = Lc;
    if (col_stages < 0)
        col_stages = Lr;
    /* every row: cols points, elements adjacent, rows cols apart */
    int rc = oracle_lines_threaded(z, cols, rows, 1, cols, sign, row_stages,
                                   nthreads);
    if (rc != ORACLE_OK)
        return rc;
    /* every column: rows points, elements cols apart, columns adjacent */
    rc = oracle_lines_threaded(z, rows, cols, cols, 1, sign, col_stages,
                               nthreads);
    if (rc != ORACLE_OK)
        return rc;
    if (sign == 1 && do_scale)
        oracle_scale(z, rows * cols, 1.0 / ((double)rows * (double)cols));
    return ORACLE_OK;
}

/*
 * Gaussian low-pass of an unshifted spectrum (the filter step of the image
 * filtering workload; not part of the paper's method, which only names image
 * filtering as a use, Section 1):
 *   Z[k][l] *= exp(-d_k^2 / (2 sr^2)) * exp(-d_l^2 / (2 sc^2)),
 *   d_k = min(k, rows - k), d_l = min(l, cols - l).
 */
void oracle_gaussian_lowpass(double *z, long rows, long cols, double sr, double sc)
{
    for (long k = 0; k < rows; k++) {
        const double dk = (double)(k < rows - k ? k : rows - k);
        const double hk = exp(-dk * dk / (2.0 * sr * sr));
        for (long l = 0; l < cols; l++) {
            const double dl = (double)(l < cols - l ? l : cols - l);
            const double h = hk * exp(-dl * dl / (2.0 * sc * sc));
            z[2 * (k * cols + l)] *= h;
            z[2 * (k * cols + l) + 1] *= h;
        }
    }
}

/*
 * Section 2 eq. 1, evaluated directly in O(n^2): X(k) = sum_n x(n) W_n^{nk}.
 * The exponent n*k is reduced modulo n before the rotation factor is
 * formed.  Any n >= 1 is accepted (no power-of-two requirement).
 */
int oracle_dft_line(const double *x, long in_stride, double *X,
                    long out_stride, long n, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1))
        return ORACLE_ERR_ARG;
    for (long k = 0; k < n; k++) {
        double sr = 0.0, si = 0.0;
        for (long m = 0; m < n; m++) {
            double wr, wi;
            oracle_twiddle((m * k) % n, n, sign, &wr, &wi);
            double ar = x[2 * m * in_stride], ai = x[2 * m * in_stride + 1];
            sr += wr * ar - wi * ai;
            si += wr * ai + wi * ar;
        }
        X[2 * k * out_stride] = sr;
        X[2 * k * out_stride + 1] = si;
    }
    return ORACLE_OK;
}

/*
 * The 2D definition written out as one double sum (no separation):
 *   X[k][l] = sum_m sum_n x[m][n] W_rows^{k m} W_cols^{l n}.
 * O((rows*cols)^2): tiny inputs only.
 */
int oracle_dft2d(const double *x, double *X, long rows, long cols, int sign)
{
    if (rows < 1 || cols < 1 || (sign != 1 && sign != -1))
        return ORACLE_ERR_ARG;
    for (long k = 0; k < rows; k++) {
        for (long l = 0; l < cols; l++) {
            double sr = 0.0, si = 0.0;
            for (long m = 0; m < rows; m++) {
                double ur, ui;
                oracle_twiddle((k * m) % rows, rows, sign, &ur, &ui);
                for (long c = 0; c < cols; c++) {
                    double vr, vi;
                    oracle_twiddle((l * c) % cols, cols, sign, &vr, &vi);
                    double wr = ur * vr - ui * vi;
                    double wi = ur * vi + ui * vr;
                    const double *a = &x[2 * (m * cols + c)];
                    sr += wr * a[0] - wi * a[1];
                    si += wr * a[1] + wi * a[0];
                }
            }
            X[2 * (k * cols + l)] = sr;
            X[2 * (k * cols + l) + 1] = si;
        }
    }
    return ORACLE_OK;
}

/*
 * The discrete cosine transform, one of the "similar transforms" Section 5
 * says the method extends to (the paper gives no algorithm for it; the
 * oracle evaluates the definitions directly, with no FFT):
 *
 *   forward (DCT-II):  X[k] = sum_{j<n} x[j] cos(pi k (2j+1) / (2n)),
 *   inverse (DCT-III): x[j] = (1/n) (X[0] + 2 sum_{1<=k<n} X[k] cos(pi k (2j+1) / (2n))),
 *
 * so that the inverse undoes the forward.  Real data, doubles.  The cosine
 * of pi*m/(2n) is taken from a table over m < 4n; the integer phase
 * k*(2j+1) is reduced modulo 4n first, and the quarter turns are exact.
 */
static double *oracle_cos_table(long n)
{
    double *c = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    if (!c)
        return NULL;
    for (long m = 0; m < 4 * n; m++) {
        if (m == 0)
            c[m] = 1.0;
        else if (m == n || m == 3 * n)
            c[m] = 0.0;
        else if (m == 2 * n)
            c[m] = -1.0;
        else
            c[m] = cos(ORACLE_PI * (double)m / (2.0 * (double)n));
    }
    return c;
}

static void oracle_dct_line_tab(const double *x, long in_stride, double *X, long out_stride,
                                long n, int inverse, const double *ctab)
{
    for (long a = 0; a < n; a++) {
        double s = 0.0;
        for (long b = 0; b < n; b++) {
            /* forward: output k = a, input j = b; inverse: output j = a, input k = b */
            long k = inverse ? b : a, j = inverse ? a : b;
            double c = ctab[(k * (2 * j + 1)) % (4 * n)];
            double w = inverse ? (b == 0 ? 1.0 : 2.0) : 1.0;
            s += w * x[b * in_stride] * c;
        }
        X[a * out_stride] = inverse ? s / (double)n : s;
    }
}

int oracle_dct_line(const double *x, long in_stride, double *X, long out_stride, long n,
                    int inverse)
{
    if (n < 1)
        return ORACLE_ERR_ARG;
    double *ctab = oracle_cos_table(n);
    if (!ctab)
        return ORACLE_ERR_OOM;
    oracle_dct_line_tab(x, in_stride, X, out_stride, n, inverse, ctab);
    free(ctab);
    return ORACLE_OK;
}

/*
 * 2D transform of a rows x cols real image z (row-major), in place: every
 * row, then every column, each by the definition above.  Any sizes >= 1.
 */
int oracle_dct2d(double *z, long rows, long cols, int inverse)
{
    if (rows < 1 || cols < 1)
        return ORACLE_ERR_ARG;
    long nmax = rows > cols ? rows : cols;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)nmax);
    double *crow = oracle_cos_table(cols), *ccol = oracle_cos_table(rows);
    if (!tmp || !crow || !ccol) {
        free(tmp);
        free(crow);
        free(ccol);
        return ORACLE_ERR_OOM;
    }
    for (long r = 0; r < rows; r++) {
        oracle_dct_line_tab(z + r * cols, 1, tmp, 1, cols, inverse, crow);
        memcpy(z + r * cols, tmp, sizeof(double) * (size_t)cols);
    }
    for (long c = 0; c < cols; c++) {
        oracle_dct_line_tab(z + c, cols, tmp, 1, rows, inverse, ccol);
        for (long r = 0; r < rows; r++)
            z[r * cols + c] = tmp[r];
    }
    free(tmp);
    free(crow);
    free(ccol);
    return ORACLE_OK;
}

/*
 * One output of the forward 2D DCT as the double sum of its definition (no
 * separation): X[k][l] = sum_m sum_n x[m][n] cos(pi k (2m+1)/(2 rows))
 * cos(pi l (2n+1)/(2 cols)).  O(rows*cols) per output.
 */
double oracle_dct2d_at(const double *x, long rows, long cols, long k, long l)
{
    double s = 0.0;
    for (long m = 0; m < rows; m++) {
        long pm = (k * (2 * m + 1)) % (4 * rows);
        double cm = cos(ORACLE_PI * (double)pm / (2.0 * (double)rows));
        for (long n = 0; n < cols; n++) {
            long pn = (l * (2 * n + 1)) % (4 * cols);
            s += x[m * cols + n] * cm * cos(ORACLE_PI * (double)pn / (2.0 * (double)cols));
        }
    }
    return s;
}
