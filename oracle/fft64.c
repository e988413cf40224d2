/*
 * FP64 CPU oracle for the 3D real-to-complex FFT and its complex-to-real
 * inverse (Chatterjee, Verma & Chaudhuri, "Transpose-free Fast Fourier
 * Transform for Turbulence Simulation", arXiv:1406.5597).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the GPU library is checked against.  Nothing in the product
 * path may link, load or call it; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark do.  It shares no code, header, table or
 * constant with the CUDA path.
 *
 * What it computes (Sec. 2): a real n0 x n1 x n2 array is transformed to the
 * non-redundant complex half n0 x n1 x (n2/2+1) ("r2c", forward; n2/2 rounded
 * down for odd n2), and back
 * ("c2r", inverse).  The paper fixes neither sign nor scaling; the reading
 * used here is the FFTW convention (the paper's transforms are FFTW's, Sec. 3):
 *
 *   X[k0,k1,k2] = sum_j x[j0,j1,j2] exp(-2 pi i (k0 j0/n0 + k1 j1/n1 + k2 j2/n2))
 *   y[j]        = sum_{k2=0}^{n2/2} c_k2 Re( sum_{k0,k1} Y[k] exp(+2 pi i (...)) )
 *                 with c_k2 = 1 at k2 = 0 and (even n2) at k2 = n2/2, else 2;
 *                 unnormalised.
 *
 * The forward transform follows the three steps of Sec. 2.1 in order: a 2D
 * transform of every n0-plane (here: axis n2, then axis n1) followed by the
 * 1D transform along n0.  The inverse runs the same steps in reverse order
 * (Sec. 2.1, last sentence): n0, then n1, then the real synthesis along n2.
 * On one processor the transpose/exchange of step 2 is the identity, so it
 * does not appear.  Deliberately, the n2 axis uses a full-length complex FFT
 * of the real row (not the half-length packing trick the GPU uses), so the
 * two implementations are structurally different.
 *
 * The 1D building block is a plain recursive mixed-radix decimation-in-time
 * FFT: a length-n transform with smallest prime factor p is p transforms of
 * length n/p on the decimated inputs, combined by a direct p-point sum with
 * twiddles W_n^{r k}.  Lengths whose remaining factor is a prime larger than
 * 5 fall back to the direct O(n^2) sum.  Twiddles come from one table of
 * exp(sign 2 pi i m / n), m = 0..n-1, computed with the C library's cos/sin
 * of the exactly reduced argument m/n.
 *
 * Also here: the naive O(N^2) 3D DFT and its inverse straight from the
 * definitions above (compensated summation), used to pin the fast oracle on
 * tiny shapes, and O(N)-per-value spot evaluations (single spectral bins of
 * an FP32 field, single real points of an FP32 half-spectrum) used where the
 * full oracle is too large.
 *
 * Layout everywhere: C row-major, n2 fastest, batch outermost; complex values
 * are interleaved (re, im) doubles (or floats for the *_f32 / *_c64 entry
 * points).  All functions return 0 on success, -1 on a bad argument and -2
 * on allocation failure.
 */
#include <complex.h>
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

static const double TWO_PI = 6.283185307179586476925286766559;

/* ------------------------------------------------------------------------ */
/* Twiddle table: w[m] = exp(sign * 2 pi i m / n), m in [0, n).             */
/* ------------------------------------------------------------------------ */
static cplx* make_table(int n, int sign)
{
    cplx* w = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!w) return NULL;
    for (int m = 0; m < n; ++m) {
        double a = TWO_PI * (double)m / (double)n;
        w[m] = cos(a) + (double)sign * sin(a) * I;
    }
    return w;
}

static int smallest_factor(int n)
{
    if (n % 2 == 0) return 2;
    if (n % 3 == 0) return 3;
    if (n % 5 == 0) return 5;
    return n; /* 1 or a prime (>5) or a product of primes >5: direct sum */
}

/*
 * y[k] = sum_{j<n} x[j*xs] W_n^{j k}, with W_n^m = w[(m mod n) * ws]
 * (w is the table of the top-level length; ws = top_n / n).
 * y must not alias x.  scratch holds at least n entries.
 */
static void fft_rec(const cplx* x, size_t xs, cplx* y, int n,
                    const cplx* w, size_t ws, cplx* scratch)
{
    if (n == 1) { y[0] = x[0]; return; }
    int p = smallest_factor(n);
    if (p == n) { /* direct DFT */
        for (int k = 0; k < n; ++k) {
            cplx s = 0;
            for (int j = 0; j < n; ++j)
                s += x[(size_t)j * xs] * w[(size_t)(((long long)j * k) % n) * ws];
            y[k] = s;
        }
        return;
    }
    int m = n / p;
    /* p sub-transforms of length m on x[r], x[r+p], ... stored at y[r*m..] */
    for (int r = 0; r < p; ++r)
        fft_rec(x + (size_t)r * xs, xs * (size_t)p, y + (size_t)r * m, m,
                w, ws * (size_t)p, scratch);
    /* combine: X[k + q m] = sum_r W_n^{r (k + q m)} Y_r[k] */
    for (int k = 0; k < m; ++k) {
        cplx in[5];
        for (int r = 0; r < p; ++r) in[r] = y[(size_t)r * m + k];
        for (int q = 0; q < p; ++q) {
            int kk = k + q * m;
            cplx s = 0;
            for (int r = 0; r < p; ++r)
                s += in[r] * w[(size_t)(((long long)r * kk) % n) * ws];
            scratch[kk] = s;
        }
    }
    memcpy(y, scratch, sizeof(cplx) * (size_t)n);
}

/* One line: out[k] = sum_j in[j] W^{jk}; in/out strided (complex elements). */
static void line_fft(const cplx* in, size_t is, cplx* out, size_t os, int n,
                     const cplx* w, cplx* buf /* 3n */)
{
    cplx* a = buf;          /* gathered input */
    cplx* b = buf + n;      /* result */
    cplx* s = buf + 2 * n;  /* recursion scratch */
    for (int j = 0; j < n; ++j) a[j] = in[(size_t)j * is];
    fft_rec(a, 1, b, n, w, 1, s);
    for (int k = 0; k < n; ++k) out[(size_t)k * os] = b[k];
}

int oracle_fft1d(const double* x, double* y, int n, int sign)
{
    if (n < 1 || (sign != 1 && sign != -1) || !x || !y) return -1;
    cplx* w = make_table(n, sign);
    cplx* buf = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
    if (!w || !buf) { free(w); free(buf); return -2; }
    line_fft((const cplx*)x, 1, (cplx*)y, 1, n, w, buf);
    free(w); free(buf);
    return 0;
}

/*
 * In-place 1D transform along one axis of a complex volume.  The volume is
 * viewed as [outer][n][inner]: element (o, j, i) sits at o*n*inner + j*inner + i.
 * Each (o, i) line is independent; lines are shared out across threads, and
 * the order of the arithmetic inside a line does not depend on the thread count.
 */
static int axis_fft(cplx* v, size_t outer, int n, size_t inner, int sign)
{
    cplx* w = make_table(n, sign);
    if (!w) return -2;
    long long lines = (long long)(outer * inner);
    int err = 0;
#pragma omp parallel
    {
        cplx* buf = (cplx*)malloc(sizeof(cplx) * 3 * (size_t)n);
        if (!buf) {
#pragma omp atomic write
            err = -2;
        } else {
#pragma omp for schedule(static)
            for (long long l = 0; l < lines; ++l) {
                size_t o = (size_t)l / inner, i = (size_t)l % inner;
                cplx* base = v + o * (size_t)n * inner + i;
                line_fft(base, inner, base, inner, n, w, buf);
            }
            free(buf);
        }
    }
    free(w);
    return err;
}

/* Forward r2c (Sec. 2, Sec. 2.1 steps 1 and 3). x: batch*n0*n1*n2 doubles;
 * X: batch*n0*n1*(n2/2+1) interleaved complex. */
int oracle_r2c3d(const double* x, double* Xout, int n0, int n1, int n2, int batch)
{
    if (!x || !Xout || n0 < 1 || n1 < 1 || n2 < 2 || batch < 1) return -1;
    const int H = n2 / 2 + 1;
    const size_t rows = (size_t)batch * n0 * n1;
    cplx* X = (cplx*)Xout;
    /* Step 1a: every real row -> full complex FFT of length n2, keep k2 <= n2/2. */
    cplx* w = make_table(n2, -1);
    if (!w) return -2;
    int err = 0;
#pragma omp parallel
    {
        cplx* buf = (cplx*)malloc(sizeof(cplx) * 4 * (size_t)n2);
        if (!buf) {
#pragma omp atomic write
            err = -2;
        } else {
            cplx* row = buf + 3 * n2;
#pragma omp for schedule(static)
            for (long long r = 0; r < (long long)rows; ++r) {
                const double* xr = x + (size_t)r * n2;
                for (int j = 0; j < n2; ++j) row[j] = xr[j];
                line_fft(row, 1, row, 1, n2, w, buf);
                cplx* Xr = X + (size_t)r * H;
                for (int k = 0; k < H; ++k) Xr[k] = row[k];
            }
            free(buf);
        }
    }
    free(w);
    if (err) return err;
    /* Step 1b: axis n1 (per plane, per k2). */
    if ((err = axis_fft(X, (size_t)batch * n0, n1, (size_t)H, -1))) return err;
    /* Step 3: axis n0 (per (k1, k2) column). */
    return axis_fft(X, (size_t)batch, n0, (size_t)n1 * H, -1);
}

/* Inverse c2r: the forward steps in reverse order (Sec. 2.1).  Y is not
 * modified (the oracle works on a copy). */
int oracle_c2r3d(const double* Yin, double* y, int n0, int n1, int n2, int batch)
{
    if (!Yin || !y || n0 < 1 || n1 < 1 || n2 < 2 || batch < 1) return -1;
    const int H = n2 / 2 + 1;
    const size_t rows = (size_t)batch * n0 * n1;
    cplx* A = (cplx*)malloc(sizeof(cplx) * rows * H);
    if (!A) return -2;
    memcpy(A, Yin, sizeof(cplx) * rows * H);
    int err;
    if ((err = axis_fft(A, (size_t)batch, n0, (size_t)n1 * H, +1))) { free(A); return err; }
    if ((err = axis_fft(A, (size_t)batch * n0, n1, (size_t)H, +1))) { free(A); return err; }
    /* Real synthesis along n2: y[j2] = sum_k2 c_k2 Re(A[k2] e^{+2 pi i k2 j2/n2}),
     * done as the inverse complex FFT of the Hermitian extension Z of the row:
     * Z[0] = Re A[0], Z[k] = A[k], Z[n2-k] = conj A[k] for 1 <= k <= (n2-1)/2,
     * and for even n2 the Nyquist bin Z[n2/2] = Re A[n2/2]. */
    cplx* w = make_table(n2, +1);
    if (!w) { free(A); return -2; }
    err = 0;
#pragma omp parallel
    {
        cplx* buf = (cplx*)malloc(sizeof(cplx) * 4 * (size_t)n2);
        if (!buf) {
#pragma omp atomic write
            err = -2;
        } else {
            cplx* row = buf + 3 * n2;
#pragma omp for schedule(static)
            for (long long r = 0; r < (long long)rows; ++r) {
                const cplx* Ar = A + (size_t)r * H;
                row[0] = creal(Ar[0]);
                if ((n2 & 1) == 0) row[n2 / 2] = creal(Ar[n2 / 2]);
                for (int k = 1; k <= (n2 - 1) / 2; ++k) {
                    row[k] = Ar[k];
                    row[n2 - k] = conj(Ar[k]);
                }
                line_fft(row, 1, row, 1, n2, w, buf);
                double* yr = y + (size_t)r * n2;
                for (int j = 0; j < n2; ++j) yr[j] = creal(row[j]);
            }
            free(buf);
        }
    }
    free(w);
    free(A);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Naive definitions (pins for the fast oracle on tiny shapes).             */
/* ------------------------------------------------------------------------ */

/* exp(sign 2 pi i (a0/n0 + a1/n1 + a2/n2)) with each a_i already reduced mod n_i.
 * The phase is formed as one exactly reduced fraction of the common period. */
static cplx phase3(long long a0, long long a1, long long a2, int n0, int n1, int n2, int sign)
{
    /* fraction f = a0/n0 + a1/n1 + a2/n2 reduced to [0,1) over the lcm-free
     * denominator n0*n1*n2 (exact in 64-bit for the tiny shapes used here) */
    long long D = (long long)n0 * n1 * n2;
    long long num = a0 * (long long)n1 * n2 + a1 * (long long)n0 * n2 + a2 * (long long)n0 * n1;
    num %= D;
    double a = TWO_PI * (double)num / (double)D;
    return cos(a) + (double)sign * sin(a) * I;
}

/* Compensated (Kahan) complex accumulator. */
typedef struct { cplx s, c; } kahan_c;
static void kahan_add(kahan_c* k, cplx v)
{
    cplx y = v - k->c;
    cplx t = k->s + y;
    k->c = (t - k->s) - y;
    k->s = t;
}

/* X[k] for every k in the half spectrum, straight from the definition. */
int oracle_r2c3d_naive(const double* x, double* Xout, int n0, int n1, int n2)
{
    if (!x || !Xout || n0 < 1 || n1 < 1 || n2 < 2) return -1;
    if ((long long)n0 * n1 * n2 > 8192) return -1; /* O(N^2): tiny shapes only */
    const int H = n2 / 2 + 1;
    cplx* X = (cplx*)Xout;
    for (int k0 = 0; k0 < n0; ++k0)
    for (int k1 = 0; k1 < n1; ++k1)
    for (int k2 = 0; k2 < H; ++k2) {
        kahan_c acc = {0, 0};
        for (int j0 = 0; j0 < n0; ++j0)
        for (int j1 = 0; j1 < n1; ++j1)
        for (int j2 = 0; j2 < n2; ++j2) {
            double v = x[((size_t)j0 * n1 + j1) * n2 + j2];
            kahan_add(&acc, v * phase3((long long)k0 * j0 % n0, (long long)k1 * j1 % n1,
                                       (long long)k2 * j2 % n2, n0, n1, n2, -1));
        }
        X[((size_t)k0 * n1 + k1) * H + k2] = acc.s;
    }
    return 0;
}

/* y[j] = sum_{k2<=n2/2} c_k2 Re(sum_{k0,k1} Y[k] exp(+...)), straight from the definition. */
int oracle_c2r3d_naive(const double* Yin, double* y, int n0, int n1, int n2)
{
    if (!Yin || !y || n0 < 1 || n1 < 1 || n2 < 2) return -1;
    if ((long long)n0 * n1 * n2 > 8192) return -1;
    const int H = n2 / 2 + 1;
    const cplx* Y = (const cplx*)Yin;
    for (int j0 = 0; j0 < n0; ++j0)
    for (int j1 = 0; j1 < n1; ++j1)
    for (int j2 = 0; j2 < n2; ++j2) {
        double s = 0.0, c = 0.0; /* Kahan on the real sum */
        for (int k0 = 0; k0 < n0; ++k0)
        for (int k1 = 0; k1 < n1; ++k1)
        for (int k2 = 0; k2 < H; ++k2) {
            double ck = (k2 == 0 || 2 * k2 == n2) ? 1.0 : 2.0;
            cplx t = Y[((size_t)k0 * n1 + k1) * H + k2] *
                     phase3((long long)k0 * j0 % n0, (long long)k1 * j1 % n1,
                            (long long)k2 * j2 % n2, n0, n1, n2, +1);
            double v = ck * creal(t) - c;
            double u = s + v;
            c = (u - s) - v;
            s = u;
        }
        y[((size_t)j0 * n1 + j1) * n2 + j2] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Spot evaluations for large shapes (O(N) per value, FP64 arithmetic).     */
/* ------------------------------------------------------------------------ */

/* For nb bins k = (k[3b], k[3b+1], k[3b+2]) (0 <= k2 <= n2/2), the exact
 * forward transform X[k] of the FP32 field x (one batch entry), promoted to
 * FP64.  Separable evaluation: for every row (j0, j1) the n2-sum, then the
 * n1-sum per plane, then the n0-sum; same value as the definition. */
int oracle_r2c_bins_f32(const float* x, int n0, int n1, int n2,
                        const int* k, int nb, double* out)
{
    if (!x || !k || !out || n0 < 1 || n1 < 1 || n2 < 2 || nb < 0) return -1;
    for (int b = 0; b < nb; ++b)
        if (k[3*b] < 0 || k[3*b] >= n0 || k[3*b+1] < 0 || k[3*b+1] >= n1 ||
            k[3*b+2] < 0 || k[3*b+2] > n2 / 2) return -1;
    cplx* w0 = make_table(n0, -1);
    cplx* w1 = make_table(n1, -1);
    cplx* w2 = make_table(n2, -1);
    if (!w0 || !w1 || !w2) { free(w0); free(w1); free(w2); return -2; }
    for (int b = 0; b < nb; ++b) {
        const int k0 = k[3*b], k1 = k[3*b+1], k2 = k[3*b+2];
        double re = 0.0, im = 0.0;
#pragma omp parallel for schedule(static) reduction(+:re,im)
        for (int j0 = 0; j0 < n0; ++j0) {
            cplx plane = 0;
            for (int j1 = 0; j1 < n1; ++j1) {
                const float* xr = x + ((size_t)j0 * n1 + j1) * n2;
                cplx row = 0;
                for (int j2 = 0; j2 < n2; ++j2)
                    row += (double)xr[j2] * w2[(size_t)(((long long)k2 * j2) % n2)];
                plane += row * w1[(size_t)(((long long)k1 * j1) % n1)];
            }
            cplx t = plane * w0[(size_t)(((long long)k0 * j0) % n0)];
            re += creal(t);
            im += cimag(t);
        }
        out[2*b] = re;
        out[2*b+1] = im;
    }
    free(w0); free(w1); free(w2);
    return 0;
}

/* For np points j = (j[3p], j[3p+1], j[3p+2]), the exact inverse c2r value
 * y[j] of the complex64 half-spectrum Y (one batch entry), in FP64. */
int oracle_c2r_points_c64(const float* Yf, int n0, int n1, int n2,
                          const int* j, int np, double* out)
{
    if (!Yf || !j || !out || n0 < 1 || n1 < 1 || n2 < 2 || np < 0) return -1;
    for (int p = 0; p < np; ++p)
        if (j[3*p] < 0 || j[3*p] >= n0 || j[3*p+1] < 0 || j[3*p+1] >= n1 ||
            j[3*p+2] < 0 || j[3*p+2] >= n2) return -1;
    const int H = n2 / 2 + 1;
    cplx* w0 = make_table(n0, +1);
    cplx* w1 = make_table(n1, +1);
    cplx* w2 = make_table(n2, +1);
    if (!w0 || !w1 || !w2) { free(w0); free(w1); free(w2); return -2; }
    for (int p = 0; p < np; ++p) {
        const int j0 = j[3*p], j1 = j[3*p+1], j2 = j[3*p+2];
        double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+:acc)
        for (int k0 = 0; k0 < n0; ++k0) {
            cplx e0 = w0[(size_t)(((long long)k0 * j0) % n0)];
            double part = 0.0;
            for (int k1 = 0; k1 < n1; ++k1) {
                const float* Yr = Yf + 2 * (((size_t)k0 * n1 + k1) * H);
                cplx row = 0;
                for (int k2 = 0; k2 < H; ++k2) {
                    double ck = (k2 == 0 || 2 * k2 == n2) ? 1.0 : 2.0;
                    cplx v = (double)Yr[2*k2] + (double)Yr[2*k2+1] * I;
                    row += ck * v * w2[(size_t)(((long long)k2 * j2) % n2)];
                }
                part += creal(row * w1[(size_t)(((long long)k1 * j1) % n1)] * e0);
            }
            acc += part;
        }
        out[p] = acc;
    }
    free(w0); free(w1); free(w2);
    return 0;
}

/* Threads the oracle's parallel loops use (1 when built without OpenMP). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
