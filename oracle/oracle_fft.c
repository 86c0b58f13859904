/*
 * CPU FP64 reference FFT for the sp-DBA oracle.  TEST INFRASTRUCTURE ONLY:
 * nothing in the product path links or calls this file; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg do.
 *
 * What it computes: the discrete Fourier transform
 *     X[k] = sum_{n=0}^{N-1} x[n] exp(s * 2*pi*i * n*k / N),   s = -1 forward, +1 inverse,
 * with an optional 1/N on the inverse, applied one axis at a time to a
 * row-major (last axis fastest) array of interleaved (re, im) doubles.  This is
 * the transform the pseudo-spectral solvers of the paper (Methods; S3.2, S4.2,
 * S5.2) apply between real space and the transformed field.
 *
 * How: a plain recursive decimation-in-time FFT.  A length-n transform whose
 * smallest prime factor is p in {2, 3} is split into p interleaved
 * subsequences x[p*m + r], each transformed recursively, and recombined as
 *     X[k] = sum_r W_n^{r k} X_r[k mod n/p],     W_n = exp(s * 2*pi*i / n).
 * Lengths with a prime factor above 3 fall back to the O(n^2) definition.
 * Twiddles are cos/sin of 2*pi*m/n in double precision for the integer
 * m = (r*k) mod n, reduced before the multiply.  Nothing is blocked or fused.
 * A single long 1-D transform runs its top recursion levels' sub-transforms
 * as parallel tasks; that changes the schedule, not one operation.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } cplx;

static cplx cmul(cplx a, cplx b) {
    cplx r = { a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re };
    return r;
}

/* table[m] = exp(s*2*pi*i*m/n), m in [0, n) */
static cplx* make_table(long n, int sign) {
    cplx* t = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!t) return NULL;
    const double two_pi = 6.283185307179586476925286766559;
    for (long m = 0; m < n; ++m) {
        double ang = two_pi * (double)m / (double)n;
        t[m].re = cos(ang);
        t[m].im = (double)sign * sin(ang);
    }
    return t;
}

/*
 * Recombination of the p sub-transforms X_r (in out[r*q .. r*q+q-1], q = n/p):
 * X[k] = sum_r W_n^{r k} X_r[k mod q], formed in scratch and copied back to out.
 */
static void recombine(long n, long p, const cplx* tab, long ts, cplx* out, cplx* scratch) {
    long q = n / p;
    for (long k = 0; k < n; ++k) {
        cplx acc = {0.0, 0.0};
        for (long r = 0; r < p; ++r) {
            long m = (r * k) % n;
            cplx v = cmul(out[r * q + (k % q)], tab[m * ts]);
            acc.re += v.re; acc.im += v.im;
        }
        scratch[k] = acc;
    }
    memcpy(out, scratch, sizeof(cplx) * (size_t)n);
}

/*
 * Transform n values x[0], x[xs], x[2 xs], ... into out[0..n-1].
 * tab holds W_{n0}^m for the top-level length n0; this level uses
 * W_n^m = tab[m * ts] with ts = n0 / n.  scratch has room for n values.
 */
static void fft_rec(const cplx* x, long xs, long n, const cplx* tab, long ts, long n0,
                    cplx* out, cplx* scratch) {
    if (n == 1) { out[0] = x[0]; return; }
    long p = (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : 0;
    if (p == 0) {
        /* direct definition for a length with no factor 2 or 3 */
        for (long k = 0; k < n; ++k) {
            cplx acc = {0.0, 0.0};
            for (long j = 0; j < n; ++j) {
                long m = (j * k) % n;
                cplx w = tab[m * ts];
                cplx v = cmul(x[j * xs], w);
                acc.re += v.re; acc.im += v.im;
            }
            out[k] = acc;
        }
        return;
    }
    long q = n / p;
    /* sub-transforms X_r of the subsequences x[p*m + r] land in out[r*q .. r*q+q-1] */
    for (long r = 0; r < p; ++r)
        fft_rec(x + r * xs, xs * p, q, tab, ts * p, n0, out + r * q, scratch + r * q);
    recombine(n, p, tab, ts, out, scratch);
}

/*
 * fft_rec with the p sub-transforms of the top `depth_left` levels run as
 * OpenMP tasks (they read disjoint inputs and write disjoint parts of out and
 * scratch).  Every output is formed by exactly the same operations in the same
 * order as in fft_rec: only the schedule differs.  Call inside a parallel
 * region, from one thread.
 */
static void fft_rec_tasks(const cplx* x, long xs, long n, const cplx* tab, long ts, long n0,
                          cplx* out, cplx* scratch, int depth_left) {
    long p = (n % 2 == 0) ? 2 : (n % 3 == 0) ? 3 : 0;
    if (depth_left <= 0 || p == 0 || n < 4096) {
        fft_rec(x, xs, n, tab, ts, n0, out, scratch);
        return;
    }
    long q = n / p;
    for (long r = 0; r < p; ++r) {
#pragma omp task firstprivate(r)
        fft_rec_tasks(x + r * xs, xs * p, q, tab, ts * p, n0, out + r * q, scratch + r * q, depth_left - 1);
    }
#pragma omp taskwait
    recombine(n, p, tab, ts, out, scratch);
}

/*
 * In-place multi-dimensional transform of `data` (interleaved complex
 * doubles), shape dims[0..ndim-1], last axis fastest.  sign = -1 forward,
 * +1 inverse; normalize != 0 multiplies by 1/(total size) at the end.
 * Returns 0 on success, -1 on bad arguments, -2 if memory ran out.
 */
int oracle_fftn(double* data, int ndim, const long* dims, int sign, int normalize) {
    if (!data || ndim < 1 || ndim > 3 || (sign != 1 && sign != -1)) return -1;
    long total = 1;
    for (int a = 0; a < ndim; ++a) { if (dims[a] < 1) return -1; total *= dims[a]; }
    cplx* z = (cplx*)data;
    int err = 0;
    for (int axis = 0; axis < ndim; ++axis) {
        long n = dims[axis];
        if (n == 1) continue;
        long inner = 1, outer = 1;
        for (int a = axis + 1; a < ndim; ++a) inner *= dims[a];
        for (int a = 0; a < axis; ++a) outer *= dims[a];
        cplx* tab = make_table(n, sign);
        if (!tab) return -2;
        long npencil = outer * inner;
        if (npencil == 1) {
            /* one long transform: its recursion's sub-transforms run as tasks */
            cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n * 3);
            if (!buf) { free(tab); return -2; }
            memcpy(buf, z, sizeof(cplx) * (size_t)n);
#pragma omp parallel
#pragma omp single
            fft_rec_tasks(buf, 1, n, tab, 1, n, buf + n, buf + 2 * n, 4);
            memcpy(z, buf + n, sizeof(cplx) * (size_t)n);
            free(buf);
            free(tab);
            continue;
        }
#pragma omp parallel
        {
            cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n * 3);
            if (!buf) {
#pragma omp atomic write
                err = -2;
            }
#pragma omp for schedule(static)
            for (long pc = 0; pc < npencil; ++pc) {
                if (!buf) continue;
                long o = pc / inner, i = pc % inner;
                cplx* base = z + o * n * inner + i;
                cplx* in = buf;
                cplx* out = buf + n;
                cplx* scr = buf + 2 * n;
                for (long j = 0; j < n; ++j) in[j] = base[j * inner];
                fft_rec(in, 1, n, tab, 1, n, out, scr);
                for (long j = 0; j < n; ++j) base[j * inner] = out[j];
            }
            free(buf);
        }
        free(tab);
        if (err) return err;
    }
    if (normalize) {
        double s = 1.0 / (double)total;
        for (long t = 0; t < 2 * total; ++t) data[t] *= s;
    }
    return 0;
}

/* Batched 1-D transform: `batch` independent signals of length n, contiguous. */
int oracle_fft1_batch(double* data, long batch, long n, int sign, int normalize) {
    long dims[2] = { batch, n };
    if (batch < 1 || n < 1) return -1;
    /* axis 0 has length `batch`: transform only the last axis */
    cplx* z = (cplx*)data;
    cplx* tab = make_table(n, sign);
    if (!tab) return -2;
    int err = 0;
#pragma omp parallel
    {
        cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n * 3);
        if (!buf) {
#pragma omp atomic write
            err = -2;
        }
#pragma omp for schedule(static)
        for (long b = 0; b < batch; ++b) {
            if (!buf) continue;
            cplx* base = z + b * n;
            memcpy(buf, base, sizeof(cplx) * (size_t)n);
            fft_rec(buf, 1, n, tab, 1, n, buf + n, buf + 2 * n);
            memcpy(base, buf + n, sizeof(cplx) * (size_t)n);
        }
        free(buf);
    }
    free(tab);
    (void)dims;
    if (err) return err;
    if (normalize) {
        double s = 1.0 / (double)n;
        for (long t = 0; t < 2 * batch * n; ++t) data[t] *= s;
    }
    return 0;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
