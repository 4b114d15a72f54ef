/*
 * CPU oracle for the AM-QFT complex DFT ("A class of AM-QFT algorithms for
 * power-of-two FFT", Pasquini).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is called by the tests, by the
 * smoke check and by the bench's CPU-baseline leg.  The product (the CUDA
 * library) never links, loads or calls it, and the two share no code.
 *
 * What it provides:
 *   - orc_naive_dft: the DFT of Eq. qft_0A written out, O(N^2), long double
 *     accumulation, angles reduced exactly from the integer n*k mod N.
 *   - orc_dft_bin: one bin of the same definition, O(N), for spot checks.
 *   - orc_cdft: the AM-QFT recursion of Sect. 3-6 for each of the 8 variants
 *     in float, double or long double (amqft_rec.inc), with an operation
 *     tally (sums, multiplications, binary translations) as Sect. 7 counts.
 *   - orc_sub: any single function of the recursion (rdft, dct, dst, dct_ot,
 *     dst_ot, dct_to, dst_to, dct_oo, dst_oo) for per-function checks.
 *   - orc_mv_time / orc_mv_freq: the two phases of M1..M8 (Tab. 5-6).
 *   - orc_angles: which trig-constant angles a transform uses (Sect. 7.1).
 *   - orc_set_fault: plants one of a few deliberate mistakes so the tests can
 *     show that the pins catch them.
 * Inverse (sign = +1) is conj(F(conj x)), unnormalised: the paper defines
 * only the forward transform.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define PI_L 3.14159265358979323846264338327950288419716939937510L

enum { FAM_COS2 = 0, FAM_SEC2 = 1, FAM_SIN2 = 2, FAM_CSC2 = 3 };
enum {
    FAULT_NONE = 0,
    FAULT_DC_MISPRINT = 1,  /* sign of Eq. qft_19A as printed */
    FAULT_DR_SIGN = 2,      /* D_r difference taken the wrong way round */
    FAULT_DK_DROP = 3,      /* D_k sum loses its second term */
    FAULT_M4_NEIGHBOUR = 4, /* M4 frequency relation uses E(k-1) twice */
    FAULT_CONST_INDEX = 5,  /* trig constant taken at n+2 instead of n */
    FAULT_DN_SIGN = 6,      /* D_n backward: S(M/2-k) = E+O instead of E-O */
    FAULT_M1_HALVING = 7    /* M1 drops the binary translation at k = 1 */
};

static int g_fault = FAULT_NONE;
static __thread long long t_add, t_mul, t_half;
static __thread int t_count;
static __thread unsigned char *t_angles;
static __thread long t_top_n;

static inline int fault_is(int f) { return g_fault == f; }
static inline void tally_add(void) { if (t_count) t_add++; }
static inline void tally_mul(void) { if (t_count) t_mul++; }
static inline void tally_half(void) { if (t_count) t_half++; }

/* Record the angle 2*pi*p/M as q/N of the top-level transform. */
static void note_angle(long M, long p) {
    if (!t_angles || M > t_top_n) return;
    long q = p * (t_top_n / M);
    if (q > 0 && q < t_top_n) t_angles[q] = 1;
}

/* cos(2*pi*p/M), M = 1 or even, with the argument reduced exactly to
 * [0, pi/4] before calling the long double libm routine. */
static long double cos_turn(long long p, long long M) {
    if (M == 1) return 1.0L;
    long long a = p % M;
    if (a < 0) a += M;
    if (2 * a > M) a = M - a;            /* cos is even and M-periodic: a in [0, M/2] */
    long double sgn = 1.0L;
    if (4 * a > M) { a = M / 2 - a; sgn = -1.0L; }   /* cos(pi - x) = -cos(x): a in [0, M/4] */
    if (8 * a > M)                        /* cos(x) = sin(pi/2 - x) */
        return sgn * sinl(2.0L * PI_L * (long double)(M - 4 * a) / (4.0L * (long double)M));
    return sgn * cosl(2.0L * PI_L * (long double)a / (long double)M);
}

/* sin(2*pi*p/M) = cos(2*pi*(4p - M)/(4M)). */
static long double sin_turn(long long p, long long M) { return cos_turn(4 * p - M, 4 * M); }

#define REAL float
#define SFX f
#include "amqft_rec.inc"
#undef REAL
#undef SFX

#define REAL double
#define SFX d
#include "amqft_rec.inc"
#undef REAL
#undef SFX

#define REAL long double
#define SFX l
#include "amqft_rec.inc"
#undef REAL
#undef SFX

/* ------------------------------------------------------------------ */
/* public entry points                                                  */
/* ------------------------------------------------------------------ */

int orc_version(void) { return 1; }
void orc_set_fault(int f) { g_fault = f; }

static int bad_args(int prec, int variant, int log2n) {
    if (prec < 0 || prec > 2) return -1;
    if (variant < 1 || variant > 8) return -2;
    if (log2n < 0 || log2n > 26) return -3;
    return 0;
}

static void tally_begin(long long *tally) {
    t_count = tally != NULL;
    t_add = t_mul = t_half = 0;
}
static void tally_end(long long *tally) {
    if (tally) { tally[0] = t_add; tally[1] = t_mul; tally[2] = t_half; }
    t_count = 0;
}

/* One complex transform of length 2^log2n, interleaved (re, im) doubles.
 * prec: 0 float, 1 double, 2 long double.  sign: -1 forward (Eq. qft_0A),
 * +1 unnormalised inverse.  tally (optional): [sums, mults, halvings]. */
int orc_cdft(int prec, int variant, int log2n, const double *in, double *out, int sign,
             long long *tally) {
    int rc = bad_args(prec, variant, log2n);
    if (rc) return rc;
    const long N = 1L << log2n;
    const double cj = sign > 0 ? -1.0 : 1.0;
    tally_begin(tally);
    if (prec == 0) {
        float *z = malloc(sizeof(float) * 2 * N), *Z = malloc(sizeof(float) * 2 * N);
        for (long i = 0; i < N; i++) { z[2 * i] = (float)in[2 * i]; z[2 * i + 1] = (float)(cj * in[2 * i + 1]); }
        cdft_f(variant, N, z, Z);
        for (long i = 0; i < N; i++) { out[2 * i] = Z[2 * i]; out[2 * i + 1] = cj * Z[2 * i + 1]; }
        free(z); free(Z);
    } else if (prec == 1) {
        double *z = malloc(sizeof(double) * 2 * N), *Z = malloc(sizeof(double) * 2 * N);
        for (long i = 0; i < N; i++) { z[2 * i] = in[2 * i]; z[2 * i + 1] = cj * in[2 * i + 1]; }
        cdft_d(variant, N, z, Z);
        for (long i = 0; i < N; i++) { out[2 * i] = Z[2 * i]; out[2 * i + 1] = cj * Z[2 * i + 1]; }
        free(z); free(Z);
    } else {
        long double *z = malloc(sizeof(long double) * 2 * N), *Z = malloc(sizeof(long double) * 2 * N);
        for (long i = 0; i < N; i++) { z[2 * i] = in[2 * i]; z[2 * i + 1] = cj * in[2 * i + 1]; }
        cdft_l(variant, N, z, Z);
        for (long i = 0; i < N; i++) { out[2 * i] = (double)Z[2 * i]; out[2 * i + 1] = cj * (double)Z[2 * i + 1]; }
        free(z); free(Z);
    }
    tally_end(tally);
    return 0;
}

/* A batch of transforms, parallel over the batch with OpenMP (nthreads <= 0:
 * the OpenMP default).  Returns the number of threads used, or < 0. */
int orc_cdft_batch(int prec, int variant, int log2n, long long batch, const double *in, double *out,
                   int sign, int nthreads) {
    int rc = bad_args(prec, variant, log2n);
    if (rc) return rc;
    const long N = 1L << log2n;
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (long long b = 0; b < batch; b++)
            orc_cdft(prec, variant, log2n, in + 2 * N * b, out + 2 * N * b, sign, NULL);
    }
#else
    (void)nthreads;
    for (long long b = 0; b < batch; b++)
        orc_cdft(prec, variant, log2n, in + 2 * N * b, out + 2 * N * b, sign, NULL);
#endif
    return used;
}

/* Single functions of the recursion, for per-function checks against the
 * pruned DCT-0/DST-0 definitions.  kind: 0 rdft, 1 dct, 2 dst, 3 dct_ot,
 * 4 dst_ot, 5 dct_to, 6 dst_to, 7 dct_oo, 8 dst_oo.  Arrays in the storage
 * of Tab. 2 (0-based).  rdft writes Re R(0..M/2) then Im R(1..M/2-1). */
int orc_sub(int prec, int variant, int kind, int log2m, const double *in, double *out,
            long long *tally) {
    int rc = bad_args(prec, variant, log2m);
    if (rc) return rc;
    const long M = 1L << log2m;
    long nin, nout;
    switch (kind) {
    case 0:
        if (M < 2) return -4;
        nin = M; nout = M;
        break;
    case 1:
        if (M < 2) return -4;
        nin = nout = M / 2 + 1;
        break;
    case 2:
        if (M < 4) return -4;
        nin = nout = M / 2 - 1;
        break;
    case 3: case 4: case 5: case 6:
        if (M < 4) return -4;
        nin = nout = M / 4;
        break;
    case 7: case 8:
        if (M < 8) return -4;
        nin = nout = M / 8;
        break;
    default: return -5;
    }
    int is_to = (variant == 2 || variant == 3 || variant == 6 || variant == 7);
    if ((kind == 3 || kind == 4) && is_to) return -6;   /* ot functions belong to 1,4,5,8 */
    if ((kind == 5 || kind == 6) && !is_to) return -6;  /* to functions belong to 2,3,6,7 */
    tally_begin(tally);
#define RUN_SUB(T, S)                                                                 \
    do {                                                                              \
        T *x = malloc(sizeof(T) * (nin + 1)), *y = malloc(sizeof(T) * (nout + 1));     \
        for (long i = 0; i < nin; i++) x[i] = (T)in[i];                               \
        switch (kind) {                                                               \
        case 0: rdft_##S(variant, M, x, y, y + M / 2 + 1); break;                     \
        case 1: dct_##S(variant, M, x, y); break;                                     \
        case 2: dst_##S(variant, M, x, y); break;                                     \
        case 3: dct_ot_##S(variant, M, x, y); break;                                  \
        case 4: dst_ot_##S(variant, M, x, y); break;                                  \
        case 5: dct_to_##S(variant, M, x, y); break;                                  \
        case 6: dst_to_##S(variant, M, x, y); break;                                  \
        case 7: dct_oo_##S(variant, M, x, y); break;                                  \
        default: dst_oo_##S(variant, M, x, y); break;                                 \
        }                                                                             \
        for (long i = 0; i < nout; i++) out[i] = (double)y[i];                         \
        free(x); free(y);                                                             \
    } while (0)
    if (prec == 0) RUN_SUB(float, f);
    else if (prec == 1) RUN_SUB(double, d);
    else RUN_SUB(long double, l);
#undef RUN_SUB
    tally_end(tally);
    return 0;
}

/* M_v phases on their own (double), M = 2^log2m >= 16, ctx 0 = DCT (Tab. 5),
 * 1 = DST (Tab. 6).  x: the oo signal (M/8 values); y: the child signal. */
int orc_mv_time(int variant, int ctx, int log2m, const double *x, double *y) {
    if (variant < 1 || variant > 8 || log2m < 4 || log2m > 26 || (ctx != 0 && ctx != 1)) return -1;
    mv_time_d(variant, ctx, 1L << log2m, x, y);
    return 0;
}
int orc_mv_freq(int variant, int ctx, int log2m, const double *e, double *o) {
    if (variant < 1 || variant > 8 || log2m < 4 || log2m > 26 || (ctx != 0 && ctx != 1)) return -1;
    mv_freq_d(variant, ctx, 1L << log2m, e, o);
    return 0;
}

/* Marks used[q] = 1 for every angle 2*pi*q/N (0 < q < N) that the
 * double-precision AM-QFT of length N = 2^log2n reads a constant at. */
int orc_angles(int variant, int log2n, unsigned char *used) {
    if (variant < 1 || variant > 8 || log2n < 1 || log2n > 22) return -1;
    const long N = 1L << log2n;
    memset(used, 0, (size_t)N);
    double *z = calloc((size_t)(2 * N), sizeof(double)), *Z = calloc((size_t)(2 * N), sizeof(double));
    t_angles = used;
    t_top_n = N;
    cdft_d(variant, N, z, Z);
    t_angles = NULL;
    free(z); free(Z);
    return 0;
}

/* Naive DFT (Eq. qft_0A), long double accumulation, exact angle reduction.
 * sign -1: forward, +1: unnormalised inverse.  Intended for N <= 2^13. */
int orc_naive_dft(int log2n, const double *in, double *out, int sign) {
    if (log2n < 0 || log2n > 16) return -1;
    const long N = 1L << log2n;
    long double *ct = malloc(sizeof(long double) * N), *st = malloc(sizeof(long double) * N);
    for (long j = 0; j < N; j++) { ct[j] = cos_turn(j, N); st[j] = sin_turn(j, N); }
    for (long k = 0; k < N; k++) {
        long double ar = 0.0L, ai = 0.0L;
        for (long n = 0; n < N; n++) {
            long j = (long)(((unsigned long)n * (unsigned long)k) & (unsigned long)(N - 1));
            long double c = ct[j], s = (long double)sign * st[j];
            long double xr = in[2 * n], xi = in[2 * n + 1];
            ar += xr * c - xi * s;
            ai += xr * s + xi * c;
        }
        out[2 * k] = (double)ar;
        out[2 * k + 1] = (double)ai;
    }
    free(ct); free(st);
    return 0;
}

/* One bin X(k) of Eq. qft_0A in long double, O(N): for spot checks at any N. */
int orc_dft_bin(int log2n, const double *in, long long k, double *out2, int sign) {
    if (log2n < 0 || log2n > 30) return -1;
    const long long N = 1LL << log2n;
    long double ar = 0.0L, ai = 0.0L;
    for (long long n = 0; n < N; n++) {
        long long j = (long long)(((unsigned long long)n * (unsigned long long)k) & (unsigned long long)(N - 1));
        long double c = cos_turn(j, N), s = (long double)sign * sin_turn(j, N);
        long double xr = in[2 * n], xi = in[2 * n + 1];
        ar += xr * c - xi * s;
        ai += xr * s + xi * c;
    }
    out2[0] = (double)ar;
    out2[1] = (double)ai;
    return 0;
}

/* Long-double size, so the tests can state which truth they ran against. */
int orc_long_double_digits(void) { return (int)__LDBL_MANT_DIG__; }
