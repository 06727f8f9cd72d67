/*
 * Oracle for mixed-datatype gemm, C := beta*C + alpha*op(A)*op(B).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow CPU statement of what the
 * mixed-datatype gemm computes. Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may build or call it; the library never does.
 * It shares no code, header or constant with the CUDA path.
 *
 * Everything is computed in binary64 / complex binary64, following the paper
 * (Van Zee, Parikh, van de Geijn, "Supporting mixed-datatype matrix multiplication
 * within the BLIS framework", arXiv 1901.06015):
 *
 *  1. Load op(A), op(B) and C from their storage datatype through (rs, cs) and the
 *     trans value (N, T, conj-only, conj-transpose) -- Sec. 2.2.1 (row/column/general
 *     strides), Sec. 2.2.2 (induced transposition), Sec. 2.2.3 and Sec. 3
 *     (conjugation without transposition). Widening to binary64 is exact; a real
 *     operand has imaginary part zero.
 *  2. Cast each real component of A and B to the computation precision
 *     (Sec. 5.1.1: the computation precision, defaulting to C's storage precision;
 *     Sec. 5.1.2: the target datatype = own domain + computation precision).
 *     alpha is cast to the computation precision, beta to C's storage precision
 *     (Sec. 7.1, option 1 for both). Rounding is round-to-nearest-even (the paper
 *     does not name a rounding mode; this is the reading we take).
 *  3. Domain rule (Fig. "mixeddom", Sec. 4.2, Sec. 7.2), one statement for all 8 cases:
 *     form P = Ahat * Bhat in complex arithmetic (real operands have Im = 0), then
 *       C real:    C_new = Re(beta) * C + Re(alpha) * Re(P)
 *       C complex: C_new = beta * C + alpha * P
 *     Imaginary alpha is an error in cases 1a, 1b, 1c, 2ab, 2ac, 2bc (Sec. 7.2); in
 *     case 0 it is dropped (projected), in case 3 it is honoured.
 *     With literal_alpha set, the "literal interpretation" that Sec. 7.2 describes is
 *     taken instead: every operand's domain at face value, so no case rejects a
 *     complex alpha and, with C real, C_new = Re(beta) * C + Re(alpha * P).
 *     beta == 0 means C is not read, and alpha == 0 (after its cast) means A and B
 *     are not read (BLAS conventions; the paper is silent on both).
 *  4. The length-k sums use the compensated dot product Dot2 of Ogita, Rump and
 *     Oishi (SIAM J. Sci. Comput. 26(6), 2005), so the oracle's own error is about
 *     one unit roundoff of binary64 plus O(k u^2).
 *  5. Output: C_new in complex binary64 (column-major m x n, "exact"), and C itself
 *     overwritten with C_new rounded (RN-even) to C's storage datatype.
 *
 * Datatype codes: 0 = s (real single), 1 = d (real double), 2 = c (complex single),
 * 3 = z (complex double), 4 = h (real binary16), 5 = k (complex binary16), 6 = b (real
 * bfloat16), 7 = w (complex bfloat16); a complex element stores (re, im).
 * Trans codes: 0 = N, 1 = T, 2 = conj only, 3 = conj-trans.
 * Computation precision: 0 = single, 1 = double, 2 = that of C, 3 = binary16, 4 =
 * bfloat16 (Sec. 5.3: a further precision; A and B are rounded to it, and, as on the
 * hardware that computes it, the sums are formed in a wider format -- here exactly).
 * Return: 0 ok, 1 invalid argument, 2 imaginary alpha in a case that forbids it.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

typedef struct { double re, im; } zval;

static int dt_is_complex(int dt) { return dt == 2 || dt == 3 || dt == 5 || dt == 7; }
/* storage precision of a datatype: 0 single, 1 double, 3 binary16, 4 bfloat16 */
static int dt_prec(int dt) {
    switch (dt) {
    case 1: case 3: return 1;
    case 4: case 5: return 3;
    case 6: case 7: return 4;
    default: return 0;
    }
}

/* Round x (binary64) to a binary format with p significant bits, smallest normal
 * 2^emin and largest finite value (2 - 2^(1-p)) 2^emax: round-to-nearest, ties to
 * even, gradual underflow, values beyond the largest finite round to infinity (IEEE
 * 754 semantics written out). Scaling by powers of two is exact, so the quotient and
 * product below introduce no rounding besides nearbyint's. */
static double rnd_fmt(double x, int p, int emin, int emax) {
    double a, q, r, maxv;
    int e, ex;
    if (x != x || x == 0.0 || isinf(x)) return x;
    a = fabs(x);
    (void)frexp(a, &e);                 /* a in [2^(e-1), 2^e) */
    ex = e - 1;
    if (ex < emin) ex = emin;           /* subnormal range: fixed quantum */
    q = ldexp(1.0, ex - (p - 1));
    r = nearbyint(a / q) * q;           /* default rounding mode: nearest, ties to even */
    maxv = ldexp(2.0 - ldexp(1.0, 1 - p), emax);
    if (r > maxv) r = INFINITY;
    return copysign(r, x);
}
static double rnd_half(double x) { return rnd_fmt(x, 11, -14, 15); }
static double rnd_bf16(double x) { return rnd_fmt(x, 8, -126, 127); }

/* binary16 bit pattern <-> value */
static double half_value(uint16_t h) {
    const int e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m | 1024), e - 25);
    return (h & 0x8000) ? -v : v;
}
static uint16_t half_bits(double x) {   /* x: already a binary16 value, inf or NaN */
    const uint16_t sgn = signbit(x) ? 0x8000 : 0;
    const double a = fabs(x);
    int e, ex;
    if (a != a) return (uint16_t)(sgn | 0x7e00);
    if (isinf(a)) return (uint16_t)(sgn | 0x7c00);
    if (a == 0.0) return sgn;
    (void)frexp(a, &e);
    ex = e - 1;
    if (ex < -14) return (uint16_t)(sgn | (uint16_t)ldexp(a, 24));        /* subnormal: m 2^-24 */
    return (uint16_t)(sgn | ((ex + 15) << 10) | (uint16_t)((ldexp(a, -ex) - 1.0) * 1024.0));
}
/* bfloat16: the upper half of a binary32 pattern */
static double bf16_value(uint16_t b) {
    const uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}
static uint16_t bf16_bits(double x) {   /* x: already a bfloat16 value, inf or NaN */
    const float f = (float)x;           /* exact */
    uint32_t u;
    memcpy(&u, &f, 4);
    if (x != x) return (uint16_t)((u >> 16) | 0x40);
    return (uint16_t)(u >> 16);
}

/* Read element at linear offset off (in elements of dt), widened to complex binary64. */
static zval load_elem(const void* base, int dt, int64_t off) {
    zval v = {0.0, 0.0};
    switch (dt) {
    case 0: v.re = (double)((const float*)base)[off]; break;
    case 1: v.re = ((const double*)base)[off]; break;
    case 2: v.re = (double)((const float*)base)[2 * off];
            v.im = (double)((const float*)base)[2 * off + 1]; break;
    case 3: v.re = ((const double*)base)[2 * off];
            v.im = ((const double*)base)[2 * off + 1]; break;
    case 4: v.re = half_value(((const uint16_t*)base)[off]); break;
    case 5: v.re = half_value(((const uint16_t*)base)[2 * off]);
            v.im = half_value(((const uint16_t*)base)[2 * off + 1]); break;
    case 6: v.re = bf16_value(((const uint16_t*)base)[off]); break;
    case 7: v.re = bf16_value(((const uint16_t*)base)[2 * off]);
            v.im = bf16_value(((const uint16_t*)base)[2 * off + 1]); break;
    }
    return v;
}

static void store_elem(void* base, int dt, int64_t off, zval v) {
    switch (dt) {
    case 0: ((float*)base)[off] = (float)v.re; break;
    case 1: ((double*)base)[off] = v.re; break;
    case 2: ((float*)base)[2 * off] = (float)v.re;
            ((float*)base)[2 * off + 1] = (float)v.im; break;
    case 3: ((double*)base)[2 * off] = v.re;
            ((double*)base)[2 * off + 1] = v.im; break;
    case 4: ((uint16_t*)base)[off] = half_bits(rnd_half(v.re)); break;
    case 5: ((uint16_t*)base)[2 * off] = half_bits(rnd_half(v.re));
            ((uint16_t*)base)[2 * off + 1] = half_bits(rnd_half(v.im)); break;
    case 6: ((uint16_t*)base)[off] = bf16_bits(rnd_bf16(v.re)); break;
    case 7: ((uint16_t*)base)[2 * off] = bf16_bits(rnd_bf16(v.re));
            ((uint16_t*)base)[2 * off + 1] = bf16_bits(rnd_bf16(v.im)); break;
    }
}

/* Round a binary64 value to a precision (0 = single, 1 = double, 3 = binary16,
 * 4 = bfloat16). */
static double rnd_prec(double x, int prec) {
    switch (prec) {
    case 0: return (double)(float)x;
    case 3: return rnd_half(x);
    case 4: return rnd_bf16(x);
    default: return x;
    }
}

double oracle_round(double x, int prec) { return rnd_prec(x, prec); }

/* Element (i, p) of op(X), where X is stored with strides (rs, cs) and trans in
 * {0:N, 1:T, 2:conj, 3:conj-trans}. For T and conj-trans, X is stored transposed. */
static zval load_op(const void* x, int dt, int64_t rs, int64_t cs, int trans, int64_t i, int64_t p) {
    int64_t off = (trans == 1 || trans == 3) ? (p * rs + i * cs) : (i * rs + p * cs);
    zval v = load_elem(x, dt, off);
    if (trans == 2 || trans == 3) v.im = -v.im;
    return v;
}

/* Error-free transformations (Knuth's TwoSum; TwoProduct via fused multiply-add). */
static void two_sum(double a, double b, double* s, double* e) {
    double z;
    *s = a + b;
    z = *s - a;
    *e = (a - (*s - z)) + (b - z);
}
static void two_prod(double a, double b, double* p, double* e) {
    *p = a * b;
    *e = fma(a, b, -*p);
}

/* Compensated dot-product accumulator (Algorithm Dot2). */
typedef struct { double p, s; } dot2;
static void dot2_init(dot2* d) { d->p = 0.0; d->s = 0.0; }
static void dot2_add(dot2* d, double x, double y) {
    double h, r, q;
    two_prod(x, y, &h, &r);
    two_sum(d->p, h, &d->p, &q);
    d->s += q + r;
}
static double dot2_result(const dot2* d) { return d->p + d->s; }

int oracle_case_of(int dtC, int dtA, int dtB) {
    /* Fig. "mixeddom": 0 RRR, 1 RRC (1b), 2 RCR (1a), 3 RCC (2ab),
     *                  4 CRR (1c), 5 CRC (2bc), 6 CCR (2ac), 7 CCC (3). */
    return (dt_is_complex(dtC) << 2) | (dt_is_complex(dtA) << 1) | dt_is_complex(dtB);
}

int oracle_mxgemm(int transa, int transb, int64_t m, int64_t n, int64_t k,
                  double alpha_re, double alpha_im,
                  const void* A, int dtA, int64_t rsA, int64_t csA,
                  const void* B, int dtB, int64_t rsB, int64_t csB,
                  double beta_re, double beta_im,
                  void* C, int dtC, int64_t rsC, int64_t csC,
                  int comp, double* c_exact, int nthreads, int literal_alpha) {
    if (transa < 0 || transa > 3 || transb < 0 || transb > 3) return 1;
    if (dtA < 0 || dtA > 7 || dtB < 0 || dtB > 7 || dtC < 0 || dtC > 7) return 1;
    if (comp < 0 || comp > 4 || m < 0 || n < 0 || k < 0) return 1;
    {
        int cse = oracle_case_of(dtC, dtA, dtB);
        if (!literal_alpha && alpha_im != 0.0 && cse != 0 && cse != 7) return 2;  /* Sec. 7.2 */
    }
    if (comp == 2) comp = dt_prec(dtC);                        /* Sec. 5.1.1 */
    {
        const int c_cplx = dt_is_complex(dtC);
        const int precC = dt_prec(dtC);
        /* Sec. 7.1: alpha to the computation precision, beta to C's precision. */
        const double ar = rnd_prec(alpha_re, comp), ai = rnd_prec(alpha_im, comp);
        const double br = rnd_prec(beta_re, precC), bi = rnd_prec(beta_im, precC);
        const int beta_zero = (br == 0.0 && bi == 0.0);
        const int alpha_zero = (ar == 0.0 && ai == 0.0);
        int64_t j;
        (void)nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
        for (j = 0; j < n; ++j) {
            int64_t i, p;
            for (i = 0; i < m; ++i) {
                dot2 pre, pim, out_re, out_im;
                double Pre, Pim;
                zval c = {0.0, 0.0}, cn;
                dot2_init(&pre); dot2_init(&pim);
                for (p = 0; p < (alpha_zero ? 0 : k); ++p) {
                    zval a = load_op(A, dtA, rsA, csA, transa, i, p);
                    zval b = load_op(B, dtB, rsB, csB, transb, p, j);
                    /* cast each component to the computation precision (Sec. 5.1.2) */
                    a.re = rnd_prec(a.re, comp); a.im = rnd_prec(a.im, comp);
                    b.re = rnd_prec(b.re, comp); b.im = rnd_prec(b.im, comp);
                    /* complex product: (ar + i ai)(br + i bi) */
                    dot2_add(&pre, a.re, b.re);
                    dot2_add(&pre, -a.im, b.im);
                    dot2_add(&pim, a.re, b.im);
                    dot2_add(&pim, a.im, b.re);
                }
                Pre = dot2_result(&pre);
                Pim = dot2_result(&pim);
                if (!beta_zero) c = load_elem(C, dtC, i * rsC + j * csC);
                dot2_init(&out_re); dot2_init(&out_im);
                if (!c_cplx) {
                    /* C real: project beta and alpha, keep Re(P) (cases 0, 1a, 1b, 2ab);
                     * literally, Re(alpha * P). */
                    if (!beta_zero) dot2_add(&out_re, br, c.re);
                    dot2_add(&out_re, ar, Pre);
                    if (literal_alpha) dot2_add(&out_re, -ai, Pim);
                    cn.re = dot2_result(&out_re);
                    cn.im = 0.0;
                } else {
                    /* C complex: beta*C + alpha*P (cases 1c, 2ac, 2bc, 3). */
                    if (!beta_zero) {
                        dot2_add(&out_re, br, c.re);
                        dot2_add(&out_re, -bi, c.im);
                        dot2_add(&out_im, br, c.im);
                        dot2_add(&out_im, bi, c.re);
                    }
                    dot2_add(&out_re, ar, Pre);
                    dot2_add(&out_re, -ai, Pim);
                    dot2_add(&out_im, ar, Pim);
                    dot2_add(&out_im, ai, Pre);
                    cn.re = dot2_result(&out_re);
                    cn.im = dot2_result(&out_im);
                }
                if (c_exact) {
                    c_exact[2 * (i + j * m)] = cn.re;
                    c_exact[2 * (i + j * m) + 1] = cn.im;
                }
                store_elem(C, dtC, i * rsC + j * csC, cn);
            }
        }
    }
    return 0;
}
