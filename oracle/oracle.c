/*
 * CPU oracle for the parallel reduction of X = {x_0..x_{n-1}} under an
 * associative combiner (Section 1.1, "Problem Definition").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA path and is deliberately slow:
 * every function is a plain sequential loop over the input in index order,
 * i.e. Algorithm 1 ("Summation") with its accumulator and "+" replaced by the
 * combiner at hand.
 *
 * What each function computes (and how it is pinned, see tests/test_oracle.py):
 *   orc_reduce_int      integer/bitwise combiners, exact (two's-complement
 *                       wrap-around where the output type wraps).
 *   orc_sum_f64_loop    Algorithm 1 verbatim with a double accumulator.
 *   orc_sum_f64_chunked the same loop over contiguous chunks on several host
 *                       threads, chunk sums added in order (the multi-core
 *                       CPU baseline the benchmark times beside the GPU).
 *   orc_exact_sum       the exact sum of the inputs (every binary16/bfloat16/
 *                       binary32/binary64 value is an integer multiple of
 *                       2^-1074, so a fixed-point accumulator of 32-bit limbs
 *                       holds the sum exactly) rounded once to double.  This is
 *                       the definition of "sum" that Section 1.1's footnote on
 *                       floating-point reordering says no single order attains.
 *   orc_prod            the product, carried as a double-double significand
 *                       with a separate integer exponent (no intermediate
 *                       overflow/underflow), rounded once to double.
 *   orc_maxmin          max / min with NaN propagation and -0 < +0.
 *   orc_argext          (extremum, first index attaining it).
 *   orc_prod_aux        product of the non-zero elements, zero count and the
 *                       index of the first zero (the forward state that the
 *                       product's gradient needs).
 *   orc_prod_except     prod_{j != i} x_j, the derivative of the product with
 *                       respect to x_i, straight from its definition.
 *   orc_scan            the prefix combinations y_i = x_0 (x) ... (x) x_i
 *                       (inclusive) or x_0 (x) ... (x) x_{i-1} (exclusive, y_0 the
 *                       identity): Algorithm 1's loop, storing the accumulator
 *                       after every step.  Integer/bitwise combiners and float
 *                       max/min (the combiners whose result is exact).
 *
 * Build: gcc -std=c11 -O2 -ffp-contract=off -fPIC -shared -pthread (ISO C, no FMA
 * contraction, so that x86-64 and AArch64 hosts give identical results).
 */
#include <stdint.h>
#include <string.h>
#include <math.h>

/* dtype codes (this file's own numbering; the Python wrapper maps names). */
enum { O_F32 = 0, O_F16 = 1, O_BF16 = 2, O_F64 = 3, O_I32 = 4, O_U32 = 5, O_I64 = 6 };
/* combiner codes */
enum { O_SUM = 0, O_PROD = 1, O_MAX = 2, O_MIN = 3, O_AND = 4, O_OR = 5, O_XOR = 6 };

/* ------------------------------------------------------------------ */
/* Decoding one element to double (exact for every supported float).  */
/* ------------------------------------------------------------------ */

/* IEEE 754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
static double half_bits_to_double(uint16_t h) {
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 0x1f;
    int f = h & 0x3ff;
    double v;
    if (e == 0)            v = ldexp((double)f, -24);              /* subnormal: f * 2^-14 * 2^-10 */
    else if (e == 31)      v = f ? NAN : INFINITY;
    else                   v = ldexp((double)(f | 0x400), e - 25); /* (1024+f) * 2^(e-15-10) */
    return sign ? -v : v;
}

/* bfloat16 is the upper half of a binary32. */
static double bf16_bits_to_double(uint16_t b) {
    uint32_t u = (uint32_t)b << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double elem_as_double(const void* x, int64_t i, int dtype) {
    switch (dtype) {
    case O_F32: return (double)((const float*)x)[i];
    case O_F16: return half_bits_to_double(((const uint16_t*)x)[i]);
    case O_BF16: return bf16_bits_to_double(((const uint16_t*)x)[i]);
    case O_F64: return ((const double*)x)[i];
    case O_I32: return (double)((const int32_t*)x)[i];
    case O_U32: return (double)((const uint32_t*)x)[i];
    default: return (double)((const int64_t*)x)[i];
    }
}

/* ------------------------------------------------------------------ */
/* Exact summation: fixed-point accumulator over 2^-1074 .. 2^1150.     */
/* ------------------------------------------------------------------ */

#define SA_LIMBS 72          /* 72 * 32 = 2304 bits >= 1074 + 1024 + headroom */
#define SA_EMIN (-1074)

typedef struct {
    int64_t d[SA_LIMBS];     /* value = sum_k d[k] * 2^(32k + SA_EMIN) */
    int64_t pending;         /* additions since the last carry pass */
    int nan, pinf, ninf;
} superacc;

static void sa_init(superacc* s) { memset(s, 0, sizeof *s); }

/* Carry pass: every limb but the last ends in [0, 2^32); the last keeps the sign. */
static void sa_normalize(superacc* s) {
    for (int k = 0; k < SA_LIMBS - 1; k++) {
        int64_t c = s->d[k] >> 32;            /* floor division by 2^32 */
        s->d[k] -= c * ((int64_t)1 << 32);
        s->d[k + 1] += c;
    }
    s->pending = 0;
}

/* Add v (a finite double, or a special value recorded by flag). */
static void sa_add(superacc* s, double v) {
    if (isnan(v)) { s->nan = 1; return; }
    if (isinf(v)) { if (v > 0) s->pinf = 1; else s->ninf = 1; return; }
    if (v == 0.0) return;
    uint64_t bits;
    memcpy(&bits, &v, 8);
    int neg = (int)(bits >> 63);
    int ebits = (int)((bits >> 52) & 0x7ff);
    uint64_t m = bits & 0xfffffffffffffull;
    int e;                                   /* v = +-m * 2^e, m an integer */
    if (ebits == 0) e = SA_EMIN;             /* subnormal */
    else { m |= (uint64_t)1 << 52; e = ebits - 1075; }
    int q = e - SA_EMIN;                     /* bit offset of m's lsb, >= 0 */
    int k = q / 32, r = q % 32;
    int64_t c0 = (int64_t)(uint32_t)(m << r);
    int64_t c1 = (int64_t)(uint32_t)((m << r) >> 32);
    int64_t c2 = r ? (int64_t)(uint32_t)(m >> (64 - r)) : 0;
    if (neg) { s->d[k] -= c0; s->d[k + 1] -= c1; s->d[k + 2] -= c2; }
    else     { s->d[k] += c0; s->d[k + 1] += c1; s->d[k + 2] += c2; }
    if (++s->pending >= ((int64_t)1 << 28)) sa_normalize(s);
}

/* Round the exact value to the nearest double (ties to even). */
static double sa_round(superacc* s) {
    if (s->nan || (s->pinf && s->ninf)) return NAN;
    if (s->pinf) return INFINITY;
    if (s->ninf) return -INFINITY;
    sa_normalize(s);
    int64_t d[SA_LIMBS];
    memcpy(d, s->d, sizeof d);
    int neg = d[SA_LIMBS - 1] < 0;
    if (neg) {                               /* negate, then carry again */
        for (int k = 0; k < SA_LIMBS; k++) d[k] = -d[k];
        for (int k = 0; k < SA_LIMBS - 1; k++) {
            int64_t c = d[k] >> 32;
            d[k] -= c * ((int64_t)1 << 32);
            d[k + 1] += c;
        }
    }
    int t = SA_LIMBS - 1;
    while (t >= 0 && d[t] == 0) t--;
    if (t < 0) return 0.0;
    /* Gather the 96-bit window d[t], d[t-1], d[t-2] (limbs below index 0 are 0). */
    uint64_t w2 = (uint64_t)d[t];
    uint64_t w1 = t >= 1 ? (uint64_t)d[t - 1] : 0;
    uint64_t w0 = t >= 2 ? (uint64_t)d[t - 2] : 0;
    int sticky = 0;
    for (int k = t - 3; k >= 0; k--) if (d[k]) { sticky = 1; break; }
    /* top limb has lz leading zeros within its 32 bits */
    int lz = 0;
    while (!((w2 << lz) & 0x80000000ull)) lz++;
    /* 64-bit significand window starting at the leading one */
    uint64_t hi = (w2 << (32 + lz)) | (w1 << lz) | (lz ? (w0 >> (32 - lz)) : 0);
    uint64_t rest = lz ? (w0 & ((1ull << (32 - lz)) - 1)) : w0;
    if (rest) sticky = 1;
    if (sticky) hi |= 1;                     /* bit 0 lies far below the rounding point */
    /* value of bit 0 of hi: the leading one sits at 2^(32t + 31 - lz + SA_EMIN) = bit 63 */
    int exp0 = 32 * t + 31 - lz + SA_EMIN - 63;
    double r = ldexp((double)hi, exp0);
    return neg ? -r : r;
}

double orc_exact_sum(const void* x, int64_t n, int dtype) {
    superacc s;
    sa_init(&s);
    for (int64_t i = 0; i < n; i++) sa_add(&s, elem_as_double(x, i, dtype));
    return sa_round(&s);
}

/* exact sum of |x_i| */
double orc_exact_abs_sum(const void* x, int64_t n, int dtype) {
    superacc s;
    sa_init(&s);
    for (int64_t i = 0; i < n; i++) sa_add(&s, fabs(elem_as_double(x, i, dtype)));
    return sa_round(&s);
}

/* exact (sum_i x_i) - r, rounded once: the error of a computed sum r */
double orc_exact_sum_minus(const void* x, int64_t n, int dtype, double r) {
    superacc s;
    sa_init(&s);
    for (int64_t i = 0; i < n; i++) sa_add(&s, elem_as_double(x, i, dtype));
    sa_add(&s, -r);
    return sa_round(&s);
}

/* Algorithm 1 verbatim: accumulator <- 0; accumulator <- accumulator + a_i. */
double orc_sum_f64_loop(const void* x, int64_t n, int dtype) {
    double acc = 0.0;
    for (int64_t i = 0; i < n; i++) acc = acc + elem_as_double(x, i, dtype);
    return acc;
}

/* ------------------------------------------------------------------ */
/* Multi-core CPU baseline: Algorithm 1 per chunk, chunks in order.     */
/* ------------------------------------------------------------------ */

/* The input is cut into `nthreads` contiguous chunks of (nearly) equal
 * length; thread k runs Algorithm 1 with a double accumulator over chunk k,
 * and the chunk sums are then added in chunk order.  With one thread this is
 * orc_sum_f64_loop.  This is the timed multi-core CPU baseline, not a
 * reference value: its error is that of a double summation (within
 * (n - 1) 2^-53 sum |x| of the exact sum). */
#include <pthread.h>

typedef struct { const void* x; int64_t lo, hi; int dtype; double sum; } sum_chunk;

static void* sum_chunk_run(void* arg) {
    sum_chunk* c = (sum_chunk*)arg;
    double acc = 0.0;
    for (int64_t i = c->lo; i < c->hi; i++) acc = acc + elem_as_double(c->x, i, c->dtype);
    c->sum = acc;
    return NULL;
}

double orc_sum_f64_chunked(const void* x, int64_t n, int dtype, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    sum_chunk ch[256];
    pthread_t th[256];
    int started[256];
    for (int k = 0; k < nthreads; k++) {
        ch[k].x = x;
        ch[k].lo = n * k / nthreads;
        ch[k].hi = n * (k + 1) / nthreads;
        ch[k].dtype = dtype;
        ch[k].sum = 0.0;
        started[k] = k > 0 && pthread_create(&th[k], NULL, sum_chunk_run, &ch[k]) == 0;
    }
    sum_chunk_run(&ch[0]);
    for (int k = 1; k < nthreads; k++) {
        if (started[k]) pthread_join(th[k], NULL);
        else sum_chunk_run(&ch[k]);                 /* no thread: run it here */
    }
    double acc = 0.0;
    for (int k = 0; k < nthreads; k++) acc = acc + ch[k].sum;
    return acc;
}

/* ------------------------------------------------------------------ */
/* Integer and bitwise combiners (exact).                               */
/* ------------------------------------------------------------------ */

/* int32 input: SUM -> int64 (exact), others -> int32 (PROD wraps mod 2^32). */
/* uint32 input: all -> uint32 (SUM and PROD wrap mod 2^32).                */
/* int64 input: all -> int64 (SUM and PROD wrap mod 2^64).                  */
/* Result is written to *out with the output type's width.                  */
int orc_reduce_int(const void* x, int64_t n, int dtype, int op, void* out) {
    if (dtype == O_I32) {
        const int32_t* a = (const int32_t*)x;
        if (op == O_SUM) {
            int64_t acc = 0;
            for (int64_t i = 0; i < n; i++) acc = acc + a[i];
            *(int64_t*)out = acc;
            return 0;
        }
        uint32_t acc;                                  /* two's-complement bits */
        switch (op) {
        case O_PROD: acc = 1; for (int64_t i = 0; i < n; i++) acc = acc * (uint32_t)a[i]; break;
        case O_MAX: { int32_t m = INT32_MIN; for (int64_t i = 0; i < n; i++) if (a[i] > m) m = a[i]; acc = (uint32_t)m; break; }
        case O_MIN: { int32_t m = INT32_MAX; for (int64_t i = 0; i < n; i++) if (a[i] < m) m = a[i]; acc = (uint32_t)m; break; }
        case O_AND: acc = 0xffffffffu; for (int64_t i = 0; i < n; i++) acc = acc & (uint32_t)a[i]; break;
        case O_OR: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc | (uint32_t)a[i]; break;
        case O_XOR: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc ^ (uint32_t)a[i]; break;
        default: return -1;
        }
        memcpy(out, &acc, 4);
        return 0;
    }
    if (dtype == O_U32) {
        const uint32_t* a = (const uint32_t*)x;
        uint32_t acc;
        switch (op) {
        case O_SUM: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc + a[i]; break;
        case O_PROD: acc = 1; for (int64_t i = 0; i < n; i++) acc = acc * a[i]; break;
        case O_MAX: acc = 0; for (int64_t i = 0; i < n; i++) if (a[i] > acc) acc = a[i]; break;
        case O_MIN: acc = 0xffffffffu; for (int64_t i = 0; i < n; i++) if (a[i] < acc) acc = a[i]; break;
        case O_AND: acc = 0xffffffffu; for (int64_t i = 0; i < n; i++) acc = acc & a[i]; break;
        case O_OR: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc | a[i]; break;
        case O_XOR: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc ^ a[i]; break;
        default: return -1;
        }
        *(uint32_t*)out = acc;
        return 0;
    }
    if (dtype == O_I64) {
        const int64_t* a = (const int64_t*)x;
        uint64_t acc;
        switch (op) {
        case O_SUM: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc + (uint64_t)a[i]; break;
        case O_PROD: acc = 1; for (int64_t i = 0; i < n; i++) acc = acc * (uint64_t)a[i]; break;
        case O_MAX: { int64_t m = INT64_MIN; for (int64_t i = 0; i < n; i++) if (a[i] > m) m = a[i]; acc = (uint64_t)m; break; }
        case O_MIN: { int64_t m = INT64_MAX; for (int64_t i = 0; i < n; i++) if (a[i] < m) m = a[i]; acc = (uint64_t)m; break; }
        case O_AND: acc = ~0ull; for (int64_t i = 0; i < n; i++) acc = acc & (uint64_t)a[i]; break;
        case O_OR: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc | (uint64_t)a[i]; break;
        case O_XOR: acc = 0; for (int64_t i = 0; i < n; i++) acc = acc ^ (uint64_t)a[i]; break;
        default: return -1;
        }
        memcpy(out, &acc, 8);
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Float max / min.  NaN propagates; -0 is ordered below +0.            */
/* ------------------------------------------------------------------ */

/* 1 if a is strictly greater than b in the order -inf < ... < -0 < +0 < ... < +inf */
static int float_gt(double a, double b) {
    if (a == 0.0 && b == 0.0) return !signbit(a) && signbit(b);
    return a > b;
}

/* Extremum and the first index attaining it.  For op == O_MAX a NaN is the
 * extremum (first NaN wins); likewise for O_MIN.  Empty input: identity and -1. */
int orc_argext(const void* x, int64_t n, int dtype, int op, double* val, int64_t* idx) {
    double best = (op == O_MAX) ? -INFINITY : INFINITY;
    int64_t bi = -1;
    for (int64_t i = 0; i < n; i++) {
        double v = elem_as_double(x, i, dtype);
        if (bi < 0) { best = v; bi = i; if (isnan(v)) break; continue; }
        if (isnan(v)) { best = v; bi = i; break; }          /* the first NaN is final */
        int better = (op == O_MAX) ? float_gt(v, best) : float_gt(best, v);
        if (better) { best = v; bi = i; }
    }
    *val = best;
    *idx = bi;
    return 0;
}

double orc_maxmin(const void* x, int64_t n, int dtype, int op) {
    double v;
    int64_t i;
    orc_argext(x, n, dtype, op, &v, &i);
    return v;
}

/* argmax / argmin over integer types: first index attaining the extremum. */
int orc_argext_int(const void* x, int64_t n, int dtype, int op, int64_t* idx) {
    int64_t bi = -1;
    for (int64_t i = 0; i < n; i++) {
        int better;
        if (bi < 0) better = 1;
        else if (dtype == O_I32) {
            int32_t a = ((const int32_t*)x)[i], b = ((const int32_t*)x)[bi];
            better = (op == O_MAX) ? a > b : a < b;
        } else if (dtype == O_U32) {
            uint32_t a = ((const uint32_t*)x)[i], b = ((const uint32_t*)x)[bi];
            better = (op == O_MAX) ? a > b : a < b;
        } else {
            int64_t a = ((const int64_t*)x)[i], b = ((const int64_t*)x)[bi];
            better = (op == O_MAX) ? a > b : a < b;
        }
        if (better) bi = i;
    }
    *idx = bi;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Product in double-double with a separate exponent.                   */
/* ------------------------------------------------------------------ */

/* Error-free product a*b = p + e (Dekker's TwoProduct, here via fma). */
static void two_prod(double a, double b, double* p, double* e) {
    *p = a * b;
    *e = fma(a, b, -*p);
}
/* Error-free sum a+b = s + e (Knuth's TwoSum). */
static void two_sum(double a, double b, double* s, double* e) {
    *s = a + b;
    double bb = *s - a;
    *e = (a - (*s - bb)) + (b - bb);
}

/* (hi, lo) * 2^ex, with hi kept in [0.5, 1). */
typedef struct { double hi, lo; int64_t ex; } ddexp;

static void dde_mul(ddexp* a, double v) {          /* v finite, non-zero */
    int ve;
    double vm = frexp(v, &ve);                        /* v = vm * 2^ve, |vm| in [0.5,1) */
    double p, e;
    two_prod(a->hi, vm, &p, &e);
    e += a->lo * vm;
    double s, t;
    two_sum(p, e, &s, &t);
    int se;
    double sm = frexp(s, &se);
    a->hi = sm;
    a->lo = ldexp(t, -se);
    a->ex += ve + se;
}

static double dde_to_double(const ddexp* a) {
    /* hi + lo rounded to double, then scaled.  ldexp is exact unless the result
     * over/underflows, where it gives the IEEE result of scaling. */
    double m = a->hi + a->lo;
    if (a->ex > 2000) return m > 0 ? INFINITY : -INFINITY;
    if (a->ex < -2200) return m > 0 ? 0.0 : -0.0;
    return ldexp(m, (int)a->ex);
}

/* Product of all elements.  Sign is the xor of the signs (IEEE rule for
 * multiplication, zeros included); NaN if any NaN or if inf meets zero. */
double orc_prod(const void* x, int64_t n, int dtype) {
    ddexp a = {0.5, 0.0, 1};                          /* 1.0 */
    int neg = 0, zero = 0, inf = 0, nan = 0;
    for (int64_t i = 0; i < n; i++) {
        double v = elem_as_double(x, i, dtype);
        if (isnan(v)) { nan = 1; continue; }
        if (signbit(v)) neg ^= 1;
        if (isinf(v)) { inf = 1; continue; }
        if (v == 0.0) { zero = 1; continue; }
        dde_mul(&a, fabs(v));
    }
    if (nan || (inf && zero)) return NAN;
    if (inf) return neg ? -INFINITY : INFINITY;
    if (zero) return neg ? -0.0 : 0.0;
    double r = dde_to_double(&a);
    return neg ? -r : r;
}

/* Same product but returned as significand in [0.5,1) and exponent, so a
 * caller can round to a narrower type (binary32) without double rounding of
 * the exponent range.  Only for finite non-zero products. */
int orc_prod_scaled(const void* x, int64_t n, int dtype, double* mant, int64_t* ex) {
    ddexp a = {0.5, 0.0, 1};
    int neg = 0;
    for (int64_t i = 0; i < n; i++) {
        double v = elem_as_double(x, i, dtype);
        if (!isfinite(v) || v == 0.0) return -1;
        if (signbit(v)) neg ^= 1;
        dde_mul(&a, fabs(v));
    }
    *mant = neg ? -(a.hi + a.lo) : (a.hi + a.lo);
    *ex = a.ex;
    return 0;
}

/* Product of the non-zero elements, the zero count and the first zero index
 * (-1 if none): everything the product's gradient needs. */
int orc_prod_aux(const void* x, int64_t n, int dtype, double* p_nz, int64_t* zcount, int64_t* zidx) {
    ddexp a = {0.5, 0.0, 1};
    int neg = 0;
    int64_t zc = 0, zi = -1;
    for (int64_t i = 0; i < n; i++) {
        double v = elem_as_double(x, i, dtype);
        if (v == 0.0) { if (zi < 0) zi = i; zc++; continue; }
        if (signbit(v)) neg ^= 1;
        dde_mul(&a, fabs(v));
    }
    double r = dde_to_double(&a);
    *p_nz = neg ? -r : r;
    *zcount = zc;
    *zidx = zi;
    return 0;
}

/* d/dx_i of prod_j x_j = prod_{j != i} x_j, straight from the definition. */
double orc_prod_except(const void* x, int64_t n, int dtype, int64_t skip) {
    ddexp a = {0.5, 0.0, 1};
    int neg = 0, zero = 0;
    for (int64_t i = 0; i < n; i++) {
        if (i == skip) continue;
        double v = elem_as_double(x, i, dtype);
        if (signbit(v)) neg ^= 1;
        if (v == 0.0) { zero = 1; continue; }
        dde_mul(&a, fabs(v));
    }
    if (zero) return neg ? -0.0 : 0.0;
    double r = dde_to_double(&a);
    return neg ? -r : r;
}

/* ------------------------------------------------------------------ */
/* Prefix scan (exact combiners)                                       */
/* ------------------------------------------------------------------ */

/* One step of an integer combiner on 64-bit two's-complement bits; `sgn`
 * selects signed order for max / min.  Sums and products wrap (the caller
 * truncates to the output width). */
static uint64_t int_step(uint64_t acc, uint64_t v, int op, int sgn) {
    switch (op) {
    case O_SUM: return acc + v;
    case O_PROD: return acc * v;
    case O_MAX: return sgn ? ((int64_t)v > (int64_t)acc ? v : acc) : (v > acc ? v : acc);
    case O_MIN: return sgn ? ((int64_t)v < (int64_t)acc ? v : acc) : (v < acc ? v : acc);
    case O_AND: return acc & v;
    case O_OR: return acc | v;
    default: return acc ^ v;
    }
}

/* y: int64 per element for i32 SUM (the sum widens), else the input's own
 * width for integers (two's complement); double values for float max/min. */
int orc_scan(const void* x, int64_t n, int dtype, int op, int exclusive, void* y) {
    if (dtype == O_I32 || dtype == O_U32 || dtype == O_I64) {
        const int sgn = dtype != O_U32;
        const int wide = dtype == O_I64 || (dtype == O_I32 && op == O_SUM);
        uint64_t acc;
        switch (op) {
        case O_SUM: case O_OR: case O_XOR: acc = 0; break;
        case O_PROD: acc = 1; break;
        case O_AND: acc = ~0ull; break;
        case O_MAX: acc = dtype == O_I64 ? (uint64_t)INT64_MIN : (dtype == O_I32 ? (uint64_t)(int64_t)INT32_MIN : 0); break;
        case O_MIN: acc = dtype == O_I64 ? (uint64_t)INT64_MAX : (dtype == O_I32 ? (uint64_t)INT32_MAX : 0xffffffffull); break;
        default: return -1;
        }
        for (int64_t i = 0; i < n; i++) {
            uint64_t v;
            if (dtype == O_I32) v = (uint64_t)(int64_t)((const int32_t*)x)[i];
            else if (dtype == O_U32) v = ((const uint32_t*)x)[i];
            else v = (uint64_t)((const int64_t*)x)[i];
            if (exclusive) {
                if (wide) ((uint64_t*)y)[i] = acc; else ((uint32_t*)y)[i] = (uint32_t)acc;
            }
            acc = int_step(acc, v, op, sgn);
            if (!wide && dtype == O_I32 && (op == O_MAX || op == O_MIN)) acc = (uint64_t)(int64_t)(int32_t)acc;
            if (!exclusive) {
                if (wide) ((uint64_t*)y)[i] = acc; else ((uint32_t*)y)[i] = (uint32_t)acc;
            }
        }
        return 0;
    }
    if (op != O_MAX && op != O_MIN) return -1;
    double best = (op == O_MAX) ? -INFINITY : INFINITY;
    for (int64_t i = 0; i < n; i++) {
        const double v = elem_as_double(x, i, dtype);
        if (exclusive) ((double*)y)[i] = best;
        if (!isnan(best)) {
            if (isnan(v)) best = v;                              /* NaN is final */
            else if ((op == O_MAX) ? float_gt(v, best) : float_gt(best, v)) best = v;
        }
        if (!exclusive) ((double*)y)[i] = best;
    }
    return 0;
}
