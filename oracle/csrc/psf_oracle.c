/*
 * psf_oracle.c -- plain, slow CPU FP64 reference for the filtered
 * Paterson-Stockmeyer scheme (PSSCF) of "A filtering technique for the matrix
 * power series being near-sparse" (Wu, Zhu, Zhao, Zhang).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code, header or table
 * with the CUDA library.
 *
 * Conventions (fixed readings of the paper, written out once here):
 *  - Matrices are square CSR, 0-based, columns strictly increasing per row,
 *    and hold only nonzero values: an entry that evaluates to exactly 0 is
 *    not stored (the sparse-matrix semantics the paper's experiments use).
 *  - Every product C = Init + A*B is Gustavson's row-by-row form: for output
 *    row r the accumulator starts from Init's row r, then for each k in A's
 *    row r in ascending column order, every entry (k, j) of B is folded in as
 *    acc[j] = fma(a_rk, b_kj, acc[j]).  fma() is the IEEE-754 fused
 *    multiply-add (one rounding).  This fixes the rounding order.
 *  - The matrix norm is the 1-norm (largest column sum of absolute values),
 *    the norm Higham's normest1 estimates (Sec. 2.2, Sec. 3.2.2).  Column sums
 *    are computed EXACTLY and rounded once to nearest-even, by a fixed-point
 *    accumulator that spans the whole double range; the result is therefore
 *    independent of summation order.
 *  - Algorithm 1 (Sec. 3.1.1) keeps an entry iff |x| > eps_f (strict), and
 *    always runs its first pass (eps_f = eps_g); see or_alg1().
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ENOMEM 2
#define OR_ENOTCONV 4

/* ------------------------------------------------------------------------ */
/* Exact sum of non-negative doubles.                                        */
/* A double x >= 0 equals M * 2^(s - 1074) with M < 2^53 an integer and s the */
/* bit position of M's least significant bit above 2^-1074:                  */
/*   normal    (biased exponent E >= 1): M = 2^52 | fraction, s = E - 1      */
/*   subnormal (E == 0):                 M = fraction,        s = 0          */
/* so every double is an integer multiple of 2^-1074 that fits below 2^2098. */
/* The accumulator is that integer, in 64-bit words, with 78 spare bits.     */
/* ------------------------------------------------------------------------ */
#define XS_WORDS 34 /* 34 * 64 = 2176 bits */

static void xs_add(uint64_t* w, double x) {
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    uint64_t E = (bits >> 52) & 0x7ffu;
    uint64_t frac = bits & ((1ull << 52) - 1);
    if (E == 0 && frac == 0) return;
    uint64_t M = E ? (frac | (1ull << 52)) : frac;
    int s = E ? (int)E - 1 : 0;
    int word = s / 64, sh = s % 64;
    uint64_t lo = M << sh;
    uint64_t hi = sh ? (M >> (64 - sh)) : 0;
    /* add lo into w[word], hi into w[word+1], ripple the carries upward */
    uint64_t old = w[word];
    w[word] = old + lo;
    uint64_t carry = (w[word] < old);
    int i = word + 1;
    uint64_t add = hi;
    while ((add | carry) && i < XS_WORDS) {
        old = w[i];
        uint64_t t = old + add;
        uint64_t c1 = (t < old);
        uint64_t t2 = t + carry;
        uint64_t c2 = (t2 < t);
        w[i] = t2;
        carry = c1 | c2;
        add = 0;
        ++i;
    }
}

static int xs_bit(const uint64_t* w, int p) { return (int)((w[p / 64] >> (p % 64)) & 1u); }

/* Round the accumulated integer (times 2^-1074) to the nearest double, ties
 * to even. */
static double xs_round(const uint64_t* w) {
    int top = -1;
    for (int i = XS_WORDS - 1; i >= 0 && top < 0; --i)
        if (w[i]) top = i * 64 + 63 - __builtin_clzll(w[i]);
    if (top < 0) return 0.0;
    uint64_t bits;
    if (top <= 52) {
        /* value < 2^53 * 2^-1074: representable as is; as a bit pattern the
         * integer itself is the subnormal (or smallest-normal) encoding */
        bits = w[0];
    } else {
        int shift = top - 52; /* bits [shift, top] form the 53-bit significand */
        uint64_t M = 0;
        for (int p = top; p >= shift; --p) M = (M << 1) | (uint64_t)xs_bit(w, p);
        int round = xs_bit(w, shift - 1);
        int sticky = 0;
        for (int p = shift - 2; p >= 0 && !sticky; --p) sticky = xs_bit(w, p);
        if (round && (sticky || (M & 1u))) {
            M += 1;
            if (M == (1ull << 53)) {
                M >>= 1;
                shift += 1;
            }
        }
        uint64_t E = (uint64_t)shift + 1; /* value = M * 2^(E - 1075) */
        if (E >= 2047) return INFINITY;
        bits = (E << 52) | (M & ((1ull << 52) - 1));
    }
    double out;
    memcpy(&out, &bits, sizeof out);
    return out;
}

/* exact, correctly rounded sum of |x[i]|, i < len (used by the tests to pin
 * the accumulator against an independent correctly rounded sum) */
double or_exact_abs_sum(const double* x, int64_t len) {
    uint64_t w[XS_WORDS];
    memset(w, 0, sizeof w);
    for (int64_t i = 0; i < len; ++i) xs_add(w, fabs(x[i]));
    return xs_round(w);
}

/* Largest exact column sum of |x| over the entries of a CSR matrix whose
 * magnitude is <= limit (limit = INFINITY takes every entry): the 1-norm of
 * that sub-matrix. */
static double colsum_max(int32_t n, const int32_t* rp, const int32_t* ci, const double* v,
                         double limit, int* err) {
    uint64_t* acc = (uint64_t*)calloc((size_t)n * XS_WORDS + 1, sizeof(uint64_t));
    if (!acc) {
        *err = OR_ENOMEM;
        return 0.0;
    }
    for (int32_t r = 0; r < n; ++r)
        for (int32_t p = rp[r]; p < rp[r + 1]; ++p) {
            double a = fabs(v[p]);
            if (a <= limit) xs_add(acc + (size_t)ci[p] * XS_WORDS, a);
        }
    double best = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        double s = xs_round(acc + (size_t)j * XS_WORDS);
        if (s > best) best = s;
    }
    free(acc);
    return best;
}

/* ||M||_1, exact column sums rounded once (Sec. 2.2: z_i bounds ||Z^i||). */
int or_norm1(int32_t n, const int32_t* rp, const int32_t* ci, const double* v, double* out) {
    int err = OR_OK;
    *out = colsum_max(n, rp, ci, v, INFINITY, &err);
    return err;
}

void or_free(void* p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Sparse kernels (all results hold nonzero values only, sorted columns).    */
/* ------------------------------------------------------------------------ */

/* Emit the nonzero entries of a dense accumulator row, in column order, for
 * the columns listed in `mark_list` (unsorted) -- sorted here by a counting
 * pass over the marker array. */
typedef struct {
    int32_t n;
    double* acc;      /* n */
    int32_t* mark;    /* n, stamp of the row that last touched the column */
    int32_t* touched; /* n, columns touched by the current row */
    int32_t ntouched;
} dense_row_t;

static int dense_row_init(dense_row_t* d, int32_t n) {
    d->n = n;
    d->acc = (double*)calloc((size_t)n + 1, sizeof(double));
    d->mark = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    d->touched = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    d->ntouched = 0;
    if (!d->acc || !d->mark || !d->touched) return OR_ENOMEM;
    for (int32_t j = 0; j < n; ++j) d->mark[j] = -1;
    return OR_OK;
}

static void dense_row_free(dense_row_t* d) {
    free(d->acc);
    free(d->mark);
    free(d->touched);
}

static void touch(dense_row_t* d, int32_t r, int32_t j) {
    if (d->mark[j] != r) {
        d->mark[j] = r;
        d->acc[j] = 0.0;
        d->touched[d->ntouched++] = j;
    }
}

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* growable CSR output */
typedef struct {
    int32_t n;
    int32_t* rp;
    int32_t* ci;
    double* v;
    int64_t nnz, cap;
} out_csr_t;

static int out_init(out_csr_t* o, int32_t n) {
    o->n = n;
    o->nnz = 0;
    o->cap = 1024;
    o->rp = (int32_t*)malloc(((size_t)n + 1) * sizeof(int32_t));
    o->ci = (int32_t*)malloc((size_t)o->cap * sizeof(int32_t));
    o->v = (double*)malloc((size_t)o->cap * sizeof(double));
    if (!o->rp || !o->ci || !o->v) return OR_ENOMEM;
    o->rp[0] = 0;
    return OR_OK;
}

static int out_push(out_csr_t* o, int32_t j, double x) {
    if (o->nnz == o->cap) {
        int64_t cap = o->cap * 2;
        int32_t* ci = (int32_t*)realloc(o->ci, (size_t)cap * sizeof(int32_t));
        if (!ci) return OR_ENOMEM;
        o->ci = ci;
        double* v = (double*)realloc(o->v, (size_t)cap * sizeof(double));
        if (!v) return OR_ENOMEM;
        o->v = v;
        o->cap = cap;
    }
    o->ci[o->nnz] = j;
    o->v[o->nnz] = x;
    o->nnz++;
    return OR_OK;
}

/* flush the accumulator row r: nonzero values, ascending columns */
static int flush_row(dense_row_t* d, out_csr_t* o, int32_t r) {
    qsort(d->touched, (size_t)d->ntouched, sizeof(int32_t), cmp_i32);
    for (int32_t t = 0; t < d->ntouched; ++t) {
        int32_t j = d->touched[t];
        double x = d->acc[j];
        if (x != 0.0)
            if (out_push(o, j, x)) return OR_ENOMEM;
    }
    d->ntouched = 0;
    if (o->nnz > INT32_MAX) return OR_ENOMEM;
    o->rp[r + 1] = (int32_t)o->nnz;
    return OR_OK;
}

static void out_export(out_csr_t* o, int32_t** rp, int32_t** ci, double** v, int64_t* nnz) {
    *rp = o->rp;
    *ci = o->ci;
    *v = o->v;
    *nnz = o->nnz;
}

static void out_free(out_csr_t* o) {
    free(o->rp);
    free(o->ci);
    free(o->v);
}

/*
 * C = Init + A * B.  Init may be absent (irp == NULL).  The accumulator of
 * row r is seeded with Init's row r, then folds the products in the order
 * stated at the top of this file.  Used for every matrix product of the
 * scheme: Eq. (11) (Init absent) and Eq. (14) (Init = B-hat).
 */
int or_matmul_add(int32_t n, const int32_t* arp, const int32_t* aci, const double* av,
                  const int32_t* brp, const int32_t* bci, const double* bv, const int32_t* irp,
                  const int32_t* ici, const double* iv, int32_t** orp, int32_t** oci,
                  double** ov, int64_t* onnz) {
    dense_row_t d;
    out_csr_t o;
    int err = dense_row_init(&d, n);
    if (!err) err = out_init(&o, n);
    if (err) {
        dense_row_free(&d);
        return OR_ENOMEM;
    }
    for (int32_t r = 0; r < n && !err; ++r) {
        if (irp)
            for (int32_t p = irp[r]; p < irp[r + 1]; ++p) {
                touch(&d, r, ici[p]);
                d.acc[ici[p]] = iv[p];
            }
        for (int32_t p = arp[r]; p < arp[r + 1]; ++p) {
            int32_t k = aci[p];
            double a = av[p];
            for (int32_t e = brp[k]; e < brp[k + 1]; ++e) {
                int32_t j = bci[e];
                touch(&d, r, j);
                d.acc[j] = fma(a, bv[e], d.acc[j]);
            }
        }
        err = flush_row(&d, &o, r);
    }
    dense_row_free(&d);
    if (err) {
        out_free(&o);
        return err;
    }
    out_export(&o, orp, oci, ov, onnz);
    return OR_OK;
}

/*
 * Y = alpha * M + X, entry by entry as y = fma(alpha, m, x) (x = 0 where X has
 * no entry), with M = I when mrp == NULL.  X may be absent (xrp == NULL).
 * B-hat_i of Eq. (13) / Alg. 2 is built by repeated calls in ascending j.
 */
int or_axpy(int32_t n, double alpha, const int32_t* mrp, const int32_t* mci, const double* mv,
            const int32_t* xrp, const int32_t* xci, const double* xv, int32_t** orp,
            int32_t** oci, double** ov, int64_t* onnz) {
    dense_row_t d;
    out_csr_t o;
    int err = dense_row_init(&d, n);
    if (!err) err = out_init(&o, n);
    if (err) {
        dense_row_free(&d);
        return OR_ENOMEM;
    }
    for (int32_t r = 0; r < n && !err; ++r) {
        if (xrp)
            for (int32_t p = xrp[r]; p < xrp[r + 1]; ++p) {
                touch(&d, r, xci[p]);
                d.acc[xci[p]] = xv[p];
            }
        if (mrp) {
            for (int32_t p = mrp[r]; p < mrp[r + 1]; ++p) {
                touch(&d, r, mci[p]);
                d.acc[mci[p]] = fma(alpha, mv[p], d.acc[mci[p]]);
            }
        } else {
            touch(&d, r, r);
            d.acc[r] = fma(alpha, 1.0, d.acc[r]);
        }
        err = flush_row(&d, &o, r);
    }
    dense_row_free(&d);
    if (err) {
        out_free(&o);
        return err;
    }
    out_export(&o, orp, oci, ov, onnz);
    return OR_OK;
}

/*
 * Algorithm 1 (Sec. 3.1.1): adaptive filter with filtering-norm-threshold
 * eps_g and tolerance e_r.  State: the scalar m_i, the norm c_i of the
 * candidate matrix c_i (entries of C not yet kept), the threshold eps_f.
 *
 *   i = 0, m_0 = 1, candidate matrix = C
 *   repeat (the first pass always runs):
 *       eps_f <- eps_g / m_i
 *       entries of the candidate matrix with |x| > eps_f leave it (kept)
 *       c_{i+1} <- || candidate matrix ||_1
 *       m_{i+1} <- c_{i+1} / eps_f
 *       i <- i + 1
 *   while c_i > eps_g (1 + e_r)
 *   C-hat = C - candidate matrix  (= entries with |x| > final eps_f)
 *
 * Since eps_f only decreases, the candidate matrix after a pass is exactly
 * the set of entries of C with |x| <= eps_f, and its norm is computed over
 * that set directly.  Returns OR_ENOTCONV after maxit passes.
 * Outputs: kept matrix, final eps_f, pass count, final c (dropped norm).
 */
int or_alg1(int32_t n, const int32_t* rp, const int32_t* ci, const double* v, double eps_g,
            double e_r, int32_t maxit, int32_t** orp, int32_t** oci, double** ov,
            int64_t* onnz, double* eps_f_out, int32_t* iters_out, double* c_out) {
    double bound = eps_g * (1.0 + e_r);
    double m = 1.0;
    double eps_f = eps_g;
    double c = 0.0;
    int32_t it = 0;
    int err = OR_OK;
    for (;;) {
        eps_f = eps_g / m;
        c = colsum_max(n, rp, ci, v, eps_f, &err);
        if (err) return err;
        m = c / eps_f;
        ++it;
        if (!(c > bound)) break;
        if (it >= maxit) {
            err = OR_ENOTCONV;
            break;
        }
    }
    out_csr_t o;
    if (out_init(&o, n)) return OR_ENOMEM;
    for (int32_t r = 0; r < n; ++r) {
        for (int32_t p = rp[r]; p < rp[r + 1]; ++p)
            if (fabs(v[p]) > eps_f)
                if (out_push(&o, ci[p], v[p])) {
                    out_free(&o);
                    return OR_ENOMEM;
                }
        o.rp[r + 1] = (int32_t)o.nnz;
    }
    out_export(&o, orp, oci, ov, onnz);
    *eps_f_out = eps_f;
    *iters_out = it;
    *c_out = c;
    return err;
}

/*
 * Dense Horner evaluation P_N(Z) = sum_{i<N} a_i Z^i (Eq. 1, the Qin/Horner
 * scheme named in Sec. 1): S <- a_{N-1} I; S <- a_i I + Z S for i = N-2..0.
 * Z and the result are n x n row-major.  Used by tests on small matrices.
 */
int or_horner_dense(int32_t n, const double* Z, const double* a, int32_t N, double* out) {
    double* S = (double*)calloc((size_t)n * n, sizeof(double));
    double* T = (double*)calloc((size_t)n * n, sizeof(double));
    if (!S || !T) {
        free(S);
        free(T);
        return OR_ENOMEM;
    }
    for (int32_t r = 0; r < n; ++r) S[(size_t)r * n + r] = a[N - 1];
    for (int32_t i = N - 2; i >= 0; --i) {
        for (int32_t r = 0; r < n; ++r)
            for (int32_t c = 0; c < n; ++c) {
                double acc = (r == c) ? a[i] : 0.0;
                for (int32_t k = 0; k < n; ++k)
                    acc = fma(Z[(size_t)r * n + k], S[(size_t)k * n + c], acc);
                T[(size_t)r * n + c] = acc;
            }
        double* t = S;
        S = T;
        T = t;
    }
    memcpy(out, S, (size_t)n * n * sizeof(double));
    free(S);
    free(T);
    return OR_OK;
}

/*
 * y = M x for a CSR matrix M (n rows): each y_r is a chain of fma() over
 * row r's entries in stored order, starting from +0.  The 1-norm estimator
 * (oracle/normest.py) applies Z^k and its transpose with it.
 */
void or_spmv(int32_t n, const int32_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
    for (int32_t r = 0; r < n; ++r) {
        double acc = 0.0;
        for (int32_t p = rp[r]; p < rp[r + 1]; ++p) acc = fma(v[p], x[ci[p]], acc);
        y[r] = acc;
    }
}
