/*
 * trx oracle — plain FP64 CPU reference for BLAS TRSM and TRMM.
 *
 * TEST INFRASTRUCTURE ONLY. The library's product path never links, loads or
 * calls this file; only the test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes is the plain definition of the two operations of the paper
 * (Section 2.1):
 *   TRMM  B := alpha*op(A)*B            (side = 'L', Eq. 1)
 *         B := alpha*B*op(A)            (side = 'R', Eq. 2)
 *   TRSM  op(A)*X = alpha*B, X -> B     (side = 'L', Eq. 3)
 *         X*op(A) = alpha*B, X -> B     (side = 'R', Eq. 4)
 * with A triangular (upper/lower, unit/non-unit diagonal), op(A) = A or A^T
 * ('C' means A^T for real data). TRSM is forward or back substitution, one
 * right-hand side at a time; TRMM is a double loop over the referenced
 * triangle. Nothing is blocked, fused or reordered beyond that definition.
 * The recursive splitting of Section 3.1 reaches the same result (up to
 * rounding), which is why the plain definition is the oracle.
 *
 * Storage follows BLAS: column-major, element (i,j) of A at A[i + j*lda].
 * Only the referenced triangle of A is read; with diag = 'U' the diagonal is
 * not read and taken as 1. alpha == 0 sets B to zero without reading A (the
 * BLAS quick return). Arguments are checked in BLAS order; an illegal i-th
 * argument returns -i (side=1 ... ldb=11), nothing is written.
 *
 * Every right-hand side (column for side = 'L', row for side = 'R') is
 * independent, so the OpenMP loop over them gives bit-identical results for
 * any thread count.
 *
 * Parity status: pinned (exact rational brute force on tiny integer systems,
 * closed forms, round-trip and side-duality invariants, and a BLAS library
 * cross-check; see tests/test_oracle_pins.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int upc(char c) { return (c >= 'a' && c <= 'z') ? c - 'a' + 'A' : c; }

typedef struct {
    int left;    /* side == 'L' */
    int lower;   /* uplo == 'L' (storage) */
    int trans;   /* transa in {'T','C'} */
    int unit;    /* diag == 'U' */
    int64_t k;   /* order of A */
    const double* A;
    int64_t lda;
} tri_t;

/* Argument check in BLAS order (side, uplo, transa, diag, m, n, alpha, A,
 * lda, B, ldb). Returns 0 or -position. */
static int check_args(char side, char uplo, char transa, char diag,
                      int64_t m, int64_t n, const void* A, int64_t lda,
                      const void* B, int64_t ldb) {
    int s = upc(side), u = upc(uplo), t = upc(transa), d = upc(diag);
    if (s != 'L' && s != 'R') return -1;
    if (u != 'L' && u != 'U') return -2;
    if (t != 'N' && t != 'T' && t != 'C') return -3;
    if (d != 'N' && d != 'U') return -4;
    if (m < 0) return -5;
    if (n < 0) return -6;
    int64_t k = (s == 'L') ? m : n;
    if (m > 0 && n > 0 && A == NULL) return -8;
    if (lda < (k > 1 ? k : 1)) return -9;
    if (m > 0 && n > 0 && B == NULL) return -10;
    if (ldb < (m > 1 ? m : 1)) return -11;
    return 0;
}

static tri_t make_tri(char side, char uplo, char transa, char diag,
                      int64_t m, int64_t n, const double* A, int64_t lda) {
    tri_t t;
    t.left = upc(side) == 'L';
    t.lower = upc(uplo) == 'L';
    t.trans = upc(transa) != 'N';
    t.unit = upc(diag) == 'U';
    t.k = t.left ? m : n;
    t.A = A;
    t.lda = lda;
    return t;
}

/* op(A) is lower triangular iff (lower, no transpose) or (upper, transpose). */
static int op_lower(const tri_t* t) { return t->lower != t->trans; }

/* Element (i,l) of op(A), honouring the triangle and the diagonal rule:
 * zero outside the referenced triangle (A is not read there), 1 on the
 * diagonal when unit (A is not read there either). */
static double opa(const tri_t* t, int64_t i, int64_t l) {
    if (i == l && t->unit) return 1.0;
    int64_t r = t->trans ? l : i;   /* stored row    */
    int64_t c = t->trans ? i : l;   /* stored column */
    if (t->lower ? (r < c) : (r > c)) return 0.0;
    return t->A[r + c * t->lda];
}

static void zero_b(int64_t m, int64_t n, double* B, int64_t ldb) {
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) B[i + j * ldb] = 0.0;
}

int oracle_nthreads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* TRSM, Eq. 3-4: substitution in the order op(A)'s triangle dictates. */
int oracle_dtrsm(char side, char uplo, char transa, char diag, int64_t m,
                 int64_t n, double alpha, const double* A, int64_t lda,
                 double* B, int64_t ldb) {
    int info = check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (info) return info;
    if (m == 0 || n == 0) return 0;
    if (alpha == 0.0) { zero_b(m, n, B, ldb); return 0; }
    tri_t t = make_tri(side, uplo, transa, diag, m, n, A, lda);
    int lo = op_lower(&t);
    if (t.left) {
        /* op(A) x = alpha b for every column b of B; x overwrites b. */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t j = 0; j < n; ++j) {
            double* x = B + j * ldb;
            if (lo) {
                for (int64_t i = 0; i < m; ++i) {          /* forward */
                    double s = alpha * x[i];
                    for (int64_t l = 0; l < i; ++l) s -= opa(&t, i, l) * x[l];
                    x[i] = t.unit ? s : s / opa(&t, i, i);
                }
            } else {
                for (int64_t i = m - 1; i >= 0; --i) {     /* backward */
                    double s = alpha * x[i];
                    for (int64_t l = i + 1; l < m; ++l) s -= opa(&t, i, l) * x[l];
                    x[i] = t.unit ? s : s / opa(&t, i, i);
                }
            }
        }
    } else {
        /* x op(A) = alpha b for every row b of B: column i of the product
         * reads sum_l x_l op(A)(l,i). For lower op(A) that sum runs over
         * l >= i (solve from the last column), for upper over l <= i. */
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r = 0; r < m; ++r) {
            double* x = B + r;   /* element i at x[i*ldb] */
            if (lo) {
                for (int64_t i = n - 1; i >= 0; --i) {
                    double s = alpha * x[i * ldb];
                    for (int64_t l = i + 1; l < n; ++l) s -= x[l * ldb] * opa(&t, l, i);
                    x[i * ldb] = t.unit ? s : s / opa(&t, i, i);
                }
            } else {
                for (int64_t i = 0; i < n; ++i) {
                    double s = alpha * x[i * ldb];
                    for (int64_t l = 0; l < i; ++l) s -= x[l * ldb] * opa(&t, l, i);
                    x[i * ldb] = t.unit ? s : s / opa(&t, i, i);
                }
            }
        }
    }
    return 0;
}

/* TRMM, Eq. 1-2: each output element is alpha times the sum over the
 * referenced triangle; a per-thread temporary keeps the inputs intact. */
int oracle_dtrmm(char side, char uplo, char transa, char diag, int64_t m,
                 int64_t n, double alpha, const double* A, int64_t lda,
                 double* B, int64_t ldb) {
    int info = check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (info) return info;
    if (m == 0 || n == 0) return 0;
    if (alpha == 0.0) { zero_b(m, n, B, ldb); return 0; }
    tri_t t = make_tri(side, uplo, transa, diag, m, n, A, lda);
    int lo = op_lower(&t);
    int64_t len = t.left ? m : n;
    int err = 0;
#pragma omp parallel
    {
        double* tmp = (double*)malloc((size_t)len * sizeof(double));
        if (!tmp) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t v = 0; v < (t.left ? n : m); ++v) {
            if (!tmp) continue;
            if (t.left) {
                double* b = B + v * ldb;              /* column v */
                for (int64_t i = 0; i < m; ++i) {
                    int64_t l0 = lo ? 0 : i, l1 = lo ? i : m - 1;
                    double s = 0.0;
                    for (int64_t l = l0; l <= l1; ++l) s += opa(&t, i, l) * b[l];
                    tmp[i] = alpha * s;
                }
                for (int64_t i = 0; i < m; ++i) b[i] = tmp[i];
            } else {
                double* b = B + v;                    /* row v, stride ldb */
                for (int64_t i = 0; i < n; ++i) {
                    /* (b op(A))_i = sum_l b_l op(A)(l,i) */
                    int64_t l0 = lo ? i : 0, l1 = lo ? n - 1 : i;
                    double s = 0.0;
                    for (int64_t l = l0; l <= l1; ++l) s += b[l * ldb] * opa(&t, l, i);
                    tmp[i] = alpha * s;
                }
                for (int64_t i = 0; i < n; ++i) b[i * ldb] = tmp[i];
            }
        }
        free(tmp);
    }
    return err ? 1 : 0;
}

/* ---- error metrics ------------------------------------------------------
 * The residual of a computed solution has to be formed more accurately than
 * the working precision of the result it judges, or an FP64 result could not
 * be judged at all. Sums use the compensated dot product "Dot2" of Ogita,
 * Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005): error-free TwoSum
 * (Knuth) and TwoProduct (via a fused multiply-add), which returns the dot
 * product as if computed in twice the working precision. */
typedef struct { double s, c; } acc2_t;

static void acc2_add_prod(acc2_t* a, double x, double y) {
    double p = x * y;
    double pe = fma(x, y, -p);          /* x*y = p + pe exactly */
    double s = a->s + p;
    double z = s - a->s;
    double se = (a->s - (s - z)) + (p - z); /* a->s + p = s + se exactly */
    a->s = s;
    a->c += pe + se;
}

/* Normwise backward error of a computed TRSM result X (Eq. 3-4):
 *   side L: ||op(A) X - alpha B||_inf / (||op(A)||_inf ||X||_inf)
 *   side R: ||X op(A) - alpha B||_inf / (||X||_inf ||op(A)||_inf)
 * B is the original right-hand side. out[0] = eta, out[1] = ||R||,
 * out[2] = ||op(A)||, out[3] = ||X||. Returns an argument code as above. */
int oracle_trsm_backward_error(char side, char uplo, char transa, char diag,
                               int64_t m, int64_t n, double alpha,
                               const double* A, int64_t lda, const double* X,
                               int64_t ldx, const double* B, int64_t ldb,
                               double* out) {
    int info = check_args(side, uplo, transa, diag, m, n, A, lda, B, ldb);
    if (info) return info;
    if (ldx < (m > 1 ? m : 1)) return -12;
    tri_t t = make_tri(side, uplo, transa, diag, m, n, A, lda);
    int64_t k = t.k;
    double na = 0.0, nx = 0.0, nr = 0.0;
    for (int64_t i = 0; i < k; ++i) {
        double s = 0.0;
        for (int64_t l = 0; l < k; ++l) s += fabs(opa(&t, i, l));
        if (s > na || isnan(s)) na = s;
    }
    for (int64_t i = 0; i < m; ++i) {
        double s = 0.0;
        for (int64_t j = 0; j < n; ++j) s += fabs(X[i + j * ldx]);
        if (s > nx || isnan(s)) nx = s;
    }
    int any_nan = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(max : nr) reduction(| : any_nan)
    for (int64_t i = 0; i < m; ++i) {
        double rowsum = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            acc2_t a = {0.0, 0.0};
            if (t.left) {
                for (int64_t l = 0; l < m; ++l) {
                    double e = opa(&t, i, l);
                    if (e != 0.0) acc2_add_prod(&a, e, X[l + j * ldx]);
                }
            } else {
                for (int64_t l = 0; l < n; ++l) {
                    double e = opa(&t, l, j);
                    if (e != 0.0) acc2_add_prod(&a, X[i + l * ldx], e);
                }
            }
            acc2_add_prod(&a, -alpha, B[i + j * ldb]);
            double r = a.s + a.c;
            rowsum += fabs(r);
            if (isnan(r)) any_nan = 1;
        }
        if (rowsum > nr) nr = rowsum;
    }
    if (any_nan) nr = NAN;
    out[1] = nr;
    out[2] = na;
    out[3] = nx;
    out[0] = (na > 0.0 && nx > 0.0) ? nr / (na * nx) : (nr == 0.0 ? 0.0 : INFINITY);
    return 0;
}

/* ||op(A)||_inf for the referenced triangle (1 on a unit diagonal). */
double oracle_op_norm_inf(char uplo, char transa, char diag, int64_t k,
                          const double* A, int64_t lda) {
    tri_t t = make_tri('L', uplo, transa, diag, k, 1, A, lda);
    double na = 0.0;
    for (int64_t i = 0; i < k; ++i) {
        double s = 0.0;
        for (int64_t l = 0; l < k; ++l) s += fabs(opa(&t, i, l));
        if (s > na) na = s;
    }
    return na;
}
