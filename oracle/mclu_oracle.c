/*
 * mclu_oracle.c - CPU oracle for complex multi-component (DD/TD/QD) LU with
 * partial pivoting, the matching solve, complex ZGEMM (3M/4M) and the solve's
 * adjoint.  TEST INFRASTRUCTURE ONLY: it is called by the test-suite, by the
 * package's smoke check and by the benchmark's CPU-baseline leg, never by the
 * library.  It shares no code with the CUDA path.
 *
 * Build: plain C11, binary64 round-to-nearest-even, -ffp-contract=off (no
 * contraction of a*b+c), no -ffast-math, OpenMP for the outer loops only.
 *
 * Multi-component arithmetic (the paper's DD/TD/QD types, Sec. 1-2: a value is
 * the unevaluated sum of L binary64 limbs, L = 2, 3, 4).  The paper cites its
 * DD/TD/QD operations but does not print them, so this oracle defines every
 * real operation as "the exact result, rounded to L limbs":
 *   - sums and products of limbs are expanded without error with TwoSum
 *     (Knuth) and FMA-based TwoProd (a*b = p + e exactly),
 *   - the resulting vector of doubles is normalised by repeating the
 *     bottom-up VecSum pass (Ogita, Rump & Oishi 2005, "Accurate sum and dot
 *     product", Alg. 4.3) until a pass changes nothing.  Every pass is
 *     error-free, and at the fixed point each component is the rounded sum of
 *     itself and the next one, which is therefore below half its ulp: a
 *     nonoverlapping expansion in decreasing order,
 *   - the first L components are the result; only the dropped tail is lost
 *     (relative error below ~2^(-52L)).
 * Division is long division with exact remainders (L+1 quotient digits).
 *
 * Complex operations follow Sec. 2.1: 4M product, Eq. (1); 3M product, Eq. (2)
 * with Im = T3 - (T1 + T2); 3M matrix product, Eq. (3).  Reciprocal of a + bi is
 * (a - bi)/(a^2 + b^2), the complex counterpart of the "inv" operation of Sec. 2.2.
 *
 * LU (Sec. 3): unblocked right-looking Gaussian elimination ("Normal LU"),
 * k-i-j order, partial pivoting on cabs1(z) = |Re z| + |Im z| evaluated exactly,
 * ties to the lowest row index, column scaled by the reciprocal of the pivot,
 * info = first exactly-zero pivot (1-based), LAPACK-style ipiv (1-based, row k
 * swapped with row ipiv[k]-1, applied for k = 0..n-1).
 *
 * Solve (Sec. 4, "forward and backward substitutions"): P b, unit-lower
 * forward substitution, upper back substitution with division by u_kk; the
 * conjugate-transpose solve applies U^H, L^H, then P^T.
 *
 * Exact residual: b - A x accumulated without any rounding in a fixed-point
 * superaccumulator over the exact TwoProd parts of every limb product, then
 * rounded greedily to binary64 limbs.
 *
 * Storage: complex L-limb matrices as 2L column-major binary64 planes; plane
 * (c, l) (c = 0 real, 1 imaginary) starts at A + (c*L + l)*ld*ncols and element
 * (i, j) of a plane is at offset j*ld + i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXL 4
#define MAXT 96

static int g_err = 0; /* sticky: a normalisation did not reach its fixed point or a buffer overflowed */

/* g_err is set from OpenMP threads: every access is atomic */
static void set_err(int bit) { __atomic_fetch_or(&g_err, bit, __ATOMIC_RELAXED); }
int orc_error_flag(void) { return __atomic_load_n(&g_err, __ATOMIC_RELAXED); }
void orc_clear_error(void) { __atomic_store_n(&g_err, 0, __ATOMIC_RELAXED); }
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------- EFTs -- */

/* Knuth's TwoSum: s = RN(a+b), e = (a+b) - s exactly, for any a, b. */
static void two_sum(double a, double b, double *s, double *e) {
  double x = a + b;
  double bv = x - a;
  double av = x - bv;
  double br = b - bv;
  double ar = a - av;
  *s = x;
  *e = ar + br;
}

/* TwoProd with a fused multiply-add: p = RN(a*b), e = a*b - p exactly
 * (when no underflow occurs in e). */
static void two_prod(double a, double b, double *p, double *e) {
  double x = a * b;
  *p = x;
  *e = fma(a, b, -x);
}

/* --------------------------------------------------- normalisation -- */

/* Drop zeros, sort by decreasing magnitude, then repeat the bottom-up VecSum
 * pass until it leaves the vector unchanged.  The exact sum is preserved.
 * Returns the number of nonzero components. */
static int normalize(double *v, int m) {
  int k = 0;
  for (int i = 0; i < m; i++)
    if (v[i] != 0.0) v[k++] = v[i];
  m = k;
  for (int i = 1; i < m; i++) {
    double x = v[i];
    int j = i - 1;
    while (j >= 0 && fabs(v[j]) < fabs(x)) {
      v[j + 1] = v[j];
      j--;
    }
    v[j + 1] = x;
  }
  int limit = 8 * m + 16;
  for (int pass = 0; pass < limit; pass++) {
    if (m <= 1) return m;
    int changed = 0;
    double s = v[m - 1];
    for (int i = m - 2; i >= 0; i--) {
      double hi, lo;
      two_sum(v[i], s, &hi, &lo);
      if (lo != v[i + 1]) changed = 1;
      v[i + 1] = lo;
      s = hi;
    }
    if (s != v[0]) changed = 1;
    v[0] = s;
    /* zeros created by the pass are removed (order of the rest is kept) */
    k = 0;
    for (int i = 0; i < m; i++)
      if (v[i] != 0.0) v[k++] = v[i];
    if (k != m) changed = 1;
    m = k;
    if (!changed) return m;
  }
  set_err(1);
  return m;
}

/* First L components of the normalised expansion (zero padded). */
static void round_to_limbs(double *v, int m, int L, double *z) {
  m = normalize(v, m);
  for (int i = 0; i < L; i++) z[i] = i < m ? v[i] : 0.0;
}

/* ------------------------------------------------ real MC operations -- */

static void mc_add(int L, const double *a, const double *b, double *z) {
  double t[2 * MAXL];
  int m = 0;
  for (int i = 0; i < L; i++) t[m++] = a[i];
  for (int i = 0; i < L; i++) t[m++] = b[i];
  round_to_limbs(t, m, L, z);
}

static void mc_neg(int L, const double *a, double *z) {
  for (int i = 0; i < L; i++) z[i] = -a[i];
}

static void mc_sub(int L, const double *a, const double *b, double *z) {
  double nb[MAXL] = {0};
  mc_neg(L, b, nb);
  mc_add(L, a, nb, z);
}

/* Exact product of all limb pairs, rounded to L limbs. */
static void mc_mul(int L, const double *a, const double *b, double *z) {
  double t[2 * MAXL * MAXL];
  int m = 0;
  for (int i = 0; i < L; i++)
    for (int j = 0; j < L; j++) {
      double p, e;
      two_prod(a[i], b[j], &p, &e);
      t[m++] = p;
      t[m++] = e;
    }
  round_to_limbs(t, m, L, z);
}

/* Long division: q_k = RN(r_k[0] / b[0]) and r_{k+1} = r_k - q_k*b, kept as an
 * exact normalised expansion; L+1 digits, then rounded to L limbs. */
static void mc_div(int L, const double *a, const double *b, double *z) {
  double bn[MAXT];
  for (int i = 0; i < L; i++) bn[i] = b[i];
  int mb = normalize(bn, L);
  if (mb == 0) { /* division by zero: IEEE semantics on the leading limb */
    z[0] = a[0] / 0.0;
    for (int i = 1; i < L; i++) z[i] = 0.0;
    return;
  }
  double r[MAXT];
  int mr = 0;
  for (int i = 0; i < L; i++) r[mr++] = a[i];
  mr = normalize(r, mr);
  double q[MAXL + 2];
  int nq = 0;
  for (int k = 0; k <= L; k++) {
    if (mr == 0) break;
    double qk = r[0] / bn[0];
    q[nq++] = qk;
    if (mr + 2 * mb > MAXT) { set_err(2); break; }
    for (int j = 0; j < mb; j++) {
      double p, e;
      two_prod(qk, bn[j], &p, &e);
      r[mr++] = -p;
      r[mr++] = -e;
    }
    mr = normalize(r, mr);
  }
  round_to_limbs(q, nq, L, z);
}

/* Sign of the exact value of an L-limb number. */
static int mc_sign(int L, const double *a) {
  double t[MAXL];
  for (int i = 0; i < L; i++) t[i] = a[i];
  int m = normalize(t, L);
  if (m == 0) return 0;
  return t[0] > 0 ? 1 : -1;
}

static void mc_abs(int L, const double *a, double *z) {
  if (mc_sign(L, a) < 0)
    mc_neg(L, a, z);
  else
    for (int i = 0; i < L; i++) z[i] = a[i];
}

/* Exact comparison of a and b: sign of the exact difference. */
static int mc_cmp(int L, const double *a, const double *b) {
  double t[2 * MAXL];
  int m = 0;
  for (int i = 0; i < L; i++) t[m++] = a[i];
  for (int i = 0; i < L; i++) t[m++] = -b[i];
  m = normalize(t, m);
  if (m == 0) return 0;
  return t[0] > 0 ? 1 : -1;
}

/* --------------------------------------------- complex MC operations -- */

typedef struct {
  double re[MAXL], im[MAXL];
} cmc;

static void c_add(int L, const cmc *a, const cmc *b, cmc *z) {
  mc_add(L, a->re, b->re, z->re);
  mc_add(L, a->im, b->im, z->im);
}

static void c_sub(int L, const cmc *a, const cmc *b, cmc *z) {
  mc_sub(L, a->re, b->re, z->re);
  mc_sub(L, a->im, b->im, z->im);
}

/* Eq. (1): (Re a Re b - Im a Im b) + (Im a Re b + Re a Im b) i */
static void c_mul4m(int L, const cmc *a, const cmc *b, cmc *z) {
  double t1[MAXL], t2[MAXL], t3[MAXL], t4[MAXL];
  mc_mul(L, a->re, b->re, t1);
  mc_mul(L, a->im, b->im, t2);
  mc_mul(L, a->im, b->re, t3);
  mc_mul(L, a->re, b->im, t4);
  mc_sub(L, t1, t2, z->re);
  mc_add(L, t3, t4, z->im);
}

/* Eq. (2): t1 = Re a Re b, t2 = Im a Im b, Re = t1 - t2,
 * Im = (Re a + Im a)(Re b + Im b) - (t1 + t2). */
static void c_mul3m(int L, const cmc *a, const cmc *b, cmc *z) {
  double t1[MAXL], t2[MAXL], sa[MAXL], sb[MAXL], t3[MAXL], t12[MAXL];
  mc_mul(L, a->re, b->re, t1);
  mc_mul(L, a->im, b->im, t2);
  mc_add(L, a->re, a->im, sa);
  mc_add(L, b->re, b->im, sb);
  mc_mul(L, sa, sb, t3);
  mc_add(L, t1, t2, t12);
  mc_sub(L, t1, t2, z->re);
  mc_sub(L, t3, t12, z->im);
}

/* 1/(a + b i) = (a - b i)/(a^2 + b^2) */
static void c_inv(int L, const cmc *a, cmc *z) {
  double aa[MAXL], bb[MAXL], d[MAXL], one[MAXL] = {1.0, 0.0, 0.0, 0.0}, r[MAXL];
  mc_mul(L, a->re, a->re, aa);
  mc_mul(L, a->im, a->im, bb);
  mc_add(L, aa, bb, d);
  mc_div(L, one, d, r);
  double nim[MAXL];
  mc_mul(L, a->re, r, z->re);
  mc_mul(L, a->im, r, nim);
  mc_neg(L, nim, z->im);
}

/* a / b = a conj(b) / |b|^2, with the real divisions done by long division */
static void c_div(int L, const cmc *a, const cmc *b, cmc *z) {
  cmc cb, num;
  for (int i = 0; i < L; i++) {
    cb.re[i] = b->re[i];
    cb.im[i] = -b->im[i];
  }
  c_mul4m(L, a, &cb, &num);
  double aa[MAXL], bb[MAXL], d[MAXL];
  mc_mul(L, b->re, b->re, aa);
  mc_mul(L, b->im, b->im, bb);
  mc_add(L, aa, bb, d);
  mc_div(L, num.re, d, z->re);
  mc_div(L, num.im, d, z->im);
}

/* cabs1(z) = |Re z| + |Im z| rounded to L limbs */
static void c_abs1(int L, const cmc *a, double *z) {
  double x[MAXL], y[MAXL];
  mc_abs(L, a->re, x);
  mc_abs(L, a->im, y);
  mc_add(L, x, y, z);
}

/* Exact cabs1 as a normalised expansion (for pivot comparisons). */
static int c_abs1_exact(int L, const cmc *a, double *t) {
  int m = 0;
  int sr = mc_sign(L, a->re), si = mc_sign(L, a->im);
  for (int i = 0; i < L; i++) t[m++] = sr < 0 ? -a->re[i] : a->re[i];
  for (int i = 0; i < L; i++) t[m++] = si < 0 ? -a->im[i] : a->im[i];
  return normalize(t, m);
}

static int exp_cmp(double *a, int ma, double *b, int mb) {
  double t[4 * MAXL];
  int m = 0;
  for (int i = 0; i < ma; i++) t[m++] = a[i];
  for (int i = 0; i < mb; i++) t[m++] = -b[i];
  m = normalize(t, m);
  if (m == 0) return 0;
  return t[0] > 0 ? 1 : -1;
}

/* ------------------------------------------------------ matrix access -- */

static inline size_t pofs(int L, int c, int l, int64_t ld, int64_t ncols) {
  return ((size_t)(c * L + l)) * (size_t)ld * (size_t)ncols;
}

static void ld_elem(int L, const double *A, int64_t ld, int64_t ncols, int64_t i, int64_t j, cmc *z) {
  size_t o = (size_t)j * ld + i;
  for (int l = 0; l < L; l++) {
    z->re[l] = A[pofs(L, 0, l, ld, ncols) + o];
    z->im[l] = A[pofs(L, 1, l, ld, ncols) + o];
  }
}

static void st_elem(int L, double *A, int64_t ld, int64_t ncols, int64_t i, int64_t j, const cmc *z) {
  size_t o = (size_t)j * ld + i;
  for (int l = 0; l < L; l++) {
    A[pofs(L, 0, l, ld, ncols) + o] = z->re[l];
    A[pofs(L, 1, l, ld, ncols) + o] = z->im[l];
  }
}

static void swap_rows(int L, double *A, int64_t ld, int64_t ncols, int64_t r1, int64_t r2) {
  if (r1 == r2) return;
  for (int c = 0; c < 2; c++)
    for (int l = 0; l < L; l++) {
      double *P = A + pofs(L, c, l, ld, ncols);
      for (int64_t j = 0; j < ncols; j++) {
        double t = P[j * ld + r1];
        P[j * ld + r1] = P[j * ld + r2];
        P[j * ld + r2] = t;
      }
    }
}

/* ------------------------------------------- elementwise entry points -- */

/* Real ops on arrays of L-limb values stored limb-major: x[l*count + e]. */
enum { ORC_ADD = 0, ORC_SUB = 1, ORC_MUL = 2, ORC_DIV = 3 };

int orc_real_op(int op, int L, int64_t count, const double *x, const double *y, double *z) {
  if (L < 2 || L > MAXL) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < count; e++) {
    double a[MAXL] = {0}, b[MAXL] = {0}, r[MAXL] = {0};
    for (int l = 0; l < L; l++) {
      a[l] = x[l * count + e];
      b[l] = y[l * count + e];
    }
    switch (op) {
      case ORC_ADD: mc_add(L, a, b, r); break;
      case ORC_SUB: mc_sub(L, a, b, r); break;
      case ORC_MUL: mc_mul(L, a, b, r); break;
      default: mc_div(L, a, b, r); break;
    }
    for (int l = 0; l < L; l++) z[l * count + e] = r[l];
  }
  return 0;
}

/* Complex ops on vectors in plane layout [2][L][count]. */
enum { ORC_CADD = 0, ORC_CSUB = 1, ORC_CMUL4M = 2, ORC_CMUL3M = 3, ORC_CDIV = 4, ORC_CINV = 5, ORC_CABS1 = 6 };

int orc_cplx_op(int op, int L, int64_t count, const double *x, const double *y, double *z) {
  if (L < 2 || L > MAXL) return -2;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < count; e++) {
    cmc a, b, r;
    ld_elem(L, x, count, 1, e, 0, &a);
    if (y) ld_elem(L, y, count, 1, e, 0, &b);
    memset(&r, 0, sizeof r);
    switch (op) {
      case ORC_CADD: c_add(L, &a, &b, &r); break;
      case ORC_CSUB: c_sub(L, &a, &b, &r); break;
      case ORC_CMUL4M: c_mul4m(L, &a, &b, &r); break;
      case ORC_CMUL3M: c_mul3m(L, &a, &b, &r); break;
      case ORC_CDIV: c_div(L, &a, &b, &r); break;
      case ORC_CINV: c_inv(L, &a, &r); break;
      default: c_abs1(L, &a, r.re); break;
    }
    st_elem(L, z, count, 1, e, 0, &r);
  }
  return 0;
}

/* EFT exposure for pinning: s,e = TwoSum(a,b); p,f = TwoProd(a,b). */
void orc_eft(int64_t count, const double *a, const double *b, double *s, double *e, double *p, double *f) {
  for (int64_t i = 0; i < count; i++) {
    two_sum(a[i], b[i], &s[i], &e[i]);
    two_prod(a[i], b[i], &p[i], &f[i]);
  }
}

/* Normalise each row of a [count][m] array in place; returns the lengths. */
void orc_normalize_rows(int64_t count, int m, double *v, int32_t *len) {
  for (int64_t i = 0; i < count; i++) len[i] = normalize(v + i * m, m);
}

/* ------------------------------------------------------------- LU -- */

/*
 * Unblocked right-looking complex GEPP (Sec. 3, "Normal LU").
 * A: n x n planes, leading dimension lda (plane stride lda*n), overwritten by
 * L\U.  ipiv: int32[n], 1-based.  info: first zero pivot (1-based) or 0.
 * gap (optional, double[n]): for each step the relative gap between the two
 * largest exact cabs1 keys, (k1 - k2)/k1 in binary64 (1 if fewer than two
 * candidates or k1 = 0).
 */
int orc_zgetrf(int L, int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, double *gap) {
  if (L < 2 || L > MAXL) return -1;
  if (n < 0) return -2;
  if (lda < (n > 1 ? n : 1)) return -4;
  *info = 0;
  double *keys = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * 2 * MAXL);
  int *klen = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!keys || !klen) { free(keys); free(klen); return -100; }
  for (int64_t k = 0; k < n; k++) {
    /* exact cabs1 keys of the candidates */
#pragma omp parallel for schedule(static)
    for (int64_t i = k; i < n; i++) {
      cmc z;
      ld_elem(L, A, lda, n, i, k, &z);
      klen[i] = c_abs1_exact(L, &z, keys + (size_t)i * 2 * MAXL);
    }
    int64_t p = k;
    for (int64_t i = k + 1; i < n; i++)
      if (exp_cmp(keys + (size_t)i * 2 * MAXL, klen[i], keys + (size_t)p * 2 * MAXL, klen[p]) > 0) p = i;
    if (gap) {
      double k1 = klen[p] ? keys[(size_t)p * 2 * MAXL] : 0.0, k2 = 0.0;
      int have2 = 0;
      for (int64_t i = k; i < n; i++) {
        if (i == p) continue;
        double v = klen[i] ? keys[(size_t)i * 2 * MAXL] : 0.0;
        if (!have2 || v > k2) k2 = v;
        have2 = 1;
      }
      gap[k] = (have2 && k1 > 0.0) ? (k1 - k2) / k1 : 1.0;
    }
    ipiv[k] = (int32_t)(p + 1);
    if (klen[p] == 0) {
      if (*info == 0) *info = (int32_t)(k + 1);
      continue;
    }
    swap_rows(L, A, lda, n, k, p);
    cmc piv, r;
    ld_elem(L, A, lda, n, k, k, &piv);
    c_inv(L, &piv, &r);
#pragma omp parallel for schedule(static)
    for (int64_t i = k + 1; i < n; i++) {
      cmc a, l;
      ld_elem(L, A, lda, n, i, k, &a);
      c_mul4m(L, &a, &r, &l);
      st_elem(L, A, lda, n, i, k, &l);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = k + 1; j < n; j++) {
      cmc u;
      ld_elem(L, A, lda, n, k, j, &u);
      for (int64_t i = k + 1; i < n; i++) {
        cmc l, a, t, z;
        ld_elem(L, A, lda, n, i, k, &l);
        ld_elem(L, A, lda, n, i, j, &a);
        c_mul4m(L, &l, &u, &t);
        c_sub(L, &a, &t, &z);
        st_elem(L, A, lda, n, i, j, &z);
      }
    }
  }
  free(keys);
  free(klen);
  return orc_error_flag() ? 1 : 0;
}

/*
 * Solve with the factors of orc_zgetrf.  trans 'N': A X = B; 'C': A^H X = B.
 * B: n x nrhs planes (plane stride ldb*nrhs), overwritten by X.
 */
int orc_zgetrs(int L, char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv,
               double *B, int64_t ldb) {
  if (L < 2 || L > MAXL) return -1;
  if (trans != 'N' && trans != 'C') return -2;
  if (n < 0) return -3;
  if (nrhs < 0) return -4;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nrhs; c++) {
    cmc x, y, a, t;
    if (trans == 'N') {
      for (int64_t k = 0; k < n; k++) {
        int64_t p = ipiv[k] - 1;
        if (p != k) {
          ld_elem(L, B, ldb, nrhs, k, c, &x);
          ld_elem(L, B, ldb, nrhs, p, c, &y);
          st_elem(L, B, ldb, nrhs, k, c, &y);
          st_elem(L, B, ldb, nrhs, p, c, &x);
        }
      }
      for (int64_t k = 0; k < n; k++) { /* unit lower */
        ld_elem(L, B, ldb, nrhs, k, c, &x);
        for (int64_t i = k + 1; i < n; i++) {
          ld_elem(L, A, lda, n, i, k, &a);
          ld_elem(L, B, ldb, nrhs, i, c, &y);
          c_mul4m(L, &a, &x, &t);
          c_sub(L, &y, &t, &y);
          st_elem(L, B, ldb, nrhs, i, c, &y);
        }
      }
      for (int64_t k = n - 1; k >= 0; k--) { /* upper */
        ld_elem(L, B, ldb, nrhs, k, c, &x);
        ld_elem(L, A, lda, n, k, k, &a);
        c_div(L, &x, &a, &x);
        st_elem(L, B, ldb, nrhs, k, c, &x);
        for (int64_t i = 0; i < k; i++) {
          ld_elem(L, A, lda, n, i, k, &a);
          ld_elem(L, B, ldb, nrhs, i, c, &y);
          c_mul4m(L, &a, &x, &t);
          c_sub(L, &y, &t, &y);
          st_elem(L, B, ldb, nrhs, i, c, &y);
        }
      }
    } else {
      /* U^H w = b: lower triangular, row k of U^H is conj(U[:, k]) */
      for (int64_t k = 0; k < n; k++) {
        ld_elem(L, B, ldb, nrhs, k, c, &x);
        ld_elem(L, A, lda, n, k, k, &a);
        for (int l = 0; l < L; l++) a.im[l] = -a.im[l];
        c_div(L, &x, &a, &x);
        st_elem(L, B, ldb, nrhs, k, c, &x);
        for (int64_t i = k + 1; i < n; i++) {
          ld_elem(L, A, lda, n, k, i, &a); /* U[k, i] -> (U^H)[i, k] = conj */
          for (int l = 0; l < L; l++) a.im[l] = -a.im[l];
          ld_elem(L, B, ldb, nrhs, i, c, &y);
          c_mul4m(L, &a, &x, &t);
          c_sub(L, &y, &t, &y);
          st_elem(L, B, ldb, nrhs, i, c, &y);
        }
      }
      /* L^H z = w: unit upper, (L^H)[i, k] = conj(L[k, i]) */
      for (int64_t k = n - 1; k >= 0; k--) {
        ld_elem(L, B, ldb, nrhs, k, c, &x);
        for (int64_t i = 0; i < k; i++) {
          ld_elem(L, A, lda, n, k, i, &a);
          for (int l = 0; l < L; l++) a.im[l] = -a.im[l];
          ld_elem(L, B, ldb, nrhs, i, c, &y);
          c_mul4m(L, &a, &x, &t);
          c_sub(L, &y, &t, &y);
          st_elem(L, B, ldb, nrhs, i, c, &y);
        }
      }
      /* x = P^T z: undo the swaps in reverse order */
      for (int64_t k = n - 1; k >= 0; k--) {
        int64_t p = ipiv[k] - 1;
        if (p != k) {
          ld_elem(L, B, ldb, nrhs, k, c, &x);
          ld_elem(L, B, ldb, nrhs, p, c, &y);
          st_elem(L, B, ldb, nrhs, k, c, &y);
          st_elem(L, B, ldb, nrhs, p, c, &x);
        }
      }
    }
  }
  return orc_error_flag() ? 1 : 0;
}

/*
 * C = A B (beta_mode 0) or C = C - A B (beta_mode 1), A m x k, B k x n, plain
 * triple loop with k ascending (Sec. 2.2 "simple matrix multiplication").
 * method 0: 4M, each product by Eq. (1) and accumulated in L-limb arithmetic;
 * method 1: 3M at the matrix level, Eq. (3): T1 = ReA ReB, T2 = ImA ImB,
 * T3 = (ReA + ImA)(ReB + ImB), Re = T1 - T2, Im = T3 - (T1 + T2).
 */
int orc_zgemm(int L, int method, int beta_mode, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
              const double *B, int64_t ldb, double *C, int64_t ldc) {
  if (L < 2 || L > MAXL) return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; j++) {
    for (int64_t i = 0; i < m; i++) {
      cmc acc, a, b, t, c;
      memset(&acc, 0, sizeof acc);
      if (method == 0) {
        for (int64_t q = 0; q < k; q++) {
          ld_elem(L, A, lda, k, i, q, &a);
          ld_elem(L, B, ldb, n, q, j, &b);
          c_mul4m(L, &a, &b, &t);
          c_add(L, &acc, &t, &acc);
        }
      } else {
        double T1[MAXL] = {0}, T2[MAXL] = {0}, T3[MAXL] = {0}, p[MAXL], sa[MAXL], sb[MAXL];
        for (int64_t q = 0; q < k; q++) {
          ld_elem(L, A, lda, k, i, q, &a);
          ld_elem(L, B, ldb, n, q, j, &b);
          mc_mul(L, a.re, b.re, p);
          mc_add(L, T1, p, T1);
          mc_mul(L, a.im, b.im, p);
          mc_add(L, T2, p, T2);
          mc_add(L, a.re, a.im, sa);
          mc_add(L, b.re, b.im, sb);
          mc_mul(L, sa, sb, p);
          mc_add(L, T3, p, T3);
        }
        double T12[MAXL];
        mc_sub(L, T1, T2, acc.re);
        mc_add(L, T1, T2, T12);
        mc_sub(L, T3, T12, acc.im);
      }
      if (beta_mode == 1) {
        ld_elem(L, C, ldc, n, i, j, &c);
        c_sub(L, &c, &acc, &acc);
      }
      st_elem(L, C, ldc, n, i, j, &acc);
    }
  }
  return orc_error_flag() ? 1 : 0;
}

/* ------------------------------------------------- superaccumulator -- */

#define SA_BIAS 1280
#define SA_WORDS 82

typedef struct {
  int64_t w[SA_WORDS];
  int64_t adds;
} superacc;

static void sa_carry(superacc *s) {
  for (int k = 0; k < SA_WORDS - 1; k++) {
    int64_t c = s->w[k] >> 32; /* arithmetic shift: floor division */
    s->w[k] -= c * ((int64_t)1 << 32);
    s->w[k + 1] += c;
  }
  s->adds = 0;
}

static void sa_add(superacc *s, double v) {
  if (v == 0.0) return;
  int e;
  double m = frexp(v, &e);
  int64_t mi = (int64_t)ldexp(m, 53);
  int p = e - 53 + SA_BIAS;
  uint64_t a = mi < 0 ? (uint64_t)(-mi) : (uint64_t)mi;
  int wi = p >> 5, sh = p & 31;
  unsigned __int128 x = ((unsigned __int128)a) << sh;
  int64_t d0 = (int64_t)(uint64_t)(x & 0xffffffffu);
  int64_t d1 = (int64_t)(uint64_t)((x >> 32) & 0xffffffffu);
  int64_t d2 = (int64_t)(uint64_t)(x >> 64);
  if (mi < 0) {
    s->w[wi] -= d0;
    s->w[wi + 1] -= d1;
    s->w[wi + 2] -= d2;
  } else {
    s->w[wi] += d0;
    s->w[wi + 1] += d1;
    s->w[wi + 2] += d2;
  }
  if (++s->adds >= ((int64_t)1 << 28)) sa_carry(s);
}

static void sa_add_prod(superacc *s, double a, double b) {
  double p, e;
  two_prod(a, b, &p, &e);
  sa_add(s, p);
  sa_add(s, e);
}

/* Round the exact value to the nearest binary64 (ties to even). */
static double sa_round(superacc *s) {
  sa_carry(s);
  int neg = s->w[SA_WORDS - 1] < 0;
  uint64_t mag[SA_WORDS];
  if (neg) { /* two's complement negation of the base-2^32 digits */
    int64_t carry = 0;
    for (int k = 0; k < SA_WORDS; k++) {
      int64_t v = -s->w[k] + carry;
      carry = v >> 32;
      mag[k] = (uint64_t)(v - carry * ((int64_t)1 << 32));
    }
  } else {
    for (int k = 0; k < SA_WORDS; k++) mag[k] = (uint64_t)s->w[k];
  }
  int h = SA_WORDS - 1;
  while (h >= 0 && mag[h] == 0) h--;
  if (h < 0) return 0.0;
  int tb = 31;
  while (!((mag[h] >> tb) & 1)) tb--;
  int top = h * 32 + tb; /* position of the leading bit */
  int lsb = top - 52;    /* position of the last kept bit */
  uint64_t mant = 0;
  for (int b = top; b >= lsb; b--) {
    uint64_t bit = b >= 0 ? (mag[b >> 5] >> (b & 31)) & 1 : 0;
    mant = (mant << 1) | bit;
  }
  int round = 0, sticky = 0;
  int rb = lsb - 1; /* round bit position; everything below it is sticky */
  if (rb >= 0) {
    round = (int)((mag[rb >> 5] >> (rb & 31)) & 1);
    uint64_t below = mag[rb >> 5] & ((((uint64_t)1) << (rb & 31)) - 1);
    sticky = below != 0;
    for (int q = (rb >> 5) - 1; q >= 0 && !sticky; q--)
      if (mag[q]) sticky = 1;
  }
  if (round && (sticky || (mant & 1))) mant += 1;
  double r = ldexp((double)mant, lsb - SA_BIAS);
  return neg ? -r : r;
}

/* Greedy rounding to L limbs: l_k = RN(v - l_0 - ... - l_{k-1}). */
static void sa_round_limbs(superacc *s, int L, double *out) {
  for (int l = 0; l < L; l++) {
    double r = sa_round(s);
    out[l] = r;
    sa_add(s, -r);
  }
}

/*
 * R = B - A X exactly, rounded to Lr limbs (Lr <= 4): A n x n (L limbs), X
 * n x nrhs (Lx limbs), B n x nrhs (Lb limbs), R planes [2][Lr][nrhs][n].
 */
int orc_exact_residual(int L, int Lx, int Lb, int Lr, int64_t n, int64_t nrhs, const double *A, int64_t lda,
                       const double *X, int64_t ldx, const double *B, int64_t ldb, double *R) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < n * nrhs; t++) {
    int64_t i = t % n, c = t / n;
    superacc sr, si;
    memset(&sr, 0, sizeof sr);
    memset(&si, 0, sizeof si);
    for (int l = 0; l < Lb; l++) {
      sa_add(&sr, B[pofs(Lb, 0, l, ldb, nrhs) + (size_t)c * ldb + i]);
      sa_add(&si, B[pofs(Lb, 1, l, ldb, nrhs) + (size_t)c * ldb + i]);
    }
    for (int64_t j = 0; j < n; j++) {
      for (int la = 0; la < L; la++) {
        double ar = A[pofs(L, 0, la, lda, n) + (size_t)j * lda + i];
        double ai = A[pofs(L, 1, la, lda, n) + (size_t)j * lda + i];
        for (int lx = 0; lx < Lx; lx++) {
          double xr = X[pofs(Lx, 0, lx, ldx, nrhs) + (size_t)c * ldx + j];
          double xi = X[pofs(Lx, 1, lx, ldx, nrhs) + (size_t)c * ldx + j];
          sa_add_prod(&sr, -ar, xr);
          sa_add_prod(&sr, ai, xi);
          sa_add_prod(&si, -ar, xi);
          sa_add_prod(&si, -ai, xr);
        }
      }
    }
    double lr[MAXL], li[MAXL];
    sa_round_limbs(&sr, Lr, lr);
    sa_round_limbs(&si, Lr, li);
    for (int l = 0; l < Lr; l++) {
      R[pofs(Lr, 0, l, n, nrhs) + (size_t)c * n + i] = lr[l];
      R[pofs(Lr, 1, l, n, nrhs) + (size_t)c * n + i] = li[l];
    }
  }
  return 0;
}

/*
 * Exact complex dot products at sampled positions: out_s = beta*C[r,c] + sum_q
 * A[r,q] B[q,c] (beta in {0, -1} meaning C - AB when -1 is applied to the
 * product: sign = -1 gives C - AB, sign = +1 gives AB), rounded to 4 limbs.
 * A: m x k (La limbs), B: k x n (Lb limbs), C: m x n (Lc limbs) or NULL.
 * out: [nsamp][2][4].
 * If lower_unit != 0, A is treated as unit lower triangular (the L factor of an
 * LU: A[r,q] = 0 for q > r, 1 for q == r) and B as upper (B[q,c] = 0 for q > c).
 */
int orc_exact_entries(int La, int Lb, int Lc, int64_t m, int64_t n, int64_t k, const double *A, int64_t lda,
                      const double *B, int64_t ldb, const double *C, int64_t ldc, int sign, int lower_unit,
                      int64_t nsamp, const int64_t *rows, const int64_t *cols, double *out) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < nsamp; s++) {
    int64_t r = rows[s], c = cols[s];
    superacc sr, si;
    memset(&sr, 0, sizeof sr);
    memset(&si, 0, sizeof si);
    if (C) {
      for (int l = 0; l < Lc; l++) {
        sa_add(&sr, C[pofs(Lc, 0, l, ldc, n) + (size_t)c * ldc + r]);
        sa_add(&si, C[pofs(Lc, 1, l, ldc, n) + (size_t)c * ldc + r]);
      }
    }
    double sg = sign < 0 ? -1.0 : 1.0;
    for (int64_t q = 0; q < k; q++) {
      if (lower_unit && (q > r || q > c)) break;
      if (lower_unit && q == r) { /* unit diagonal of L: add B[q, c] */
        for (int lb = 0; lb < Lb; lb++) {
          sa_add(&sr, sg * B[pofs(Lb, 0, lb, ldb, n) + (size_t)c * ldb + q]);
          sa_add(&si, sg * B[pofs(Lb, 1, lb, ldb, n) + (size_t)c * ldb + q]);
        }
        continue;
      }
      for (int la = 0; la < La; la++) {
        double ar = A[pofs(La, 0, la, lda, k) + (size_t)q * lda + r];
        double ai = A[pofs(La, 1, la, lda, k) + (size_t)q * lda + r];
        for (int lb = 0; lb < Lb; lb++) {
          double br = B[pofs(Lb, 0, lb, ldb, n) + (size_t)c * ldb + q];
          double bi = B[pofs(Lb, 1, lb, ldb, n) + (size_t)c * ldb + q];
          sa_add_prod(&sr, sg * ar, br);
          sa_add_prod(&sr, -sg * ai, bi);
          sa_add_prod(&si, sg * ar, bi);
          sa_add_prod(&si, sg * ai, br);
        }
      }
    }
    double lr[MAXL], li[MAXL];
    sa_round_limbs(&sr, 4, lr);
    sa_round_limbs(&si, 4, li);
    for (int l = 0; l < 4; l++) {
      out[s * 8 + l] = lr[l];
      out[s * 8 + 4 + l] = li[l];
    }
  }
  return 0;
}

/* Exact sum of each row of a [count][m] array, rounded greedily to L limbs. */
void orc_exact_sum_rows(int64_t count, int m, const double *v, int L, double *out) {
  for (int64_t i = 0; i < count; i++) {
    superacc s;
    memset(&s, 0, sizeof s);
    for (int j = 0; j < m; j++) sa_add(&s, v[i * m + j]);
    sa_round_limbs(&s, L, out + i * L);
  }
}

/*
 * Adjoint of x = A^{-1} b for a real loss with gradient xbar = dLoss/dx
 * (conjugate-Wirtinger convention): lambda = A^{-H} xbar, bbar = lambda,
 * Abar = -lambda x^H.  LU, ipiv: factors of A.  xbar is overwritten by lambda
 * (planes n x 1), Abar: n x n planes (leading dimension ldab).
 */
int orc_adjoint(int L, int64_t n, const double *LU, int64_t lda, const int32_t *ipiv, const double *x,
                double *xbar, double *Abar, int64_t ldab) {
  int rc = orc_zgetrs(L, 'C', n, 1, LU, lda, ipiv, xbar, n);
  if (rc < 0) return rc;
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; j++) {
    cmc xj, li, t;
    ld_elem(L, x, n, 1, j, 0, &xj);
    for (int l = 0; l < L; l++) xj.im[l] = -xj.im[l];
    for (int64_t i = 0; i < n; i++) {
      ld_elem(L, xbar, n, 1, i, 0, &li);
      c_mul4m(L, &li, &xj, &t);
      for (int l = 0; l < L; l++) {
        t.re[l] = -t.re[l];
        t.im[l] = -t.im[l];
      }
      st_elem(L, Abar, ldab, n, i, j, &t);
    }
  }
  return orc_error_flag() ? 1 : 0;
}

/*
 * Ill-conditioned test matrix A = Q1 diag(sigma) Q2^H in L-limb arithmetic
 * (Lout = L): Q = H_1 ... H_h, H = I - 2 v v^H / (v^H v), from binary64
 * vectors V1, V2 ([h][2][n]); sigma_i = r^i (r binary64, powers in L-limb
 * arithmetic).  A: n x n planes (ld = n).  Formation: start from diag(sigma),
 * apply Q2^H from the right (A <- A H_j for j = h..1, H Hermitian), then Q1
 * from the left (A <- H_j A for j = h..1).
 */
static void apply_reflector(int L, int64_t n, double *A, const double *v, int left) {
  /* w = 2 / (v^H v) */
  double nrm[MAXL] = {0}, t[MAXL], two[MAXL] = {2.0, 0, 0, 0}, w[MAXL];
  for (int64_t i = 0; i < n; i++) {
    double vr[MAXL] = {v[i], 0, 0, 0}, vi[MAXL] = {v[n + i], 0, 0, 0};
    mc_mul(L, vr, vr, t);
    mc_add(L, nrm, t, nrm);
    mc_mul(L, vi, vi, t);
    mc_add(L, nrm, t, nrm);
  }
  mc_div(L, two, nrm, w);
#pragma omp parallel for schedule(static)
  for (int64_t s = 0; s < n; s++) {
    /* left: column s of A: a <- a - w v (v^H a);  right: row s of A: a <- a - w (a v) v^H */
    cmc acc, e, vv, p;
    memset(&acc, 0, sizeof acc);
    for (int64_t i = 0; i < n; i++) {
      memset(&vv, 0, sizeof vv);
      vv.re[0] = v[i];
      vv.im[0] = left ? -v[n + i] : v[n + i]; /* conj(v_i) for v^H a */
      if (left)
        ld_elem(L, A, n, n, i, s, &e);
      else
        ld_elem(L, A, n, n, s, i, &e);
      c_mul4m(L, &vv, &e, &p);
      c_add(L, &acc, &p, &acc);
    }
    cmc ws;
    mc_mul(L, acc.re, w, ws.re);
    mc_mul(L, acc.im, w, ws.im);
    for (int64_t i = 0; i < n; i++) {
      memset(&vv, 0, sizeof vv);
      vv.re[0] = v[i];
      vv.im[0] = left ? v[n + i] : -v[n + i]; /* v_i (left) or conj(v_i) (right) */
      c_mul4m(L, &ws, &vv, &p);
      if (left) {
        ld_elem(L, A, n, n, i, s, &e);
        c_sub(L, &e, &p, &e);
        st_elem(L, A, n, n, i, s, &e);
      } else {
        ld_elem(L, A, n, n, s, i, &e);
        c_sub(L, &e, &p, &e);
        st_elem(L, A, n, n, s, i, &e);
      }
    }
  }
}

int orc_make_ill_conditioned(int L, int64_t n, int h, const double *V1, const double *V2, double r, double *A) {
  memset(A, 0, sizeof(double) * 2 * L * (size_t)n * (size_t)n);
  double sig[MAXL] = {1.0, 0, 0, 0}, rr[MAXL] = {r, 0, 0, 0};
  for (int64_t i = 0; i < n; i++) {
    for (int l = 0; l < L; l++) A[pofs(L, 0, l, n, n) + (size_t)i * n + i] = sig[l];
    mc_mul(L, sig, rr, sig);
  }
  for (int j = h - 1; j >= 0; j--) apply_reflector(L, n, A, V2 + (size_t)j * 2 * n, 0);
  for (int j = h - 1; j >= 0; j--) apply_reflector(L, n, A, V1 + (size_t)j * 2 * n, 1);
  return orc_error_flag() ? 1 : 0;
}

/* ------------------------------------------------ real LU and solve -- */

/*
 * The real multi-component LU that the complex one builds on (the author's
 * earlier real DD/TD/QD LU, Sec. 1; the same blocked/"Normal" structure,
 * Sec. 3), one plane per limb: limb plane l of a real L-limb matrix starts at
 * A + l*ld*ncols, element (i, j) at offset j*ld + i.  Pivot = argmax of the
 * exact |a_ik| over i >= k, ties to the lowest row; the column is scaled by
 * the MC reciprocal 1/a_kk (long division of 1 by the pivot, the "inv" of
 * Sec. 2.2); a_ij -= l_ik u_kj with the MC product and difference; info =
 * first exactly-zero pivot; gap as in orc_zgetrf.
 */
static inline size_t rofs(int l, int64_t ld, int64_t ncols) { return (size_t)l * (size_t)ld * (size_t)ncols; }

static void ld_rel(int L, const double *A, int64_t ld, int64_t ncols, int64_t i, int64_t j, double *z) {
  size_t o = (size_t)j * ld + i;
  for (int l = 0; l < L; l++) z[l] = A[rofs(l, ld, ncols) + o];
}

static void st_rel(int L, double *A, int64_t ld, int64_t ncols, int64_t i, int64_t j, const double *z) {
  size_t o = (size_t)j * ld + i;
  for (int l = 0; l < L; l++) A[rofs(l, ld, ncols) + o] = z[l];
}

static void swap_rows_real(int L, double *A, int64_t ld, int64_t ncols, int64_t r1, int64_t r2) {
  if (r1 == r2) return;
  for (int l = 0; l < L; l++) {
    double *P = A + rofs(l, ld, ncols);
    for (int64_t j = 0; j < ncols; j++) {
      double t = P[j * ld + r1];
      P[j * ld + r1] = P[j * ld + r2];
      P[j * ld + r2] = t;
    }
  }
}

/* Exact |a| as a normalised expansion (for pivot comparisons). */
static int abs_exact(int L, const double *a, double *t) {
  int s = mc_sign(L, a);
  for (int i = 0; i < L; i++) t[i] = s < 0 ? -a[i] : a[i];
  return normalize(t, L);
}

int orc_dgetrf(int L, int64_t n, double *A, int64_t lda, int32_t *ipiv, int32_t *info, double *gap) {
  if (L < 2 || L > MAXL) return -1;
  if (n < 0) return -2;
  if (lda < (n > 1 ? n : 1)) return -4;
  *info = 0;
  double *keys = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * MAXL);
  int *klen = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  if (!keys || !klen) { free(keys); free(klen); return -100; }
  const double one[MAXL] = {1.0, 0.0, 0.0, 0.0};
  for (int64_t k = 0; k < n; k++) {
#pragma omp parallel for schedule(static)
    for (int64_t i = k; i < n; i++) {
      double z[MAXL];
      ld_rel(L, A, lda, n, i, k, z);
      klen[i] = abs_exact(L, z, keys + (size_t)i * MAXL);
    }
    int64_t p = k;
    for (int64_t i = k + 1; i < n; i++)
      if (exp_cmp(keys + (size_t)i * MAXL, klen[i], keys + (size_t)p * MAXL, klen[p]) > 0) p = i;
    if (gap) {
      double k1 = klen[p] ? keys[(size_t)p * MAXL] : 0.0, k2 = 0.0;
      int have2 = 0;
      for (int64_t i = k; i < n; i++) {
        if (i == p) continue;
        double v = klen[i] ? keys[(size_t)i * MAXL] : 0.0;
        if (!have2 || v > k2) k2 = v;
        have2 = 1;
      }
      gap[k] = (have2 && k1 > 0.0) ? (k1 - k2) / k1 : 1.0;
    }
    ipiv[k] = (int32_t)(p + 1);
    if (klen[p] == 0) {
      if (*info == 0) *info = (int32_t)(k + 1);
      continue;
    }
    swap_rows_real(L, A, lda, n, k, p);
    double piv[MAXL], r[MAXL];
    ld_rel(L, A, lda, n, k, k, piv);
    mc_div(L, one, piv, r);
#pragma omp parallel for schedule(static)
    for (int64_t i = k + 1; i < n; i++) {
      double a[MAXL], l[MAXL];
      ld_rel(L, A, lda, n, i, k, a);
      mc_mul(L, a, r, l);
      st_rel(L, A, lda, n, i, k, l);
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = k + 1; j < n; j++) {
      double u[MAXL];
      ld_rel(L, A, lda, n, k, j, u);
      for (int64_t i = k + 1; i < n; i++) {
        double l[MAXL], a[MAXL], t[MAXL], z[MAXL];
        ld_rel(L, A, lda, n, i, k, l);
        ld_rel(L, A, lda, n, i, j, a);
        mc_mul(L, l, u, t);
        mc_sub(L, a, t, z);
        st_rel(L, A, lda, n, i, j, z);
      }
    }
  }
  free(keys);
  free(klen);
  return orc_error_flag() ? 1 : 0;
}

/*
 * Solve with the factors of orc_dgetrf.  trans 'N': A X = B; 'T': A^T X = B
 * (U^T, then L^T, then P^T).  B: n x nrhs limb planes (plane stride
 * ldb*nrhs), overwritten by X.
 */
int orc_dgetrs(int L, char trans, int64_t n, int64_t nrhs, const double *A, int64_t lda, const int32_t *ipiv,
               double *B, int64_t ldb) {
  if (L < 2 || L > MAXL) return -1;
  if (trans != 'N' && trans != 'T') return -2;
  if (n < 0) return -3;
  if (nrhs < 0) return -4;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nrhs; c++) {
    double x[MAXL], y[MAXL], a[MAXL], t[MAXL];
    if (trans == 'N') {
      for (int64_t k = 0; k < n; k++) {
        int64_t p = ipiv[k] - 1;
        if (p != k) {
          ld_rel(L, B, ldb, nrhs, k, c, x);
          ld_rel(L, B, ldb, nrhs, p, c, y);
          st_rel(L, B, ldb, nrhs, k, c, y);
          st_rel(L, B, ldb, nrhs, p, c, x);
        }
      }
      for (int64_t k = 0; k < n; k++) { /* unit lower */
        ld_rel(L, B, ldb, nrhs, k, c, x);
        for (int64_t i = k + 1; i < n; i++) {
          ld_rel(L, A, lda, n, i, k, a);
          ld_rel(L, B, ldb, nrhs, i, c, y);
          mc_mul(L, a, x, t);
          mc_sub(L, y, t, y);
          st_rel(L, B, ldb, nrhs, i, c, y);
        }
      }
      for (int64_t k = n - 1; k >= 0; k--) { /* upper */
        ld_rel(L, B, ldb, nrhs, k, c, x);
        ld_rel(L, A, lda, n, k, k, a);
        mc_div(L, x, a, x);
        st_rel(L, B, ldb, nrhs, k, c, x);
        for (int64_t i = 0; i < k; i++) {
          ld_rel(L, A, lda, n, i, k, a);
          ld_rel(L, B, ldb, nrhs, i, c, y);
          mc_mul(L, a, x, t);
          mc_sub(L, y, t, y);
          st_rel(L, B, ldb, nrhs, i, c, y);
        }
      }
    } else {
      /* U^T w = b: lower triangular, (U^T)[i, k] = U[k, i] */
      for (int64_t k = 0; k < n; k++) {
        ld_rel(L, B, ldb, nrhs, k, c, x);
        ld_rel(L, A, lda, n, k, k, a);
        mc_div(L, x, a, x);
        st_rel(L, B, ldb, nrhs, k, c, x);
        for (int64_t i = k + 1; i < n; i++) {
          ld_rel(L, A, lda, n, k, i, a);
          ld_rel(L, B, ldb, nrhs, i, c, y);
          mc_mul(L, a, x, t);
          mc_sub(L, y, t, y);
          st_rel(L, B, ldb, nrhs, i, c, y);
        }
      }
      /* L^T z = w: unit upper, (L^T)[i, k] = L[k, i] */
      for (int64_t k = n - 1; k >= 0; k--) {
        ld_rel(L, B, ldb, nrhs, k, c, x);
        for (int64_t i = 0; i < k; i++) {
          ld_rel(L, A, lda, n, k, i, a);
          ld_rel(L, B, ldb, nrhs, i, c, y);
          mc_mul(L, a, x, t);
          mc_sub(L, y, t, y);
          st_rel(L, B, ldb, nrhs, i, c, y);
        }
      }
      /* x = P^T z: undo the swaps in reverse order */
      for (int64_t k = n - 1; k >= 0; k--) {
        int64_t p = ipiv[k] - 1;
        if (p != k) {
          ld_rel(L, B, ldb, nrhs, k, c, x);
          ld_rel(L, B, ldb, nrhs, p, c, y);
          st_rel(L, B, ldb, nrhs, k, c, y);
          st_rel(L, B, ldb, nrhs, p, c, x);
        }
      }
    }
  }
  return orc_error_flag() ? 1 : 0;
}
