/*
 * Blockwise (Schur-complement) matrix inversion: CPU reference oracle.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * FP64 statement of what the GPU library computes. Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it. The GPU
 * library neither links nor calls it, and it shares no code with the GPU
 * library (no headers, helpers or tables).
 *
 * Paper: R. Thiru Senthil, "Blockwise inversion and algorithms for inverting
 * large partitioned matrices" (arXiv 2305.11103).
 *
 *   oracle_gj_inverse        textbook Gauss-Jordan with partial pivoting on
 *                            the augmented matrix [M | I]; the paper calls the
 *                            method for the diagonal blocks arbitrary (Sec. 5,
 *                            discussion of performance).
 *   oracle_small_inverse     closed-form (adjugate / determinant) inverse of
 *                            orders 1..3, the "algebraic expressions" the paper
 *                            uses for its small diagonal blocks (Sec. 5.1).
 *   oracle_block_inverse     Eq. (a) applied recursively: the leading diagonal
 *                            block plays A, the rest of the matrix plays D, and
 *                            the Schur complement S_A = D - C A^-1 B is inverted
 *                            by the same procedure on the remaining blocks. The
 *                            products are taken in the out-of-place order of the
 *                            paper's `invertor_by_a` procedure (Sec. 4.1): first
 *                            A^-1 B and C A^-1, then the Schur complement, then
 *                            the three blocks that use S_A^-1 - six two-matrix
 *                            products and two reductions per level.
 *   oracle_paper_partition   the paper's partition rule, Eq. (blocking) and
 *                            Table 2: N_k = 2^(int(log2 m) - 1) diagonal blocks
 *                            with orders in {2,3,4}, the remainder going to the
 *                            last blocks.
 *   oracle_quarter_partition four diagonal blocks of order floor(m/4), the last
 *                            (m mod 4) of them one larger (the same remainder
 *                            to the last blocks pattern as Table 2).
 *   oracle_residual          rho = ||A X - I||_F / (||A||_F ||X||_F) in FP64.
 *   oracle_ns_step           one Newton-Schulz step X <- X (2I - A X), written
 *                            as X + X (I - A X), in FP64 (a refinement the
 *                            paper does not use; plain definition).
 *
 * Products are plain triple loops summed in index order. Build with
 * -O2 -ffp-contract=off so that no FMA contraction changes the rounding.
 * OpenMP (if enabled) splits only the rows of a product's output.
 *
 * Status codes: 0 = success; -2 = a pivot block or Schur complement is
 * singular (an exact zero pivot or a non-finite entry); -1 = bad argument;
 * -4 = out of memory. *failing_block receives the global index of the block
 * whose inverse failed.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_INVALID (-1)
#define OR_SINGULAR (-2)
#define OR_NOMEM (-4)

/* Mutation switch used by the self-test of the pin suite: when the oracle is
 * built with -DORACLE_MUTANT=k a deliberate, plausible mistake is planted so
 * that the tests can show that their pins catch it. 0 = the real oracle. */
#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0
#endif

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int oracle_mutant(void) { return ORACLE_MUTANT; }

/* C (m x n) = A (m x k) * B (k x n), all row-major with leading dimensions. */
static void matmul(int m, int n, int k, const double* A, long lda,
                   const double* B, long ldb, double* C, long ldc) {
  long i;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (i = 0; i < m; ++i) {
    double* c = C + i * ldc;
    for (int j = 0; j < n; ++j) c[j] = 0.0;
    for (int l = 0; l < k; ++l) {
      double a = A[i * lda + l];
      const double* b = B + (long)l * ldb;
      for (int j = 0; j < n; ++j) c[j] += a * b[j];
    }
  }
}

/* Gauss-Jordan elimination with partial pivoting on [M | I]. The pivot is the
 * entry of largest magnitude in the current column at or below the diagonal;
 * on ties the lowest row index wins. Singular: an exact zero or non-finite
 * pivot. */
int oracle_gj_inverse(int m, const double* M, long ldm, double* out, long ldo) {
  if (m <= 0 || !M || !out || ldm < m || ldo < m) return OR_INVALID;
  long w = 2L * m;
  double* aug = (double*)malloc(sizeof(double) * (size_t)m * (size_t)w);
  if (!aug) return OR_NOMEM;
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j < m; ++j) {
      aug[i * w + j] = M[i * ldm + j];
      aug[i * w + m + j] = (i == j) ? 1.0 : 0.0;
    }
  }
  int status = OR_OK;
  for (int c = 0; c < m; ++c) {
    int r = c;
    double best = fabs(aug[(long)c * w + c]);
    for (int i = c + 1; i < m; ++i) {
      double v = fabs(aug[(long)i * w + c]);
      if (v > best) { best = v; r = i; }
    }
    double piv = aug[(long)r * w + c];
    if (piv == 0.0 || !isfinite(piv)) { status = OR_SINGULAR; break; }
    if (r != c) {
#if ORACLE_MUTANT == 5
      /* planted mistake: the row swap skips the identity half */
      for (long j = 0; j < m; ++j) {
#else
      for (long j = 0; j < w; ++j) {
#endif
        double t = aug[(long)r * w + j];
        aug[(long)r * w + j] = aug[(long)c * w + j];
        aug[(long)c * w + j] = t;
      }
    }
    for (long j = 0; j < w; ++j) aug[(long)c * w + j] /= piv;
    for (int i = 0; i < m; ++i) {
      if (i == c) continue;
      double f = aug[(long)i * w + c];
      if (f == 0.0) continue;
      for (long j = 0; j < w; ++j) aug[(long)i * w + j] -= f * aug[(long)c * w + j];
    }
  }
  if (status == OR_OK) {
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        double v = aug[(long)i * w + m + j];
        if (!isfinite(v)) status = OR_SINGULAR;
        out[i * ldo + j] = v;
      }
  }
  free(aug);
  return status;
}

/* Closed-form inverse of orders 1, 2 and 3: adjugate divided by determinant. */
int oracle_small_inverse(int m, const double* M, long ldm, double* out, long ldo) {
#define E(i, j) M[(i) * ldm + (j)]
#define O(i, j) out[(i) * ldo + (j)]
  if (m == 1) {
    double a = E(0, 0);
    if (a == 0.0 || !isfinite(a)) return OR_SINGULAR;
    O(0, 0) = 1.0 / a;
    return OR_OK;
  }
  if (m == 2) {
    double a = E(0, 0), b = E(0, 1), c = E(1, 0), d = E(1, 1);
    double det = a * d - b * c;
    if (det == 0.0 || !isfinite(det)) return OR_SINGULAR;
    O(0, 0) = d / det;
    O(0, 1) = -b / det;
    O(1, 0) = -c / det;
    O(1, 1) = a / det;
    return OR_OK;
  }
  if (m == 3) {
    /* cofactors C_ij; inverse = C^T / det */
    double c00 = E(1, 1) * E(2, 2) - E(1, 2) * E(2, 1);
    double c01 = -(E(1, 0) * E(2, 2) - E(1, 2) * E(2, 0));
    double c02 = E(1, 0) * E(2, 1) - E(1, 1) * E(2, 0);
    double c10 = -(E(0, 1) * E(2, 2) - E(0, 2) * E(2, 1));
    double c11 = E(0, 0) * E(2, 2) - E(0, 2) * E(2, 0);
    double c12 = -(E(0, 0) * E(2, 1) - E(0, 1) * E(2, 0));
    double c20 = E(0, 1) * E(1, 2) - E(0, 2) * E(1, 1);
    double c21 = -(E(0, 0) * E(1, 2) - E(0, 2) * E(1, 0));
    double c22 = E(0, 0) * E(1, 1) - E(0, 1) * E(1, 0);
    double det = E(0, 0) * c00 + E(0, 1) * c01 + E(0, 2) * c02;
    if (det == 0.0 || !isfinite(det)) return OR_SINGULAR;
#if ORACLE_MUTANT == 6
    /* planted mistake: the cofactor matrix used without its transpose */
    O(0, 0) = c00 / det; O(0, 1) = c01 / det; O(0, 2) = c02 / det;
    O(1, 0) = c10 / det; O(1, 1) = c11 / det; O(1, 2) = c12 / det;
    O(2, 0) = c20 / det; O(2, 1) = c21 / det; O(2, 2) = c22 / det;
#else
    O(0, 0) = c00 / det; O(0, 1) = c10 / det; O(0, 2) = c20 / det;
    O(1, 0) = c01 / det; O(1, 1) = c11 / det; O(1, 2) = c21 / det;
    O(2, 0) = c02 / det; O(2, 1) = c12 / det; O(2, 2) = c22 / det;
#endif
    return OR_OK;
  }
#undef E
#undef O
  return OR_INVALID;
}

/* Inverse of one diagonal block: closed form for orders <= 3, else GJ. */
static int block_base_inverse(int m, const double* M, long ldm, double* out, long ldo) {
  if (m <= 3) return oracle_small_inverse(m, M, ldm, out, ldo);
  return oracle_gj_inverse(m, M, ldm, out, ldo);
}

/* Eq. (a), recursively. `depth` is the global index of this sub-problem's
 * first diagonal block. */
static int inv_rec(int n, int p, const int* sizes, const double* M, long ldm,
                   double* X, long ldx, int depth, int* failing_block) {
  if (p == 1) {
    int st = block_base_inverse(n, M, ldm, X, ldx);
    if (st == OR_SINGULAR && failing_block) *failing_block = depth;
    return st;
  }
  int m0 = sizes[0], m1 = n - m0;
  const double* A = M;
  const double* B = M + m0;
  const double* C = M + (long)m0 * ldm;
  const double* D = M + (long)m0 * ldm + m0;

  size_t need = (size_t)m0 * m0 + 2 * (size_t)m0 * m1 + 2 * (size_t)m1 * m1 + (size_t)m1 * m0;
  double* buf = (double*)malloc(sizeof(double) * need);
  if (!buf) return OR_NOMEM;
  double* Ai = buf;                       /* m0 x m0 : A^-1            */
  double* P = Ai + (size_t)m0 * m0;       /* m0 x m1 : A^-1 B          */
  double* Q = P + (size_t)m0 * m1;        /* m1 x m0 : C A^-1          */
  double* S = Q + (size_t)m1 * m0;        /* m1 x m1 : S_A, then C P   */
  double* Si = S + (size_t)m1 * m1;       /* m1 x m1 : S_A^-1          */

  int st = block_base_inverse(m0, A, ldm, Ai, m0);
  if (st != OR_OK) {
    if (st == OR_SINGULAR && failing_block) *failing_block = depth;
    free(buf);
    return st;
  }
  matmul(m0, m1, m0, Ai, m0, B, ldm, P, m1);          /* A^-1 B        */
  matmul(m1, m0, m0, C, ldm, Ai, m0, Q, m0);          /* C A^-1        */
  matmul(m1, m1, m0, C, ldm, P, m1, S, m1);           /* C (A^-1 B)    */
  for (int i = 0; i < m1; ++i)                        /* S_A = D - C A^-1 B */
    for (int j = 0; j < m1; ++j)
#if ORACLE_MUTANT == 2
      /* planted mistake: wrong sign in the Schur complement */
      S[(long)i * m1 + j] = D[(long)i * ldm + j] + S[(long)i * m1 + j];
#else
      S[(long)i * m1 + j] = D[(long)i * ldm + j] - S[(long)i * m1 + j];
#endif

  st = inv_rec(m1, p - 1, sizes + 1, S, m1, Si, m1, depth + 1, failing_block);
  if (st != OR_OK) { free(buf); return st; }

  /* Top-right: -A^-1 B S_A^-1 */
  double* TR = X + m0;
  matmul(m0, m1, m1, P, m1, Si, m1, TR, ldx);
#if ORACLE_MUTANT == 1
  /* planted mistake: sign of the top-right block dropped */
#else
  for (int i = 0; i < m0; ++i)
    for (int j = 0; j < m1; ++j) TR[(long)i * ldx + j] = -TR[(long)i * ldx + j];
#endif
  /* Bottom-left: -S_A^-1 C A^-1 */
  double* BL = X + (long)m0 * ldx;
  matmul(m1, m0, m1, Si, m1, Q, m0, BL, ldx);
  for (int i = 0; i < m1; ++i)
    for (int j = 0; j < m0; ++j) BL[(long)i * ldx + j] = -BL[(long)i * ldx + j];
  /* Top-left: A^-1 + A^-1 B S_A^-1 C A^-1 = A^-1 - TR Q */
  double* TL = X;
  matmul(m0, m0, m1, TR, ldx, Q, m0, TL, ldx);
  for (int i = 0; i < m0; ++i)
    for (int j = 0; j < m0; ++j) {
#if ORACLE_MUTANT == 3
      /* planted mistake: the A^-1 term of the top-left block dropped */
      TL[(long)i * ldx + j] = -TL[(long)i * ldx + j];
#else
      TL[(long)i * ldx + j] = Ai[(long)i * m0 + j] - TL[(long)i * ldx + j];
#endif
    }
  /* Bottom-right: S_A^-1 */
  for (int i = 0; i < m1; ++i)
    for (int j = 0; j < m1; ++j) {
#if ORACLE_MUTANT == 4
      /* planted mistake: S_A^-1 stored transposed */
      X[(long)(m0 + i) * ldx + m0 + j] = Si[(long)j * m1 + i];
#else
      X[(long)(m0 + i) * ldx + m0 + j] = Si[(long)i * m1 + j];
#endif
    }
  free(buf);
  return OR_OK;
}

/* Inverse of the n x n matrix A (row-major, leading dimension lda) partitioned
 * into p diagonal blocks of orders sizes[0..p-1] (sum = n). X receives A^-1
 * (row-major, leading dimension ldx); X must not alias A. */
int oracle_block_inverse(int n, int p, const int* sizes, const double* A, long lda,
                         double* X, long ldx, int* failing_block) {
  if (failing_block) *failing_block = -1;
  if (n <= 0 || p <= 0 || !sizes || !A || !X || lda < n || ldx < n) return OR_INVALID;
  long sum = 0;
  for (int i = 0; i < p; ++i) {
    if (sizes[i] <= 0) return OR_INVALID;
    sum += sizes[i];
  }
  if (sum != n) return OR_INVALID;
  return inv_rec(n, p, sizes, A, lda, X, ldx, 0, failing_block);
}

/* The paper's partition rule (Eq. (blocking), Table 2): for order m >= 2 the
 * number of diagonal blocks is N_k = 2^(int(log2 m) - 1); each block starts at
 * order 2 and the remaining m - 2 N_k units go to the last blocks first, one
 * per block per round. Returns N_k, or -1 if m < 2 or the output is too small. */
int oracle_paper_partition(int m, int* sizes, int cap) {
  if (m < 2) return OR_INVALID;
  int e = (int)log2((double)m);          /* (int) of the double log2, as stated */
  int nk = 1 << (e - 1);
  if (nk > cap) return OR_INVALID;
  for (int i = 0; i < nk; ++i) sizes[i] = 2;
  int r = m - 2 * nk;
#if ORACLE_MUTANT == 9
  /* planted mistake: the remainder handed out from the first block */
  int pos = 0;
  while (r > 0) {
    sizes[pos] += 1;
    r -= 1;
    pos = (pos == nk - 1) ? 0 : pos + 1;
  }
#else
  int pos = nk - 1;
  while (r > 0) {                         /* hand out one unit per block from the end */
    sizes[pos] += 1;
    r -= 1;
    pos = (pos == 0) ? nk - 1 : pos - 1;
  }
#endif
  return nk;
}

/* Four diagonal blocks of order floor(m/4); the last (m mod 4) blocks get one
 * more. Returns 4, or -1 if m < 4. */
int oracle_quarter_partition(int m, int* sizes) {
  if (m < 4) return OR_INVALID;
  int q = m / 4, r = m % 4;
#if ORACLE_MUTANT == 10
  /* planted mistake: the larger blocks placed first */
  for (int i = 0; i < 4; ++i) sizes[i] = q + ((i < r) ? 1 : 0);
#else
  for (int i = 0; i < 4; ++i) sizes[i] = q + ((i >= 4 - r) ? 1 : 0);
#endif
  return 4;
}

/* rho = ||A X - I||_F / (||A||_F ||X||_F), all in FP64. */
double oracle_residual(int n, const double* A, long lda, const double* X, long ldx) {
  double* R = (double*)malloc(sizeof(double) * (size_t)n * n);
  if (!R) return NAN;
  matmul(n, n, n, A, lda, X, ldx, R, n);
  double r2 = 0.0, a2 = 0.0, x2 = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double e = R[(long)i * n + j] - (i == j ? 1.0 : 0.0);
      r2 += e * e;
      double a = A[(long)i * lda + j], x = X[(long)i * ldx + j];
      a2 += a * a;
      x2 += x * x;
    }
  free(R);
#if ORACLE_MUTANT == 7
  /* planted mistake: the square root of the numerator dropped */
  return r2 / (sqrt(a2) * sqrt(x2));
#else
  return sqrt(r2) / (sqrt(a2) * sqrt(x2));
#endif
}

/* One Newton-Schulz step: Xn = X + X (I - A X). */
int oracle_ns_step(int n, const double* A, long lda, const double* X, long ldx,
                   double* Xn, long ldn) {
  double* E = (double*)malloc(sizeof(double) * (size_t)n * n);
  double* F = (double*)malloc(sizeof(double) * (size_t)n * n);
  if (!E || !F) { free(E); free(F); return OR_NOMEM; }
  matmul(n, n, n, A, lda, X, ldx, E, n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) E[(long)i * n + j] = (i == j ? 1.0 : 0.0) - E[(long)i * n + j];
#if ORACLE_MUTANT == 8
  /* planted mistake: the correction multiplied on the wrong side, E X */
  matmul(n, n, n, E, n, X, ldx, F, n);
#else
  matmul(n, n, n, X, ldx, E, n, F, n);
#endif
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Xn[(long)i * ldn + j] = X[(long)i * ldx + j] + F[(long)i * n + j];
  free(E);
  free(F);
  return OR_OK;
}
