/*
 * CPU FP64 oracle for SPD block-tridiagonal solves.  TEST INFRASTRUCTURE ONLY:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load or run this file.  It shares no code with the CUDA path.
 *
 * Problem (Eq. 1, Sec. 1): A is SPD block-tridiagonal with N diagonal blocks
 * A_{i,i} (n x n) and N-1 sub-diagonal blocks A_{i+1,i}; the block above the
 * diagonal is A_{i+1,i}^T.  X and B are (N*n) x d.  Layout (0-based blocks):
 *   A_diag[i*n*n + r*n + c]   = (A_{i,i})_{r,c}, read as sym(A_{i,i})
 *   A_sub [i*n*n + r*n + c]   = (A_{i+1,i})_{r,c}
 *   B/X   [(i*n + r)*d + k]
 *
 * The diagonal blocks are read as sym(A_ii) = (A_ii + A_ii^T)/2; for exactly
 * symmetric input this equals reading one triangle.
 *
 * The method computes X = A^{-1} B, which has a plain definition, so the
 * oracle is that definition carried out by the serial base case of the paper:
 * the block-Cholesky sweep of Algorithm 1 and the block forward/backward
 * substitution of Algorithm 2 with a single segment (K = 1, J = N), i.e. the
 * block-Thomas algorithm.  Dense kernels are unblocked textbook loops.
 *
 * Built with -O2 -ffp-contract=off so that x86 and Arm hosts round alike.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define AT(M, n, r, c) ((M)[(size_t)(r) * (size_t)(n) + (size_t)(c)])

/* Cholesky-Crout of an n x n SPD matrix, in place (lower triangle = L, upper
 * zeroed): L_kk = sqrt(S_kk - sum_p L_kp^2), L_ik = (S_ik - sum_p L_ip L_kp)/L_kk.
 * This is the "cholesky" (potrf) step of Algorithm 1.  Returns 0, or k+1 if
 * pivot k is not positive and finite. */
static int chol_inplace(int n, double *S) {
  for (int k = 0; k < n; ++k) {
    double dkk = AT(S, n, k, k);
    for (int p = 0; p < k; ++p) dkk -= AT(S, n, k, p) * AT(S, n, k, p);
    if (!(dkk > 0.0) || !isfinite(dkk)) return k + 1;
    const double lkk = sqrt(dkk);
    AT(S, n, k, k) = lkk;
    for (int i = k + 1; i < n; ++i) {
      double s = AT(S, n, i, k);
      for (int p = 0; p < k; ++p) s -= AT(S, n, i, p) * AT(S, n, k, p);
      AT(S, n, i, k) = s / lkk;
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = r + 1; c < n; ++c) AT(S, n, r, c) = 0.0;
  return 0;
}

/* Forward substitution L Y = M for an n x m right-hand side (trsm with L). */
static void trsv_lower(int n, int m, const double *L, double *M) {
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < n; ++i) {
      double s = AT(M, m, i, c);
      for (int p = 0; p < i; ++p) s -= AT(L, n, i, p) * AT(M, m, p, c);
      AT(M, m, i, c) = s / AT(L, n, i, i);
    }
}

/* Backward substitution L^T X = M for an n x m right-hand side. */
static void trsv_lower_t(int n, int m, const double *L, double *M) {
  for (int c = 0; c < m; ++c)
    for (int i = n - 1; i >= 0; --i) {
      double s = AT(M, m, i, c);
      for (int p = i + 1; p < n; ++p) s -= AT(L, n, p, i) * AT(M, m, p, c);
      AT(M, m, i, c) = s / AT(L, n, i, i);
    }
}

/*
 * Block-Cholesky factorisation A = Lt Lt^T with Lt block lower bidiagonal:
 * diagonal blocks L_j (lower triangular) and sub-diagonal blocks C_j.
 * Algorithm 1 (Sec. 3.2) with K = 1, J = N:
 *   L_0 = chol(sym A_00);
 *   for j = 0..N-2:  C_j^T = L_j^{-1} A_{j+1,j}^T   (trsm)
 *                    S = sym A_{j+1,j+1} - C_j C_j^T (gemm)
 *                    L_{j+1} = chol(S)             (potrf)
 * L: (N,n,n), C: (N-1,n,n), both written.  Returns 0, or 1 + (first failing
 * block index) if a pivot is not positive and finite.
 */
int oracle_factor(int64_t N, int n, const double *A_diag, const double *A_sub,
                  double *L, double *C) {
  const size_t nn = (size_t)n * n;
  double *T = (double *)malloc(nn * sizeof(double));
  if (!T) return -1;
  for (int64_t j = 0; j < N; ++j) {
    double *Lj = L + (size_t)j * nn;
    const double *Aj = A_diag + (size_t)j * nn;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) AT(Lj, n, r, c) = 0.5 * (AT(Aj, n, r, c) + AT(Aj, n, c, r));
    if (j > 0) {
      const double *Cp = C + (size_t)(j - 1) * nn;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          double s = 0.0;
          for (int p = 0; p < n; ++p) s += AT(Cp, n, r, p) * AT(Cp, n, c, p);
          AT(Lj, n, r, c) -= s;
        }
    }
    if (chol_inplace(n, Lj) != 0) { free(T); return (int)(j + 1); }
    if (j < N - 1) {
      /* T = A_{j+1,j}^T, then T <- L_j^{-1} T, C_j = T^T */
      const double *Asj = A_sub + (size_t)j * nn;
      double *Cj = C + (size_t)j * nn;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) AT(T, n, r, c) = AT(Asj, n, c, r);
      trsv_lower(n, n, Lj, T);
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) AT(Cj, n, r, c) = AT(T, n, c, r);
    }
  }
  free(T);
  return 0;
}

/*
 * Block forward/backward substitution, Algorithm 2 (Sec. 3.2) with K = 1:
 *   Y_0 = L_0^{-1} B_0,  Y_j = L_j^{-1}(B_j - C_{j-1} Y_{j-1});
 *   X_{N-1} = L_{N-1}^{-T} Y_{N-1},  X_j = L_j^{-T}(Y_j - C_j^T X_{j+1}).
 * B and X are (N,n,d); X may alias B.
 */
void oracle_solve(int64_t N, int n, int d, const double *L, const double *C,
                  const double *B, double *X) {
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  if (X != B) memcpy(X, B, (size_t)N * nd * sizeof(double));
  for (int64_t j = 0; j < N; ++j) {
    double *Xj = X + (size_t)j * nd;
    if (j > 0) {
      const double *Cp = C + (size_t)(j - 1) * nn;
      const double *Xp = X + (size_t)(j - 1) * nd;
      for (int r = 0; r < n; ++r)
        for (int k = 0; k < d; ++k) {
          double s = 0.0;
          for (int p = 0; p < n; ++p) s += AT(Cp, n, r, p) * AT(Xp, d, p, k);
          AT(Xj, d, r, k) -= s;
        }
    }
    trsv_lower(n, d, L + (size_t)j * nn, Xj);
  }
  for (int64_t j = N - 1; j >= 0; --j) {
    double *Xj = X + (size_t)j * nd;
    if (j < N - 1) {
      const double *Cj = C + (size_t)j * nn;
      const double *Xn = X + (size_t)(j + 1) * nd;
      for (int r = 0; r < n; ++r)
        for (int k = 0; k < d; ++k) {
          double s = 0.0;
          for (int p = 0; p < n; ++p) s += AT(Cj, n, p, r) * AT(Xn, d, p, k);
          AT(Xj, d, r, k) -= s;
        }
    }
    trsv_lower_t(n, d, L + (size_t)j * nn, Xj);
  }
}

/* log det A = 2 sum_j sum_k log (L_j)_kk, since det A = prod_j det(L_j)^2.
 * The N n terms are summed with Neumaier's compensated summation (Neumaier
 * 1974): a plain running sum of 10^6 terms loses ~N n u of the total. */
double oracle_logdet(int64_t N, int n, const double *L) {
  const size_t nn = (size_t)n * n;
  double s = 0.0, c = 0.0;
  for (int64_t j = 0; j < N; ++j)
    for (int k = 0; k < n; ++k) {
      const double t = log(AT(L + (size_t)j * nn, n, k, k));
      const double u = s + t;
      c += (fabs(s) >= fabs(t)) ? (s - u) + t : (t - u) + s;
      s = u;
    }
  return 2.0 * (s + c);
}

/* ---- compensated residual (Ogita, Rump and Oishi 2005, "Accurate sum and
 * dot product": TwoSum, TwoProduct via fma, and Dot2) ---- */
static inline void two_sum(double a, double b, double *s, double *e) {
  const double x = a + b;
  const double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static inline void two_prod(double a, double b, double *p, double *e) {
  const double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}
typedef struct { double s, c; } dot2_acc;
static inline void dot2_add(dot2_acc *acc, double a, double b) {
  double p, ep, s, es;
  two_prod(a, b, &p, &ep);
  two_sum(acc->s, p, &s, &es);
  acc->s = s;
  acc->c += ep + es;
}

/*
 * R = B - A X, each entry accumulated with Dot2 (result as accurate as if
 * computed in twice the working precision, then rounded).  sym(A_ii) enters
 * as 0.5*A_ii[r][p] + 0.5*A_ii[p][r]; halving is exact, so no rounding is
 * introduced before the products.
 */
void oracle_residual(int64_t N, int n, int d, const double *A_diag, const double *A_sub,
                     const double *X, const double *B, double *R) {
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  for (int64_t i = 0; i < N; ++i) {
    const double *Ad = A_diag + (size_t)i * nn;
    const double *Xi = X + (size_t)i * nd;
    for (int r = 0; r < n; ++r)
      for (int k = 0; k < d; ++k) {
        dot2_acc acc = {B[(size_t)i * nd + (size_t)r * d + k], 0.0};
        for (int p = 0; p < n; ++p) {
          dot2_add(&acc, -0.5 * AT(Ad, n, r, p), AT(Xi, d, p, k));
          dot2_add(&acc, -0.5 * AT(Ad, n, p, r), AT(Xi, d, p, k));
        }
        if (i > 0) { /* A_{i,i-1} X_{i-1} */
          const double *As = A_sub + (size_t)(i - 1) * nn;
          const double *Xp = X + (size_t)(i - 1) * nd;
          for (int p = 0; p < n; ++p) dot2_add(&acc, -AT(As, n, r, p), AT(Xp, d, p, k));
        }
        if (i < N - 1) { /* A_{i+1,i}^T X_{i+1} */
          const double *As = A_sub + (size_t)i * nn;
          const double *Xn = X + (size_t)(i + 1) * nd;
          for (int p = 0; p < n; ++p) dot2_add(&acc, -AT(As, n, p, r), AT(Xn, d, p, k));
        }
        R[(size_t)i * nd + (size_t)r * d + k] = acc.s + acc.c;
      }
  }
}

/* ||A||_inf: the largest absolute row sum of the full Nn x Nn operator. */
double oracle_norm_inf_A(int64_t N, int n, const double *A_diag, const double *A_sub) {
  const size_t nn = (size_t)n * n;
  double best = 0.0;
  for (int64_t i = 0; i < N; ++i)
    for (int r = 0; r < n; ++r) {
      double s = 0.0;
      const double *Ad = A_diag + (size_t)i * nn;
      for (int p = 0; p < n; ++p) s += fabs(0.5 * (AT(Ad, n, r, p) + AT(Ad, n, p, r)));
      if (i > 0)
        for (int p = 0; p < n; ++p) s += fabs(AT(A_sub + (size_t)(i - 1) * nn, n, r, p));
      if (i < N - 1)
        for (int p = 0; p < n; ++p) s += fabs(AT(A_sub + (size_t)i * nn, n, p, r));
      if (s > best) best = s;
    }
  return best;
}

/*
 * Gradients of a scalar loss through X = A^{-1} B, given the adjoint
 * Lambda = A^{-1} dL/dX.  With dL/dA_full = -Lambda X^T and the diagonal blocks
 * entering as sym(A_ii) and A_{i+1,i} entering at (i+1,i) and, transposed, at
 * (i,i+1):
 *   dL/dA_ii      = -sym(Lambda_i X_i^T)
 *   dL/dA_{i+1,i} = -(Lambda_{i+1} X_i^T + X_{i+1} Lambda_i^T)
 * (dL/dB = Lambda needs no arithmetic).
 */
void oracle_adjoint_grads(int64_t N, int n, int d, const double *Lam, const double *X,
                          double *dA_diag, double *dA_sub) {
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  for (int64_t i = 0; i < N; ++i) {
    const double *Li = Lam + (size_t)i * nd, *Xi = X + (size_t)i * nd;
    double *G = dA_diag + (size_t)i * nn;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) {
        double s = 0.0;
        for (int k = 0; k < d; ++k) s += AT(Li, d, r, k) * AT(Xi, d, c, k) + AT(Xi, d, r, k) * AT(Li, d, c, k);
        AT(G, n, r, c) = -0.5 * s;
      }
    if (i < N - 1) {
      const double *Ln = Lam + (size_t)(i + 1) * nd, *Xn = X + (size_t)(i + 1) * nd;
      double *Gs = dA_sub + (size_t)i * nn;
      for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
          double s = 0.0;
          for (int k = 0; k < d; ++k) s += AT(Ln, d, r, k) * AT(Xi, d, c, k) + AT(Xn, d, r, k) * AT(Li, d, c, k);
          AT(Gs, n, r, c) = -s;
        }
    }
  }
}

/*
 * Operation tally of the block-Thomas sweep above (flops, counting a fused
 * multiply-add as two): per block Cholesky n^3/3 + n^2/2 + n/6, per coupling
 * trsm n^3 and Schur update (symmetric) n^2 (n+1); per block solve 6 n^2 d
 * less the coupling terms at the two ends.  out[0] = factor, out[1] = solve.
 */
void oracle_tally(int64_t N, int n, int d, double *out) {
  const double nd = (double)n;
  const double chol = nd * nd * nd / 3.0 + nd * nd / 2.0 + nd / 6.0;
  const double trsm = nd * nd * nd;
  const double syrk = nd * nd * (nd + 1.0);
  out[0] = (double)N * chol + (double)(N - 1) * (trsm + syrk);
  /* two triangular solves per block (n^2 d each) and two coupling gemms per
   * interior link (2 n^2 d each) */
  out[1] = (double)N * 2.0 * nd * nd * d + (double)(N - 1) * 4.0 * nd * nd * d;
}

/* Batched convenience for the CPU baseline: factor + solve K independent
 * systems, one per thread.  Per-instance arrays are passed as pointer lists.
 * info[k] receives the factor status.  Scratch per instance is malloc'ed. */
void oracle_factor_solve_batched(int K, const int64_t *Nk, const int *nk, int d,
                                 const double *const *A_diag, const double *const *A_sub,
                                 const double *const *B, double *const *X, int *info) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int k = 0; k < K; ++k) {
    const size_t nn = (size_t)nk[k] * nk[k];
    double *L = (double *)malloc((size_t)Nk[k] * nn * sizeof(double));
    double *C = (double *)malloc(((size_t)(Nk[k] > 1 ? Nk[k] - 1 : 1)) * nn * sizeof(double));
    if (!L || !C) { info[k] = -1; free(L); free(C); continue; }
    info[k] = oracle_factor(Nk[k], nk[k], A_diag[k], A_sub[k], L, C);
    if (info[k] == 0) oracle_solve(Nk[k], nk[k], d, L, C, B[k], X[k]);
    free(L);
    free(C);
  }
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  extern int omp_get_max_threads(void);
  return omp_get_max_threads();
#else
  return 1;
#endif
}
