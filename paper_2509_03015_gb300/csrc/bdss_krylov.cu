// Preconditioned conjugate gradients in FP64 with the FP32 factorisation as
// the preconditioner: the refinement of the mixed-precision path for systems
// whose condition number defeats plain iterative refinement.  Plain
// refinement X += M^-1 (B - A X) with an FP32 factor M contracts the error
// only while kappa(A) u_32 stays below one; CG on A dX = B - A X with M^-1 as
// preconditioner keeps converging beyond that, because M^-1 A differs from I
// mainly on the few eigenvectors of A's smallest eigenvalues, which CG
// removes in about as many iterations (Krylov-based refinement: Carson and
// Higham, SIAM J. Sci. Comput. 2018, GMRES-IR; Higham and Pranesh, SIAM J.
// Sci. Comput. 2021, the symmetric positive definite case).
//
// M^-1 is applied in finite precision and so changes slightly between
// applications; beta uses the flexible (Polak-Ribiere) form
//   beta_k = z_{k+1}^T (r_{k+1} - r_k) / z_k^T r_k = -alpha_k z_{k+1}^T q_k / rho_k
// (r_{k+1} = r_k - alpha_k q_k), which tolerates that.  Every right-hand-side
// column runs its own CG (its own alpha, beta, rho).
//
// Kernels, all FP64 and HBM / latency bound:
//   k_btd_apply      out = B - A P, or A P  (sym(A_ii) on the diagonal, Eq. 1)
//   k_col_dots       per-CTA partial sums of x1.y1 and x2.y2 per column
//   k_pcg_scalars    one CTA: the partials summed in a fixed order (results
//                    do not depend on scheduling), then rho, alpha or beta, or
//                    the norms
//   k_pcg_update     X += alpha P, R -= alpha Q, per-CTA maxima of the row
//                    sums of |R| and |X| (infinity norms of the (N n) x d blocks)
//   k_pcg_direction  P = Z + beta P
#include <cfloat>

#include "bdss_device.cuh"
#include "bdss_krylov.h"

namespace bdss {

namespace {

__global__ void __launch_bounds__(kThreads) k_btd_apply(long long N, int n, int d, const double *A_diag,
                                                        const double *A_sub, const double *P, const double *B,
                                                        double *out) {
  const long long nd = (long long)n * d, nn = (long long)n * n, total = N * nd;
  // consecutive threads take consecutive rows r of one column c of one block
  // row i: the column reads A[q][r] are coalesced
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const long long i = g / nd;
    const int e = (int)(g - i * nd), c = e / n, r = e - c * n;
    const double *Ad = A_diag + i * nn;
    const double *p0 = P + i * nd + c;
    double s = 0.0;
    for (int q = 0; q < n; ++q)
      s = fma(__ldg(Ad + (long long)r * n + q) + __ldg(Ad + (long long)q * n + r), __ldg(p0 + (long long)q * d), s);
    double ax = 0.5 * s;
    if (i > 0) {  // A_{i,i-1} p_{i-1}
      const double *Al = A_sub + (i - 1) * nn + (long long)r * n, *pm = P + (i - 1) * nd + c;
      double t = 0.0;
      for (int q = 0; q < n; ++q) t = fma(__ldg(Al + q), __ldg(pm + (long long)q * d), t);
      ax += t;
    }
    if (i + 1 < N) {  // A_{i+1,i}^T p_{i+1}
      const double *Au = A_sub + i * nn + r, *pp = P + (i + 1) * nd + c;
      double t = 0.0;
      for (int q = 0; q < n; ++q) t = fma(__ldg(Au + (long long)q * n), __ldg(pp + (long long)q * d), t);
      ax += t;
    }
    const long long o = i * nd + (long long)r * d + c;
    out[o] = B ? __ldg(B + o) - ax : ax;
  }
}

// Block (d, kThreads / d): thread (c, y) sums column c over rows y, y + ny, ...
__global__ void __launch_bounds__(kThreads) k_col_dots(long long rows, int d, const double *x1, const double *y1,
                                                       const double *x2, const double *y2, double *part) {
  __shared__ double red[2][kThreads];
  const int c = threadIdx.x, ty = threadIdx.y, ny = blockDim.y;
  double s1 = 0.0, s2 = 0.0;
  for (long long row = (long long)blockIdx.x * ny + ty; row < rows; row += (long long)gridDim.x * ny) {
    const long long o = row * d + c;
    s1 = fma(x1[o], y1[o], s1);
    if (x2) s2 = fma(x2[o], y2[o], s2);
  }
  red[0][ty * d + c] = s1;
  red[1][ty * d + c] = s2;
  __syncthreads();
  if (ty == 0) {
    double a = 0.0, b = 0.0;
    for (int y = 0; y < ny; ++y) {
      a += red[0][y * d + c];
      b += red[1][y * d + c];
    }
    part[((size_t)blockIdx.x * 2 + 0) * kKrylovMaxD + c] = a;
    part[((size_t)blockIdx.x * 2 + 1) * kKrylovMaxD + c] = b;
  }
}

__global__ void k_pcg_scalars(int nparts, int d, const double *part, int step, double *sc) {
  const int c = threadIdx.x;
  if (step == kPcgNorms) {
    if (c == 0) {
      const double *pm = part + (size_t)kKrylovGrid * 2 * kKrylovMaxD;
      double rn = 0.0, xn = 0.0;
      for (int g = 0; g < nparts; ++g) {
        rn = fmax(rn, pm[2 * g]);
        xn = fmax(xn, pm[2 * g + 1]);
      }
      sc[kScNorm] = rn;
      sc[kScNorm + 1] = xn;
    }
    return;
  }
  if (c >= d) return;
  double s0 = 0.0, s1 = 0.0;
  for (int g = 0; g < nparts; ++g) {
    s0 += part[((size_t)g * 2 + 0) * kKrylovMaxD + c];
    s1 += part[((size_t)g * 2 + 1) * kKrylovMaxD + c];
  }
  const double rho = sc[kScRho + c];
  if (step == kPcgStart) {
    sc[kScRho + c] = s0;                                  // z.r
  } else if (step == kPcgAlpha) {
    sc[kScAlpha + c] = s0 > 0.0 ? rho / s0 : 0.0;         // rho / p.q (0: column done)
  } else {
    sc[kScBeta + c] = rho != 0.0 ? -sc[kScAlpha + c] * s1 / rho : 0.0;  // -alpha z.q / rho
    sc[kScRho + c] = s0;                                  // z.r
  }
}

__global__ void __launch_bounds__(kThreads) k_pcg_update(long long rows, int d, const double *sc, const double *P,
                                                         const double *Q, double *X, double *R, double *part) {
  __shared__ double red[2][kThreads];
  __shared__ double alpha[kKrylovMaxD];
  for (int c = threadIdx.x; c < d; c += blockDim.x) alpha[c] = sc[kScAlpha + c];
  __syncthreads();
  double rmax = 0.0, xmax = 0.0;
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (long long)gridDim.x * blockDim.x) {
    double rs = 0.0, xs = 0.0;
    for (int c = 0; c < d; ++c) {
      const long long o = row * d + c;
      const double x = fma(alpha[c], P[o], X[o]);
      const double r = fma(-alpha[c], Q[o], R[o]);
      X[o] = x;
      R[o] = r;
      rs += fabs(r);
      xs += fabs(x);
    }
    // a NaN must not vanish in fmax: report it as infinite
    rmax = fmax(rmax, rs <= DBL_MAX ? rs : INFINITY);
    xmax = fmax(xmax, xs <= DBL_MAX ? xs : INFINITY);
  }
  red[0][threadIdx.x] = rmax;
  red[1][threadIdx.x] = xmax;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[0][threadIdx.x] = fmax(red[0][threadIdx.x], red[0][threadIdx.x + w]);
      red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double *pm = part + (size_t)kKrylovGrid * 2 * kKrylovMaxD;
    pm[2 * blockIdx.x] = red[0][0];
    pm[2 * blockIdx.x + 1] = red[1][0];
  }
}

__global__ void __launch_bounds__(kThreads) k_pcg_direction(long long total, int d, const double *sc,
                                                            const double *Z, double *P, int init) {
  for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
       o += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(o % d);
    P[o] = init ? Z[o] : fma(sc[kScBeta + c], P[o], Z[o]);
  }
}

int flat_grid(long long total, int sms) {
  long long g = (total + kThreads - 1) / kThreads;
  const long long cap = 8LL * (sms > 0 ? sms : 1);
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_btd_apply(long long N, int n, int d, const double *A_diag, const double *A_sub, const double *P,
                             const double *B, double *out, int sms, cudaStream_t s) {
  k_btd_apply<<<flat_grid(N * n * d, sms), kThreads, 0, s>>>(N, n, d, A_diag, A_sub, P, B, out);
  return cudaGetLastError();
}

int col_dots_grid(long long rows, int d) {
  const int ny = kThreads / d;
  long long g = (rows + ny - 1) / ny;
  if (g > kKrylovGrid) g = kKrylovGrid;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_col_dots(long long rows, int d, const double *x1, const double *y1, const double *x2,
                            const double *y2, double *part, int grid, cudaStream_t s) {
  if (d < 1 || d > kKrylovMaxD || grid < 1 || grid > kKrylovGrid) return cudaErrorInvalidValue;
  k_col_dots<<<grid, dim3(d, kThreads / d), 0, s>>>(rows, d, x1, y1, x2, y2, part);
  return cudaGetLastError();
}

int pcg_update_grid(long long rows) {
  long long g = (rows + kThreads - 1) / kThreads;
  if (g > kKrylovGrid) g = kKrylovGrid;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_pcg_update(long long rows, int d, const double *sc, const double *P, const double *Q, double *X,
                              double *R, double *part, int grid, cudaStream_t s) {
  if (d < 1 || d > kKrylovMaxD || grid < 1 || grid > kKrylovGrid) return cudaErrorInvalidValue;
  k_pcg_update<<<grid, kThreads, 0, s>>>(rows, d, sc, P, Q, X, R, part);
  return cudaGetLastError();
}

cudaError_t launch_pcg_scalars(int nparts, int d, const double *part, int step, double *sc, cudaStream_t s) {
  if (d < 1 || d > kKrylovMaxD || nparts < 1 || nparts > kKrylovGrid) return cudaErrorInvalidValue;
  k_pcg_scalars<<<1, kKrylovMaxD, 0, s>>>(nparts, d, part, step, sc);
  return cudaGetLastError();
}

cudaError_t launch_pcg_direction(long long rows, int d, const double *sc, const double *Z, double *P, int init,
                                 int sms, cudaStream_t s) {
  k_pcg_direction<<<flat_grid(rows * d, sms), kThreads, 0, s>>>(rows * d, d, sc, Z, P, init);
  return cudaGetLastError();
}

// Shifted copy of the diagonal blocks for the shifted FP32 factorisation:
// out = A_diag with every diagonal entry scaled by (1 + sigma), i.e.
// A + sigma diag(A) (the off-diagonal blocks are used unchanged).
__global__ void k_shift_diag(long long N, int n, const double *A_diag, double sigma, double *out) {
  const long long nn = (long long)n * n, total = N * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long w = e % nn;
    const double v = A_diag[e];
    out[e] = (w / n == w % n) ? v + sigma * v : v;
  }
}

cudaError_t launch_shift_diag(long long N, int n, const double *A_diag, double sigma, double *out, int sms,
                              cudaStream_t s) {
  k_shift_diag<<<4 * sms, 256, 0, s>>>(N, n, A_diag, sigma, out);
  return cudaGetLastError();
}

}  // namespace bdss
