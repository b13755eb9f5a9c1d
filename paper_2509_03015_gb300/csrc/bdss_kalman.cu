// Assembly of the Kalman-smoother normal equations of Sec. 4.2 on the device,
// so that a smoother built on the solver never forms its Hessian on the host.
// Step k (0-based) has transition G_k (n x n), observation H_k (m x n),
// precisions Qinv_k (n x n), Rinv_k (m x m), measurement z_k and process
// offset zeta_k; with G_N = 0 the MAP normal equations are block tridiagonal:
//   A_kk      = Qinv_k + G_{k+1}^T Qinv_{k+1} G_{k+1} + H_k^T Rinv_k H_k
//   A_{k+1,k} = -Qinv_{k+1} G_{k+1}
//   b_k       = H_k^T Rinv_k z_k + Qinv_k zeta_k - G_{k+1}^T Qinv_{k+1} zeta_{k+1}
// Two launches, each a flat grid of (step, task) CTAs whose tasks of one step
// are adjacent so that step's operands are shared through L2:
//   products  A_{k+1,k} tiles (-Qinv G), U_k = Rinv_k H_k tiles (a row
//             scaling when Rinv_k is diagonal), and the vectors
//             v_k = Rinv_k z_k, w_k = Qinv_k zeta_k;
//   diagonal  A_kk tiles = Qinv_k + H_k^T U_k - G_{k+1}^T A_{k+1,k}, and b_k.
// All arithmetic is FP64, 64 x 64 output tiles through gemm_nt_tile.
#include "bdss_large.cuh"
#include "bdss_kalman.h"

namespace bdss {

namespace {

__device__ void store_tile(double *out, long long ld, int rows, int cols, int r0, int c0,
                           const double (&acc)[4][4], double sign, const double *add) {
  const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + 4 * tm + i;
    if (r >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + 4 * tn + j;
      if (c >= cols) continue;
      const long long o = (long long)r * ld + c;
      out[o] = (add ? add[o] : 0.0) + sign * acc[i][j];
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_kalman_products(KalmanArgs a) {
  __shared__ double sA[kKc * kTilePad], sB[kKc * kTilePad];
  const int n = a.n, m = a.m, nt = ntiles(n), mt = ntiles(m);
  const int tasks = nt * nt + mt * nt + 1;
  const long long k = (long long)blockIdx.x / tasks;
  const int t = (int)((long long)blockIdx.x - k * tasks);
  const long long nn = (long long)n * n, mn = (long long)m * n;
  const long long mm = a.rinv_diag ? (long long)m : (long long)m * m;  // Rinv stride per step
  double acc[4][4] = {};
  if (t < nt * nt) {
    if (k + 1 >= a.N) return;
    const int r0 = (t / nt) * kTile, c0 = (t % nt) * kTile;
    const View<double> Q{a.Qinv + (k + 1) * nn, n, 1, n, n};   // (r, j) -> Qinv_{k+1}[r][j]
    const View<double> Gt{a.G + (k + 1) * nn, 1, n, n, n};     // (c, j) -> G_{k+1}[j][c]
    gemm_nt_tile(acc, Q, r0, Gt, c0, n, sA, sB);
    store_tile(a.A_sub + k * nn, n, n, n, r0, c0, acc, -1.0, nullptr);
  } else if (t < nt * nt + mt * nt) {
    const int u = t - nt * nt, r0 = (u / nt) * kTile, c0 = (u % nt) * kTile;
    if (a.rinv_diag) {
      const double *rk = a.Rinv + k * mm, *Hk = a.H + k * mn;
      double *Uk = a.U + k * mn;
      for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = r0 + e / kTile, c = c0 + e % kTile;
        if (r < m && c < n) Uk[(long long)r * n + c] = rk[r] * Hk[(long long)r * n + c];
      }
      return;
    }
    const View<double> R{a.Rinv + k * mm, m, 1, m, m};         // (r, j) -> Rinv_k[r][j]
    const View<double> Ht{a.H + k * mn, 1, n, n, m};           // (c, j) -> H_k[j][c]
    gemm_nt_tile(acc, R, r0, Ht, c0, m, sA, sB);
    store_tile(a.U + k * mn, n, m, n, r0, c0, acc, 1.0, nullptr);
  } else {
    if (!a.B) return;
    const double *Rk = a.Rinv + k * mm, *zk = a.z + k * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double s = 0.0;
      if (a.rinv_diag)
        s = Rk[i] * zk[i];
      else
        for (int j = 0; j < m; ++j) s = fma(Rk[(long long)i * m + j], zk[j], s);
      a.v[k * m + i] = s;
    }
    const double *Qk = a.Qinv + k * nn, *ek = a.zeta ? a.zeta + k * n : nullptr;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = 0.0;
      if (ek)
        for (int j = 0; j < n; ++j) s = fma(Qk[(long long)i * n + j], ek[j], s);
      a.w[k * n + i] = s;
    }
  }
}

__global__ void __launch_bounds__(kThreads) k_kalman_diag(KalmanArgs a) {
  __shared__ double sA[kKc * kTilePad], sB[kKc * kTilePad];
  const int n = a.n, m = a.m, nt = ntiles(n);
  const int tasks = nt * nt + 1;
  const long long k = (long long)blockIdx.x / tasks;
  const int t = (int)((long long)blockIdx.x - k * tasks);
  const long long nn = (long long)n * n, mn = (long long)m * n;
  if (t < nt * nt) {
    const int r0 = (t / nt) * kTile, c0 = (t % nt) * kTile;
    double acc[4][4] = {};
    const View<double> Hc{a.H + k * mn, 1, n, n, m};           // (r, j) -> H_k[j][r]
    const View<double> Uc{a.U + k * mn, 1, n, n, m};           // (c, j) -> U_k[j][c]
    gemm_nt_tile(acc, Hc, r0, Uc, c0, m, sA, sB);
    if (k + 1 < a.N) {
      double acc2[4][4] = {};
      const View<double> Gc{a.G + (k + 1) * nn, 1, n, n, n};   // (r, j) -> G_{k+1}[j][r]
      const View<double> Sc{a.A_sub + k * nn, 1, n, n, n};     // (c, j) -> A_{k+1,k}[j][c]
      gemm_nt_tile(acc2, Gc, r0, Sc, c0, n, sA, sB);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] -= acc2[i][j];
    }
    store_tile(a.A_diag + k * nn, n, n, n, r0, c0, acc, 1.0, a.Qinv + k * nn);
  } else {
    if (!a.B) return;
    const double *Hk = a.H + k * mn, *vk = a.v + k * m, *wk = a.w + k * n;
    const bool next = k + 1 < a.N;
    const double *G1 = a.G + (k + 1) * nn, *w1 = a.w + (k + 1) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s = fma(Hk[(long long)j * n + i], vk[j], s);
      double g = 0.0;
      if (next)
        for (int j = 0; j < n; ++j) g = fma(G1[(long long)j * n + i], w1[j], g);
      a.B[k * n + i] = s + wk[i] - g;
    }
  }
}

}  // namespace

long long kalman_max_steps(int n, int m) {
  const int nt = ntiles(n), mt = ntiles(m);
  return 0x7fffffffLL / (nt * nt + mt * nt + 1);
}

cudaError_t launch_kalman_assemble(const KalmanArgs &a, cudaStream_t s) {
  const int nt = ntiles(a.n), mt = ntiles(a.m);
  const long long g1 = a.N * (long long)(nt * nt + mt * nt + 1);
  const long long g2 = a.N * (long long)(nt * nt + 1);
  if (a.N > kalman_max_steps(a.n, a.m)) return cudaErrorInvalidValue;
  k_kalman_products<<<(unsigned)g1, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_kalman_diag<<<(unsigned)g2, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bdss
