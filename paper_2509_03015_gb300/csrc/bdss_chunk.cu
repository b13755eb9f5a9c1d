// Kernels of the partitioned solve (one chunk of a system split over ranks):
// the coupling right-hand sides, the small n x n products that form a
// chunk's contribution to the reduced system of its boundary separators
// (Sec. 3.1, Eq. 5 with the chunk interior as A_uu), and the right-hand side
// of the back-solve.  All FP64; these are O(n^3) per chunk, next to the
// chunk's factorisation, so they are plain one-thread-per-output loops.
#include <cuda_runtime.h>

#include "bdss_chunk.h"

namespace bdss {

namespace {

// Z (Nb x n x dc) = 0 except block `blk`: Z[blk][r][c] = M[r][c0 + c]
// (trans = 0) or M[c0 + c][r] (trans = 1), M n x n.
__global__ void k_chunk_rhs(long long Nb, int n, int dc, int blk, const double *M, int trans, int c0, double *Z) {
  const long long total = Nb * n * dc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / ((long long)n * dc);
    const int rem = (int)(e - b * n * dc), r = rem / dc, c = rem - r * dc;
    double v = 0.0;
    if (b == blk) v = trans ? M[(size_t)(c0 + c) * n + r] : M[(size_t)r * n + c0 + c];
    Z[e] = v;
  }
}

// C[r][c0 + c] = sum_k op(P)[r][k] Q[k][c] for r < n, c < m: op(P) = P
// (trans = 0) or P^T (trans = 1), P n x n; Q n x m (row-major, leading
// dimension m); C with leading dimension ldc.
__global__ void k_chunk_product(int n, int m, const double *P, int trans, const double *Q, double *C, int ldc,
                                int c0) {
  const int total = n * m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int r = e / m, c = e - r * m;
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      const double p = trans ? P[(size_t)k * n + r] : P[(size_t)r * n + k];
      s = fma(p, Q[(size_t)k * m + c], s);
    }
    C[(size_t)r * ldc + c0 + c] = s;
  }
}

// Bp = B, then Bp[0] -= A_left x_left and Bp[Nb-1] -= A_right^T x_right
// (either term absent when its pointer is null).
__global__ void k_chunk_fix_rhs(long long Nb, int n, int d, const double *B, const double *A_left,
                                const double *A_right, const double *x_left, const double *x_right, double *Bp) {
  const long long total = Nb * n * d;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / ((long long)n * d);
    const int rem = (int)(e - b * n * d), r = rem / d, c = rem - r * d;
    double v = B[e];
    if (b == 0 && A_left)
      for (int k = 0; k < n; ++k) v = fma(-A_left[(size_t)r * n + k], x_left[(size_t)k * d + c], v);
    if (b == Nb - 1 && A_right)
      for (int k = 0; k < n; ++k) v = fma(-A_right[(size_t)k * n + r], x_right[(size_t)k * d + c], v);
    Bp[e] = v;
  }
}

int grid_for(long long total) {
  long long g = (total + 255) / 256;
  if (g > 4096) g = 4096;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t launch_chunk_rhs(long long Nb, int n, int dc, int blk, const double *M, int trans, int c0, double *Z,
                             cudaStream_t s) {
  k_chunk_rhs<<<grid_for(Nb * n * dc), 256, 0, s>>>(Nb, n, dc, blk, M, trans, c0, Z);
  return cudaGetLastError();
}

cudaError_t launch_chunk_product(int n, int m, const double *P, int trans, const double *Q, double *C, int ldc,
                                 int c0, cudaStream_t s) {
  k_chunk_product<<<grid_for((long long)n * m), 256, 0, s>>>(n, m, P, trans, Q, C, ldc, c0);
  return cudaGetLastError();
}

cudaError_t launch_chunk_fix_rhs(long long Nb, int n, int d, const double *B, const double *A_left,
                                 const double *A_right, const double *x_left, const double *x_right, double *Bp,
                                 cudaStream_t s) {
  k_chunk_fix_rhs<<<grid_for(Nb * n * d), 256, 0, s>>>(Nb, n, d, B, A_left, A_right, x_left, x_right, Bp);
  return cudaGetLastError();
}

}  // namespace bdss
