// Kernels of the large-block path (64 < n <= 256).  Each level runs three
// sub-phases of tile tasks -- A1 (Cholesky per eliminated block), A2
// (forward substitution per vector tile), B (Schur update per output tile) --
// then the FP64 top block, then the downward tasks C per level.  The
// persistent kernel separates sub-phases with the bounded grid barrier; the
// per-level mode launches one kernel per sub-phase.
#include "bdss_large.cuh"
#include "bdss_launch.h"

namespace bdss {

enum { kSubA1 = 0, kSubA2 = 1, kSubB = 2, kSubC = 3 };

template <typename T>
__device__ bool large_sub(const Args<T> &a, int l, int sub, bool factor, T *smem, int *s_flag) {
  const int n = a.p.n, d = a.d;
  const long long Nl = a.p.Nl[l];
  const long long nE = Nl / 2, nS = (Nl + 1) / 2;
  if (sub == kSubA1) {
    for (long long m = blockIdx.x; m < nE; m += gridDim.x)
      if (!largeA1(a, l, 2 * m + 1, smem, s_flag)) return false;
  } else if (sub == kSubA2) {
    const int VT = vec_tile(sizeof(T));
    const int nvt = ((factor ? 2 * n : 0) + d + VT - 1) / VT;
    for (long long t = blockIdx.x; t < nE * nvt; t += gridDim.x) {
      const long long j = 2 * (t / nvt) + 1;
      const int v = (int)(t % nvt);
      if (v * VT < largeA2_vectors(a, l, j, factor)) largeA2(a, l, j, v, factor, smem);
    }
  } else if (sub == kSubB) {
    const int nTB = largeB_tiles(n, factor, d);
    for (long long t = blockIdx.x; t < nS * nTB; t += gridDim.x) largeB(a, l, t / nTB, (int)(t % nTB), factor, smem);
  } else {
    for (long long m = blockIdx.x; m < nE; m += gridDim.x) largeC(a, l, 2 * m + 1, smem);
  }
  return true;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_large_persistent(const __grid_constant__ Args<T> a, int factor,
                                                               int rhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  T *smem = reinterpret_cast<T *>(smem_raw);
  int bar = 0;
  for (int l = 0; l < a.p.L; ++l) {
    if (factor) {
      large_sub(a, l, kSubA1, true, smem, &s_flag);
      if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
    }
    large_sub(a, l, kSubA2, factor != 0, smem, &s_flag);
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
    large_sub(a, l, kSubB, factor != 0, smem, &s_flag);
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
  if (blockIdx.x == 0) largeTop(a, factor != 0, reinterpret_cast<double *>(smem_raw), &s_flag);
  if (!rhs || a.p.L == 0) return;
  if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  for (int l = a.p.L - 1; l >= 0; --l) {
    large_sub(a, l, kSubC, false, smem, &s_flag);
    if (l > 0 && !grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_large_sub(const __grid_constant__ Args<T> a, int l, int sub,
                                                        int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  if (ld_relaxed_i32(&a.st->status) != 0) return;
  large_sub(a, l, sub, factor != 0, reinterpret_cast<T *>(smem_raw), &s_flag);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_large_top(const __grid_constant__ Args<T> a, int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  if (ld_relaxed_i32(&a.st->status) != 0) return;
  largeTop(a, factor != 0, reinterpret_cast<double *>(smem_raw), &s_flag);
}

// FP64 residual for large blocks: one CTA per block row, one thread per row r
// of the block with up to 16 right-hand-side columns in registers:
//   R[r][c] = B[r][c] - 0.5 sum_p (A[r][p] + A[p][r]) x_i[p][c]
//             - sum_p A_{i,i-1}[r][p] x_{i-1}[p][c] - sum_p A_{i+1,i}[p][r] x_{i+1}[p][c]
constexpr int kResCols = 16;

__global__ void __launch_bounds__(kThreads) k_residual_rows(long long N, int n, int d, const double *A_diag,
                                                            const double *A_sub, const double *X, const double *B,
                                                            float *R32, DevStatus *st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sX = reinterpret_cast<double *>(smem_raw);  // x_{i-1}, x_i, x_{i+1}: [3][n][d]
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    for (int e = threadIdx.x; e < 3 * n * d; e += blockDim.x) {
      const int w = e / (n * d), rem = e - w * n * d;
      const long long blk = i - 1 + w;
      sX[e] = (blk >= 0 && blk < N) ? ldcg(X + blk * nd + rem) : 0.0;
    }
    __syncthreads();
    const double *xm = sX, *x0 = sX + nd, *xp = sX + 2 * nd;
    const double *D = A_diag + i * nn;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      double rs = 0.0, xs = 0.0;
      for (int c0 = 0; c0 < d; c0 += kResCols) {
        const int dc = min(kResCols, d - c0);
        double accD[kResCols], acc[kResCols];
#pragma unroll
        for (int c = 0; c < kResCols; ++c) accD[c] = acc[c] = 0.0;
        for (int p = 0; p < n; ++p) {
          const double sp = __ldg(D + (size_t)r * n + p) + __ldg(D + (size_t)p * n + r);
#pragma unroll
          for (int c = 0; c < kResCols; ++c)
            if (c < dc) accD[c] = fma(sp, x0[p * d + c0 + c], accD[c]);
        }
        if (i > 0) {
          const double *Al = A_sub + (i - 1) * nn;
          for (int p = 0; p < n; ++p) {
            const double v = __ldg(Al + (size_t)r * n + p);
#pragma unroll
            for (int c = 0; c < kResCols; ++c)
              if (c < dc) acc[c] = fma(v, xm[p * d + c0 + c], acc[c]);
          }
        }
        if (i + 1 < N) {
          const double *Au = A_sub + i * nn;
          for (int p = 0; p < n; ++p) {
            const double v = __ldg(Au + (size_t)p * n + r);
#pragma unroll
            for (int c = 0; c < kResCols; ++c)
              if (c < dc) acc[c] = fma(v, xp[p * d + c0 + c], acc[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < kResCols; ++c)
          if (c < dc) {
            const size_t o = i * nd + (size_t)r * d + c0 + c;
            const double rv = (ldcg(B + o) - acc[c]) - 0.5 * accD[c];
            R32[o] = (float)rv;
            rs += fabs(rv);
            xs += fabs(x0[r * d + c0 + c]);
          }
      }
      atomicMax(&st->nrm[0], (unsigned long long)__double_as_longlong(rs));
      atomicMax(&st->nrm[1], (unsigned long long)__double_as_longlong(xs));
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
template <typename T>
size_t smem_bytes_large(int n, int d) {
  size_t b = smem_large(n, d, (int)sizeof(T)) * sizeof(T);
  const size_t top = smem_large_top(n, d) * sizeof(double);
  if (top > b) b = top;
  return (b + 15) & ~(size_t)15;
}

template <typename T>
cudaError_t configure_large(int n, int d, size_t *smem, int *blocks_per_sm) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void *kernels[] = {(const void *)k_large_persistent<T>, (const void *)k_large_sub<T>,
                           (const void *)k_large_top<T>, (const void *)k_residual_rows};
  for (const void *k : kernels) {
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  }
  const size_t sm = smem_bytes_large<T>(n, d);
  int occ = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_large_persistent<T>, kThreads, sm);
  if (e != cudaSuccess) return e;
  *smem = sm;
  *blocks_per_sm = occ;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_large_persistent(const Args<T> &a, int factor, int rhs, int grid, size_t smem, cudaStream_t s) {
  Args<T> copy = a;
  if (!rhs) copy.d = 0;
  int f = factor, r = rhs;
  void *params[] = {(void *)&copy, (void *)&f, (void *)&r};
  return cudaLaunchCooperativeKernel((const void *)k_large_persistent<T>, dim3(grid), dim3(kThreads), params, smem,
                                     s);
}

template <typename T>
cudaError_t launch_large_sub(const Args<T> &a, int l, int sub, int factor, int grid, size_t smem, cudaStream_t s) {
  k_large_sub<T><<<grid, kThreads, smem, s>>>(a, l, sub, factor);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_large_top(const Args<T> &a, int factor, size_t smem, cudaStream_t s) {
  k_large_top<T><<<1, kThreads, smem, s>>>(a, factor);
  return cudaGetLastError();
}

long long large_sub_tasks(const Plan &p, int l, int sub, int factor, int d, int esz) {
  const long long Nl = p.Nl[l], nE = Nl / 2, nS = (Nl + 1) / 2;
  if (sub == kSubA1 || sub == kSubC) return nE;
  if (sub == kSubA2) {
    const int VT = vec_tile(esz);
    return nE * (((factor ? 2 * p.n : 0) + d + VT - 1) / VT);
  }
  return nS * largeB_tiles(p.n, factor != 0, d);
}

cudaError_t launch_residual_rows(long long N, int n, int d, const double *A_diag, const double *A_sub,
                                 const double *X, const double *B, float *R32, DevStatus *st, int grid,
                                 cudaStream_t s) {
  const size_t sm = (size_t)3 * n * d * sizeof(double);
  k_residual_rows<<<grid, kThreads, sm, s>>>(N, n, d, A_diag, A_sub, X, B, R32, st);
  return cudaGetLastError();
}

#define BDSS_INSTANTIATE_LARGE(T)                                                                        \
  template size_t smem_bytes_large<T>(int, int);                                                         \
  template cudaError_t configure_large<T>(int, int, size_t *, int *);                                    \
  template cudaError_t launch_large_persistent<T>(const Args<T> &, int, int, int, size_t, cudaStream_t); \
  template cudaError_t launch_large_sub<T>(const Args<T> &, int, int, int, int, size_t, cudaStream_t);   \
  template cudaError_t launch_large_top<T>(const Args<T> &, int, size_t, cudaStream_t);

BDSS_INSTANTIATE_LARGE(double)
BDSS_INSTANTIATE_LARGE(float)

}  // namespace bdss
