// Kernels and their host launchers.  Two launch structures share the same
// device phases:
//   persistent : one cooperative launch runs every level; grid barriers
//                separate the phases (the fully fused recursion that Sec. 5
//                names as the way past per-level launch overhead);
//   per-level  : one launch per level and phase, the structure of
//                Algorithms 4 and 7.
#include "bdss_device.cuh"
#include "bdss_launch.h"

namespace bdss {

enum { kModeFactor = 1, kModeRhs = 2 };

template <typename T>
__global__ void __launch_bounds__(kThreads) k_persistent(const __grid_constant__ Args<T> a, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  T *smem = reinterpret_cast<T *>(smem_raw);
  const bool factor = (mode & kModeFactor) != 0;
  const bool rhs = (mode & kModeRhs) != 0 && a.d > 0;  // the host sets a.d = 0 without RHS
  int bar = 0;
  for (int l = 0; l < a.p.L; ++l) {
    const long long Nl = a.p.Nl[l];
    const long long nElim = Nl / 2, nSep = (Nl + 1) / 2;
    for (long long m = blockIdx.x; m < nElim; m += gridDim.x)
      if (!phaseA(a, l, 2 * m + 1, factor, smem, &s_flag)) break;
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
    for (long long k = blockIdx.x; k < nSep; k += gridDim.x) phaseB(a, l, k, factor, smem);
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
  if (blockIdx.x == 0) top_block(a, factor, reinterpret_cast<double *>(smem_raw), &s_flag);
  if (!rhs || a.p.L == 0) return;
  if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  for (int l = a.p.L - 1; l >= 0; --l) {
    const long long nElim = a.p.Nl[l] / 2;
    for (long long m = blockIdx.x; m < nElim; m += gridDim.x) phaseC(a, l, 2 * m + 1, smem);
    if (l > 0 && !grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
}

__device__ __forceinline__ bool status_set(const DevStatus *st) {
  return ld_relaxed_i32(&st->status) != 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_phaseA(const __grid_constant__ Args<T> a, int l, int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  if (status_set(a.st)) return;
  const long long nElim = a.p.Nl[l] / 2;
  for (long long m = blockIdx.x; m < nElim; m += gridDim.x)
    if (!phaseA(a, l, 2 * m + 1, factor != 0, reinterpret_cast<T *>(smem_raw), &s_flag)) return;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_phaseB(const __grid_constant__ Args<T> a, int l, int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (status_set(a.st)) return;
  const long long nSep = (a.p.Nl[l] + 1) / 2;
  for (long long k = blockIdx.x; k < nSep; k += gridDim.x)
    phaseB(a, l, k, factor != 0, reinterpret_cast<T *>(smem_raw));
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_top(const __grid_constant__ Args<T> a, int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  if (status_set(a.st)) return;
  top_block(a, factor != 0, reinterpret_cast<double *>(smem_raw), &s_flag);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_phaseC(const __grid_constant__ Args<T> a, int l) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (status_set(a.st)) return;
  const long long nElim = a.p.Nl[l] / 2;
  for (long long m = blockIdx.x; m < nElim; m += gridDim.x)
    phaseC(a, l, 2 * m + 1, reinterpret_cast<T *>(smem_raw));
}

// ---------------------------------------------------------------------------
// FP64 residual of the refinement loop: R = B - A X, one CTA per block row,
// one thread per row of the block.  Also max-norms ||R||_inf, ||X||_inf
// (max over rows of the absolute row sums), accumulated with atomicMax on
// the bit patterns of non-negative doubles, which order like the values.
// R is written in FP32 (the right-hand side of the FP32 correction solve).
// ---------------------------------------------------------------------------
constexpr int kResMaxD = 16;

__global__ void __launch_bounds__(kThreads) k_residual(long long N, int n, int d, const double *A_diag,
                                                       const double *A_sub, const double *X, const double *B,
                                                       float *R32, DevStatus *st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = ldstride(n);
  double *sD = reinterpret_cast<double *>(smem_raw);  // A_ii (full)
  double *sS = sD + (size_t)n * ld;                     // A_{i,i-1}
  double *sX = sS + (size_t)n * ld;                     // x_{i-1}, x_i, x_{i+1}: [3][n][d]
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    stage_rows(sD, ld, A_diag + i * nn, n);
    if (i > 0) stage_rows(sS, ld, A_sub + (i - 1) * nn, n);
    for (int e = threadIdx.x; e < 3 * n * d; e += blockDim.x) {
      const int w = e / (n * d), rem = e - w * n * d;
      const long long blk = i - 1 + w;
      sX[e] = (blk >= 0 && blk < N) ? ldcg(X + blk * nd + rem) : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r < n) {
      double rs = 0.0, xs = 0.0;  // absolute row sums of R and X over all d columns
      for (int c0 = 0; c0 < d; c0 += kResMaxD) {
        const int dc = min(kResMaxD, d - c0);
        double accD[kResMaxD], acc[kResMaxD];
#pragma unroll
        for (int c = 0; c < kResMaxD; ++c) { accD[c] = 0.0; acc[c] = 0.0; }
        const double *xm = sX, *x0 = sX + nd, *xp = sX + 2 * nd;
        // sym(A_ii) x_i = 0.5 * sum_p (A[r][p] + A[p][r]) x_p
        for (int p = 0; p < n; ++p) {
          const double sp = sD[r * ld + p] + sD[p * ld + r];
#pragma unroll
          for (int c = 0; c < kResMaxD; ++c)
            if (c < dc) accD[c] = fma(sp, x0[p * d + c0 + c], accD[c]);
        }
        if (i > 0)
          for (int p = 0; p < n; ++p) {
            const double a = sS[r * ld + p];
#pragma unroll
            for (int c = 0; c < kResMaxD; ++c)
              if (c < dc) acc[c] = fma(a, xm[p * d + c0 + c], acc[c]);
          }
        if (i + 1 < N) {
          const double *Au = A_sub + i * nn;  // A_{i+1,i}^T: element (r,p) = Au[p][r]
          for (int p = 0; p < n; ++p) {
            const double a = ldcg(Au + (size_t)p * n + r);
#pragma unroll
            for (int c = 0; c < kResMaxD; ++c)
              if (c < dc) acc[c] = fma(a, xp[p * d + c0 + c], acc[c]);
          }
        }
        const double *Bi = B + i * nd + (size_t)r * d + c0;
        float *Ri = R32 + i * nd + (size_t)r * d + c0;
#pragma unroll
        for (int c = 0; c < kResMaxD; ++c)
          if (c < dc) {
            const double rv = (ldcg(Bi + c) - acc[c]) - 0.5 * accD[c];
            Ri[c] = (float)rv;
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

// ||A||_inf of the full operator: one CTA per block row, thread per row.
__global__ void __launch_bounds__(kThreads) k_norm_A(long long N, int n, const double *A_diag,
                                                     const double *A_sub, DevStatus *st) {
  const size_t nn = (size_t)n * n;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    const int r = threadIdx.x;
    if (r < n) {
      double s = 0.0;
      const double *D = A_diag + i * nn;
      for (int p = 0; p < n; ++p) s += fabs(ldcg(D + r * n + p) + ldcg(D + p * n + r));
      s *= 0.5;
      if (i > 0) {
        const double *S = A_sub + (i - 1) * nn;
        for (int p = 0; p < n; ++p) s += fabs(ldcg(S + r * n + p));
      }
      if (i + 1 < N) {
        const double *S = A_sub + i * nn;
        for (int p = 0; p < n; ++p) s += fabs(ldcg(S + (size_t)p * n + r));
      }
      atomicMax(&st->nrm[2], (unsigned long long)__double_as_longlong(s));
    }
  }
}

// log det: sum over eliminated blocks (every original block i >= 1) of
// -2 sum_k log(1/L_kk) plus the top block's; reduced per CTA into out[blockIdx].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_logdet(long long N, int n, const T *Ld, const double *Ltop,
                                                     double *partial) {
  __shared__ double red[kThreads];
  double s = 0.0;
  const size_t nn = (size_t)n * n;
  const long long total = N * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / n;
    const int k = (int)(t - i * n);
    const double rd = (i == 0) ? Ltop[k * n + k] : (double)Ld[i * nn + (size_t)k * n + k];
    s -= 2.0 * log(rd);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
template <typename T>
size_t smem_bytes(int n, int d) {
  size_t w = smem_phaseA(n, d);
  if (smem_phaseB(n, d) > w) w = smem_phaseB(n, d);
  if (smem_down(n, d) > w) w = smem_down(n, d);
  size_t b = w * sizeof(T);
  if (smem_top_bytes(n, d) > b) b = smem_top_bytes(n, d);
  return (b + 15) & ~(size_t)15;
}

// The dynamic shared-memory limit of every kernel is raised once to the
// device's opt-in maximum, so that handles of different sizes never lower
// it under one another; each launch still requests only what it needs.
static cudaError_t raise_smem_limits() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const void *kernels[] = {
      (const void *)k_persistent<double>, (const void *)k_phaseA<double>, (const void *)k_phaseB<double>,
      (const void *)k_top<double>,        (const void *)k_phaseC<double>, (const void *)k_persistent<float>,
      (const void *)k_phaseA<float>,      (const void *)k_phaseB<float>,  (const void *)k_top<float>,
      (const void *)k_phaseC<float>,      (const void *)k_residual};
  for (const void *k : kernels) {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t configure(int n, int d, size_t *smem, int *blocks_per_sm) {
  const size_t sm = smem_bytes<T>(n, d);
  cudaError_t e0 = raise_smem_limits();
  if (e0 != cudaSuccess) return e0;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persistent<T>, kThreads, sm);
  if (e != cudaSuccess) return e;
  *smem = sm;
  *blocks_per_sm = occ;
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_persistent(const Args<T> &a, int factor, int rhs, int grid, size_t smem, cudaStream_t s) {
  Args<T> copy = a;
  if (!rhs) copy.d = 0;
  int mode = (factor ? kModeFactor : 0) | (rhs ? kModeRhs : 0);
  void *params[] = {(void *)&copy, (void *)&mode};
  return cudaLaunchCooperativeKernel((const void *)k_persistent<T>, dim3(grid), dim3(kThreads), params, smem, s);
}

template <typename T>
cudaError_t launch_phaseA(const Args<T> &a, int l, int factor, int grid, size_t smem, cudaStream_t s) {
  k_phaseA<T><<<grid, kThreads, smem, s>>>(a, l, factor);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_phaseB(const Args<T> &a, int l, int factor, int grid, size_t smem, cudaStream_t s) {
  k_phaseB<T><<<grid, kThreads, smem, s>>>(a, l, factor);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_top(const Args<T> &a, int factor, size_t smem, cudaStream_t s) {
  k_top<T><<<1, kThreads, smem, s>>>(a, factor);
  return cudaGetLastError();
}
template <typename T>
cudaError_t launch_phaseC(const Args<T> &a, int l, int grid, size_t smem, cudaStream_t s) {
  k_phaseC<T><<<grid, kThreads, smem, s>>>(a, l);
  return cudaGetLastError();
}

cudaError_t launch_residual(long long N, int n, int d, const double *A_diag, const double *A_sub, const double *X,
                            const double *B, float *R32, DevStatus *st, int grid, cudaStream_t s) {
  const size_t sm = ((size_t)2 * n * ldstride(n) + (size_t)3 * n * d) * sizeof(double);
  k_residual<<<grid, kThreads, sm, s>>>(N, n, d, A_diag, A_sub, X, B, R32, st);
  return cudaGetLastError();
}

cudaError_t launch_norm_A(long long N, int n, const double *A_diag, const double *A_sub, DevStatus *st, int grid,
                          cudaStream_t s) {
  k_norm_A<<<grid, kThreads, 0, s>>>(N, n, A_diag, A_sub, st);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_logdet(long long N, int n, const T *Ld, const double *Ltop, double *partial, int grid,
                          cudaStream_t s) {
  k_logdet<T><<<grid, kThreads, 0, s>>>(N, n, Ld, Ltop, partial);
  return cudaGetLastError();
}

#define BDSS_INSTANTIATE(T)                                                                                   \
  template size_t smem_bytes<T>(int, int);                                                                    \
  template cudaError_t configure<T>(int, int, size_t *, int *);                                               \
  template cudaError_t launch_persistent<T>(const Args<T> &, int, int, int, size_t, cudaStream_t);            \
  template cudaError_t launch_phaseA<T>(const Args<T> &, int, int, int, size_t, cudaStream_t);                \
  template cudaError_t launch_phaseB<T>(const Args<T> &, int, int, int, size_t, cudaStream_t);                \
  template cudaError_t launch_top<T>(const Args<T> &, int, size_t, cudaStream_t);                             \
  template cudaError_t launch_phaseC<T>(const Args<T> &, int, int, size_t, cudaStream_t);                     \
  template cudaError_t launch_logdet<T>(long long, int, const T *, const double *, double *, int, cudaStream_t);

BDSS_INSTANTIATE(double)
BDSS_INSTANTIATE(float)

}  // namespace bdss
