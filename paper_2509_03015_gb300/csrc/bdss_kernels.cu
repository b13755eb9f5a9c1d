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

// Resident CTAs per SM the persistent kernel is compiled for (register
// budget): FP64 is shared-memory limited to 3 at n = 64; FP32 fits 4.
template <typename T> struct PersistentOcc { static constexpr int value = sizeof(T) == 4 ? 4 : 3; };

template <typename T>
__global__ void __launch_bounds__(kThreads, PersistentOcc<T>::value)
    k_persistent(const __grid_constant__ Args<T> a, int mode) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  T *smem = reinterpret_cast<T *>(smem_raw);
  const bool factor = (mode & kModeFactor) != 0;
  const bool rhs = (mode & kModeRhs) != 0 && a.d > 0;  // the host sets a.d = 0 without RHS
  int bar = 0;
  const int rank = spread_rank(a.st, a.timeout_ns);
  if (rank < 0) return;
  for (int l = 0; l < a.p.L; ++l) {
    const long long Nl = a.p.Nl[l];
    const long long nElim = Nl / 2, nSep = (Nl + 1) / 2;
    // task t -> block t % count, part t / count: the parts of one block sit
    // `count` ranks apart, i.e. on different SMs
    const int pA = parts_A<T>(a.p, l, factor, a.capacity);
    for (long long t = rank; t < nElim * pA; t += gridDim.x) {
      if (l == 0 && factor && t + gridDim.x < nElim * pA) prefetch_elim_inputs(a, 2 * ((t + gridDim.x) % nElim) + 1);
      if (!phaseA(a, l, 2 * (t % nElim) + 1, factor, smem, &s_flag, (int)(t / nElim), pA)) break;
    }
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
    const int pB = parts_B<T>(a.p, l, factor, a.capacity);
    for (long long t = rank; t < nSep * pB; t += gridDim.x) {
      if (l == 0 && factor && t + gridDim.x < nSep * pB) prefetch_sep_inputs(a, 2 * ((t + gridDim.x) % nSep));
      phaseB(a, l, t % nSep, factor, smem, (int)(t / nSep), pB);
    }
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
  if (rank == 0) top_block(a, factor, reinterpret_cast<double *>(smem_raw), &s_flag);
  if (!rhs || a.p.L == 0) return;
  if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  for (int l = a.p.L - 1; l >= 0; --l) {
    const long long nElim = a.p.Nl[l] / 2;
    for (long long m = rank; m < nElim; m += gridDim.x) phaseC(a, l, 2 * m + 1, smem);
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
  const int pA = parts_A<T>(a.p, l, factor != 0, a.capacity);
  for (long long t = blockIdx.x; t < nElim * pA; t += gridDim.x) {
    if (l == 0 && factor && t + gridDim.x < nElim * pA) prefetch_elim_inputs(a, 2 * ((t + gridDim.x) % nElim) + 1);
    if (!phaseA(a, l, 2 * (t % nElim) + 1, factor != 0, reinterpret_cast<T *>(smem_raw), &s_flag, (int)(t / nElim),
                pA))
      return;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_phaseB(const __grid_constant__ Args<T> a, int l, int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (status_set(a.st)) return;
  const long long nSep = (a.p.Nl[l] + 1) / 2;
  const int pB = parts_B<T>(a.p, l, factor != 0, a.capacity);
  for (long long t = blockIdx.x; t < nSep * pB; t += gridDim.x) {
    if (l == 0 && factor && t + gridDim.x < nSep * pB) prefetch_sep_inputs(a, 2 * ((t + gridDim.x) % nSep));
    phaseB(a, l, t % nSep, factor != 0, reinterpret_cast<T *>(smem_raw), (int)(t / nSep), pB);
  }
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
// FP64 residual of the refinement loop: R = B - A X, one CTA per block row.
// sym(A_ii) is staged once in shared memory as S = A_ii + A_ii^T; every
// thread then owns one (row r, column c) output
//   R[r][c] = B[r][c] - ((A_{i,i-1} x_{i-1})[r][c] + (A_{i+1,i}^T x_{i+1})[r][c])
//                     - 0.5 (S x_i)[r][c]
// with the three products accumulated as independent chains (the coupling
// blocks read through L1; a missing neighbour multiplies zeros).  Also the
// max-norms ||R||_inf and ||X||_inf (max over rows of absolute row sums),
// reduced in the CTA and merged with one atomicMax per CTA.  R is written in
// FP32 for the FP32 correction solve.  With with_norm, also ||A||_inf from
// the same reads (row r sums |sym(A_ii)[r][:]|, |A_{i,i-1}[r][:]| and
// |A_{i+1,i}[:][r]|), in FP32 arithmetic on magnitudes taken from the FP64
// bit fields (abs_f32_bits): it only scales the refinement's stopping test,
// where a relative error of 1e-6 is immaterial.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_residual(long long N, int n, int d, const double *A_diag,
                                                       const double *A_sub, const double *X, const double *B,
                                                       float *R32, DevStatus *st, int with_norm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = ldstride(n);
  double *sS = reinterpret_cast<double *>(smem_raw);  // A_ii + A_ii^T
  double *sX = sS + (size_t)n * ld;                     // x_{i-1}, x_i, x_{i+1}: [3][n][d]
  double *sA = sX + (size_t)3 * n * d;                  // |R| entries: [n][d]
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  double maxR = 0.0, maxX = 0.0, maxA = 0.0;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    stage_rows(sS, ld, A_diag + i * nn, n);
    for (int e = threadIdx.x; e < 3 * n * d; e += blockDim.x) {
      const int w = e / (n * d), rem = e - w * n * d;
      const long long blk = i - 1 + w;
      sX[e] = (blk >= 0 && blk < N) ? ldcg(X + blk * nd + rem) : 0.0;
    }
    __syncthreads();
    // S = A + A^T in place: each unordered pair (r, p) belongs to one thread
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e / n, p = e - r * n;
      if (p <= r) {
        const double v = sS[r * ld + p] + sS[p * ld + r];
        sS[r * ld + p] = v;
        sS[p * ld + r] = v;
      }
    }
    __syncthreads();
    const double *xm = sX, *x0 = sX + nd, *xp = sX + 2 * nd;
    // missing neighbours: any valid finite block times the zero x staged above
    const double *Al = i > 0 ? A_sub + (i - 1) * nn : A_diag;  // A_{i,i-1}
    const double *Au = i + 1 < N ? A_sub + i * nn : A_diag;    // A_{i+1,i}
    for (int t = threadIdx.x; t < n * d; t += blockDim.x) {
      const int r = t / d, c = t - r * d;
      double accD = 0.0, accL = 0.0, accU = 0.0;
      const double *Sr = sS + r * ld;
      const double *Alr = Al + (size_t)r * n, *Aur = Au + r;
      if (with_norm) {  // uniform over the launch: no divergence
        const bool hl = i > 0, hu = i + 1 < N;
        float na = 0.0f;
#pragma unroll 4
        for (int p = 0; p < n; ++p) {
          const double s_ = Sr[p], l_ = __ldg(Alr + p), u_ = __ldg(Aur + (size_t)p * n);
          accD = fma(s_, x0[p * d + c], accD);
          accL = fma(l_, xm[p * d + c], accL);
          accU = fma(u_, xp[p * d + c], accU);
          na += 0.5f * abs_f32_bits(s_) + (hl ? abs_f32_bits(l_) : 0.0f) + (hu ? abs_f32_bits(u_) : 0.0f);
        }
        maxA = fmax(maxA, (double)na);
      } else {
#pragma unroll 4
        for (int p = 0; p < n; ++p) {
          accD = fma(Sr[p], x0[p * d + c], accD);
          accL = fma(__ldg(Alr + p), xm[p * d + c], accL);
          accU = fma(__ldg(Aur + (size_t)p * n), xp[p * d + c], accU);
        }
      }
      const double rv = (ldcg(B + i * nd + t) - (accL + accU)) - 0.5 * accD;
      R32[i * nd + t] = (float)rv;
      sA[t] = fabs(rv);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      double rs = 0.0, xs = 0.0;
      for (int c = 0; c < d; ++c) {
        rs += sA[r * d + c];
        xs += fabs(x0[r * d + c]);
      }
      maxR = fmax(maxR, rs);
      maxX = fmax(maxX, xs);
    }
    __syncthreads();
  }
  cta_max_to(&st->nrm[0], maxR);
  cta_max_to(&st->nrm[1], maxX);
  if (with_norm) cta_max_to(&st->nrm[2], maxA);
}


// log det: sum over eliminated blocks (every original block i >= 1) of
// -2 sum_k log(1/L_kk) plus the top block's; reduced per CTA into out[blockIdx].
template <typename T>
__global__ void __launch_bounds__(kThreads) k_logdet(long long N, int n, int Ltop_level, const T *Ld,
                                                     const double *Ltop, double *partial) {
  __shared__ double red[kThreads];
  double s = 0.0;
  const size_t nn = (size_t)n * n;
  const long long total = N * n;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long i = t / n;
    const int k = (int)(t - i * n);
    // blocks of the top level (positions j 2^L) were factored into Ltop
    const bool top = (i & ((1LL << Ltop_level) - 1)) == 0;
    const double rd = top ? Ltop[(size_t)(i >> Ltop_level) * nn + (size_t)k * n + k]
                          : (double)Ld[i * nn + (size_t)k * n + k];
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

// Adjoint gradients of a scalar loss through X = A^{-1} B, given
// Lambda = A^{-1} dL/dX (one CTA per block row, one thread per entry):
//   dL/dA_ii      = -sym(Lambda_i X_i^T)
//   dL/dA_{i+1,i} = -(Lambda_{i+1} X_i^T + X_{i+1} Lambda_i^T)
// (the diagonal blocks enter the operator as sym(A_ii); A_{i+1,i} enters at
// (i+1, i) and, transposed, at (i, i+1)).
__global__ void __launch_bounds__(kThreads) k_adjoint_grads(long long N, int n, int d, const double *Lam,
                                                            const double *X, double *dA_diag, double *dA_sub) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sL0 = reinterpret_cast<double *>(smem_raw);  // Lambda_i   [n][d]
  double *sX0 = sL0 + (size_t)n * d;                    // X_i
  double *sL1 = sX0 + (size_t)n * d;                    // Lambda_{i+1}
  double *sX1 = sL1 + (size_t)n * d;                    // X_{i+1}
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  for (long long i = blockIdx.x; i < N; i += gridDim.x) {
    const bool next = (i + 1 < N);
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      sL0[e] = ldcg(Lam + i * nd + e);
      sX0[e] = ldcg(X + i * nd + e);
      sL1[e] = next ? ldcg(Lam + (i + 1) * nd + e) : 0.0;
      sX1[e] = next ? ldcg(X + (i + 1) * nd + e) : 0.0;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      double g = 0.0;
      for (int k = 0; k < d; ++k) {
        g = fma(sL0[r * d + k], sX0[c * d + k], g);
        g = fma(sX0[r * d + k], sL0[c * d + k], g);
      }
      dA_diag[i * nn + e] = -0.5 * g;
      if (next) {
        double h = 0.0;
        for (int k = 0; k < d; ++k) {
          h = fma(sL1[r * d + k], sX0[c * d + k], h);
          h = fma(sX1[r * d + k], sL0[c * d + k], h);
        }
        dA_sub[i * nn + e] = -h;
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_adjoint_grads(long long N, int n, int d, const double *Lam, const double *X, double *dA_diag,
                                 double *dA_sub, int grid, cudaStream_t s) {
  const size_t sm = (size_t)4 * n * d * sizeof(double);
  k_adjoint_grads<<<grid, kThreads, sm, s>>>(N, n, d, Lam, X, dA_diag, dA_sub);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
template <typename T>
size_t smem_bytes(int n, int d) {
  size_t w = smem_phaseA(n, d);
  const size_t wb = smem_phaseB(n, d, (int)sizeof(T));
  if (wb > w) w = wb;
  if (smem_down(n, d) > w) w = smem_down(n, d);
  size_t b = w * sizeof(T);
  if (smem_top_bytes(n, d) > b) b = smem_top_bytes(n, d);
  return (b + 15) & ~(size_t)15;
}

// The dynamic shared-memory limit of every kernel is raised once to the
// device's opt-in maximum, so that handles of different sizes never lower
// it under one another; each launch still requests only what it needs.
cudaError_t raise_smem_limits() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const void *kernels[] = {
      (const void *)k_persistent<double>, (const void *)k_phaseA<double>, (const void *)k_phaseB<double>,
      (const void *)k_top<double>,        (const void *)k_phaseC<double>, (const void *)k_persistent<float>,
      (const void *)k_phaseA<float>,      (const void *)k_phaseB<float>,  (const void *)k_top<float>,
      (const void *)k_phaseC<float>,      (const void *)k_residual,       (const void *)k_adjoint_grads};
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
  cudaError_t e0 = raise_smem_limits();
  if (e0 != cudaSuccess) return e0;
  return occupancy<T>(n, d, smem, blocks_per_sm);
}

template <typename T>
cudaError_t occupancy(int n, int d, size_t *smem, int *blocks_per_sm) {
  const size_t sm = smem_bytes<T>(n, d);
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
                            const double *B, float *R32, DevStatus *st, int with_norm, int grid, cudaStream_t s) {
  const size_t sm = ((size_t)n * ldstride(n) + (size_t)3 * n * d + (size_t)n * d) * sizeof(double);
  k_residual<<<grid, kThreads, sm, s>>>(N, n, d, A_diag, A_sub, X, B, R32, st, with_norm);
  return cudaGetLastError();
}


template <typename T>
cudaError_t launch_logdet(long long N, int n, int Ltop_level, const T *Ld, const double *Ltop, double *partial, int grid,
                          cudaStream_t s) {
  k_logdet<T><<<grid, kThreads, 0, s>>>(N, n, Ltop_level, Ld, Ltop, partial);
  return cudaGetLastError();
}

#define BDSS_INSTANTIATE(T)                                                                                   \
  template size_t smem_bytes<T>(int, int);                                                                    \
  template cudaError_t configure<T>(int, int, size_t *, int *);                                               \
  template cudaError_t occupancy<T>(int, int, size_t *, int *);                                               \
  template cudaError_t launch_persistent<T>(const Args<T> &, int, int, int, size_t, cudaStream_t);            \
  template cudaError_t launch_phaseA<T>(const Args<T> &, int, int, int, size_t, cudaStream_t);                \
  template cudaError_t launch_phaseB<T>(const Args<T> &, int, int, int, size_t, cudaStream_t);                \
  template cudaError_t launch_top<T>(const Args<T> &, int, size_t, cudaStream_t);                             \
  template cudaError_t launch_phaseC<T>(const Args<T> &, int, int, size_t, cudaStream_t);                     \
  template cudaError_t launch_logdet<T>(long long, int, int, const T *, const double *, double *, int, cudaStream_t);

BDSS_INSTANTIATE(double)
BDSS_INSTANTIATE(float)

}  // namespace bdss
