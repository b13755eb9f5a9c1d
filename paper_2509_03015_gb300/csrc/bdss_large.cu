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

template <typename T, bool kTc>
__device__ bool large_sub(const Args<T> &a, int l, int sub, bool factor, T *smem, int *s_flag, TcState *tc,
                          int rank) {
  const int n = a.p.n, d = a.d;
  const long long Nl = a.p.Nl[l];
  const long long nE = Nl / 2, nS = (Nl + 1) / 2;
  if (sub == kSubA1) {
    for (long long m = rank; m < nE; m += gridDim.x)
      if (!largeA1(a, l, 2 * m + 1, smem, s_flag)) return false;
  } else if (sub == kSubA2 && !factor && a.Li) {
    // solve pass with the stored inverses: y_j = L_j^{-1} b_j, a thread per row
    if constexpr (sizeof(T) == 4)
      for (long long m = rank; m < nE; m += gridDim.x) largeA2_rows(a, l, 2 * m + 1, smem);
  } else if (sub == kSubA2) {
    const int VT = vec_tile(sizeof(T));
    const int nvt = (largeA2_slots(a, factor) + VT - 1) / VT;
    for (long long t = rank; t < nE * nvt; t += gridDim.x) {
      const long long j = 2 * (t / nvt) + 1;
      const int v = (int)(t % nvt);
      if (largeA2_live(a, l, j, factor, v * VT)) largeA2(a, l, j, v, factor, smem);
    }
  } else if (sub == kSubB) {
    if constexpr (kTc) {
      if (tc && factor) {
        // D and E tiles on the tensor cores, RHS tiles on CUDA cores
        const int nTC = largeB_tc_tiles(n), nR = largeB_tiles(n, false, d), nTB = nTC + nR;
        for (long long t = rank; t < nS * nTB; t += gridDim.x) {
          const long long k = t / nTB;
          const int u = (int)(t % nTB);
          if (u < nTC) {
            if (!largeB_tc(a, l, k, u, *tc)) return false;
          } else {
            largeB(a, l, k, u - nTC, false, smem);
          }
        }
        return true;
      }
    }
    if constexpr (sizeof(T) == 4) {
      if (!factor) {  // solve pass: the separator RHS updates, a thread per row
        for (long long k = rank; k < nS; k += gridDim.x) largeB_rows(a, l, k, smem);
        return true;
      }
    }
    const int nTB = largeB_tiles(n, factor, d);
    for (long long t = rank; t < nS * nTB; t += gridDim.x) largeB(a, l, t / nTB, (int)(t % nTB), factor, smem);
  } else if (sub == kSubBRhsOnly) {
    const int nR = largeB_tiles(n, false, d);
    for (long long t = rank; t < nS * nR; t += gridDim.x) largeB(a, l, t / nR, (int)(t % nR), false, smem);
  } else {
    if constexpr (sizeof(T) == 4) {
      if (a.Li) {  // with the stored inverses, a thread per row
        for (long long m = rank; m < nE; m += gridDim.x) largeC_rows(a, l, 2 * m + 1, smem);
        return true;
      }
    }
    for (long long m = rank; m < nE; m += gridDim.x) largeC(a, l, 2 * m + 1, smem);
  }
  return true;
}

template <typename T, bool kTc>
__device__ void large_body(const Args<T> &a, int factor, int rhs, unsigned char *smem_raw, int *s_flag,
                           TcState *tc) {
  T *smem = reinterpret_cast<T *>(smem_raw);
  int bar = 0;
  const int rank = spread_rank(a.st, a.timeout_ns);
  if (rank < 0) return;
  for (int l = 0; l < a.p.L; ++l) {
    if (factor) {
      large_sub<T, kTc>(a, l, kSubA1, true, smem, s_flag, tc, rank);
      if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
    }
    large_sub<T, kTc>(a, l, kSubA2, factor != 0, smem, s_flag, tc, rank);
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
    large_sub<T, kTc>(a, l, kSubB, factor != 0, smem, s_flag, tc, rank);
    if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
  if (rank == 0) largeTop(a, factor != 0, reinterpret_cast<double *>(smem_raw), s_flag);
  if (!rhs || a.p.L == 0) return;
  if (!grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  for (int l = a.p.L - 1; l >= 0; --l) {
    large_sub<T, kTc>(a, l, kSubC, false, smem, s_flag, tc, rank);
    if (l > 0 && !grid_barrier(a.st, a.timeout_ns, ++bar, a.skip_barrier)) return;
  }
}

// The tensor-core state (TMEM, mbarriers) is set up once per CTA when the
// TF32 mode factors and released on every way out of the kernel body.  The
// tensor-core variant (kTc) is a separate kernel: the occupancy calculator
// allows one CTA per SM for a kernel that contains tcgen05 code, while the
// FP32 tiles without it fit two.
// Register cap: FP32 tiles fit two CTAs per SM in shared memory, so the
// registers must allow two as well; FP64 is shared-memory limited to one.
#define BDSS_LARGE_MAXNREG(T) __maxnreg__(sizeof(T) == 4 ? 120 : 255)

template <typename T, bool kTc>
__global__ void __launch_bounds__(kThreads) BDSS_LARGE_MAXNREG(T)
    k_large_persistent(const __grid_constant__ Args<T> a, int factor, int rhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  if constexpr (kTc) {
    __shared__ uint64_t s_bars[3];
    __shared__ uint32_t s_tmem;
    TcState tc;
    const bool use_tc = a.tf32 && factor;
    if (use_tc) tc_begin(tc, smem_raw, s_bars, &s_tmem);
    large_body<T, true>(a, factor, rhs, smem_raw, &s_flag, use_tc ? &tc : nullptr);
    if (use_tc) tc_end(tc, a.timeout_ns);
  } else {
    large_body<T, false>(a, factor, rhs, smem_raw, &s_flag, nullptr);
  }
}

template <typename T, bool kTc>
__global__ void __launch_bounds__(kThreads) BDSS_LARGE_MAXNREG(T)
    k_large_sub(const __grid_constant__ Args<T> a, int l, int sub, int factor) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  if (ld_relaxed_i32(&a.st->status) != 0) return;
  if constexpr (kTc) {
    __shared__ uint64_t s_bars[3];
    __shared__ uint32_t s_tmem;
    TcState tc;
    const bool use_tc = a.tf32 && factor && sub == kSubB;
    if (use_tc) tc_begin(tc, smem_raw, s_bars, &s_tmem);
    large_sub<T, true>(a, l, sub, factor != 0, reinterpret_cast<T *>(smem_raw), &s_flag, use_tc ? &tc : nullptr,
                       (int)blockIdx.x);
    if (use_tc) tc_end(tc, a.timeout_ns);
  } else {
    large_sub<T, false>(a, l, sub, factor != 0, reinterpret_cast<T *>(smem_raw), &s_flag, nullptr, (int)blockIdx.x);
  }
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
                                                            float *R32, DevStatus *st, int with_norm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sX = reinterpret_cast<double *>(smem_raw);  // x_{i-1}, x_i, x_{i+1}: [3][n][d]
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  double maxR = 0.0, maxX = 0.0, maxA = 0.0;
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
      float na = 0.0f;  // ||A||_inf row sum (with_norm), FP32 as it only scales the stop test
      for (int c0 = 0; c0 < d; c0 += kResCols) {
        const bool nrm = with_norm && c0 == 0;
        const int dc = min(kResCols, d - c0);
        double accD[kResCols], acc[kResCols];
#pragma unroll
        for (int c = 0; c < kResCols; ++c) accD[c] = acc[c] = 0.0;
        for (int p = 0; p < n; ++p) {
          const double sp = __ldg(D + (size_t)r * n + p) + __ldg(D + (size_t)p * n + r);
          if (nrm) na += 0.5f * abs_f32_bits(sp);
#pragma unroll
          for (int c = 0; c < kResCols; ++c)
            if (c < dc) accD[c] = fma(sp, x0[p * d + c0 + c], accD[c]);
        }
        if (i > 0) {
          const double *Al = A_sub + (i - 1) * nn;
          for (int p = 0; p < n; ++p) {
            const double v = __ldg(Al + (size_t)r * n + p);
            if (nrm) na += abs_f32_bits(v);
#pragma unroll
            for (int c = 0; c < kResCols; ++c)
              if (c < dc) acc[c] = fma(v, xm[p * d + c0 + c], acc[c]);
          }
        }
        if (i + 1 < N) {
          const double *Au = A_sub + i * nn;
          for (int p = 0; p < n; ++p) {
            const double v = __ldg(Au + (size_t)p * n + r);
            if (nrm) na += abs_f32_bits(v);
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
      maxR = fmax(maxR, rs);
      maxX = fmax(maxX, xs);
      maxA = fmax(maxA, (double)na);
    }
    __syncthreads();
  }
  cta_max_to(&st->nrm[0], maxR);
  cta_max_to(&st->nrm[1], maxX);
  if (with_norm) cta_max_to(&st->nrm[2], maxA);
}

__global__ void k_tc_selftest(const __grid_constant__ CUtensorMap map, const float *W, int n, double *err,
                              int *status, long long timeout_ns);

// ---------------------------------------------------------------------------
template <typename T>
size_t smem_bytes_large(int n, int d) {
  size_t b = smem_large(n, d, (int)sizeof(T)) * sizeof(T);
  const size_t top = smem_large_top(n, d) * sizeof(double);
  if (top > b) b = top;
  if (sizeof(T) == 4 && kTcSmemBytes > b) b = kTcSmemBytes;
  return (b + 15) & ~(size_t)15;
}

template <typename T>
cudaError_t configure_large(int n, int d, size_t *smem, int *blocks_per_sm, int *blocks_per_sm_tc) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void *kernels[] = {(const void *)k_large_persistent<T, false>, (const void *)k_large_sub<T, false>,
                           (const void *)k_large_persistent<float, true>, (const void *)k_large_sub<float, true>,
                           (const void *)k_large_top<T>, (const void *)k_residual_rows,
                           (const void *)k_tc_selftest};
  for (const void *k : kernels) {
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  }
  const size_t sm = smem_bytes_large<T>(n, d);
  int occ = 0, occ_tc = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_large_persistent<T, false>, kThreads, sm);
  if (e == cudaSuccess && sizeof(T) == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_tc, k_large_persistent<float, true>, kThreads, sm);
  if (e != cudaSuccess) return e;
  *smem = sm;
  *blocks_per_sm = occ;
  *blocks_per_sm_tc = sizeof(T) == 4 ? occ_tc : occ;
  return cudaSuccess;
}

// The tensor-core kernel runs only when the TF32 mode factors.
template <typename T>
bool large_uses_tc(const Args<T> &a, int factor) {
  return sizeof(T) == 4 && a.tf32 && factor;
}

template <typename T>
cudaError_t launch_large_persistent(const Args<T> &a, int factor, int rhs, int grid, size_t smem, cudaStream_t s) {
  Args<T> copy = a;
  if (!rhs) copy.d = 0;
  int f = factor, r = rhs;
  void *params[] = {(void *)&copy, (void *)&f, (void *)&r};
  const void *k = (const void *)k_large_persistent<T, false>;
  if constexpr (sizeof(T) == 4)
    if (large_uses_tc(a, factor)) k = (const void *)k_large_persistent<float, true>;
  return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(kThreads), params, smem, s);
}

template <typename T>
cudaError_t launch_large_sub(const Args<T> &a, int l, int sub, int factor, int grid, size_t smem, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (large_uses_tc(a, factor) && sub == kSubB) {
      k_large_sub<float, true><<<grid, kThreads, smem, s>>>(a, l, sub, factor);
      return cudaGetLastError();
    }
  }
  k_large_sub<T, false><<<grid, kThreads, smem, s>>>(a, l, sub, factor);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_large_top(const Args<T> &a, int factor, size_t smem, cudaStream_t s) {
  k_large_top<T><<<1, kThreads, smem, s>>>(a, factor);
  return cudaGetLastError();
}

long long large_sub_tasks(const Plan &p, int l, int sub, int factor, int d, int esz, int tf32, int inv) {
  const long long Nl = p.Nl[l], nE = Nl / 2, nS = (Nl + 1) / 2;
  if (sub == kSubBRhsOnly) return nS * largeB_tiles(p.n, false, d);
  if (sub == kSubA1 || sub == kSubC) return nE;
  if (sub == kSubA2) {
    if (!factor && inv) return nE;
    const int VT = vec_tile(esz);
    return nE * (((factor ? (inv ? 3 : 2) * p.n : 0) + d + VT - 1) / VT);
  }
  if (tf32 && factor) return nS * (largeB_tc_tiles(p.n) + largeB_tiles(p.n, false, d));
  if (!factor && esz == 4) return nS;  // a thread per row (largeB_rows)
  return nS * largeB_tiles(p.n, factor != 0, d);
}

// ---------------------------------------------------------------------------
// Tensor map of the coupling buffer for the TMA loads of the TF32 tiles.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t make_w_tensor_map(CUtensorMap *out, const float *Wb, long long rows, int n) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = (EncodeTiledFn)p;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)Wb, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Self-check of the tensor-core tile: one 128 x 128 tile C = A B^T, K = 256,
// 3xTF32 on tcgen05 against an FP64 CUDA-core product of the same FP32
// inputs.  err[0] = max |C_tc - C_ref| / max(sum_k |a||b|).
__global__ void __launch_bounds__(kThreads) k_tc_selftest(const __grid_constant__ CUtensorMap map, const float *W,
                                                          int n, double *err, int *status, long long timeout_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t s_bars[3];
  __shared__ uint32_t s_tmem;
  TcState tc;
  tc_begin(tc, smem_raw, s_bars, &s_tmem);
  // rows 0..127 (A) against rows 128..255 (B) of the n x n matrix W
  const bool ok = tc_accumulate(tc, &map, 0, 128, n, true, timeout_ns);
  if (!ok) {
    if (threadIdx.x == 0) *status = kStTimeout;
  } else {
    float v[64];
    int row, col0;
    tc_read_row(tc, v, row, col0);
    double worst = 0.0;
    for (int j = 0; j < 64; ++j) {
      const int c = col0 + j;
      double ref = 0.0, mag = 0.0;
      for (int k = 0; k < n; ++k) {
        const double x = W[(size_t)row * n + k], y = W[(size_t)(128 + c) * n + k];
        ref = fma(x, y, ref);
        mag += fabs(x * y);
      }
      const double e = fabs((double)v[j] - ref) / (mag > 0 ? mag : 1.0);
      worst = e > worst ? e : worst;
    }
    atomicMax(reinterpret_cast<unsigned long long *>(err), (unsigned long long)__double_as_longlong(worst));
  }
  tc_end(tc, timeout_ns);
}

cudaError_t run_tc_selftest(double *max_err, int *status) {
  const int n = 256;
  float *W = nullptr;
  double *d_err = nullptr;
  int *d_status = nullptr;
  cudaError_t e = cudaMalloc(&W, (size_t)n * n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_err, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&d_status, sizeof(int));
  float *h = nullptr;
  if (e == cudaSuccess) h = (float *)malloc((size_t)n * n * sizeof(float));
  if (e == cudaSuccess && h) {
    unsigned s = 12345u;
    for (int i = 0; i < n * n; ++i) {  // deterministic values in (-1, 1), full FP32 mantissas
      s = s * 1664525u + 1013904223u;
      h[i] = (float)((double)(s >> 8) / (double)(1u << 24) * 2.0 - 1.0);
    }
    e = cudaMemcpy(W, h, (size_t)n * n * sizeof(float), cudaMemcpyHostToDevice);
  }
  free(h);
  CUtensorMap map;
  if (e == cudaSuccess) e = make_w_tensor_map(&map, W, n, n);
  if (e == cudaSuccess) e = cudaMemset(d_err, 0, sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(d_status, 0, sizeof(int));
  if (e == cudaSuccess) {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void *)k_tc_selftest);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute((const void *)k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
  }
  if (e == cudaSuccess) {
    k_tc_selftest<<<1, kThreads, kTcSmemBytes>>>(map, W, n, d_err, d_status, 2000000000LL);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(max_err, d_err, sizeof(double), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(status, d_status, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(W);
  cudaFree(d_err);
  cudaFree(d_status);
  return e;
}

cudaError_t launch_residual_rows(long long N, int n, int d, const double *A_diag, const double *A_sub,
                                 const double *X, const double *B, float *R32, DevStatus *st, int with_norm,
                                 int grid, cudaStream_t s) {
  const size_t sm = (size_t)3 * n * d * sizeof(double);
  k_residual_rows<<<grid, kThreads, sm, s>>>(N, n, d, A_diag, A_sub, X, B, R32, st, with_norm);
  return cudaGetLastError();
}

#define BDSS_INSTANTIATE_LARGE(T)                                                                        \
  template size_t smem_bytes_large<T>(int, int);                                                         \
  template cudaError_t configure_large<T>(int, int, size_t *, int *, int *);                             \
  template cudaError_t launch_large_persistent<T>(const Args<T> &, int, int, int, size_t, cudaStream_t); \
  template cudaError_t launch_large_sub<T>(const Args<T> &, int, int, int, int, size_t, cudaStream_t);   \
  template cudaError_t launch_large_top<T>(const Args<T> &, int, size_t, cudaStream_t);

BDSS_INSTANTIATE_LARGE(double)
BDSS_INSTANTIATE_LARGE(float)

}  // namespace bdss
