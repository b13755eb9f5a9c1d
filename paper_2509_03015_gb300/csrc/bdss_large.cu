// Kernels of the large-block path (64 < n <= 256).  Each level runs three
// sub-phases of tile tasks -- A1 (Cholesky per eliminated block), A2
// (forward substitution per vector tile), B (Schur update per output tile) --
// then the FP64 top block, then the downward tasks C per level.  The
// persistent kernel separates sub-phases with the bounded grid barrier; the
// per-level mode launches one kernel per sub-phase.
#include "bdss_large.cuh"
#include "bdss_launch.h"

namespace bdss {


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

// ---------------------------------------------------------------------------
// Solve passes of the mixed-precision refinement with the stored inverses,
// streamed (FP32, n % 4 == 0, d <= 16).  Every product of a pass reads one
// n x n FP32 block once against an n x 16 operand in shared memory, 16 FMAs
// per matrix element, so the pass is HBM-bound: the blocks are streamed
// through a ring of shared-memory stages filled by the TMA engine, about
// 128 KB in flight per CTA, instead of register loads of a few KB.
//   A2 (upward, eliminated j):  y_j = L_j^{-1} b_j        rows of L^{-1}
//   B  (upward, separator s):   b_s -= Wt(s-1) y_{s-1} + Wt(s) y_{s+1}   rows of Wt
//   C  (downward, eliminated j): t = y_j - Wt(j-1)^T x_{j-1} - Wt(j)^T x_{j+1},
//                               x_j = (L_j^{-1})^T t      columns of Wt, L^{-1}
// A row product (thread r: sum_k P[r][k] v[k]) takes chunks of 32 columns of
// all n rows as one 2-D TMA box with the 128-byte swizzle (row r's 16-byte
// group q sits at q ^ (r & 7)); a column product (thread r: sum_k P[k][r]
// v[k]) takes chunks of 32 whole rows with one bulk copy.  The zeros of L^{-1}
// above its diagonal are stored, so the triangular products run over full
// squares.  Thread 0 refills a stage as soon as the CTA has consumed it;
// every wait is bounded.
// ---------------------------------------------------------------------------
static_assert(kCorrMaxD == kRowCols, "one streamed pass carries the row tasks' 16 columns");
constexpr int kCorrKR = 32;     // columns (row products) or rows (column products) per chunk
constexpr int kCorrStages = 4;  // ring depth with one CTA per SM (levels with few blocks)
constexpr int kCorrStagesPair = 2;  // ring depth with two CTAs per SM (levels with many blocks)
constexpr size_t kCorrSmemPerSM = 233472;  // shared memory of an SM (bytes)

__host__ __device__ inline int corr_pad(int n) { return (n + kCorrKR - 1) / kCorrKR * kCorrKR; }
__host__ __device__ inline size_t corr_stage_bytes(int n) { return (size_t)kCorrKR * n * sizeof(float); }
// stage stride: a multiple of 1024 bytes, the period of the 128-byte swizzle
__host__ __device__ inline size_t corr_stage_stride(int n) { return (corr_stage_bytes(n) + 1023) & ~(size_t)1023; }
// Shared memory of a streamed pass: `stages` chunks of 32 x n/P floats, two
// operand blocks and the partial sums of q threads per row.
size_t corr_smem_bytes(int n, int stages, int q, int P) {
  return stages * corr_stage_stride(n / P) + (size_t)2 * corr_pad(n) * kRowCols * sizeof(float) +
         (size_t)(q - 1) * kThreads * kRowCols * sizeof(float) + 1024;
}
size_t corr_smem_bytes(int n) {
  const size_t a = corr_smem_bytes(n, kCorrStages, 2, 1), b = corr_smem_bytes(n, kCorrStages, 4, 4);
  return a > b ? a : b;
}

struct CorrProd {
  long long row0;  // first row of the block in its buffer (block index x n)
  int trans;       // 1: column product (bulk rows), 0: row product (2-D box)
  int inLi;        // 1: the block is in Li, 0: in Wb
};

// Products of task t of sub-phase `sub` at level l (in consumption order).
__device__ __forceinline__ int corr_prods(const Args<float> &a, int l, int sub, long long t, CorrProd (&P)[3]) {
  const int n = a.p.n;
  const long long Nl = a.p.Nl[l], off = (long long)a.p.off[l];
  if (sub == kSubA2) {
    P[0] = {((2 * t + 1) << l) * n, 0, 1};
    return 1;
  }
  if (sub == kSubB) {
    const long long s = 2 * t;
    int c = 0;
    if (s >= 2) P[c++] = {(off + s - 1) * n, 0, 0};
    if (s + 1 < Nl) P[c++] = {(off + s) * n, 0, 0};
    return c;
  }
  const long long j = 2 * t + 1;
  int c = 0;
  if (sub == kSubC2) {
    P[0] = {(j << l) * n, 1, 1};
    return 1;
  }
  P[c++] = {(off + j - 1) * n, 1, 0};
  if (j + 1 < Nl) P[c++] = {(off + j) * n, 1, 0};
  if (sub == kSubC) P[c++] = {(j << l) * n, 1, 1};
  return c;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// acc[c] += sum over the columns k0 + 4 q0 .. k0 + 4 (q0 + kG) - 1 of row r of
// a swizzled box of 32 columns (kG of its eight 16-byte groups).
template <int kG>
__device__ __forceinline__ void corr_rows_chunk(const unsigned char *stage, int r, int k0, int q0, const float *V,
                                                float (&acc)[kRowCols]) {
  const unsigned char *row = stage + (size_t)r * 128;
#pragma unroll
  for (int i = 0; i < kG; ++i) {
    const int q = q0 + i;
    const float4 f = *reinterpret_cast<const float4 *>(row + ((q ^ (r & 7)) << 4));
    const float fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float4 *v4 = reinterpret_cast<const float4 *>(V + (size_t)(k0 + 4 * q + e) * kRowCols);
#pragma unroll
      for (int c4 = 0; c4 < kRowCols / 4; ++c4) {
        const float4 w = v4[c4];
        acc[4 * c4 + 0] = fmaf(fv[e], w.x, acc[4 * c4 + 0]);
        acc[4 * c4 + 1] = fmaf(fv[e], w.y, acc[4 * c4 + 1]);
        acc[4 * c4 + 2] = fmaf(fv[e], w.z, acc[4 * c4 + 2]);
        acc[4 * c4 + 3] = fmaf(fv[e], w.w, acc[4 * c4 + 3]);
      }
    }
  }
}

// acc[c] += sum over the rows kk0 .. kk1 - 1 (k0 + kk) of column r of a row chunk.
__device__ __forceinline__ void corr_cols_chunk(const float *stage, int pitch, int r, int k0, int kk0, int kk1,
                                                const float *V, float (&acc)[kRowCols]) {
#pragma unroll 4
  for (int kk = kk0; kk < kk1; ++kk) {
    const float p = stage[(size_t)kk * pitch + r];
    const float4 *v4 = reinterpret_cast<const float4 *>(V + (size_t)(k0 + kk) * kRowCols);
#pragma unroll
    for (int c4 = 0; c4 < kRowCols / 4; ++c4) {
      const float4 w = v4[c4];
      acc[4 * c4 + 0] = fmaf(p, w.x, acc[4 * c4 + 0]);
      acc[4 * c4 + 1] = fmaf(p, w.y, acc[4 * c4 + 1]);
      acc[4 * c4 + 2] = fmaf(p, w.z, acc[4 * c4 + 2]);
      acc[4 * c4 + 3] = fmaf(p, w.w, acc[4 * c4 + 3]);
    }
  }
}

// sV[k][c] = src[k][c] for k < n, c < d; zero elsewhere (rows up to the pad).
template <typename S>
__device__ __forceinline__ void corr_stage_vec(float *sV, const S *src, int n, int np, int d) {
#pragma unroll 4
  for (int e = threadIdx.x; e < np * kRowCols; e += blockDim.x) {
    const int k = e / kRowCols, c = e - k * kRowCols;
    sV[e] = (k < n && c < d) ? (float)ldcg(src + (size_t)k * d + c) : 0.0f;
  }
}

// With kQ threads per output row (each on 32 / kQ columns or rows of every
// chunk), the partial sums meet in shared memory in a fixed order: thread
// kq = 0 adds those of kq = 1, 2, ...  All threads call it.
template <int kQ>
__device__ __forceinline__ void corr_reduce(float (&acc)[kRowCols], float *red, int rl, int kq) {
  if constexpr (kQ > 1) {
    if (kq > 0) {
      float4 *dst = reinterpret_cast<float4 *>(red + ((size_t)(kq - 1) * kThreads + rl) * kRowCols);
#pragma unroll
      for (int q = 0; q < kRowCols / 4; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
    __syncthreads();
    if (kq == 0) {
#pragma unroll
      for (int i = 1; i < kQ; ++i) {
        const float4 *src = reinterpret_cast<const float4 *>(red + ((size_t)(i - 1) * kThreads + rl) * kRowCols);
#pragma unroll
        for (int q = 0; q < kRowCols / 4; ++q) {
          const float4 v = src[q];
          acc[4 * q] += v.x;
          acc[4 * q + 1] += v.y;
          acc[4 * q + 2] += v.z;
          acc[4 * q + 3] += v.w;
        }
      }
    }
  }
}

template <int kQ>
__global__ void __launch_bounds__(kQ == 2 ? 2 * kThreads : kThreads, kQ == 1 ? 2 : 1)
    k_large_corr(const __grid_constant__ CorrMaps maps, const __grid_constant__ Args<float> a, int l, int sub,
                 int stages, int P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t full[kCorrStages], vbar;
  __shared__ int s_ok;
  // one read of the status decides for the whole CTA
  if (threadIdx.x == 0) s_ok = ld_relaxed_i32(&a.st->status) == 0;
  __syncthreads();
  if (!s_ok) return;
  const int n = a.p.n, d = a.d, np = corr_pad(n);
  // work item = (block, part h of P); thread = (row or column r of the part,
  // share kq of every chunk); g = h R + r indexes the block's data
  const int RT = blockDim.x / kQ, R = n / P;
  const int r = threadIdx.x % RT, kq = threadIdx.x / RT;
  const bool active = r < R;
  const bool cols = (sub == kSubC || sub == kSubC1 || sub == kSubC2);
  const long long Nl = a.p.Nl[l];
  const long long tasks = (sub == kSubB) ? (Nl + 1) / 2 : Nl / 2, items = tasks * P;
  const size_t SB = corr_stage_bytes(R), SS = corr_stage_stride(R), nd = (size_t)n * d;
  const int nch = (n + kCorrKR - 1) / kCorrKR;
  // 1024-byte aligned ring, by pointer arithmetic on the shared array so that
  // the compiler keeps shared-memory loads (an integer round trip would make
  // every read below a generic load)
  unsigned char *ring = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float *sV0 = reinterpret_cast<float *>(ring + stages * SS);
  float *sV1 = sV0 + (size_t)np * kRowCols;
  float *red = sV1 + (size_t)np * kRowCols;  // (kQ - 1) x 256 x 16 partial sums
  if (threadIdx.x == 0) {
    for (int s = 0; s < stages; ++s) mbar_init(&full[s], 1);
    mbar_init(&vbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  // producer cursor (thread 0): work item pt, product pp, chunk pc
  long long pt = blockIdx.x;
  int pp = 0, pc = 0, pn = 0;
  CorrProd PP[3];
  long long issued = 0;
  auto issue = [&](int stage) {
    while (pt < items && pp >= pn) {
      pt += gridDim.x;
      pp = 0;
      pc = 0;
      pn = pt < items ? corr_prods(a, l, sub, pt / P, PP) : 0;
    }
    if (pt >= items) return;
    const CorrProd &Q = PP[pp];
    const int h = (int)(pt % P);
    unsigned char *dst = ring + (size_t)stage * SS;
    if (!Q.trans) {
      // rows h R .. h R + R - 1 of the block, columns pc*32 .. +31
      mbar_expect_tx(&full[stage], (uint32_t)SB);
      tma_load_2d(dst, Q.inLi ? &maps.rowsLi : &maps.rowsW, pc * kCorrKR, (int)(Q.row0 + (long long)h * R),
                  &full[stage]);
    } else if (P > 1) {
      // rows pc*32 .. +31 of the block, columns h R .. h R + R - 1
      mbar_expect_tx(&full[stage], (uint32_t)SB);
      tma_load_2d(dst, Q.inLi ? &maps.colsLi : &maps.colsW, h * R, (int)(Q.row0 + (long long)pc * kCorrKR),
                  &full[stage]);
    } else {
      const int rows = min(kCorrKR, n - pc * kCorrKR);
      const uint32_t bytes = (uint32_t)((size_t)rows * n * sizeof(float));
      const float *src = (Q.inLi ? a.Li : a.Wb) + (size_t)(Q.row0 + (long long)pc * kCorrKR) * n;
      mbar_expect_tx(&full[stage], bytes);
      bulk_load(dst, src, bytes, &full[stage]);
    }
    ++issued;
    if (++pc == nch) {
      pc = 0;
      ++pp;
    }
  };
  if (threadIdx.x == 0) {
    pn = pt < items ? corr_prods(a, l, sub, pt / P, PP) : 0;
    for (int s = 0; s < stages; ++s) issue(s);
  }
  bool vpend = false;  // an operand copy may still be in flight (timeout path)
  int cs = 0;
  uint32_t cph = 0, vph = 0;
  long long consumed = 0;
  bool ok = true;
  const float *ys = a.Yt ? a.Yt : a.Y;  // y of the eliminated blocks in this pass
  // rows n .. np - 1 of the operands stay zero (only rows < n are written)
  for (int e = n * kRowCols + threadIdx.x; e < np * kRowCols; e += blockDim.x) sV0[e] = sV1[e] = 0.0f;
  // with 16 columns an operand block is n x 16 contiguous floats: one bulk copy
  const bool bulkV = (d == kRowCols);
  const uint32_t vbytes = (uint32_t)((size_t)n * kRowCols * sizeof(float));
  for (long long u = blockIdx.x; u < items && ok; u += gridDim.x) {
    const long long t = u / P;
    const int g = (int)(u % P) * R + r;  // row / column of the block this thread serves
    long long orig;
    bool hasM = false;
    int npr;
    const float *src0 = nullptr, *src1 = nullptr, *yj = nullptr;
    const double *src0d = nullptr;
    if (sub == kSubA2) {
      orig = (2 * t + 1) << l;
      const size_t bo = (size_t)orig * nd;
      if (l == 0 && a.B64) src0d = a.B64 + bo;
      else src0 = ((l == 0 && a.Bt) ? a.Bt : a.Y) + bo;
      npr = 1;
    } else if (sub == kSubB) {
      const long long s = 2 * t;
      orig = s << l;
      hasM = s >= 2;
      const bool hasP = s + 1 < Nl;
      if (hasM) src0 = ys + (size_t)((s - 1) << l) * nd;
      if (hasP) src1 = ys + (size_t)((s + 1) << l) * nd;
      npr = (int)hasM + (int)hasP;
    } else if (sub == kSubC2) {
      const long long j = 2 * t + 1;
      orig = j << l;
      src0 = ys + (size_t)orig * nd;  // t, formed by C1 in place of y_j
      npr = 1;
    } else {
      const long long j = 2 * t + 1;
      orig = j << l;
      const bool hasR = j + 1 < Nl;
      src0 = a.Y + (size_t)((j - 1) << l) * nd;
      if (hasR) src1 = a.Y + (size_t)((j + 1) << l) * nd;
      yj = ys + (size_t)orig * nd;  // y_j: read at the t step, fetched into L2 now
      if (active && kq == 0) prefetch_l2(yj + (size_t)g * d, (size_t)d * sizeof(float));
      npr = (sub == kSubC1) ? (hasR ? 2 : 1) : (hasR ? 3 : 2);
    }
    const uint32_t nsrc = (src0 ? 1u : 0u) + (src1 ? 1u : 0u);
    if (bulkV && !src0d) {
      if (nsrc > 0) {
        if (threadIdx.x == 0) {
          fence_proxy_async_smem();
          mbar_expect_tx(&vbar, nsrc * vbytes);
          if (src0) bulk_load(sV0, src0, vbytes, &vbar);
          if (src1) bulk_load(sV1, src1, vbytes, &vbar);
        }
        if (!mbar_wait_cta(&vbar, vph, a.timeout_ns, &s_ok)) {
          if (threadIdx.x == 0) set_status(a.st, kStTimeout, l, -1);
          vpend = true;
          ok = false;
          break;
        }
        vph ^= 1;
      }
    } else {
      if (src0d) corr_stage_vec(sV0, src0d, n, np, d);
      if (src0) corr_stage_vec(sV0, src0, n, np, d);
      if (src1) corr_stage_vec(sV1, src1, n, np, d);
      __syncthreads();
    }
    float acc[kRowCols];
#pragma unroll
    for (int c = 0; c < kRowCols; ++c) acc[c] = 0.0f;
    for (int p = 0; p < npr && ok; ++p) {
      const bool lastC = (sub == kSubC && p == npr - 1);
      if (lastC) {
        // t = y_j - (W_L x_{j-1} + W_R x_{j+1}) into sV0, free once the W
        // products are done (the last chunk ended with a barrier)
        corr_reduce<kQ>(acc, red, r, kq);
        if (active && kq == 0) {
          const float *yr = yj + (size_t)g * d;
          if (d == kRowCols) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 y4 = __ldcg(reinterpret_cast<const float4 *>(yr) + q);
              sV0[r * kRowCols + 4 * q + 0] = y4.x - acc[4 * q + 0];
              sV0[r * kRowCols + 4 * q + 1] = y4.y - acc[4 * q + 1];
              sV0[r * kRowCols + 4 * q + 2] = y4.z - acc[4 * q + 2];
              sV0[r * kRowCols + 4 * q + 3] = y4.w - acc[4 * q + 3];
            }
          } else {
#pragma unroll
            for (int c = 0; c < kRowCols; ++c) sV0[r * kRowCols + c] = (c < d) ? ldcg(yr + c) - acc[c] : 0.0f;
          }
        }
#pragma unroll
        for (int c = 0; c < kRowCols; ++c) acc[c] = 0.0f;
        __syncthreads();
      }
      const float *V = (sub == kSubA2 || sub == kSubC2) ? sV0
                       : (sub == kSubB)                  ? ((p == 0 && hasM) ? sV0 : sV1)
                       : (lastC || p == 0)               ? sV0
                                                         : sV1;
      for (int c = 0; c < nch; ++c) {
        if (!mbar_wait_cta(&full[cs], cph, a.timeout_ns, &s_ok)) {
          if (threadIdx.x == 0) set_status(a.st, kStTimeout, l, -1);
          ok = false;
          break;
        }
        const unsigned char *stage = ring + (size_t)cs * SS;
        if (active) {
          if (cols) {
            const int rows = min(kCorrKR, n - c * kCorrKR), per = kCorrKR / kQ;
            corr_cols_chunk(reinterpret_cast<const float *>(stage), P > 1 ? R : n, r, c * kCorrKR, kq * per,
                            min(rows, (kq + 1) * per), V, acc);
          } else {
            corr_rows_chunk<8 / kQ>(stage, r, c * kCorrKR, kq * (8 / kQ), V, acc);
          }
        }
        __syncthreads();  // every thread is done with the stage
        ++consumed;
        if (threadIdx.x == 0) {
          fence_proxy_async_smem();
          issue(cs);
        }
        if (++cs == stages) {
          cs = 0;
          cph ^= 1;
        }
      }
    }
    if (!ok) continue;
    corr_reduce<kQ>(acc, red, r, kq);
    if (!active || kq != 0) continue;
    const size_t o = (size_t)orig * nd + (size_t)g * d;
    if (d == kRowCols) {
      // a thread's row of the block is 16 contiguous values
      if (sub == kSubA2) {
        float4 *dst = reinterpret_cast<float4 *>(a.Yt + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
      } else if (sub == kSubB) {
        float base[kRowCols];
        if (l == 0 && a.B64) {
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const double2 b2 = __ldcg(reinterpret_cast<const double2 *>(a.B64 + o) + q);
            base[2 * q] = (float)b2.x;
            base[2 * q + 1] = (float)b2.y;
          }
        } else {
          const float *bs = (l == 0 && a.Bt) ? a.Bt : a.Y;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 b4 = __ldcg(reinterpret_cast<const float4 *>(bs + o) + q);
            base[4 * q] = b4.x;
            base[4 * q + 1] = b4.y;
            base[4 * q + 2] = b4.z;
            base[4 * q + 3] = b4.w;
          }
        }
        float4 *dst = reinterpret_cast<float4 *>(a.Y + o);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          dst[q] = make_float4(base[4 * q] - acc[4 * q], base[4 * q + 1] - acc[4 * q + 1],
                               base[4 * q + 2] - acc[4 * q + 2], base[4 * q + 3] - acc[4 * q + 3]);
      } else if (sub == kSubC1) {
        // t = y_j - (W_L x_{j-1} + W_R x_{j+1}), in place of y_j
        float4 *yt = reinterpret_cast<float4 *>(const_cast<float *>(ys) + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 y4 = __ldcg(yt + q);
          yt[q] = make_float4(y4.x - acc[4 * q], y4.y - acc[4 * q + 1], y4.z - acc[4 * q + 2], y4.w - acc[4 * q + 3]);
        }
      } else {
        float4 *dst = reinterpret_cast<float4 *>(a.Y + o);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        if (a.X64) {
          double2 *x2 = reinterpret_cast<double2 *>(a.X64 + o);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            double2 v = make_double2((double)acc[2 * q], (double)acc[2 * q + 1]);
            if (a.x_accumulate) {
              const double2 old = x2[q];
              v.x += old.x;
              v.y += old.y;
            }
            x2[q] = v;
          }
        }
      }
    } else if (sub == kSubA2) {
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c < d) a.Yt[o + c] = acc[c];
    } else if (sub == kSubC1) {
      float *yt = const_cast<float *>(ys) + o;
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c < d) yt[c] = ldcg(yt + c) - acc[c];
    } else if (sub == kSubB) {
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c < d) {
          float base;
          if (l == 0 && a.B64) base = (float)ldcg(a.B64 + o + c);
          else if (l == 0 && a.Bt) base = ldcg(a.Bt + o + c);
          else base = ldcg(a.Y + o + c);
          a.Y[o + c] = base - acc[c];
        }
    } else {
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c < d) {
          a.Y[o + c] = acc[c];
          if (a.X64) a.X64[o + c] = a.x_accumulate ? a.X64[o + c] + (double)acc[c] : (double)acc[c];
        }
    }
  }
  // after a timeout: wait out the copies still in flight before the CTA ends
  if (threadIdx.x == 0 && vpend) mbar_wait(&vbar, vph, a.timeout_ns);
  if (threadIdx.x == 0 && issued > consumed) {
    int s = cs;
    uint32_t ph = cph;
    for (long long k = consumed; k < issued; ++k) {
      mbar_wait(&full[s], ph, a.timeout_ns);
      if (++s == stages) {
        s = 0;
        ph ^= 1;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// TF32 Schur products on the tensor cores, pipelined (the separator update of
// Algorithm 3 in the TF32 mode of the tiled path).  An output tile of
// 128 x 128 (D's lower part: one round per eliminated neighbour, accumulated;
// E: one round) takes, per K chunk of 32, twelve tcgen05.mma (kind::tf32,
// K = 8): hi*hi + hi*lo + lo*hi, the 3xTF32 product, into an FP32
// accumulator in TMEM, where hi is W rounded to TF32 and lo = W - hi.
// Roles (320 threads):
//   warp 0     TMA: the raw W slabs of the A and B rows (2 x 16 KB per chunk)
//              into a ring of two stages;
//   warps 6-9  split each raw stage into hi and lo slabs (the swizzled
//              layout is element-position preserving) in a second ring;
//   warp 1     one thread issues the MMAs of a split stage and commits it;
//   warps 2-5  drain the accumulator, two buffers, so that a tile's
//              epilogue runs under the next tile's products.
// Every wait is bounded; a timed-out wait aborts every role.
// ---------------------------------------------------------------------------
constexpr int kTsRaw = 2 * kTcSlab;     // raw A | B of one chunk
constexpr int kTsSplit = 4 * kTcSlab;   // A hi | A lo | B hi | B lo
constexpr int kTsStages = 2;            // stages of each ring
constexpr int kTsThreads = 320;
constexpr int kTsSplitters = 128;       // warps 6-9
constexpr uint32_t kTsTmemCols = 2 * kTcN;
constexpr size_t kTsSmem = (size_t)kTsStages * (kTsRaw + kTsSplit) + 1024;

__device__ __forceinline__ bool ts_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait; gives up early when another role aborted (abort != null).
__device__ __forceinline__ bool ts_wait(uint64_t *bar, uint32_t parity, long long timeout_ns, volatile int *abort) {
  long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    if (ts_try(bar, parity)) return true;
    if ((it & 63) == 63) {
      if (abort && *abort) return false;
      const long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive_local(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct TsTile {
  long long k;       // separator 2k
  int isD, ti, tj, nr;
  // rows (in the W buffer) of the A and B operands of rounds 0 and 1; scalar
  // fields, so that the tile stays in registers
  long long ra0, ra1, rb0, rb1;
  __device__ long long a_of(int r) const { return r == 0 ? ra0 : ra1; }
  __device__ long long b_of(int r) const { return r == 0 ? rb0 : rb1; }
};

__device__ __forceinline__ TsTile ts_tile(const Args<float> &a, int l, long long u) {
  const int n = a.p.n, nt = (n + kTcM - 1) / kTcM, nD = nt * (nt + 1) / 2, per = nD + nt * nt;
  const long long Nl = a.p.Nl[l], slot0 = a.p.off[l];
  TsTile T;
  T.k = u / per;
  const int t = (int)(u - T.k * per);
  const long long s = 2 * T.k;
  T.nr = 0;
  T.ra0 = T.ra1 = T.rb0 = T.rb1 = 0;
  if (t < nD) {
    T.isD = 1;
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    T.ti = ti;
    T.tj = t - ti * (ti + 1) / 2;
    const long long bm = (slot0 + s - 1) * n, bp = (slot0 + s) * n;
    const bool hasM = s >= 2, hasP = s + 1 < Nl;
    // round 0: the left neighbour if present, else the right one
    T.ra0 = (hasM ? bm : bp) + T.ti * kTcM;
    T.rb0 = (hasM ? bm : bp) + T.tj * kTcM;
    T.ra1 = bp + T.ti * kTcM;
    T.rb1 = bp + T.tj * kTcM;
    T.nr = (int)hasM + (int)hasP;
  } else {
    T.isD = 0;
    T.ti = (t - nD) / nt;
    T.tj = (t - nD) - T.ti * nt;
    if (s + 2 < Nl) {
      T.ra0 = (slot0 + s + 1) * n + T.ti * kTcM;
      T.rb0 = (slot0 + s) * n + T.tj * kTcM;
      T.nr = 1;
    }
  }
  return T;
}

__global__ void __launch_bounds__(kTsThreads, 1)
    k_tf32_schur(const __grid_constant__ CUtensorMap mapW, const __grid_constant__ Args<float> a, int l) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t tfull[kTsStages], tempty[kTsStages], sfull[kTsStages], sempty[kTsStages];
  __shared__ uint64_t acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort, s_go;
  if (threadIdx.x == 0) s_go = ld_relaxed_i32(&a.st->status) == 0;
  __syncthreads();
  if (!s_go) return;
  unsigned char *raw = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char *split = raw + (size_t)kTsStages * kTsRaw;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.p.n, nt = (n + kTcM - 1) / kTcM, kchunks = (n + kTcK - 1) / kTcK;
  const long long Nl = a.p.Nl[l];
  const long long tiles = ((Nl + 1) / 2) * (long long)(nt * (nt + 1) / 2 + nt * nt);
  volatile int *abort = &s_abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kTsStages; ++s) {
      mbar_init(&tfull[s], 1);
      mbar_init(&tempty[s], kTsSplitters);
      mbar_init(&sfull[s], kTsSplitters);
      mbar_init(&sempty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    mbar_init(&drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&s_tmem, kTsTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  auto fail = [&]() {
    *abort = 1;
    set_status(a.st, kStTimeout, l, -1);
  };

  if (warp == 0) {
    // ---- TMA producer: raw slabs ------------------------------------------------
    if (lane == 0) {
      int st = 0;
      uint32_t ph = 0;
      bool stop = false;
      for (long long u = blockIdx.x; u < tiles && !stop; u += gridDim.x) {
        const TsTile T = ts_tile(a, l, u);
        for (int r = 0; r < T.nr && !stop; ++r)
          for (int kc = 0; kc < kchunks; ++kc) {
            if (!ts_wait(&tempty[st], ph ^ 1, a.timeout_ns, abort)) {
              fail();
              stop = true;
              break;
            }
            unsigned char *base = raw + (size_t)st * kTsRaw;
            mbar_expect_tx(&tfull[st], kTsRaw);
            tma_load_2d(base, &mapW, kc * kTcK, (int)T.a_of(r), &tfull[st]);
            tma_load_2d(base + kTcSlab, &mapW, kc * kTcK, (int)T.b_of(r), &tfull[st]);
            if (++st == kTsStages) { st = 0; ph ^= 1; }
          }
      }
      // wait out the loads still in flight (each stage's last armed phase)
      for (int s = 0; s < kTsStages; ++s) ts_wait(&tfull[s], (s < st) ? ph : (ph ^ 1), a.timeout_ns, nullptr);
    }
  } else if (warp >= 6) {
    // ---- split warps: raw -> hi | lo -------------------------------------------
    const int sid = threadIdx.x - 6 * 32;
    int ts = 0, ss = 0;
    uint32_t tph = 0, sph = 0;
    bool stop = false;
    for (long long u = blockIdx.x; u < tiles && !stop; u += gridDim.x) {
      const TsTile T = ts_tile(a, l, u);
      for (int r = 0; r < T.nr && !stop; ++r)
        for (int kc = 0; kc < kchunks; ++kc) {
          // warp-uniform waits: lane 0 polls, the others then observe the phase
          int ok = 0;
          if (lane == 0)
            ok = (ts_wait(&tfull[ts], tph, a.timeout_ns, abort) && ts_wait(&sempty[ss], sph ^ 1, a.timeout_ns, abort))
                     ? 1
                     : 0;
          ok = __shfl_sync(0xffffffffu, ok, 0);
          if (!ok) {
            if (lane == 0) fail();
            stop = true;
            break;
          }
          if (lane != 0) {
            ts_try(&tfull[ts], tph);
            ts_try(&sempty[ss], sph ^ 1);
          }
          const float4 *src = reinterpret_cast<const float4 *>(raw + (size_t)ts * kTsRaw);
          unsigned char *dst = split + (size_t)ss * kTsSplit;
#pragma unroll 4
          for (int i = sid; i < kTsRaw / 16; i += kTsSplitters) {
            const int which = i / (kTcSlab / 16), j = i - which * (kTcSlab / 16);  // A or B, float4 in slab
            const float4 x = src[i];
            float4 h, o;
            const float xs[4] = {x.x, x.y, x.z, x.w};
            float hs[4], os[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              hs[q] = __uint_as_float((__float_as_uint(xs[q]) + 0x1000u) & 0xFFFFE000u);
              os[q] = xs[q] - hs[q];
            }
            h = make_float4(hs[0], hs[1], hs[2], hs[3]);
            o = make_float4(os[0], os[1], os[2], os[3]);
            reinterpret_cast<float4 *>(dst + (size_t)which * 2 * kTcSlab)[j] = h;
            reinterpret_cast<float4 *>(dst + (size_t)which * 2 * kTcSlab + kTcSlab)[j] = o;
          }
          fence_proxy_async_smem();  // the MMAs read the split slabs through the async proxy
          mbar_arrive_local(&tempty[ts]);
          mbar_arrive_local(&sfull[ss]);
          if (++ts == kTsStages) { ts = 0; tph ^= 1; }
          if (++ss == kTsStages) { ss = 0; sph ^= 1; }
        }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = tc_idesc_tf32(kTcM, kTcN);
      int st = 0;
      uint32_t ph = 0;
      long long i = 0;  // tiles with work so far: accumulator buffer i & 1
      bool stop = false;
      for (long long u = blockIdx.x; u < tiles && !stop; u += gridDim.x) {
        const TsTile T = ts_tile(a, l, u);
        if (T.nr == 0) continue;
        const int b = (int)(i & 1);
        if (!ts_wait(&acc_empty[b], (uint32_t)((i >> 1) & 1), a.timeout_ns, abort)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kTcN);
        bool first = true;
        for (int r = 0; r < T.nr && !stop; ++r)
          for (int kc = 0; kc < kchunks; ++kc) {
            if (!ts_wait(&sfull[st], ph, a.timeout_ns, abort)) {
              fail();
              stop = true;
              break;
            }
            tc_fence_after();
            const unsigned char *base = split + (size_t)st * kTsSplit;
            const unsigned char *Ahi = base, *Alo = base + kTcSlab, *Bhi = base + 2 * kTcSlab,
                                *Blo = base + 3 * kTcSlab;
#pragma unroll
            for (int kk = 0; kk < kTcK / 8; ++kk) {
              const int off = kk * 32;  // 8 TF32 = 32 bytes along K inside the swizzle atom
              tc_mma_tf32(d, tc_desc_sw128(Ahi, off), tc_desc_sw128(Bhi, off), idesc, first ? 0u : 1u);
              first = false;
              tc_mma_tf32(d, tc_desc_sw128(Ahi, off), tc_desc_sw128(Blo, off), idesc, 1u);
              tc_mma_tf32(d, tc_desc_sw128(Alo, off), tc_desc_sw128(Bhi, off), idesc, 1u);
            }
            tc_commit(&sempty[st]);
            if (++st == kTsStages) { st = 0; ph ^= 1; }
          }
        if (stop) break;
        tc_commit(&acc_full[b]);
        ++i;
      }
      // every MMA issued has completed before TMEM is released
      tc_commit(&drain);
      ts_wait(&drain, 0, a.timeout_ns, nullptr);
    }
  } else {
    // ---- epilogue: warps 2..5, TMEM lane quarter warp % 4 ---------------------
    const int quarter = warp & 3;
    const size_t nn = (size_t)n * n;
    tc_fence_before();
    mbar_arrive_local(&acc_empty[0]);
    mbar_arrive_local(&acc_empty[1]);
    long long i = 0;
    for (long long u = blockIdx.x; u < tiles; u += gridDim.x) {
      const TsTile T = ts_tile(a, l, u);
      if (T.nr == 0) continue;
      const int b = (int)(i & 1);
      int ok = 0;
      if (lane == 0) ok = ts_wait(&acc_full[b], (uint32_t)((i >> 1) & 1), a.timeout_ns, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      if (lane != 0) ts_try(&acc_full[b], (uint32_t)((i >> 1) & 1));
      tc_fence_after();
      const int R = T.ti * kTcM + 32 * quarter + lane;
      const long long s = 2 * T.k, orig = s << l;
      const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(b * kTcN);
#pragma unroll 1
      for (int cb = 0; cb < kTcN / 32; ++cb) {
        float v[32];
        tmem_ld32(taddr + (uint32_t)(cb * 32), v);
        if (R >= n) continue;
        const int C0 = T.tj * kTcN + cb * 32;
        if (T.isD) {
          if (C0 > R) continue;  // the block lies above the diagonal for this row
          float *Dg = a.Ld + (size_t)orig * nn + (size_t)R * n;
          float base[32];
          // every load of the block first (independent, in flight together),
          // then the stores
          if (l == 0) {
            const double *Ag = a.A_diag + (size_t)orig * nn;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int C = C0 + j;
              const bool in = C <= R && C < n;
              const double x = in ? ldcg(Ag + (size_t)R * n + C) : 0.0;
              const double y = in ? ldcg(Ag + (size_t)C * n + R) : 0.0;
              base[j] = 0.5f * ((float)x + (float)y);
            }
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int C = C0 + j;
              base[j] = (C <= R && C < n) ? ldcg(Dg + C) : 0.0f;
            }
          }
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int C = C0 + j;
            if (C <= R && C < n) Dg[C] = base[j] - v[j];
          }
        } else {
          float *Eg = a.Eb + ((size_t)a.p.off[l + 1] + (size_t)T.k) * nn + (size_t)R * n;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int C = C0 + j;
            if (C < n) Eg[C] = -v[j];
          }
        }
      }
      tc_fence_before();
      mbar_arrive_local(&acc_empty[b]);
      ++i;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTsTmemCols);
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
                           (const void *)k_tc_selftest, (const void *)k_large_corr<1>,
                           (const void *)k_large_corr<2>, (const void *)k_large_corr<4>,
                           (const void *)k_tf32_schur};
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

// Split factor of a level's streamed pass: with few blocks each block's
// output rows (or columns) are shared by P CTAs on different SMs (n a
// multiple of 32, so that every chunk stays inside its block).
int corr_split(int n, long long tasks, int sms, int max_split) {
  if (n % 32 != 0) return 1;
  if (max_split >= 4 && tasks * 4 <= sms) return 4;
  if (max_split >= 2 && tasks * 2 <= sms) return 2;
  return 1;
}

cudaError_t launch_large_corr(const CorrMaps *maps, int max_split, const Args<float> &a, int l, int sub, int sms,
                              cudaStream_t s) {
  const int n = a.p.n;
  const long long Nl = a.p.Nl[l];
  const long long tasks = (sub == kSubB) ? (Nl + 1) / 2 : Nl / 2;
  if (tasks <= 0) return cudaSuccess;
  const int P = corr_split(n, tasks, sms, max_split);
  if (P == 1 && (sub == kSubC1 || sub == kSubC2)) return cudaErrorInvalidValue;  // the fused C serves P = 1
  if (P > 1) {
    const long long items = tasks * P;
    const int grid = (int)(items < sms ? items : sms);
    const CorrMaps &m = maps[P == 2 ? 1 : 2];
    if (P == 2)
      k_large_corr<2><<<grid, kThreads, corr_smem_bytes(n, kCorrStages, 2, 2), s>>>(m, a, l, sub, kCorrStages, 2);
    else
      k_large_corr<4><<<grid, kThreads, corr_smem_bytes(n, kCorrStages, 4, 4), s>>>(m, a, l, sub, kCorrStages, 4);
    return cudaGetLastError();
  }
  // many blocks: two CTAs per SM with a two-stage ring each (more warps to
  // hide latency, the same bytes in flight);
  //   few blocks: one CTA per block, two threads per row, a deeper ring
  const bool pair =
      tasks >= 2LL * sms && 2 * (corr_smem_bytes(n, kCorrStagesPair, 1, 1) + 1024) <= kCorrSmemPerSM;
  const long long cap = pair ? 2LL * sms : (long long)sms;
  const int grid = (int)(tasks < cap ? tasks : cap);
  if (pair)
    k_large_corr<1><<<grid, kThreads, corr_smem_bytes(n, kCorrStagesPair, 1, 1), s>>>(maps[0], a, l, sub,
                                                                                   kCorrStagesPair, 1);
  else
    k_large_corr<2><<<grid, 2 * kThreads, corr_smem_bytes(n, kCorrStages, 2, 1), s>>>(maps[0], a, l, sub,
                                                                                   kCorrStages, 1);
  return cudaGetLastError();
}

cudaError_t launch_tf32_schur(const CUtensorMap &mapW, const Args<float> &a, int l, int sms, cudaStream_t s) {
  const int n = a.p.n, nt = (n + kTcM - 1) / kTcM;
  const long long tiles = ((a.p.Nl[l] + 1) / 2) * (long long)(nt * (nt + 1) / 2 + nt * nt);
  if (tiles <= 0) return cudaSuccess;
  const int grid = (int)(tiles < sms ? tiles : sms);
  k_tf32_schur<<<grid, kTsThreads, kTsSmem, s>>>(mapW, a, l);
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

cudaError_t make_f32_map(CUtensorMap *out, const float *base, long long rows, int n, int box_rows);
cudaError_t make_w_tensor_map(CUtensorMap *out, const float *Wb, long long rows, int n) {
  return make_f32_map(out, Wb, rows, n, kTcM);
}

// 2-D map over `rows` rows of n floats: boxes of 32 columns x box_rows rows,
// 128-byte swizzle.
cudaError_t make_f32_map_box(CUtensorMap *out, const float *base, long long rows, int n, int box_cols,
                             int box_rows, bool swizzle);
cudaError_t make_f32_map(CUtensorMap *out, const float *base, long long rows, int n, int box_rows) {
  return make_f32_map_box(out, base, rows, n, kTcK, box_rows, true);
}

// General form: boxes of box_cols x box_rows; the 128-byte swizzle needs
// box_cols = 32.
cudaError_t make_f32_map_box(CUtensorMap *out, const float *base, long long rows, int n, int box_cols,
                             int box_rows, bool swizzle) {
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
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, (void *)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
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
