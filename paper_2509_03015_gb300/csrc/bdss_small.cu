// One-cluster path for short systems of small blocks (FP64, n <= 32).
//
// The recursion of Sec. 3 (Algorithms 4 and 7 with interior segments of
// length one) is the same as in the persistent kernel, but the whole call is
// one launch of a single thread-block cluster (up to 16 CTAs on 16 SMs of one
// GPC): the phases are separated by the cluster's hardware barrier instead of
// grid-wide barriers on a counter in global memory, and the launch needs no
// cooperative co-residency check.  At N = 64, n = 8 a level's work is a few
// dozen blocks, so the time of a call is the chain of dependent steps: every
// task stages all of its operands with one round of loads, then computes
// (the Cholesky of phase A fused with the substitutions of both couplings and
// of the right-hand sides), then stores.
//
// The workspace and the factor storage are the handle's (Ld, Wb, Ltop, Y)
// in the same layout as the persistent kernel, so a factorisation made here
// is solved, differentiated and its log-determinant read by the other paths,
// and every entry receives the same floating-point operations in the same
// order as there: the results are bitwise those of the persistent kernel.
//
// The status word is cleared by the kernel itself and its outcome written
// to the caller's page-locked copy at the end, so a call is one launch and
// one stream synchronisation (no memset, no device-to-host copy).
#include <cooperative_groups.h>

#include <algorithm>

#include "bdss_device.cuh"
#include "bdss_launch.h"
#include "bdss_small.h"

namespace cg = cooperative_groups;

namespace bdss {

// Shared-memory words (doubles) of the phases at (n, d):
//   A: L, 2n coupling vectors, d RHS vectors;
//   B: three W^T blocks, two sets of d vectors, the separator's D and b;
//   C: L, two W^T blocks, three sets of d vectors;
//   top block / serial top sweep: (2n + d) rows.
size_t small_smem_bytes(int n, int d) {
  const size_t ld = (size_t)ldstride(n);
  size_t w = (size_t)(3 * n + d) * ld;
  w = std::max(w, (size_t)(4 * n + 2 * d) * ld + (size_t)n * d);
  w = std::max(w, (size_t)(3 * n + 3 * d) * ld);
  w = std::max(w, (size_t)(2 * n + d) * ld);
  return (w + 8) * sizeof(double);
}

__device__ __forceinline__ int round32(int x) { return (x + 31) & ~31; }

// Staging in one round.  A phase's operands come from several blocks in L2
// (or in page-locked host memory at level 0); staging them block by block
// costs one dependent round trip each (about half a microsecond in L2).
// A StageList names up to kMaxSegs row-major rows x cols sources and their
// shared-memory destinations (stride ld; as rows, or transposed so that the
// columns become rows), and stage_round has every thread issue the loads of
// up to kStageUnroll elements before any of their stores.
constexpr int kMaxSegs = 7;
constexpr int kStageUnroll = 8;
struct StageSeg {
  const double *src;
  double *dst;
  int rows, cols, ld, transpose;
};
struct StageList {
  StageSeg seg[kMaxSegs];
  int count = 0;
  __device__ void add(const double *src, double *dst, int rows, int cols, int ld, int transpose) {
    seg[count++] = StageSeg{src, dst, rows, cols, ld, transpose};
  }
};
// All threads call; no barrier inside.
__device__ void stage_round(const StageList &g) {
  int start[kMaxSegs + 1];
  start[0] = 0;
  for (int i = 0; i < g.count; ++i) start[i + 1] = start[i] + g.seg[i].rows * g.seg[i].cols;
  const int total = start[g.count];
  for (int base = 0; base < total; base += kStageUnroll * (int)blockDim.x) {
    double v[kStageUnroll];
    double *dst[kStageUnroll];
#pragma unroll
    for (int u = 0; u < kStageUnroll; ++u) {
      const int e = base + u * (int)blockDim.x + (int)threadIdx.x;
      dst[u] = nullptr;
      if (e < total) {
        int i = 0;
        while (i + 1 < g.count && e >= start[i + 1]) ++i;
        const StageSeg &sg = g.seg[i];
        const int f = e - start[i], r = f / sg.cols, c = f - r * sg.cols;
        v[u] = __ldcg(sg.src + f);
        dst[u] = sg.dst + (sg.transpose ? c * sg.ld + r : r * sg.ld + c);
      }
    }
#pragma unroll
    for (int u = 0; u < kStageUnroll; ++u)
      if (dst[u]) *dst[u] = v[u];
  }
}

// Lower triangle of a staged caller block <- sym(A) = (A + A^T) / 2, the same
// operations as stage_sym_lower.  All threads call; no barrier inside.
__device__ void sym_lower_inplace(double *s, int ld, int n) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e - i * n;
    if (c < i) s[i * ld + c] = 0.5 * (s[i * ld + c] + s[c * ld + i]);
  }
}

// Phase A, eliminated position j of level l (Algorithm 1's potrf and trsm,
// Algorithm 5's interior solve):
//   L_j = chol(D_j), W_L = L_j^{-1} A_{j,j-1}, W_R = L_j^{-1} A_{j+1,j}^T,
//   y_j = L_j^{-1} b_j,
// all in one sweep of chol_fused, with the operands staged in one round.
// Level 0 reads the caller's blocks; level l >= 1 the Schur-updated diagonal
// (Ld) and the couplings of region l, which this task then overwrites with
// its W^T.  Without factor, only y_j with the stored L_j.  Only the lower
// triangles of the staged diagonal blocks are used.
__device__ bool small_phaseA(const Args<double> &a, int l, long long j, bool factor, double *smem, int *s_flag) {
  const int n = a.p.n, ld = ldstride(n), d = a.d;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  const int nv = factor ? (hasR ? 2 * n : n) : 0;
  double *sL = smem;
  double *sV = sL + (size_t)n * ld;        // columns of A_{j,j-1}, then rows of A_{j+1,j}
  double *sB = sV + (size_t)nv * ld;       // d RHS vectors
  double *W = a.Wb + (size_t)a.p.off[l] * nn;
  StageList g;
  if (factor) {
    g.add((l == 0 ? a.A_diag : a.Ld) + (size_t)orig * nn, sL, n, n, ld, 0);
    g.add((l == 0 ? a.A_sub : W) + (size_t)(j - 1) * nn, sV, n, n, ld, 1);
    if (hasR) g.add((l == 0 ? a.A_sub : W) + (size_t)j * nn, sV + (size_t)n * ld, n, n, ld, 0);
  } else {
    g.add(a.Ld + (size_t)orig * nn, sL, n, n, ld, 0);
  }
  if (d > 0) g.add(((l == 0 && a.B64) ? a.B64 : a.Y) + (size_t)orig * nd, sB, n, d, ld, 1);
  stage_round(g);
  __syncthreads();
  if (factor && l == 0) {
    sym_lower_inplace(sL, ld, n);
    __syncthreads();
  }
  if (factor) {
    if (chol_fused(sL, ld, n, sV, nv, sB, d, s_flag)) {
      if (threadIdx.x == 0) set_status(a.st, kStNotSPD, l, orig);
      __syncthreads();
      return false;
    }
    double *Lg = a.Ld + (size_t)orig * nn;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      if (c <= r) Lg[e] = sL[r * ld + c];
    }
    // W^T rows: row c = column c of W (slot j-1: W_L, slot j: W_R)
    for (int e = threadIdx.x; e < nv * n; e += blockDim.x) {
      const int c = e / n, i = e - c * n;
      W[(size_t)(j - 1) * nn + (size_t)c * n + i] = sV[c * ld + i];
    }
  } else if (d > 0) {
    trsv_fwd_cta(sL, ld, n, sB, d);
    __syncthreads();
  }
  if (d > 0) {
    double *Yj = a.Y + (size_t)orig * nd;
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      Yj[e] = sB[c * ld + i];
    }
  }
  __syncthreads();
  return true;
}

// Phase B, separator position s = 2k of level l (Algorithm 3 + Assemble,
// Algorithm 5's separator update):
//   S_ss      = D_s - W_R(s-1)^T W_R(s-1) - W_L(s+1)^T W_L(s+1)  (lower)
//   b_s      -= W_R(s-1)^T y_{s-1} + W_L(s+1)^T y_{s+1}
//   S_{s+2,s} = -W_R(s+1)^T W_L(s+1)  -> region l+1, slot k
// Every operand (the three W^T blocks, both neighbours' y, D_s and b_s) is
// staged in one round; the three kinds of outputs start on warp boundaries
// so that no warp runs two of the inner loops.
__device__ void small_phaseB(const Args<double> &a, int l, long long k, bool factor, double *smem) {
  const int n = a.p.n, ld = ldstride(n), d = a.d;
  const long long Nl = a.p.Nl[l];
  const long long s = 2 * k;
  const bool hasM = (s >= 2), hasP = (s + 1 < Nl), hasE = factor && (s + 2 < Nl);
  const long long orig = s << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  double *sW0 = smem;                       // W_R(s-1)^T
  double *sW1 = sW0 + (size_t)n * ld;       // W_L(s+1)^T
  double *sW2 = sW1 + (size_t)n * ld;       // W_R(s+1)^T
  double *sY = sW2 + (size_t)n * ld;        // y_{s-1}, y_{s+1} as d vectors each
  double *sD = sY + (size_t)2 * d * ld;     // D_s (lower triangle used)
  double *sb = sD + (size_t)n * ld;         // b_s (n x d, row-major)
  const double *W = a.Wb + (size_t)a.p.off[l] * nn;
  StageList g;
  if (hasM) g.add(W + (size_t)(s - 1) * nn, sW0, n, n, ld, 0);
  if (hasP) g.add(W + (size_t)s * nn, sW1, n, n, ld, 0);
  if (hasE) g.add(W + (size_t)(s + 1) * nn, sW2, n, n, ld, 0);
  if (d > 0) {
    if (hasM) g.add(a.Y + (size_t)((s - 1) << l) * nd, sY, n, d, ld, 1);
    if (hasP) g.add(a.Y + (size_t)((s + 1) << l) * nd, sY + (size_t)d * ld, n, d, ld, 1);
    g.add(((l == 0 && a.B64) ? a.B64 : a.Y) + (size_t)orig * nd, sb, 1, n * d, 0, 0);
  }
  if (factor) g.add((l == 0 ? a.A_diag : a.Ld) + (size_t)orig * nn, sD, n, n, ld, 0);
  stage_round(g);
  __syncthreads();
  if (factor && l == 0) {
    sym_lower_inplace(sD, ld, n);
    __syncthreads();
  }
  const int nD = factor ? n * (n + 1) / 2 : 0, nB = n * d, nE = hasE ? n * n : 0;
  const int pD = round32(nD), pB = round32(nB);
  double *Dg = a.Ld + (size_t)orig * nn;
  double *En = a.Wb + ((size_t)a.p.off[l + 1] + (size_t)k) * nn;
  double *Yo = a.Y + (size_t)orig * nd;
  for (int t = threadIdx.x; t < pD + pB + nE; t += blockDim.x) {
    if (t < pD) {
      if (t < nD) {
        int r, c;
        tri_index(t, r, c);
        double acc = sD[r * ld + c];
        if (hasM) {
          const double *wr = sW0 + r * ld, *wc = sW0 + c * ld;
          for (int q = 0; q < n; ++q) acc = fma(-wr[q], wc[q], acc);
        }
        if (hasP) {
          const double *wr = sW1 + r * ld, *wc = sW1 + c * ld;
          for (int q = 0; q < n; ++q) acc = fma(-wr[q], wc[q], acc);
        }
        Dg[r * n + c] = acc;
      }
    } else if (t < pD + pB) {
      const int e = t - pD;
      if (e < nB) {
        const int r = e / d, c = e - r * d;
        double acc = sb[e];
        if (hasM) {
          const double *wr = sW0 + r * ld, *y = sY + (size_t)c * ld;
          for (int q = 0; q < n; ++q) acc = fma(-wr[q], y[q], acc);
        }
        if (hasP) {
          const double *wr = sW1 + r * ld, *y = sY + (size_t)(d + c) * ld;
          for (int q = 0; q < n; ++q) acc = fma(-wr[q], y[q], acc);
        }
        Yo[e] = acc;
      }
    } else {
      const int e = t - pD - pB;
      const int r = e / n, c = e - r * n;
      const double *wr = sW2 + r * ld, *wc = sW1 + c * ld;
      double acc = 0.0;
      for (int q = 0; q < n; ++q) acc = fma(-wr[q], wc[q], acc);
      En[e] = acc;
    }
  }
  __syncthreads();
}

// Top block (the base case of Algorithms 4 and 7 with N_* = 1), FP64: the
// operations of top_block with its operands staged in one round; a top
// level of several blocks (N_* > 1) goes to the serial sweep.
__device__ bool small_top(const Args<double> &a, bool factor, double *smem, int *s_flag) {
  if (a.p.Nl[a.p.L] > 1) return top_block(a, factor, smem, s_flag);
  const int n = a.p.n, ld = ldstride(n), d = a.d, L = a.p.L;
  double *sL = smem;
  double *sB = sL + (size_t)n * ld;
  StageList g;
  g.add(factor ? (L == 0 ? a.A_diag : a.Ld) : a.Ltop, sL, n, n, ld, 0);
  if (d > 0) g.add((L == 0 && a.B64) ? a.B64 : a.Y, sB, n, d, ld, 1);
  stage_round(g);
  __syncthreads();
  if (factor && L == 0) {
    sym_lower_inplace(sL, ld, n);
    __syncthreads();
  }
  if (factor) {
    if (chol_staged(sL, ld, n, s_flag)) {
      if (threadIdx.x == 0) set_status(a.st, kStNotSPD, L, 0);
      __syncthreads();
      return false;
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      a.Ltop[e] = (c <= r) ? sL[r * ld + c] : 0.0;
    }
  }
  if (d > 0) {
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int v = warp; v < d; v += nw) {
      trsv_fwd_warp<double, 1>(sL, ld, n, sB + (size_t)v * ld, 1);
      __syncwarp();
      trsv_bwd_warp<double, 1>(sL, ld, n, sB + (size_t)v * ld, 1);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      a.Y[e] = sB[c * ld + i];
    }
  }
  __syncthreads();
  return true;
}

// Downward pass at level l, eliminated position j (Algorithms 6, 2):
//   x_j = L_j^{-T} (y_j - W_L x_{j-1} - W_R x_{j+1}),
// with L_j, both W^T blocks, y_j and the neighbours' x staged in one round.
__device__ void small_phaseC(const Args<double> &a, int l, long long j, double *smem) {
  const int n = a.p.n, ld = ldstride(n), d = a.d;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  double *sL = smem;
  double *sWL = sL + (size_t)n * ld;        // W_L^T: sWL[p*ld + q] = W_L[q][p]
  double *sWR = sWL + (size_t)n * ld;       // W_R^T
  double *sT = sWR + (size_t)n * ld;        // y_j, then t, then x_j (d vectors)
  double *sXm = sT + (size_t)d * ld;        // x_{j-1}
  double *sXp = sXm + (size_t)d * ld;       // x_{j+1}
  const double *W = a.Wb + (size_t)a.p.off[l] * nn;
  StageList g;
  g.add(a.Ld + (size_t)orig * nn, sL, n, n, ld, 0);
  g.add(W + (size_t)(j - 1) * nn, sWL, n, n, ld, 0);
  if (hasR) g.add(W + (size_t)j * nn, sWR, n, n, ld, 0);
  g.add(a.Y + (size_t)orig * nd, sT, n, d, ld, 1);
  g.add(a.Y + (size_t)((j - 1) << l) * nd, sXm, n, d, ld, 1);
  if (hasR) g.add(a.Y + (size_t)((j + 1) << l) * nd, sXp, n, d, ld, 1);
  stage_round(g);
  __syncthreads();
  for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
    const int c = e / n, q = e - c * n;
    double acc = sT[c * ld + q];
    {
      const double *x = sXm + (size_t)c * ld;
      for (int p = 0; p < n; ++p) acc = fma(-sWL[p * ld + q], x[p], acc);
    }
    if (hasR) {
      const double *x = sXp + (size_t)c * ld;
      for (int p = 0; p < n; ++p) acc = fma(-sWR[p * ld + q], x[p], acc);
    }
    sT[c * ld + q] = acc;
  }
  __syncthreads();
  trsv_bwd_cta(sL, ld, n, sT, d);
  __syncthreads();
  double *Yo = a.Y + (size_t)orig * nd;
  for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
    const int i = e / d, c = e - i * d;
    Yo[e] = sT[c * ld + i];
  }
  __syncthreads();
}

// Cluster barrier, then (CTA 0, thread 0) the %globaltimer stamp of its
// release in trace slot `bar`.
__device__ __forceinline__ void small_sync(cg::cluster_group &cl, const Args<double> &a, int rank, int &bar) {
  cl.sync();
  if (rank == 0 && threadIdx.x == 0 && bar < kTraceSlots) a.st->trace[bar] = global_ns();
  ++bar;
}

// The whole call in one cluster.  Every CTA passes every cluster barrier
// (the task loops and the error checks sit between them), so a failed task
// only makes the remaining work be skipped: the failing CTA raises a flag in
// the shared memory of every CTA of the cluster, read after the next
// barrier.  `out` is the caller's page-locked status copy (device-visible
// address); it also receives the barrier stamps (start-up, phases A and B of
// each level, after the top block, each downward level, end),
// zero-terminated.
__global__ void __launch_bounds__(kSmallThreads) k_small(const __grid_constant__ Args<double> a, int mode,
                                                       DevStatus *out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag;
  __shared__ int s_err;
  double *smem = reinterpret_cast<double *>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
  const bool factor = (mode & 1) != 0;
  const bool rhs = (mode & 2) != 0 && a.d > 0;
  int bar = 0;
  if (threadIdx.x == 0) s_err = 0;
  if (rank == 0 && threadIdx.x == 0) {
    a.st->status = 0;
    a.st->level = 0;
    a.st->block = 0;
  }
  small_sync(cl, a, rank, bar);  // every CTA runs and has cleared its flag
  auto failed = [&]() { return __syncthreads_or(*(volatile int *)&s_err != 0) != 0; };
  auto raise = [&]() {
    if (threadIdx.x == 0)
      for (int r = 0; r < C; ++r) *cl.map_shared_rank(&s_err, r) = 1;
  };
  for (int l = 0; l < a.p.L; ++l) {
    const long long Nl = a.p.Nl[l];
    if (!failed())
      for (long long t = rank; t < Nl / 2; t += C)
        if (!small_phaseA(a, l, 2 * t + 1, factor, smem, &s_flag)) {
          raise();
          break;
        }
    small_sync(cl, a, rank, bar);
    if (!failed())
      for (long long k = rank; k < (Nl + 1) / 2; k += C) small_phaseB(a, l, k, factor, smem);
    small_sync(cl, a, rank, bar);
  }
  if (rank == 0 && !failed() && !small_top(a, factor, smem, &s_flag)) raise();
  if (rhs && a.p.L > 0) {
    small_sync(cl, a, rank, bar);
    for (int l = a.p.L - 1; l >= 0; --l) {
      if (!failed())
        for (long long m = rank; m < a.p.Nl[l] / 2; m += C) small_phaseC(a, l, 2 * m + 1, smem);
      if (l > 0) small_sync(cl, a, rank, bar);
    }
  }
  small_sync(cl, a, rank, bar);
  if (rank == 0 && threadIdx.x == 0) {
    volatile DevStatus *o = out;
    const int nb = bar < kTraceSlots ? bar : kTraceSlots;
    for (int i = 0; i < nb; ++i) o->trace[i] = a.st->trace[i];
    if (nb < kTraceSlots) o->trace[nb] = 0;
    o->level = __ldcg(&a.st->level);
    o->block = __ldcg(&a.st->block);
    o->status = ld_relaxed_i32(&a.st->status);
  }
}

static cudaLaunchConfig_t small_config(int cluster, size_t smem, cudaStream_t s, cudaLaunchAttribute *attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cluster, 1, 1);
  cfg.blockDim = dim3(kSmallThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

cudaError_t small_cluster_size(size_t smem, int *cluster) {
  *cluster = 0;
  cudaError_t e = cudaFuncSetAttribute(k_small, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess && smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  for (int c = 16; c >= 2; c /= 2) {
    cudaLaunchAttribute attr[1];
    const cudaLaunchConfig_t cfg = small_config(c, smem, nullptr, attr);
    int active = 0;
    if (cudaOccupancyMaxActiveClusters(&active, k_small, &cfg) == cudaSuccess && active >= 1) {
      *cluster = c;
      return cudaSuccess;
    }
    cudaGetLastError();  // an unsupported size is not an error of the call
  }
  return cudaSuccess;
}

cudaError_t launch_small(const Args<double> &a, int factor, int rhs, int cluster, size_t smem, DevStatus *out,
                         cudaStream_t s) {
  cudaLaunchAttribute attr[1];
  const cudaLaunchConfig_t cfg = small_config(cluster, smem, s, attr);
  const int mode = (factor ? 1 : 0) | (rhs ? 2 : 0);
  return cudaLaunchKernelEx(&cfg, k_small, a, mode, out);
}

}  // namespace bdss
