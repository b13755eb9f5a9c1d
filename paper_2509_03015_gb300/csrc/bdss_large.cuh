// Large-block path (64 < n <= 256): the same odd-even reduction and storage
// as the shared-memory path (bdss_device.cuh), with every n x n operation cut
// into 64 x 64 tiles staged through shared memory, so that one block's work
// can be spread over tile tasks:
//   A1  eliminated block: blocked right-looking Cholesky, in place in Ld
//       (Algorithm 1, potrf; level 0 reads sym(A_jj) on its first step);
//   A2  (eliminated block, vector tile): forward substitution of the coupling
//       vectors (W_L, W_R, Sec. 3.3 stage 2) and of the RHS (y = L^{-1} b),
//       blocked by 64-row tiles (gemm update + triangular tile solve);
//   B   (separator, output tile): Schur update and new coupling (Algorithm 3,
//       Eq. 5) and the separator RHS update (Algorithm 5);
//   C   eliminated block: x = L^{-T}(y - W_L x_{j-1} - W_R x_{j+1})
//       (Algorithms 6, 2), blocked from the bottom tile up;
//   top the remaining block, FP64, blocked, in Ltop.
#pragma once
#include <type_traits>

#include "bdss_device.cuh"
#include "bdss_tc.cuh"

namespace bdss {

// A pointer into the dynamic shared memory, re-derived from the shared array
// itself: inside a function that is not inlined a pointer parameter is
// generic, and every access through it would be a generic load or store.
template <typename T>
__device__ __forceinline__ T *as_shared(T *p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  return reinterpret_cast<T *>(smem_raw + (smem_u32(p) - smem_u32(smem_raw)));
}

constexpr int kTile = 64;   // output / triangular tile
constexpr int kKc = 32;     // k-chunk staged per gemm step
constexpr int kTilePad = kTile + 1;

__host__ __device__ inline int ntiles(int n) { return (n + kTile - 1) / kTile; }
// Vectors per forward-substitution task: one 64-wide gemm tile of them.
__host__ __device__ inline int vec_tile(int /*elem_size: the same for FP32 and FP64*/) { return 64; }

// Strided matrix view: element (r, c) at p[r * rs + c * cs]; zero outside
// rows x cols.  Global views load through L2 (written by other CTAs across
// grid barriers); shared-memory views (kSmem) load directly.
template <typename S, bool kSmem = false>
struct View {
  const S *p;
  long long rs, cs;
  int rows, cols;
  __device__ S at(int r, int c) const {
    if (r >= rows || c >= cols) return S(0);
    const S *q = p + (long long)r * rs + (long long)c * cs;
    return kSmem ? *q : ldcg(q);
  }
};

// acc[i][j] += sum_k A(r0 + 4 tm + i, k) * B(c0 + 4 tn + j, k) for the 64 x 64
// output tile at (r0, c0), k over [0, K): "NT" products of two strided views
// through shared memory (sA, sB: kKc x kTilePad each).  256 threads: thread t
// owns rows 4 (t / 16) + i and columns 4 (t % 16) + j.  The next k-chunk is
// loaded into registers (all loads of a chunk issued together) while the
// current one is multiplied, so global latency overlaps the FMAs.
template <typename T, typename VA, typename VB>
__device__ void gemm_nt_tile(T (&acc)[4][4], const VA &A, int r0, const VB &B, int c0, int K, T *sA, T *sB) {
  const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
  constexpr int kPer = kTile * kKc / kThreads;  // elements per thread and operand
  T ra[kPer], rb[kPer];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = threadIdx.x + q * kThreads, m = e / kKc, k = e - m * kKc;
      const bool kin = (k0 + k) < K;
      ra[q] = kin ? (T)A.at(r0 + m, k0 + k) : T(0);
      rb[q] = kin ? (T)B.at(c0 + m, k0 + k) : T(0);
    }
  };
  load(0);
  for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = threadIdx.x + q * kThreads, m = e / kKc, k = e - m * kKc;
      sA[k * kTilePad + m] = ra[q];
      sB[k * kTilePad + m] = rb[q];
    }
    __syncthreads();
    if (k0 + kKc < K) load(k0 + kKc);
    const int kc = min(kKc, K - k0);
    for (int k = 0; k < kc; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = sA[k * kTilePad + 4 * tm + i];
        b[i] = sB[k * kTilePad + 4 * tn + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
}

// The same product for a narrow output: rows r0..r0+63 by up to 16 columns
// from c0 (right-hand sides).  Thread t owns row t / 4 and columns
// 4 (t % 4) + j, so every thread works when d <= 16 (the square tile would
// leave three quarters of its FMAs on zero columns).  sB needs kKc x 17.
// The next chunk is prefetched into registers as in gemm_nt_tile.
constexpr int kNarrow = 16;
template <typename T, typename VA, typename VB>
__device__ void gemm_nt_narrow(T (&acc)[4], const VA &A, int r0, const VB &B, int c0, int K, T *sA, T *sB) {
  const int tr = threadIdx.x >> 2, tc = threadIdx.x & 3;
  constexpr int kPa = kTile * kKc / kThreads, kPb = kNarrow * kKc / kThreads;
  T ra[kPa], rb[kPb];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < kPa; ++q) {
      const int e = threadIdx.x + q * kThreads, m = e / kKc, k = e - m * kKc;
      ra[q] = (k0 + k) < K ? (T)A.at(r0 + m, k0 + k) : T(0);
    }
#pragma unroll
    for (int q = 0; q < kPb; ++q) {
      const int e = threadIdx.x + q * kThreads, m = e / kKc, k = e - m * kKc;
      rb[q] = (k0 + k) < K ? (T)B.at(c0 + m, k0 + k) : T(0);
    }
  };
  load(0);
  for (int k0 = 0; k0 < K; k0 += kKc) {
#pragma unroll
    for (int q = 0; q < kPa; ++q) {
      const int e = threadIdx.x + q * kThreads, m = e / kKc, k = e - m * kKc;
      sA[k * kTilePad + m] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < kPb; ++q) {
      const int e = threadIdx.x + q * kThreads, m = e / kKc, k = e - m * kKc;
      sB[k * (kNarrow + 1) + m] = rb[q];
    }
    __syncthreads();
    if (k0 + kKc < K) load(k0 + kKc);
    const int kc = min(kKc, K - k0);
    for (int k = 0; k < kc; ++k) {
      const T a = sA[k * kTilePad + tr];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fma(a, sB[k * (kNarrow + 1) + 4 * tc + j], acc[j]);
    }
    __syncthreads();
  }
}

// Shared memory (in elements of FP64) of the FP64 top block: d solution
// vectors plus the tile work area (it never stages coupling vectors).
__host__ __device__ inline size_t smem_large_top(int n, int d) {
  return (size_t)(d > 0 ? d : 1) * (n + 1) + (size_t)kTile * kTilePad + (size_t)2 * kKc * kTilePad + 16;
}

// Shared memory (in elements of T) of the large-path tasks.
__host__ __device__ inline size_t smem_large(int n, int d, int esz) {
  const size_t gemm = (size_t)2 * kKc * kTilePad;
  const size_t tile = (size_t)kTile * kTilePad;
  const int vt = vec_tile(esz);
  const size_t a2 = (size_t)vt * (n + 1) + tile + gemm;   // vectors + L tile + gemm staging
  const size_t c = (size_t)(d > 0 ? d : 1) * (n + 1) + tile + gemm;
  const size_t a1 = tile + gemm;
  size_t m = a2 > c ? a2 : c;
  if (a1 > m) m = a1;
  return m + 16;
}

// ---------------------------------------------------------------------------
// Blocked Cholesky of the n x n matrix M (row-major, leading dim n), in place
// (lower triangle; diagonal tiles get 1 / L_kk on their diagonal).  `src` is
// where the not-yet-touched tiles live before the first step (sym(A) from the
// caller's FP64 block at level 0, else M itself).  Returns 0 or a failing
// column + 1.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __noinline__ int chol_blocked(T *M, int n, const double *src_sym, T *smem, int *s_flag, T *Dinv = nullptr) {
  smem = as_shared(smem);
  s_flag = as_shared(s_flag);
  const int nt = ntiles(n);
  T *sT = smem;                              // 64 x 65 tile
  T *sA = sT + kTile * kTilePad;
  T *sB = sA + kKc * kTilePad;
  T *sP2 = sB + kKc * kTilePad;              // panel rows when Dinv is given (64 x 65)
  const int ld = kTilePad;
  auto src = [&](int r, int c) -> T {      // element of the matrix before step 0
    if (src_sym) return T(0.5) * ((T)ldcg(src_sym + (long long)r * n + c) + (T)ldcg(src_sym + (long long)c * n + r));
    return ldcg(M + (long long)r * n + c);
  };
  for (int k = 0; k < nt; ++k) {
    const int k0 = k * kTile, kb = min(kTile, n - k0);
    const bool first = (k == 0) && src_sym;
    // diagonal tile
#pragma unroll 4
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int r = e / kTile, c = e - r * kTile;
      T v = T(0);
      if (r < kb && c <= r) v = first ? src(k0 + r, k0 + c) : ldcg(M + (long long)(k0 + r) * n + k0 + c);
      sT[r * ld + c] = v;
    }
    __syncthreads();
    const int bad = blockDim.x >= 64 ? chol_fused(sT, ld, kb, sT, 0, sT, 0, s_flag) : chol_staged(sT, ld, kb, s_flag);
    if (bad) return k0 + bad;
    for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
      const int r = e / kb, c = e - r * kb;
      if (c <= r) M[(long long)(k0 + r) * n + k0 + c] = sT[r * ld + c];
    }
    if (Dinv) {
      // L_kk^{-1} (the diagonal tile of L^{-1}): unit vectors through the tile
      // substitution once, then every solve with this tile is a product
      T *sI = sA;  // 64 x 65 (sA and sB are contiguous)
      __syncthreads();
      for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = e / kTile, c = e - r * kTile;
        sI[r * ld + c] = (r == c && r < kb) ? T(1) : T(0);
      }
      __syncthreads();
      trsv_tile_fwd(sT, ld, kb, sI, ld, kb);
      for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
        const int r = e / kb, c = e - r * kb;  // (L_kk^{-1})[r][c] = entry r of solved vector c
        Dinv[(long long)(k0 + r) * n + k0 + c] = (c <= r) ? sI[c * ld + r] : T(0);
      }
      __syncthreads();
      // panel below: L_ik = S_ik L_kk^{-T}, i.e. L_ik[r][c] = sum_q S_ik[r][q] L_kk^{-1}[c][q]
      const View<T> Dk{Dinv + (long long)k0 * n + k0, n, 1, kb, kb};
      for (int i = k + 1; i < nt; ++i) {
        const int i0 = i * kTile, ib = min(kTile, n - i0);
#pragma unroll 4
        for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
          const int r = e / kTile, c = e - r * kTile;
          T v = T(0);
          if (r < ib && c < kb) v = first ? src(i0 + r, k0 + c) : ldcg(M + (long long)(i0 + r) * n + k0 + c);
          sP2[r * ld + c] = v;
        }
        __syncthreads();
        T acc[4][4] = {};
        const View<T, true> Pr{sP2, ld, 1, ib, kb};
        gemm_nt_tile(acc, Pr, 0, Dk, 0, kb, sA, sB);
        const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
#pragma unroll
        for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) {
            const int r = 4 * tm + a2, c = 4 * tn + b2;
            if (r < ib && c < kb) M[(long long)(i0 + r) * n + k0 + c] = acc[a2][b2];
          }
        __syncthreads();
      }
    }
    // panel below: L_ik = S_ik L_kk^{-T}: each row x solves L_kk x = s
    for (int i = k + 1; i < nt && !Dinv; ++i) {
      const int i0 = i * kTile, ib = min(kTile, n - i0);
      // reuse the gemm staging area for the panel rows (ib x kb)
      T *sP = sA;  // needs kTile x kTilePad: sA and sB are contiguous 2 * kKc * kTilePad = kTile * kTilePad
      __syncthreads();
#pragma unroll 4
      for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int r = e / kTile, c = e - r * kTile;
        T v = T(0);
        if (r < ib && c < kb) v = first ? src(i0 + r, k0 + c) : ldcg(M + (long long)(i0 + r) * n + k0 + c);
        sP[r * ld + c] = v;
      }
      __syncthreads();
      trsv_tile_fwd(sT, ld, kb, sP, ld, ib);  // each panel row x solves L_kk x = s
      for (int e = threadIdx.x; e < ib * kb; e += blockDim.x) {
        const int r = e / kb, c = e - r * kb;
        M[(long long)(i0 + r) * n + k0 + c] = sP[r * ld + c];
      }
    }
    __syncthreads();
    // trailing update: S_ij -= L_ik L_jk^T, k < j <= i
    for (int i = k + 1; i < nt; ++i)
      for (int j = k + 1; j <= i; ++j) {
        const int i0 = i * kTile, j0 = j * kTile;
        T acc[4][4] = {};
        const View<T> Ar{M + (long long)k0, n, 1, n, kb};
        gemm_nt_tile(acc, Ar, i0, Ar, j0, kb, sA, sB);
        const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = i0 + 4 * tm + a, c = j0 + 4 * tn + b;
            if (r < n && c < n && c <= r) {
              const T base = first ? src(r, c) : ldcg(M + (long long)r * n + c);
              M[(long long)r * n + c] = base - acc[a][b];
            }
          }
        __syncthreads();
      }
  }
  return 0;
}

// Forward substitution L v = v for `nv` vectors held as rows of sV (stride
// n + 1), L (n x n, reciprocal diagonal) in global memory, blocked by 64-row
// tiles: gemm update from the solved rows, then the triangular tile.
template <typename T>
__device__ void trsv_fwd_blocked(const T *L, int n, T *sV, int nv, T *smem, const T *Dinv = nullptr) {
  const int nt = ntiles(n), lv = n + 1;
  T *sT = smem;
  T *sA = sT + kTile * kTilePad;
  T *sB = sA + kKc * kTilePad;
  for (int R = 0; R < nt; ++R) {
    const int r0 = R * kTile, rb = min(kTile, n - r0);
    if (R > 0) {
      // sV[c][r0 + r] -= sum_{p < r0} L[r0 + r][p] sV[c][p]; output 64 rows x (up to 64) vectors
      for (int c0 = 0; c0 < nv; c0 += kTile) {
        T acc[4][4] = {};
        const View<T> Lr{L, n, 1, n, r0};
        const View<T, true> Vc{sV + (long long)c0 * lv, lv, 1, nv - c0, r0};
        gemm_nt_tile(acc, Lr, r0, Vc, 0, r0, sA, sB);
        const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = 4 * tm + a, c = c0 + 4 * tn + b;
            if (r < rb && c < nv) sV[(long long)c * lv + r0 + r] -= acc[a][b];
          }
        __syncthreads();
      }
    }
    if (Dinv) {
      // the diagonal tile's solve as a product with its stored inverse:
      // v[r0 + i] = sum_q L_RR^{-1}[i][q] v[r0 + q], 64 vectors at a time
      const View<T> Dr{Dinv + (long long)r0 * n + r0, n, 1, rb, rb};
      for (int c0 = 0; c0 < nv; c0 += kTile) {
        T acc[4][4] = {};
        const View<T, true> Vc{sV + (long long)c0 * lv + r0, lv, 1, nv - c0, rb};
        gemm_nt_tile(acc, Dr, 0, Vc, 0, rb, sA, sB);
        const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int i = 4 * tm + a, c = c0 + 4 * tn + b;
            if (i < rb && c < nv) sV[(long long)c * lv + r0 + i] = acc[a][b];
          }
        __syncthreads();
      }
      continue;
    }
#pragma unroll 4
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int r = e / kTile, c = e - r * kTile;
      sT[r * kTilePad + c] = (r < rb && c <= r) ? ldcg(L + (long long)(r0 + r) * n + r0 + c) : T(0);
    }
    __syncthreads();
    trsv_tile_fwd(sT, kTilePad, rb, sV + r0, lv, nv);
  }
}

// Backward substitution L^T z = t for `nv` vectors (rows of sV), blocked
// from the bottom tile up.
template <typename T>
__device__ void trsv_bwd_blocked(const T *L, int n, T *sV, int nv, T *smem) {
  const int nt = ntiles(n), lv = n + 1;
  T *sT = smem;
  T *sA = sT + kTile * kTilePad;
  T *sB = sA + kKc * kTilePad;
  for (int R = nt - 1; R >= 0; --R) {
    const int r0 = R * kTile, rb = min(kTile, n - r0), r1 = r0 + rb;
    if (r1 < n) {
      // sV[c][r0 + r] -= sum_{p >= r1} L[p][r0 + r] sV[c][p]
      for (int c0 = 0; c0 < nv; c0 += kTile) {
        T acc[4][4] = {};
        const View<T> Lt{L + (long long)r1 * n, 1, n, n, n - r1};  // (r, k) -> L[r1 + k][r]
        const View<T, true> Vc{sV + (long long)c0 * lv + r1, lv, 1, nv - c0, n - r1};
        gemm_nt_tile(acc, Lt, r0, Vc, 0, n - r1, sA, sB);
        const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int r = 4 * tm + a, c = c0 + 4 * tn + b;
            if (r < rb && c < nv) sV[(long long)c * lv + r0 + r] -= acc[a][b];
          }
        __syncthreads();
      }
    }
#pragma unroll 4
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int r = e / kTile, c = e - r * kTile;
      sT[r * kTilePad + c] = (r < rb && c <= r) ? ldcg(L + (long long)(r0 + r) * n + r0 + c) : T(0);
    }
    __syncthreads();
    trsv_tile_bwd(sT, kTilePad, rb, sV + r0, lv, nv);
  }
}

// ---------------------------------------------------------------------------
// Tasks
// ---------------------------------------------------------------------------

// A1: Cholesky of eliminated position j of level l.
template <typename T>
__device__ bool largeA1(const Args<T> &a, int l, long long j, T *smem, int *s_flag) {
  const int n = a.p.n;
  const long long orig = j << l;
  T *M = a.Ld + orig * (long long)n * n;
  // FP32 with stored inverses: the diagonal tiles of L^{-1} are formed here,
  // and every tile solve after them is a product
  T *Dinv = a.Li ? a.Li + orig * (long long)n * n : nullptr;
  const int bad = chol_blocked(M, n, l == 0 ? a.A_diag + orig * (long long)n * n : nullptr, smem, s_flag, Dinv);
  if (bad) {
    if (threadIdx.x == 0) set_status(a.st, kStNotSPD, l, orig);
    __syncthreads();
    return false;
  }
  __syncthreads();
  return true;
}

// Number of vectors of eliminated position j's forward substitution.
// Vector slots of an eliminated block's forward substitution: the couplings
// (2 n, the 64-vector tiles are laid out as if the right coupling existed),
// the n unit vectors whose solutions are the columns of L^{-1} (factor with
// an inverse buffer), then the RHS columns.
template <typename T>
__device__ __forceinline__ int largeA2_slots(const Args<T> &a, bool factor) {
  return (factor ? (a.Li ? 3 : 2) * a.p.n : 0) + a.d;
}

// Number of vectors of eliminated position j's forward substitution.
template <typename T>
__device__ __forceinline__ bool largeA2_live(const Args<T> &a, int l, long long j, bool factor, int c0) {
  const int n = a.p.n;
  const bool hasR = (j + 1 < a.p.Nl[l]);
  // a vector tile is idle only when it holds nothing but the absent E_R rows
  return !(factor && !hasR && c0 >= n && c0 + vec_tile(sizeof(T)) <= 2 * n);
}

// A2: vector tile v of eliminated position j.  Slots [0, n) are E_L's
// columns, [n, 2n) E_R's rows (absent for the last block of a level: those
// slots are skipped), [2n, 3n) the unit vectors of L^{-1} (with an inverse
// buffer), then the RHS columns; in a solve pass only the RHS columns.
template <typename T>
__device__ void largeA2(const Args<T> &a, int l, long long j, int v, bool factor, T *smem) {
  const int n = a.p.n, d = a.d, lv = n + 1;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n;
  const int nW = factor ? 2 * n : 0;              // coupling slots
  const int nI = (factor && a.Li) ? n : 0;        // unit-vector slots
  const int VT = vec_tile(sizeof(T));
  const int slots = nW + nI + d;
  const int c0 = v * VT, nv = min(VT, slots - c0);
  T *sV = smem;
  T *work = sV + (size_t)VT * lv;
  const T *E = (l == 0) ? nullptr : a.Eb + (size_t)a.p.off[l] * nn;  // couplings formed at level l-1
  // stage vectors
#pragma unroll 8
  for (int e = threadIdx.x; e < n * nv; e += blockDim.x) {
    const int i = e / nv, cc = e - i * nv, c = c0 + cc;
    T val;
    if (c < nW && c < n) {  // column c of A_{j,j-1}
      val = (l == 0) ? (T)ldcg(a.A_sub + (size_t)(j - 1) * nn + (size_t)i * n + c)
                     : ldcg(E + (size_t)(j - 1) * nn + (size_t)i * n + c);
    } else if (c < nW) {  // row c - n of A_{j+1,j} (zero for the last block)
      const int r = c - n;
      val = !hasR ? T(0)
                  : (l == 0) ? (T)ldcg(a.A_sub + (size_t)j * nn + (size_t)r * n + i)
                             : ldcg(E + (size_t)j * nn + (size_t)r * n + i);
    } else if (c < nW + nI) {  // unit vector e_{c - nW}
      val = (i == c - nW) ? T(1) : T(0);
    } else {  // RHS column
      const int k = c - nW - nI;
      const size_t bo = (size_t)orig * n * d + (size_t)i * d + k;
      if (l == 0 && a.B64) val = (T)ldcg(a.B64 + bo);
      else if (l == 0 && a.Bt) val = ldcg(a.Bt + bo);
      else val = ldcg(a.Y + bo);
    }
    sV[(size_t)cc * lv + i] = val;
  }
  __syncthreads();
  trsv_fwd_blocked(a.Ld + (size_t)orig * nn, n, sV, nv, work, factor && a.Li ? a.Li + (size_t)orig * nn : nullptr);
  // write back
  T *W = a.Wb + (size_t)a.p.off[l] * nn;
  for (int e = threadIdx.x; e < n * nv; e += blockDim.x) {
    const int cc = e / n, i = e - cc * n, c = c0 + cc;
    const T val = sV[(size_t)cc * lv + i];
    long long wo = -1;  // element of the coupling buffer, if this is a coupling slot
    if (c < nW && c < n) wo = (long long)((size_t)(j - 1) * nn + (size_t)c * n + i);
    else if (c < nW) { if (hasR) wo = (long long)((size_t)j * nn + (size_t)(c - n) * n + i); }
    else if (c >= nW + nI) a.Y[(size_t)orig * n * d + (size_t)i * d + (c - nW - nI)] = val;
    if (wo >= 0) W[wo] = val;
  }
  if (nI) {
    // columns u0..u1-1 of L^{-1}, row-major in Li: consecutive threads take
    // consecutive columns of one row
    const int u0 = max(c0, nW) - nW, u1 = min(c0 + nv, nW + nI) - nW;
    if (u1 > u0) {
      T *Li = a.Li + (size_t)orig * nn;
      const int nu = u1 - u0;
      for (int e = threadIdx.x; e < n * nu; e += blockDim.x) {
        const int i = e / nu, u = u0 + e - i * nu;
        // the diagonal tiles were formed by the Cholesky task and are read
        // by this level's other substitution tasks: left as they are
        if (i / kTile != u / kTile) Li[(size_t)i * n + u] = sV[(size_t)(u + nW - c0) * lv + i];
      }
    }
  }
  __syncthreads();
}

// Tiles of a separator's phase-B work.
__host__ __device__ inline int largeB_tiles(int n, bool factor, int d) {
  const int nt = ntiles(n);
  return (factor ? nt * (nt + 1) / 2 + nt * nt : 0) + (d > 0 ? nt : 0);
}

// B: output tile `t` of separator s = 2k at level l.
template <typename T>
__device__ void largeB(const Args<T> &a, int l, long long k, int t, bool factor, T *smem) {
  const int n = a.p.n, d = a.d, nt = ntiles(n);
  const long long Nl = a.p.Nl[l];
  const long long s = 2 * k;
  const bool hasM = (s >= 2), hasP = (s + 1 < Nl), hasE = (s + 2 < Nl);
  const long long orig = s << l;
  const size_t nn = (size_t)n * n;
  const T *W = a.Wb + (size_t)a.p.off[l] * nn;
  const View<T> W0{W + (size_t)(s - 1) * nn, n, 1, n, n};   // W_R(s-1)^T
  const View<T> W1{W + (size_t)s * nn, n, 1, n, n};         // W_L(s+1)^T
  const View<T> W2{W + (size_t)(s + 1) * nn, n, 1, n, n};   // W_R(s+1)^T
  T *sA = smem, *sB = sA + kKc * kTilePad;
  const int tm = threadIdx.x >> 4, tn = threadIdx.x & 15;
  const int nD = factor ? nt * (nt + 1) / 2 : 0, nE = factor ? nt * nt : 0;
  if (t < nD) {
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    const int tj = t - ti * (ti + 1) / 2;
    T acc[4][4] = {};
    if (hasM) gemm_nt_tile(acc, W0, ti * kTile, W0, tj * kTile, n, sA, sB);
    if (hasP) gemm_nt_tile(acc, W1, ti * kTile, W1, tj * kTile, n, sA, sB);
    T *Dg = a.Ld + (size_t)orig * nn;
    const double *Ag = a.A_diag + (size_t)orig * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int r = ti * kTile + 4 * tm + i, c = tj * kTile + 4 * tn + jj;
        if (r < n && c <= r) {
          const T base = (l == 0) ? T(0.5) * ((T)ldcg(Ag + (size_t)r * n + c) + (T)ldcg(Ag + (size_t)c * n + r))
                                  : ldcg(Dg + (size_t)r * n + c);
          Dg[(size_t)r * n + c] = base - acc[i][jj];
        }
      }
  } else if (t < nD + nE) {
    if (!hasE) return;
    const int u = t - nD, ti = u / nt, tj = u - ti * nt;
    T acc[4][4] = {};
    gemm_nt_tile(acc, W2, ti * kTile, W1, tj * kTile, n, sA, sB);
    T *En = a.Eb + ((size_t)a.p.off[l + 1] + (size_t)k) * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int r = ti * kTile + 4 * tm + i, c = tj * kTile + 4 * tn + jj;
        if (r < n && c < n) En[(size_t)r * n + c] = -acc[i][jj];
      }
  } else {
    const int ti = t - nD - nE;
    const size_t boff = (size_t)orig * n * d;
    for (int c0 = 0; c0 < d; c0 += kNarrow) {
      T acc[4] = {};
      // y as the "B" operand: (c, q) -> y[q][c]
      const T *ys = a.Yt ? a.Yt : a.Y;  // where this pass keeps y of the eliminated blocks
      const View<T> Ym{ys + (size_t)((s - 1) << l) * n * d + c0, 1, d, d - c0, n};
      const View<T> Yp{ys + (size_t)((s + 1) << l) * n * d + c0, 1, d, d - c0, n};
      if (hasM) gemm_nt_narrow(acc, W0, ti * kTile, Ym, 0, n, sA, sB);
      if (hasP) gemm_nt_narrow(acc, W1, ti * kTile, Yp, 0, n, sA, sB);
      const int r = ti * kTile + (threadIdx.x >> 2);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int c = c0 + 4 * (threadIdx.x & 3) + jj;
        if (r < n && c < d) {
          const size_t o = boff + (size_t)r * d + c;
          T base;
          if (l == 0 && a.B64) base = (T)ldcg(a.B64 + o);
          else if (l == 0 && a.Bt) base = ldcg(a.Bt + o);
          else base = ldcg(a.Y + o);
          a.Y[o] = base - acc[jj];
        }
      }
      __syncthreads();
    }
  }
  __syncthreads();
}

// Tensor-core tiles of a separator's Schur update (large FP32 path, TF32
// mode): 128 x 128 output tiles, lower D tiles then E tiles.
__host__ __device__ inline int largeB_tc_tiles(int n) {
  const int t = (n + kTcM - 1) / kTcM;
  return t * (t + 1) / 2 + t * t;
}

// Tile t of separator s = 2k at level l on tcgen05 (3xTF32).  Returns false on
// a timed-out wait (the status word is then set).
__device__ inline bool largeB_tc(const Args<float> &a, int l, long long k, int t, TcState &tc) {
  const int n = a.p.n, nt = (n + kTcM - 1) / kTcM, nD = nt * (nt + 1) / 2;
  const long long Nl = a.p.Nl[l];
  const long long s = 2 * k;
  const bool hasM = (s >= 2), hasP = (s + 1 < Nl), hasE = (s + 2 < Nl);
  const long long orig = s << l;
  const size_t nn = (size_t)n * n;
  const long long slot0 = a.p.off[l];
  bool ok = true;
  int ti, tj;
  if (t < nD) {
    ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
    tj = t - ti * (ti + 1) / 2;
    bool first = true;
    if (hasM) {
      const int base = (int)((slot0 + s - 1) * n);
      ok = tc_accumulate(tc, a.tmap_w, base + ti * kTcM, base + tj * kTcM, n, first, a.timeout_ns);
      first = false;
    }
    if (ok && hasP) {
      const int base = (int)((slot0 + s) * n);
      ok = tc_accumulate(tc, a.tmap_w, base + ti * kTcM, base + tj * kTcM, n, first, a.timeout_ns);
    }
  } else {
    if (!hasE) return true;
    const int u = t - nD;
    ti = u / nt;
    tj = u - ti * nt;
    ok = tc_accumulate(tc, a.tmap_w, (int)((slot0 + s + 1) * n) + ti * kTcM, (int)((slot0 + s) * n) + tj * kTcM, n,
                       true, a.timeout_ns);
  }
  if (!ok) {
    if (threadIdx.x == 0) set_status(a.st, kStTimeout, l, orig);
    return false;
  }
  float v[64];
  int row, col0;
  tc_read_row(tc, v, row, col0);
  const int R = ti * kTcM + row;
  if (t < nD) {
    float *Dg = a.Ld + (size_t)orig * nn;
    const double *Ag = a.A_diag + (size_t)orig * nn;
    if (R < n)
      for (int j = 0; j < 64; ++j) {
        const int C = tj * kTcN + col0 + j;
        if (C <= R && C < n) {
          const float base = (l == 0) ? 0.5f * ((float)ldcg(Ag + (size_t)R * n + C) + (float)ldcg(Ag + (size_t)C * n + R))
                                      : ldcg(Dg + (size_t)R * n + C);
          Dg[(size_t)R * n + C] = base - v[j];
        }
      }
  } else {
    float *En = a.Eb + ((size_t)a.p.off[l + 1] + (size_t)k) * nn;
    if (R < n)
      for (int j = 0; j < 64; ++j) {
        const int C = tj * kTcN + col0 + j;
        if (C < n) En[(size_t)R * n + C] = -v[j];
      }
  }
  tc_fence_before();
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Solve passes with the stored inverses (FP32 tiled path), one thread per
// output row: each product is an n x n matrix times up to 16 vectors that
// sit in shared memory as sV[k * 16 + c].  Thread r streams row r of the
// matrix (kTrans = false: P[r ld + k], float4 loads when aligned) or column r
// (kTrans = true: P[k ld + r], coalesced across the warp), with no barrier
// inside the product, so that the loads of a whole block are in flight
// together.
// ---------------------------------------------------------------------------
constexpr int kRowCols = 16;

template <bool kTrans>
__device__ __forceinline__ void rowprod16(float (&acc)[kRowCols], const float *P, int ld, int r, int k0, int k1,
                                          const float *sV) {
  int k = k0;
  if (!kTrans && ((ld & 3) == 0) && ((reinterpret_cast<uintptr_t>(P) & 15) == 0)) {
    for (; k < k1 && (k & 3); ++k) {
      const float a = ldcg(P + (size_t)r * ld + k);
#pragma unroll
      for (int c = 0; c < kRowCols; ++c) acc[c] = fma(a, sV[k * kRowCols + c], acc[c]);
    }
    for (; k + 4 <= k1; k += 4) {
      const float4 a4 = __ldcg(reinterpret_cast<const float4 *>(P + (size_t)r * ld + k));
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < kRowCols; ++c) acc[c] = fma(av[q], sV[(k + q) * kRowCols + c], acc[c]);
    }
  }
#pragma unroll 4
  for (; k < k1; ++k) {
    const float a = kTrans ? ldcg(P + (size_t)k * ld + r) : ldcg(P + (size_t)r * ld + k);
#pragma unroll
    for (int c = 0; c < kRowCols; ++c) acc[c] = fma(a, sV[k * kRowCols + c], acc[c]);
  }
}

// sV[k * 16 + c] = src[k * d + c0 + c] (k < n, c < 16; zero past column d).
template <typename S>
__device__ __forceinline__ void stage16(float *sV, const S *src, int n, int d, int c0) {
#pragma unroll 4
  for (int e = threadIdx.x; e < n * kRowCols; e += blockDim.x) {
    const int k = e / kRowCols, c = e - k * kRowCols;
    sV[e] = (c0 + c < d) ? (float)ldcg(src + (size_t)k * d + c0 + c) : 0.0f;
  }
}

// Upward pass, eliminated block j of level l: y_j = L_j^{-1} b_j into Yt.
__device__ inline void largeA2_rows(const Args<float> &a, int l, long long j, float *smem) {
  const int n = a.p.n, d = a.d, r = threadIdx.x;
  const long long orig = j << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  const float *Li = a.Li + (size_t)orig * nn;
  for (int c0 = 0; c0 < d; c0 += kRowCols) {
    if (l == 0 && a.B64) stage16(smem, a.B64 + (size_t)orig * nd, n, d, c0);
    else stage16(smem, ((l == 0 && a.Bt) ? a.Bt : a.Y) + (size_t)orig * nd, n, d, c0);
    __syncthreads();
    if (r < n) {
      float acc[kRowCols] = {};
      rowprod16<false>(acc, Li, n, r, 0, r + 1, smem);  // L^{-1} is lower triangular
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c0 + c < d) a.Yt[(size_t)orig * nd + (size_t)r * d + c0 + c] = acc[c];
    }
    __syncthreads();
  }
}

// Upward pass, separator s = 2k of level l: b_s -= W_R(s-1)^T y_{s-1} + W_L(s+1)^T y_{s+1}
// (Algorithm 5), with (W^T y)[r] = sum_q Wt[r][q] y[q] over the stored W^T rows.
__device__ inline void largeB_rows(const Args<float> &a, int l, long long k, float *smem) {
  const int n = a.p.n, d = a.d, r = threadIdx.x;
  const long long Nl = a.p.Nl[l], s = 2 * k;
  const bool hasM = (s >= 2), hasP = (s + 1 < Nl);
  const long long orig = s << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  const float *W = a.Wb + (size_t)a.p.off[l] * nn;
  const float *ys = a.Yt ? a.Yt : a.Y;
  float *sM = smem, *sP = smem + (size_t)n * kRowCols;
  for (int c0 = 0; c0 < d; c0 += kRowCols) {
    if (hasM) stage16(sM, ys + (size_t)((s - 1) << l) * nd, n, d, c0);
    if (hasP) stage16(sP, ys + (size_t)((s + 1) << l) * nd, n, d, c0);
    __syncthreads();
    if (r < n) {
      float acc[kRowCols] = {};
      if (hasM) rowprod16<false>(acc, W + (size_t)(s - 1) * nn, n, r, 0, n, sM);
      if (hasP) rowprod16<false>(acc, W + (size_t)s * nn, n, r, 0, n, sP);
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c0 + c < d) {
          const size_t o = (size_t)orig * nd + (size_t)r * d + c0 + c;
          float base;
          if (l == 0 && a.B64) base = (float)ldcg(a.B64 + o);
          else if (l == 0 && a.Bt) base = ldcg(a.Bt + o);
          else base = ldcg(a.Y + o);
          a.Y[o] = base - acc[c];
        }
    }
    __syncthreads();
  }
}

// Downward pass, eliminated block j of level l (Algorithms 6, 2):
// t = y_j - W_L x_{j-1} - W_R x_{j+1} with (W x)[q] = sum_p Wt[p][q] x[p], then
// x_j = L_j^{-T} t, i.e. x[r] = sum_{q >= r} L^{-1}[q][r] t[q].
__device__ inline void largeC_rows(const Args<float> &a, int l, long long j, float *smem) {
  const int n = a.p.n, d = a.d, r = threadIdx.x;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  const float *W = a.Wb + (size_t)a.p.off[l] * nn;
  const float *Li = a.Li + (size_t)orig * nn;
  const float *Yj = (a.Yt ? a.Yt : a.Y) + (size_t)orig * nd;
  float *sXm = smem, *sXp = smem + (size_t)n * kRowCols, *sT = smem + (size_t)2 * n * kRowCols;
  for (int c0 = 0; c0 < d; c0 += kRowCols) {
    stage16(sXm, a.Y + (size_t)((j - 1) << l) * nd, n, d, c0);
    if (hasR) stage16(sXp, a.Y + (size_t)((j + 1) << l) * nd, n, d, c0);
    __syncthreads();
    if (r < n) {
      float acc[kRowCols] = {};
      rowprod16<true>(acc, W + (size_t)(j - 1) * nn, n, r, 0, n, sXm);
      if (hasR) rowprod16<true>(acc, W + (size_t)j * nn, n, r, 0, n, sXp);
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        sT[r * kRowCols + c] = (c0 + c < d) ? ldcg(Yj + (size_t)r * d + c0 + c) - acc[c] : 0.0f;
    }
    __syncthreads();
    if (r < n) {
      float x[kRowCols] = {};
      rowprod16<true>(x, Li, n, r, r, n, sT);
#pragma unroll
      for (int c = 0; c < kRowCols; ++c)
        if (c0 + c < d) {
          const size_t o = (size_t)orig * nd + (size_t)r * d + c0 + c;
          a.Y[o] = x[c];
          if (a.X64) a.X64[o] = a.x_accumulate ? a.X64[o] + (double)x[c] : (double)x[c];
        }
    }
    __syncthreads();
  }
}

// C: downward pass for eliminated position j of level l.
template <typename T>
__device__ void largeC(const Args<T> &a, int l, long long j, T *smem) {
  const int n = a.p.n, d = a.d, lv = n + 1;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  T *sV = smem;                       // d vectors of length n
  T *work = sV + (size_t)d * lv;
  T *sA = work + kTile * kTilePad, *sB = sA + kKc * kTilePad;
  const T *W = a.Wb + (size_t)a.p.off[l] * nn;
  const T *Yj = (a.Yt ? a.Yt : a.Y) + (size_t)orig * nd;
  // t[q][c] = y[q][c] - sum_p W_L[q][p] x_{j-1}[p][c] - sum_p W_R[q][p] x_{j+1}[p][c],
  // W_L[q][p] = Wt_L[p][q]
  const View<T> WLq{W + (size_t)(j - 1) * nn, 1, n, n, n};
  const View<T> WRq{W + (size_t)j * nn, 1, n, n, n};
  const View<T> Xm{a.Y + (size_t)((j - 1) << l) * nd, 1, d, d, n};
  const View<T> Xp{a.Y + (size_t)((j + 1) << l) * nd, 1, d, d, n};
  for (int R = 0; R < ntiles(n); ++R)
    for (int c0 = 0; c0 < d; c0 += kNarrow) {
      T acc[4] = {};
      const View<T> Xmc{Xm.p + c0, 1, d, d - c0, n};
      const View<T> Xpc{Xp.p + c0, 1, d, d - c0, n};
      gemm_nt_narrow(acc, WLq, R * kTile, Xmc, 0, n, sA, sB);
      if (hasR) gemm_nt_narrow(acc, WRq, R * kTile, Xpc, 0, n, sA, sB);
      const int q = R * kTile + (threadIdx.x >> 2);
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int c = c0 + 4 * (threadIdx.x & 3) + jj;
        if (q < n && c < d) sV[(size_t)c * lv + q] = ldcg(Yj + (size_t)q * d + c) - acc[jj];
      }
      __syncthreads();
    }
  T *Yo = a.Y + (size_t)orig * nd;
  trsv_bwd_blocked(a.Ld + (size_t)orig * nn, n, sV, d, work);
#pragma unroll 4
  for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
    const int i = e / d, c = e - i * d;
    const T x = sV[(size_t)c * lv + i];
    Yo[e] = x;
    if (a.X64) {
      double *xo = a.X64 + (size_t)orig * nd + e;
      *xo = a.x_accumulate ? *xo + (double)x : (double)x;
    }
  }
  __syncthreads();
}

// Top block in FP64: Ltop <- D (from Ld slot 0, or sym(A_00) if no level),
// blocked Cholesky in place, then x_0 = L^{-T} L^{-1} b_0.
template <typename T>
__device__ __noinline__ bool largeTop(const Args<T> &a, bool factor, double *smem, int *s_flag) {
  smem = as_shared(smem);
  s_flag = as_shared(s_flag);
  const int n = a.p.n, d = a.d, L = a.p.L, lv = n + 1;
  const size_t nn = (size_t)n * n;
  if (factor) {
    if (L > 0) {
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) a.Ltop[e] = (double)ldcg(a.Ld + e);
      __syncthreads();
      __threadfence_block();
    }
    const int bad = chol_blocked(a.Ltop, n, L == 0 ? a.A_diag : nullptr, smem, s_flag);
    if (bad) {
      if (threadIdx.x == 0) set_status(a.st, kStNotSPD, L, 0);
      __syncthreads();
      return false;
    }
    if constexpr (sizeof(T) == 4) {
      if (a.Ltinv) {
        // the FP32 solve passes apply the top factor as products with L^{-1}:
        // float(L) into Ltinv[0 .. n^2), then its inverse into Ltinv[n^2 ..),
        // 64 unit vectors at a time through the blocked substitution
        float *Lf = a.Ltinv, *Li = a.Ltinv + nn;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) Lf[e] = (float)a.Ltop[e];
        __syncthreads();
        float *sV = reinterpret_cast<float *>(smem);
        float *work = sV + (size_t)kTile * lv;
        for (int u0 = 0; u0 < n; u0 += kTile) {
          const int nu = min(kTile, n - u0);
          for (int e = threadIdx.x; e < nu * n; e += blockDim.x) {
            const int c = e / n, i = e - c * n;
            sV[(size_t)c * lv + i] = (i == u0 + c) ? 1.0f : 0.0f;
          }
          __syncthreads();
          trsv_fwd_blocked(Lf, n, sV, nu, work);
          for (int e = threadIdx.x; e < n * nu; e += blockDim.x) {
            const int i = e / nu, c = e - i * nu;
            Li[(size_t)i * n + u0 + c] = sV[(size_t)c * lv + i];
          }
          __syncthreads();
        }
      }
    }
  }
  if constexpr (sizeof(T) == 4) {
    if (d > 0 && a.Ltinv) {
      // x_0 = L^{-T} (L^{-1} b_0), a thread per row, FP32 like the rest of the pass
      const float *Li = a.Ltinv + nn;
      float *sB = reinterpret_cast<float *>(smem), *sY = sB + (size_t)n * kRowCols;
      const int r = threadIdx.x;
      for (int c0 = 0; c0 < d; c0 += kRowCols) {
        if (L == 0 && a.B64) stage16(sB, a.B64, n, d, c0);
        else stage16(sB, (L == 0 && a.Bt) ? a.Bt : a.Y, n, d, c0);
        __syncthreads();
        if (r < n) {
          float y[kRowCols] = {};
          rowprod16<false>(y, Li, n, r, 0, r + 1, sB);
#pragma unroll
          for (int c = 0; c < kRowCols; ++c) sY[r * kRowCols + c] = y[c];
        }
        __syncthreads();
        if (r < n) {
          float x[kRowCols] = {};
          rowprod16<true>(x, Li, n, r, r, n, sY);
#pragma unroll
          for (int c = 0; c < kRowCols; ++c)
            if (c0 + c < d) {
              const size_t o = (size_t)r * d + c0 + c;
              a.Y[o] = x[c];
              if (a.X64) a.X64[o] = a.x_accumulate ? a.X64[o] + (double)x[c] : (double)x[c];
            }
        }
        __syncthreads();
      }
      return true;
    }
  }
  if (d > 0) {
    double *sV = smem;
    double *work = sV + (size_t)d * lv;
#pragma unroll 4
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      double v;
      if (L == 0 && a.B64) v = ldcg(a.B64 + e);
      else if (L == 0 && a.Bt) v = (double)ldcg(a.Bt + e);
      else v = (double)ldcg(a.Y + e);
      sV[(size_t)c * lv + i] = v;
    }
    __syncthreads();
    trsv_fwd_blocked(a.Ltop, n, sV, d, work);
    trsv_bwd_blocked(a.Ltop, n, sV, d, work);
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      const double x = sV[(size_t)c * lv + i];
      a.Y[e] = (T)x;
      if (a.X64) a.X64[e] = a.x_accumulate ? a.X64[e] + x : x;
    }
  }
  __syncthreads();
  (void)nn;
  return true;
}

}  // namespace bdss
