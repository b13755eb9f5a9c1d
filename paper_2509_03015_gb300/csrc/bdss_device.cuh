// Device side of odd-even block cyclic reduction for SPD block-tridiagonal
// systems (Sec. 3, Eq. 2-5, Algorithms 1-7, interior segments of length one).
//
// Level l holds N_l = ceil(N / 2^l) blocks; its position j is original block
// j << l.  Odd positions are eliminated, even positions are the separators
// that form level l+1.  Storage (T = double or float):
//   Ld   : N x n x n.  Slot of original block i.  After factoring, the slot of
//          every eliminated block holds its Cholesky factor L (lower
//          triangle; the diagonal holds 1 / L_kk) -- in FP32, L^{-1} with the
//          same diagonal (kStoreInverse) -- and the slot of every separator
//          holds its updated diagonal block (lower triangle) until it is
//          eliminated.  Block 0 is the top block; its FP64 factor is in Ltop
//          (same convention).
//   Wb   : coupling slots, region l = [off_l, off_l + N_l - 1).  Slot k of
//          region l couples level-l positions k and k+1.  Region 0 is written
//          only (its couplings are the caller's A_sub); region l >= 1 first
//          receives the new sub-diagonal S_{k+1,k} (row-major, like A_sub)
//          from the separators of level l-1, which the eliminated block of
//          level l that owns the slot then overwrites with its W^T:
//            eliminated j: slot j-1 <- W_L^T = (L_j^{-1} A_{j,j-1})^T,
//                          slot j   <- W_R^T = (L_j^{-1} A_{j+1,j}^T)^T.
//   Y    : N x n x d right-hand side / solution in T.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

namespace bdss {

constexpr int kMaxLevels = 48;
constexpr int kThreads = 256;
constexpr int kMaxN = 64;

enum { kStOk = 0, kStNotSPD = 2, kStTimeout = 6 };

constexpr int kSmSlots = 256;  // SM-id table of the spread rank
constexpr int kCtaSlots = 8;   // co-resident CTA classes per SM
constexpr int kTraceSlots = 256;  // grid-barrier release stamps kept per launch

struct DevStatus {
  unsigned int bar_count;  // arrivals at the current grid barrier
  unsigned int bar_gen;    // unused (the grid barrier counts arrivals only)
  int status;              // 0 = ok, else a bdss_status code
  int pad;
  long long level;         // NOT_SPD: level and original block of the pivot
  long long block;
  unsigned long long nrm[4];  // residual kernel: bit patterns of max-norms (>= 0)
  unsigned int sm_count[kSmSlots];    // CTAs seen per SM (spread rank)
  unsigned int slot_count[kCtaSlots]; // CTAs per arrival slot (spread rank)
  long long trace[kTraceSlots];       // %globaltimer (ns) at each barrier release
};
// Leading bytes of DevStatus that kernels without grid barriers use (status,
// pivot position, norms): the batched path copies only these per instance.
constexpr size_t kStatusCoreBytes = offsetof(DevStatus, sm_count);

struct Plan {
  long long N;
  int n;
  int L;                         // levels with eliminations; N_L == 1
  long long Nl[kMaxLevels + 1];  // N_l
  long long off[kMaxLevels + 1]; // first Wb slot of region l
};

template <typename T>
struct Args {
  Plan p;
  const double *A_diag;  // caller's blocks (FP64), read at level 0
  const double *A_sub;
  T *Ld;
  T *Wb;
  T *Eb;                 // large-block path: couplings S_{k+1,k} of levels >= 1,
                         // kept apart from Wb (several tasks share one block)
  double *Ltop;
  int d;                 // right-hand-side columns in this call (0: none)
  const double *B64;     // level-0 RHS source in FP64, or null
  const T *Bt;           // level-0 RHS source in T, or null
  T *Y;                  // working RHS / solution (N x n x d)
  double *X64;           // FP64 output; null if Y already is the output
  int x_accumulate;      // X64 += x instead of X64 = x
  DevStatus *st;
  long long timeout_ns;
  int skip_barrier;      // test hook: 1-based barrier index CTA 0 skips
  int capacity;          // CTAs of a full persistent grid (tail-level splits)
  int tf32;              // large FP32 path: Schur products on tcgen05 (3xTF32)
  const CUtensorMap *tmap_w;  // TMA map of Wb as (slots * n) rows x n FP32 columns
  T *Li;                 // large FP32 path: L^{-1} of every eliminated block (slot of
                         // its original index, row-major n x n, zero above the
                         // diagonal), formed by the factorisation; null elsewhere
  T *Ltinv;              // large FP32 path: float(L_top) then its inverse (2 n^2), for
                         // the solve passes' top block; null elsewhere
  T *Yt;                 // large FP32 path, solve passes: y_j = L_j^{-1} b_j of the
                         // eliminated blocks (N x n x d), kept apart from Y because
                         // row tiles of one block are formed by several CTAs
};

// Odd row stride of a staged n x n block (shared-memory bank spread).
__host__ __device__ __forceinline__ int ldstride(int n) { return (n & 1) ? n : n + 1; }

template <typename T> __device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int *p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long global_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_status(DevStatus *st, int code, long long level, long long block) {
  if (atomicCAS(&st->status, 0, code) == 0) {
    st->level = level;
    st->block = block;
  }
}

// |x| as an FP32 value built from the IEEE-754 fields of the FP64 x with
// integer operations only: the exponent is rebiased (1023 -> 127) and the
// top 20 of the 52 fraction bits are kept, so the relative error is below
// 2^-20; magnitudes below 2^-126 give 0 and from 2^128 up (and NaN) give
// +inf.  Used for norm estimates, where a conversion instruction would
// occupy the narrow FP64 pipe.
__device__ __forceinline__ float abs_f32_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x) & 0x7FFFFFFFu;  // exponent and fraction[51:32]
  if (hi < (897u << 20)) return 0.0f;
  if (hi >= (1151u << 20)) return __int_as_float(0x7F800000);
  return __uint_as_float((hi - (896u << 20)) << 3);
}

// CTA-wide maximum of a non-negative double, then one atomicMax on its bit
// pattern (non-negative doubles order like their bit patterns).  All
// threads call.
__device__ inline void cta_max_to(unsigned long long *dst, double v) {
  __shared__ double s_w[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int w = 0; w < nw; ++w) m = fmax(m, s_w[w]);
    atomicMax(dst, (unsigned long long)__double_as_longlong(m));
  }
}

// Ask L2 for `bytes` starting at p (prefetch.global.L2, one 128-byte line
// per thread and step).  Used one task ahead on the caller's level-0 inputs,
// so that blocks held in host memory cross the link while the CTA works on
// its current block.  All threads call.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
  const char *c = static_cast<const char *>(p);
  for (size_t off = (size_t)threadIdx.x * 128; off < bytes; off += (size_t)blockDim.x * 128)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(c + off));
}

// Grid-wide barrier for a cooperative launch.  Every wait is bounded: after
// timeout_ns (or an iteration cap) the waiting CTA records BDSS_ERR_TIMEOUT
// and returns false; any recorded error also makes it return false.  The
// caller must return from the kernel when it gets false.
//
// The arrival counter only grows during a launch (the host clears it before
// each launch): barrier `index` (the launch's barriers are numbered 0, 1, ...
// in order) is released once (index + 1) x gridDim arrivals have been made.
// Each CTA makes one acquire-release add (its CTA's writes, ordered before it
// by the CTA barrier, are released with it) and then polls with acquire
// loads, so no CTA resets or bumps a second word on the release path.  The
// CTA whose arrival completes the count stamps the release time.
__device__ __forceinline__ unsigned atom_add_acq_rel_u32(unsigned *p, unsigned v) {
  unsigned old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

static __device__ __noinline__ bool grid_barrier(DevStatus *st, long long timeout_ns, int index, int skip) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_relaxed_i32(&st->status) != 0) {
      ok = 0;
    } else {
      const unsigned target = (unsigned)(index + 1) * gridDim.x;
      const bool skip_me = (skip == index) && (blockIdx.x == 0);
      unsigned cur;
      if (!skip_me) {
        cur = atom_add_acq_rel_u32(&st->bar_count, 1u) + 1u;
        if (cur == target && index >= 0 && index < kTraceSlots) st->trace[index] = global_ns();
      } else {
        cur = ld_acquire_u32(&st->bar_count);
      }
      if (cur < target) {
        const long long t0 = global_ns();
        const unsigned long long cap = 1000000ull + (unsigned long long)(timeout_ns / 16);
        unsigned long long spins = 0;
        while (ld_acquire_u32(&st->bar_count) < target) {
          if (ld_relaxed_i32(&st->status) != 0) { ok = 0; break; }
          ++spins;
          if ((spins & 31) == 0 && (global_ns() - t0 > timeout_ns || spins > cap)) {
            set_status(st, kStTimeout, -1, -1);
            ok = 0;
            break;
          }
          if (spins > 64) __nanosleep(32);
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Dense rank of this CTA in a cooperative grid such that ranks 0..S-1 sit on
// S different SMs, S..2S-1 again on different SMs, and so on (S = SMs in
// use): each CTA takes an arrival slot on its SM, then an index within its
// slot class; after one grid barrier the class sizes are final and
// rank = (CTAs of lower classes) + index.  Work loops that stride by this
// rank keep a level with fewer blocks than SMs on distinct SMs (consecutive
// block indices of a launch may share an SM).  Returns -1 if the barrier
// reports an error.
static __device__ __noinline__ int spread_rank(DevStatus *st, long long timeout_ns) {
  __shared__ int s_rank;
  __shared__ unsigned s_slot, s_idx;
  if (threadIdx.x == 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    const unsigned slot = atomicAdd(&st->sm_count[smid % kSmSlots], 1u);
    const unsigned cls = slot < kCtaSlots ? slot : kCtaSlots - 1;
    s_slot = cls;
    s_idx = atomicAdd(&st->slot_count[cls], 1u);
  }
  if (!grid_barrier(st, timeout_ns, 0, -1)) return -1;
  if (threadIdx.x == 0) {
    unsigned prefix = 0;
    for (unsigned c = 0; c < s_slot; ++c) prefix += ld_acquire_u32(&st->slot_count[c]);
    s_rank = (int)(prefix + s_idx);
  }
  __syncthreads();
  return s_rank;
}

// ---------------------------------------------------------------------------
// Staging helpers (all threads of the CTA participate).
// ---------------------------------------------------------------------------

// s[i*ld + c] = sym(A)[i][c] = (A[i][c] + A[c][i]) / 2 for c <= i, from a
// caller FP64 block: the whole block is staged row by row (reads in address
// order, also over a host link), then the lower triangle is symmetrised in
// shared memory (the upper triangle is left holding A).  Contains a barrier:
// all threads call.
template <typename T>
__device__ void stage_sym_lower(T *s, int ld, const double *g, int n) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e - i * n;
    s[i * ld + c] = (T)ldcg(g + e);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e - i * n;
    if (c < i) s[i * ld + c] = T(0.5) * (s[i * ld + c] + s[c * ld + i]);
  }
}
// s[i*ld + c] = g[i][c] for c <= i (lower triangle of a workspace block).
template <typename T, typename S>
__device__ void stage_lower(T *s, int ld, const S *g, int n) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e - i * n;
    if (c <= i) s[i * ld + c] = (T)ldcg(g + e);
  }
}
// s[i*ld + c] = g[i][c] (a full n x n block).
template <typename T, typename S>
__device__ void stage_rows(T *s, int ld, const S *g, int n) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, c = e - i * n;
    s[i * ld + c] = (T)ldcg(g + e);
  }
}
// s[c*ld + i] = g[i][c]: the columns of an n x m row-major block become rows.
template <typename T, typename S>
__device__ void stage_cols(T *s, int ld, const S *g, int n, int m) {
  for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
    const int i = e / m, c = e - i * m;
    s[c * ld + i] = (T)ldcg(g + e);
  }
}

// Map a lower-triangle linear index t to (a, b), 0 <= b <= a.
__device__ __forceinline__ void tri_index(int t, int &a, int &b) {
  int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  while (r * (r + 1) / 2 > t) --r;
  a = r;
  b = t - r * (r + 1) / 2;
}

// 1/sqrt(x) for x > 0.  FP64: an FP32 seed (x inside the FP32 range)
// refined by two Newton-Raphson steps on f(y) = 1/y^2 - x, i.e.
// y <- y (3/2 - (x/2) y^2); each step roughly doubles the correct bits
// (23 -> 46 -> full precision).  About 7 FP64 instructions instead of a
// square root and a division on the narrow FP64 pipe.  FP32: rsqrtf.
__device__ __forceinline__ float rsqrt_nr(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
  const double h = 0.5 * x;
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return y;
}

// Pivot of the Cholesky sweeps: 1/sqrt(x) for a positive finite x with five
// FP64 instructions on the critical path (each holds a warp's FP64 issue for
// ~64 cycles on this GPU).  The seed is the FP32 reciprocal square root of x
// cut to FP32 by integer operations (relative error below 2^-22 together);
// one third-order step on f(y) = 1/y^2 - x,
//   e = 1 - x y^2,   y <- y + y e (1/2 + 3/8 e),
// leaves a truncation error of about (5/16) e^3 < 2^-64, so the result is
// within an ulp or two.  Outside the FP32 exponent range: 1 / sqrt(x).
__device__ __forceinline__ float rsqrt_pivot(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_pivot(double x) {
  const long long b = __double_as_longlong(x);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex < 1023 - 120 || ex > 1023 + 120) return 1.0 / sqrt(x);
  const float xf = __int_as_float(((ex - 1023 + 127) << 23) | (int)((b >> 29) & 0x7FFFFF));
  const int yb = __float_as_int(rsqrtf(xf));
  const double y = __longlong_as_double(((long long)(((yb >> 23) & 0xFF) - 127 + 1023) << 52) |
                                        ((long long)(yb & 0x7FFFFF) << 29));
  const double e = fma(-x, y * y, 1.0);
  return fma(y, e * fma(e, 0.375, 0.5), y);
}
// x > 0 and finite, from the bits (no FP64 compare on the pivot path).
__device__ __forceinline__ bool pivot_ok(float x) { return x > 0.0f && isfinite(x); }
__device__ __forceinline__ bool pivot_ok(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && (int)(b >> 52) < 0x7FF;
}

// Cholesky of the staged lower triangle (Algorithm 1, potrf), in place,
// right-looking: per column, warp 0 takes the pivot and scales the column,
// then every thread updates the trailing lower triangle, so the FP64 work
// of the update runs in whole warps.  On exit the diagonal holds 1 / L_kk.
// Returns the first failing column + 1, or 0.
template <typename T>
__device__ int chol_staged(T *s, int ld, int n, int *s_flag) {
  const int tid = threadIdx.x;
  if (tid == 0) *s_flag = 0;
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    if (tid < 32) {
      const T dkk = s[k * ld + k];
      const bool ok = (dkk > T(0)) && isfinite(dkk);
      const T r = rsqrt_nr(ok ? dkk : T(1));
      for (int i = k + 1 + tid; i < n; i += 32) s[i * ld + k] *= r;
      __syncwarp();
      if (tid == 0) {
        s[k * ld + k] = r;
        if (!ok && *s_flag == 0) *s_flag = k + 1;
      }
    }
    __syncthreads();
    if (*s_flag) break;
    const int m = n - k - 1;
    const int cnt = m * (m + 1) / 2;
    for (int t = tid; t < cnt; t += blockDim.x) {
      int a, b;
      tri_index(t, a, b);
      const int i = k + 1 + a, j = k + 1 + b;
      s[i * ld + j] = fma(-s[i * ld + k], s[j * ld + k], s[i * ld + j]);
    }
  }
  __syncthreads();
  return *s_flag;
}

// Packed lower-triangle index t -> (a, b), b <= a < kMaxN, as (a << 8) | b:
// a 4 KB read-only table (L1-resident) instead of a square root per element.
struct TriTable {
  unsigned short v[kMaxN * (kMaxN + 1) / 2];
};
constexpr TriTable make_tri_table() {
  TriTable t{};
  int k = 0;
  for (int a = 0; a < kMaxN; ++a)
    for (int b = 0; b <= a; ++b) t.v[k++] = (unsigned short)((a << 8) | b);
  return t;
}
static __device__ const TriTable g_tri = make_tri_table();

// Barrier among the update warps only (every warp but the current pivot
// warp, named barrier 1).
__device__ __forceinline__ void update_warps_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"((int)blockDim.x - 32) : "memory");
}

// Cholesky of the staged lower triangle fused with forward substitution
// (Algorithm 1's potrf and trsm in one right-looking sweep):
//   L = chol(S) in place (diagonal <- 1 / L_kk), and for every staged vector
//   w (rows of V1 and V2, stride ld): w <- L^{-1} w.
// One warp finishes the next column (its update and pivot) while the other
// warps apply the current column to the trailing triangle and to the
// vectors, so one pivot latency per column is exposed instead of a pivot
// plus a barrier-separated update and a separate substitution.  Each entry
// receives the same fused multiply-adds in the same order as the
// column-by-column factorisation followed by row-by-row substitution.
// Needs blockDim.x >= 64 (a multiple of 32).  Returns the first failing
// column + 1, or 0.
template <typename T>
__device__ int chol_fused(T *s, int ld, int n, T *V1, int nv1, T *V2, int nv2, int *s_flag) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int nv = nv1 + nv2;
  int bad = 0;
  if (tid < 32) {  // column 0
    const T dkk = s[0];
    const bool ok = pivot_ok(dkk);
    const T r = rsqrt_pivot(ok ? dkk : T(1));
    for (int i = 1 + lane; i < n; i += 32) s[i * ld] *= r;
    if (lane == 0) {
      s[0] = r;
      *s_flag = ok ? 0 : 1;
      bad = ok ? 0 : 1;
    }
  }
  if (__syncthreads_or(bad)) return 1;
  // The pivot warp of column k+1 cycles over warps 0..3, which sit on the
  // SM's four sub-partitions: every CTA's pivot chain would otherwise share
  // one sub-partition's FP64 unit with that CTA's update work.
  const int warp = tid >> 5, nw = blockDim.x >> 5, pcyc = nw < 4 ? nw : 4;
  const int un = blockDim.x - 32;  // update-thread count
  for (int k = 0; k + 1 < n; ++k) {
    const int pw = (k + 1) % pcyc;
    if (warp == pw) {
      // column k+1: apply column k, pivot, scale (rows k+1+lane, k+33+lane)
      const int i0 = k + 1 + lane, i1 = i0 + 32;
      const T lk = s[(k + 1) * ld + k];
      T v0 = T(0), v1 = T(0);
      if (i0 < n) v0 = fma(-s[i0 * ld + k], lk, s[i0 * ld + k + 1]);
      if (i1 < n) v1 = fma(-s[i1 * ld + k], lk, s[i1 * ld + k + 1]);
      const T dkk = __shfl_sync(0xffffffffu, v0, 0);
      const bool ok = pivot_ok(dkk);
      const T r = rsqrt_pivot(ok ? dkk : T(1));
      if (i0 < n) s[i0 * ld + k + 1] = lane == 0 ? r : v0 * r;
      if (i1 < n) s[i1 * ld + k + 1] = v1 * r;
      if (lane == 0 && !ok) {
        *s_flag = k + 2;
        bad = 1;
      }
    } else {
      // vectors: w[k] <- w[k] / L_kk, then w[j] -= w[k] L[j][k] for j > k;
      // trailing triangle j >= k+2: S[i][j] -= L[i][k] L[j][k]
      const int ut = warp < pw ? tid : tid - 32;  // index among the update threads
      const T rk = s[k * ld + k];
      for (int v = ut; v < nv; v += un) {
        T *w = v < nv1 ? V1 + v * ld : V2 + (v - nv1) * ld;
        w[k] *= rk;
      }
      update_warps_sync();
      const int m2 = n - k - 2, cnt = m2 * (m2 + 1) / 2;
      const int m1 = n - k - 1, tot = cnt + nv * m1;
      // (v, j) of vector entry u: v = floor(u / m1) through an FP32
      // reciprocal (exact here: u < 2^13 and the quotient is at least
      // 1/(2 m1) away from the next integer)
      const float inv_m1 = 1.0f / (float)m1;
      // kU independent entries per pass, all loads before any store (the
      // stores may not be reordered above later loads of the same array)
      constexpr int kU = sizeof(T) == 8 ? 2 : 4;
      for (int t = ut; t < tot; t += kU * un) {
        T *dst[kU];
        T x[kU], y[kU], z[kU];
#pragma unroll
        for (int q = 0; q < kU; ++q) {
          const int tq = t + q * un;
          if (tq < tot) {
            if (tq < cnt) {
              const unsigned ab = __ldg(&g_tri.v[tq]);
              const int i = k + 2 + (int)(ab >> 8), j = k + 2 + (int)(ab & 255u);
              dst[q] = s + i * ld + j;
              x[q] = s[i * ld + k];
              y[q] = s[j * ld + k];
            } else {
              const int u = tq - cnt;
              const int v = (int)(((float)u + 0.5f) * inv_m1);
              const int j = k + 1 + (u - v * m1);
              T *w = v < nv1 ? V1 + v * ld : V2 + (v - nv1) * ld;
              dst[q] = w + j;
              x[q] = w[k];
              y[q] = s[j * ld + k];
            }
            z[q] = *dst[q];
          }
        }
#pragma unroll
        for (int q = 0; q < kU; ++q)
          if (t + q * un < tot) *dst[q] = fma(-x[q], y[q], z[q]);
      }
    }
    if (__syncthreads_or(bad)) return *s_flag;
  }
  const T rl = s[(n - 1) * ld + n - 1];
  for (int v = tid; v < nv; v += blockDim.x) {
    T *w = v < nv1 ? V1 + v * ld : V2 + (v - nv1) * ld;
    w[n - 1] *= rl;
  }
  __syncthreads();
  return 0;
}

// Warp-cooperative substitutions for a few right-hand sides (n <= 64): lane
// l owns rows l and l + 32 of every vector (vectors are rows of V, stride
// ld); each pivot is finished by its owning lane and broadcast by shuffle,
// then all lanes update their rows.  One warp runs the whole solve, so the
// FP64 work of a handful of vectors fills its lanes instead of one lane per
// vector.  Call from exactly one warp.
template <typename T, int C = 4>
__device__ void trsv_fwd_warp(const T *sL, int ld, int n, T *V, int nv) {
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < nv; c0 += C) {
    const int cn = min(C, nv - c0);
    T y0[C], y1[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      y0[c] = (c < cn && lane < n) ? V[(c0 + c) * ld + lane] : T(0);
      y1[c] = (c < cn && lane + 32 < n) ? V[(c0 + c) * ld + lane + 32] : T(0);
    }
    for (int r = 0; r < n; ++r) {
      const T rd = sL[r * ld + r];
      const int owner = r & 31;
      T yr[C];
      if (r < 32) {
#pragma unroll
        for (int c = 0; c < C; ++c) yr[c] = __shfl_sync(0xffffffffu, y0[c] * rd, owner);
        if (lane == owner)
#pragma unroll
          for (int c = 0; c < C; ++c) y0[c] = yr[c];
        const T l0 = (lane > r && lane < n) ? sL[lane * ld + r] : T(0);
#pragma unroll
        for (int c = 0; c < C; ++c) y0[c] = fma(-l0, yr[c], y0[c]);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) yr[c] = __shfl_sync(0xffffffffu, y1[c] * rd, owner);
        if (lane == owner)
#pragma unroll
          for (int c = 0; c < C; ++c) y1[c] = yr[c];
      }
      if (n > 32) {
        const T l1 = (lane + 32 > r && lane + 32 < n) ? sL[(lane + 32) * ld + r] : T(0);
#pragma unroll
        for (int c = 0; c < C; ++c) y1[c] = fma(-l1, yr[c], y1[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (c < cn && lane < n) V[(c0 + c) * ld + lane] = y0[c];
      if (c < cn && lane + 32 < n) V[(c0 + c) * ld + lane + 32] = y1[c];
    }
  }
}

// L^T z = t, same organisation, from the last row up.
template <typename T, int C = 4>
__device__ void trsv_bwd_warp(const T *sL, int ld, int n, T *V, int nv) {
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < nv; c0 += C) {
    const int cn = min(C, nv - c0);
    T y0[C], y1[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      y0[c] = (c < cn && lane < n) ? V[(c0 + c) * ld + lane] : T(0);
      y1[c] = (c < cn && lane + 32 < n) ? V[(c0 + c) * ld + lane + 32] : T(0);
    }
    for (int r = n - 1; r >= 0; --r) {
      const T rd = sL[r * ld + r];
      const int owner = r & 31;
      T zr[C];
      if (r >= 32) {
#pragma unroll
        for (int c = 0; c < C; ++c) zr[c] = __shfl_sync(0xffffffffu, y1[c] * rd, owner);
        if (lane == owner)
#pragma unroll
          for (int c = 0; c < C; ++c) y1[c] = zr[c];
        const T l1 = (lane + 32 < r) ? sL[r * ld + lane + 32] : T(0);
#pragma unroll
        for (int c = 0; c < C; ++c) y1[c] = fma(-l1, zr[c], y1[c]);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) zr[c] = __shfl_sync(0xffffffffu, y0[c] * rd, owner);
        if (lane == owner)
#pragma unroll
          for (int c = 0; c < C; ++c) y0[c] = zr[c];
      }
      const T l0 = (lane < r) ? sL[r * ld + lane] : T(0);
#pragma unroll
      for (int c = 0; c < C; ++c) y0[c] = fma(-l0, zr[c], y0[c]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      if (c < cn && lane < n) V[(c0 + c) * ld + lane] = y0[c];
      if (c < cn && lane + 32 < n) V[(c0 + c) * ld + lane + 32] = y1[c];
    }
  }
}

// The same substitutions with the vectors spread over the CTA's warps, one
// vector per warp at a time: a warp issues at most one FP64 instruction per
// ~64 cycles on this GPU, so a handful of right-hand sides on one warp is
// bound by that rate while the SM's other FP64 units idle.  Same operations
// per vector as above.  All threads call; no barrier inside.
template <typename T>
__device__ void trsv_fwd_cta(const T *sL, int ld, int n, T *V, int nv) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = warp; v < nv; v += nw) trsv_fwd_warp<T, 1>(sL, ld, n, V + (size_t)v * ld, 1);
}
template <typename T>
__device__ void trsv_bwd_cta(const T *sL, int ld, int n, T *V, int nv) {
  const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = warp; v < nv; v += nw) trsv_bwd_warp<T, 1>(sL, ld, n, V + (size_t)v * ld, 1);
}

// Forward substitution L w = v for `nv` staged vectors (rows of V, stride
// ldv), L an n x n lower-triangular tile (stride ldl, reciprocal diagonal),
// both in shared memory.  On this GPU one warp issues at most one FP64
// instruction per ~64 cycles and the SM's FP64 pipe needs four or more warps
// to be full, so the work is spread over all warps: rows are taken 8 at a
// time; the update of a row block from the rows already solved runs over
// (vector, row) pairs on every thread, then one thread per vector solves the
// 8 x 8 diagonal triangle.  Each vector receives the same operations in the
// same order as the row-by-row sweep.  All threads call; ends with a barrier.
template <typename T>
__device__ void trsv_tile_fwd(const T *sL, int ldl, int n, T *V, int ldv, int nv) {
  constexpr int RB = 8;
  for (int r0 = 0; r0 < n; r0 += RB) {
    const int rb = min(RB, n - r0);
    if (r0 > 0) {
      for (int t = threadIdx.x; t < nv * rb; t += blockDim.x) {
        const int i = t / nv, v = t - i * nv;
        T *w = V + (size_t)v * ldv;
        const T *lr = sL + (size_t)(r0 + i) * ldl;
        T acc = w[r0 + i];
        for (int p = 0; p < r0; ++p) acc = fma(-lr[p], w[p], acc);
        w[r0 + i] = acc;
      }
      __syncthreads();
    }
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      T *w = V + (size_t)v * ldv + r0;
      T acc[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) acc[i] = (i < rb) ? w[i] : T(0);
#pragma unroll
      for (int i = 0; i < RB; ++i)
        if (i < rb) {
          T a = acc[i];
#pragma unroll
          for (int q = 0; q < i; ++q) a = fma(-sL[(size_t)(r0 + i) * ldl + r0 + q], acc[q], a);
          acc[i] = a * sL[(size_t)(r0 + i) * ldl + r0 + i];
        }
#pragma unroll
      for (int i = 0; i < RB; ++i)
        if (i < rb) w[i] = acc[i];
    }
    __syncthreads();
  }
}

// Backward substitution L^T z = t, same organisation from the last row block
// up: the update of a row block from the rows below runs over (vector, row)
// pairs, then one thread per vector solves the block's triangle.
template <typename T>
__device__ void trsv_tile_bwd(const T *sL, int ldl, int n, T *V, int ldv, int nv) {
  constexpr int RB = 8;
  for (int r1 = n; r1 > 0; r1 -= RB) {
    const int r0 = max(0, r1 - RB), rb = r1 - r0;
    if (r1 < n) {
      for (int t = threadIdx.x; t < nv * rb; t += blockDim.x) {
        const int i = t / nv, v = t - i * nv;
        T *w = V + (size_t)v * ldv;
        T acc = w[r0 + i];
        for (int p = r1; p < n; ++p) acc = fma(-sL[(size_t)p * ldl + r0 + i], w[p], acc);
        w[r0 + i] = acc;
      }
      __syncthreads();
    }
    for (int v = threadIdx.x; v < nv; v += blockDim.x) {
      T *w = V + (size_t)v * ldv + r0;
      T acc[RB];
#pragma unroll
      for (int i = 0; i < RB; ++i) acc[i] = (i < rb) ? w[i] : T(0);
#pragma unroll
      for (int i = RB - 1; i >= 0; --i)
        if (i < rb) {
          T a = acc[i];
#pragma unroll
          for (int q = i + 1; q < RB; ++q)
            if (q < rb) a = fma(-sL[(size_t)(r0 + q) * ldl + r0 + i], acc[q], a);
          acc[i] = a * sL[(size_t)(r0 + i) * ldl + r0 + i];
        }
#pragma unroll
      for (int i = 0; i < RB; ++i)
        if (i < rb) w[i] = acc[i];
    }
    __syncthreads();
  }
}

// Square tiles with one stride for L and the vectors.
template <typename T>
__device__ void trsv_fwd_rows(const T *sL, int ld, int n, T *V, int nv) {
  trsv_tile_fwd(sL, ld, n, V, ld, nv);
}

// Shared-memory words (in T) of each phase.
// Phase A holds L, one pass of n coupling vectors and the d RHS vectors;
// phase B holds two W^T blocks and two d-vector sets.  (Two passes / two
// stages keep a CTA near 70 KB at n = 64 in FP64, so that three CTAs share
// an SM.)
__host__ __device__ inline size_t smem_phaseA(int n, int d) {
  const int ld = ldstride(n);
  return (size_t)(2 * n + d) * ld + 8;
}
__host__ __device__ inline size_t smem_phaseB(int n, int d, int esz) {
  const int ld = ldstride(n);
  const size_t generic = (size_t)(2 * n + 2 * d) * ld + 8;
  if (esz != 4) return generic;
  const size_t fp32_tiled = (size_t)2 * 64 * 68 + (size_t)2 * d * n + 8;  // phaseB_f32
  return generic > fp32_tiled ? generic : fp32_tiled;
}
__host__ __device__ inline size_t smem_down(int n, int d) {
  const int ld = ldstride(n);
  return (size_t)n * ld + (size_t)3 * d * ld + 8;
}
__host__ __device__ inline size_t smem_top_bytes(int n, int d) {
  const int ld = ldstride(n);
  return ((size_t)n * ld + (size_t)d * ld + 8) * sizeof(double);
}

// The FP32 path (n <= 64) keeps L^{-1} instead of L in the slot of every
// eliminated block, so that its solve passes (run once per refinement step)
// apply the triangular factors as products instead of substitutions; the
// extra n^3/6 FMAs per block are FP32.  The diagonal still holds 1 / L_kk.
template <typename T> constexpr bool kStoreInverse = sizeof(T) == 4;

// CTAs per block at a level with few blocks: the persistent grid holds
// `capacity` CTAs; when a level has fewer blocks than that, each block's
// work is split over up to max_parts CTAs (one CTA per block would leave most
// SMs idle while the level's latency sets the pace).
__host__ __device__ inline int split_parts(long long items, int capacity, int max_parts) {
  if (items <= 0) return 1;
  const long long k = (long long)capacity / items;
  if (k < 2) return 1;
  return k > max_parts ? max_parts : (int)k;
}
constexpr int kMaxPartsA = 8;  // coupling columns of phase A over CTAs
constexpr int kMaxPartsB = 8;  // output entries of the FP64 phase B over CTAs

// Blocks below n = 32 hold too little work per column to be worth a CTA
// each: no split there (fewer CTAs also make the grid barriers cheaper).
constexpr int kSplitMinN = 32;
template <typename T> __host__ __device__ inline int parts_A(const Plan &p, int l, bool factor, int capacity) {
  return (factor && p.n >= kSplitMinN) ? split_parts(p.Nl[l] / 2, capacity, kMaxPartsA) : 1;
}
template <typename T> __host__ __device__ inline int parts_B(const Plan &p, int l, bool factor, int capacity) {
  return (factor && sizeof(T) == 8 && p.n >= kSplitMinN) ? split_parts((p.Nl[l] + 1) / 2, capacity, kMaxPartsB)
                                                          : 1;
}

// s[(c - c0)*ld + i] = g[i][c] for c0 <= c < c1 (columns of an n x n block).
template <typename T, typename S>
__device__ void stage_col_range(T *s, int ld, const S *g, int n, int c0, int c1) {
  const int w = c1 - c0;
  for (int e = threadIdx.x; e < n * w; e += blockDim.x) {
    const int i = e / w, c = e - i * w;
    s[c * ld + i] = (T)ldcg(g + (size_t)i * n + c0 + c);
  }
}
// s[(r - r0)*ld + c] = g[r][c] for r0 <= r < r1 (rows of an n x n block).
template <typename T, typename S>
__device__ void stage_row_range(T *s, int ld, const S *g, int n, int r0, int r1) {
  for (int e = threadIdx.x; e < (r1 - r0) * n; e += blockDim.x) {
    const int r = e / n, c = e - r * n;
    s[r * ld + c] = (T)ldcg(g + (size_t)(r0 + r) * n + c);
  }
}

// Level-0 inputs of eliminated position j (A_jj, A_{j,j-1}, A_{j+1,j}, b_j)
// and of separator position s (A_ss, b_s), for prefetch_l2.
template <typename T>
__device__ void prefetch_elim_inputs(const Args<T> &a, long long j) {
  const size_t nn = (size_t)a.p.n * a.p.n, nd = (size_t)a.p.n * a.d;
  prefetch_l2(a.A_diag + j * nn, nn * sizeof(double));
  prefetch_l2(a.A_sub + (j - 1) * nn, (j + 1 < a.p.N ? 2 : 1) * nn * sizeof(double));
  if (a.B64 && nd) prefetch_l2(a.B64 + j * nd, nd * sizeof(double));
}
template <typename T>
__device__ void prefetch_sep_inputs(const Args<T> &a, long long s) {
  const size_t nn = (size_t)a.p.n * a.p.n, nd = (size_t)a.p.n * a.d;
  prefetch_l2(a.A_diag + s * nn, nn * sizeof(double));
  if (a.B64 && nd) prefetch_l2(a.B64 + s * nd, nd * sizeof(double));
}

// ---------------------------------------------------------------------------
// Phase A: eliminated position j (odd) of level l.
//   factor:  L_j = chol(D_j); W_L^T, W_R^T via forward substitution (trsm);
//   rhs:     y_j = L_j^{-1} b_j (Algorithm 5's interior solve, fused).
// With factor == false only the RHS part runs, using the stored L_j.
// The 2n coupling columns (n of W_L, then n of W_R) may be split over
// `nparts` CTAs: each factors D_j itself (the same arithmetic, so the same
// L_j), solves its contiguous share of the columns, and part 0 alone stores
// L_j and handles the right-hand sides.  Every column is solved by the same
// operations whatever the split.
// ---------------------------------------------------------------------------
template <typename T>
__device__ bool phaseA(const Args<T> &a, int l, long long j, bool factor, T *smem, int *s_flag, int part = 0,
                       int nparts = 1) {
  const int n = a.p.n, ld = ldstride(n);
  const int d = part == 0 ? a.d : 0;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n;
  const int nW = factor ? (hasR ? 2 * n : n) : 0;
  const int c0 = (int)((long long)part * nW / nparts), c1 = (int)((long long)(part + 1) * nW / nparts);
  const int l0 = c0, l1 = min(c1, n);                   // W_L columns of this part
  const int r0 = max(c0, n) - n, r1 = c1 - n;           // W_R columns (rows of A_{j+1,j})
  if (part > 0 && c1 <= c0) return true;                // nothing to solve here
  T *sL = smem;
  T *sV = sL + (size_t)n * ld;                          // up to n coupling vectors (one pass)
  T *sB = sV + (size_t)(factor ? n : 0) * ld;           // d RHS vectors
  const T *E = (l == 0) ? nullptr : a.Wb + (size_t)a.p.off[l] * nn;
  T *W = a.Wb + (size_t)a.p.off[l] * nn;
  const T *EL = (l == 0) ? nullptr : E + (size_t)(j - 1) * nn;
  const T *ER = (l == 0) ? nullptr : E + (size_t)j * nn;
  const double *AL = a.A_sub ? a.A_sub + (size_t)(j - 1) * nn : nullptr;
  const double *AR = a.A_sub ? a.A_sub + (size_t)j * nn : nullptr;

  // vectors solved along with the factorisation: this part's W_L columns,
  // or its W_R columns if it has no W_L ones; W_R columns of a part that
  // has both follow in a second pass
  const bool passL = l1 > l0, fuseR = !passL && r1 > r0;
  if (factor) {
    if (l == 0) stage_sym_lower(sL, ld, a.A_diag + orig * nn, n);
    else stage_lower(sL, ld, a.Ld + orig * nn, n);
    if (passL) {  // columns of E_l[j-1] = A_{j,j-1}
      if (l == 0) stage_col_range(sV, ld, AL, n, l0, l1);
      else stage_col_range(sV, ld, EL, n, l0, l1);
    } else if (fuseR) {  // rows of E_l[j] = A_{j+1,j}
      if (l == 0) stage_row_range(sV, ld, AR, n, r0, r1);
      else stage_row_range(sV, ld, ER, n, r0, r1);
    }
  } else {
    stage_lower(sL, ld, a.Ld + orig * nn, n);
  }
  if (d > 0) {
    const size_t boff = (size_t)orig * n * d;
    if (l == 0 && a.B64) stage_cols(sB, ld, a.B64 + boff, n, d);
    else if (l == 0 && a.Bt) stage_cols(sB, ld, a.Bt + boff, n, d);
    else stage_cols(sB, ld, a.Y + boff, n, d);
  }
  __syncthreads();
  const int nvf = passL ? l1 - l0 : (fuseR ? r1 - r0 : 0);
  if (factor) {
    int bad;
    if (blockDim.x >= 64 && sizeof(T) == 8) {
      // FP64: the sweep carries the d right-hand sides only; the coupling
      // columns follow in the blocked substitution.  The sweep's column
      // barriers then pace the short pivot chain alone, while the
      // substitution's long (vector, row) updates run with few barriers and
      // fill the FP64 pipe for the other CTAs on the SM (level 0 of the
      // N = 16384, n = 64 system: 5.63 -> 5.35 ms).  Each entry receives the
      // same operations in the same order either way.
      bad = chol_fused(sL, ld, n, sV, 0, sB, d, s_flag);
      if (!bad && nvf > 0) trsv_fwd_rows(sL, ld, n, sV, nvf);
    } else if (blockDim.x >= 64) {
      // FP32: short FMA latency makes the separate substitution cheap
      bad = chol_fused(sL, ld, n, sV, 0, sB, 0, s_flag);
      if (!bad) {
        if (nvf > 0) trsv_fwd_rows(sL, ld, n, sV, nvf);
        if (d > 0) trsv_fwd_cta(sL, ld, n, sB, d);
        __syncthreads();
      }
    } else {
      bad = chol_staged(sL, ld, n, s_flag);
      if (!bad) {
        if (nvf > 0) trsv_fwd_rows(sL, ld, n, sV, nvf);
        if (d > 0) trsv_fwd_cta(sL, ld, n, sB, d);
        __syncthreads();
      }
    }
    if (bad) {
      if (threadIdx.x == 0) set_status(a.st, kStNotSPD, l, orig);
      __syncthreads();
      return false;
    }
    if (part == 0 && !kStoreInverse<T>) {
      T *Lg = a.Ld + orig * nn;
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        if (c <= r) Lg[e] = sL[r * ld + c];
      }
    }
  } else if (d > 0 && kStoreInverse<T>) {
    // FP32 solve pass: y = L^{-1} b as a product with the stored inverse
    T *Yj = a.Y + (size_t)orig * n * d;
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      const T *li = sL + i * ld, *b = sB + c * ld;
      T acc = T(0);
      for (int p = 0; p <= i; ++p) acc = fma(li[p], b[p], acc);
      Yj[e] = acc;
    }
    __syncthreads();
    return true;
  } else if (d > 0) {
    trsv_fwd_cta(sL, ld, n, sB, d);
    __syncthreads();
  }
  if (nvf > 0) {
    T *Wd = W + (size_t)(passL ? j - 1 : j) * nn;
    const int c0w = passL ? l0 : r0;
    for (int e = threadIdx.x; e < nvf * n; e += blockDim.x) {
      const int c = e / n, i = e - c * n;
      Wd[(size_t)(c0w + c) * n + i] = sV[c * ld + i];
    }
  }
  if (d > 0) {
    T *Yj = a.Y + (size_t)orig * n * d;
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      Yj[e] = sB[c * ld + i];
    }
  }
  if (passL && r1 > r0) {
    // pass 2: W_R from the rows of E_l[j] = A_{j+1,j}
    __syncthreads();
    if (l == 0) stage_row_range(sV, ld, AR, n, r0, r1);
    else stage_row_range(sV, ld, ER, n, r0, r1);
    __syncthreads();
    trsv_fwd_rows(sL, ld, n, sV, r1 - r0);
    __syncthreads();
    T *WR = W + (size_t)j * nn;
    for (int e = threadIdx.x; e < (r1 - r0) * n; e += blockDim.x) {
      const int c = e / n, i = e - c * n;
      WR[(size_t)(r0 + c) * n + i] = sV[c * ld + i];
    }
  }
  if (kStoreInverse<T> && factor && part == 0) {
    // FP32: store L^{-1} (its diagonal is the same 1 / L_kk): the columns of
    // the identity through the substitution
    __syncthreads();
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int c = e / n, i = e - c * n;
      sV[c * ld + i] = (i == c) ? T(1) : T(0);
    }
    __syncthreads();
    trsv_fwd_rows(sL, ld, n, sV, n);
    T *Lg = a.Ld + orig * nn;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      const int i = e / n, c = e - i * n;
      if (c <= i) Lg[e] = sV[c * ld + i];
    }
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Phase B: separator position s = 2k of level l (Algorithm 3 + Assemble,
// Algorithm 5's separator update):
//   S_ss      = D_s - W_R(s-1)^T W_R(s-1) - W_L(s+1)^T W_L(s+1)  (lower)
//   b_s      -= W_R(s-1)^T y_{s-1} + W_L(s+1)^T y_{s+1}
//   S_{s+2,s} = -W_R(s+1)^T W_L(s+1)  -> region l+1, slot k
// W_R(s+1)^T is staged over W_R(s-1)^T once the first two are done.
// ---------------------------------------------------------------------------
// FP32 phase B (n <= 64, 256 threads): the W^T blocks are staged k-major
// (sK[k][r] = W^T[r][k], rows of 68 floats, zero beyond n) so that each thread
// computes a 4 x 4 tile of the 64 x 64 products with two 128-bit shared loads
// per 16 FMAs; D is formed in full (only its lower triangle is stored).
constexpr int kPB = 68;  // k-major row stride (floats), 16-byte aligned

// g == nullptr stages zeros (a separator without that neighbour).
__device__ __forceinline__ void stage_kmajor(float *sK, const float *g, int n) {
  for (int e = threadIdx.x; e < kMaxN * kMaxN; e += blockDim.x) {
    const int r = e >> 6, kk = e & 63;   // coalesced over k
    sK[kk * kPB + r] = (g && r < n && kk < n) ? ldcg(g + (size_t)r * n + kk) : 0.0f;
  }
}

__device__ __forceinline__ void tile_acc_kmajor(float (&acc)[4][4], const float *sA, const float *sB, int n, int tr,
                                                int tc) {
  for (int kk = 0; kk < n; ++kk) {
    const float4 x = *reinterpret_cast<const float4 *>(sA + kk * kPB + 4 * tr);
    const float4 y = *reinterpret_cast<const float4 *>(sB + kk * kPB + 4 * tc);
    const float xa[4] = {x.x, x.y, x.z, x.w}, yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(xa[i], yb[j], acc[i][j]);
  }
}

__device__ inline void phaseB_f32(const Args<float> &a, int l, long long k, bool factor, float *smem) {
  const int n = a.p.n, d = a.d;
  const long long Nl = a.p.Nl[l];
  const long long s = 2 * k;
  const bool hasM = (s >= 2), hasP = (s + 1 < Nl), hasE = (s + 2 < Nl);
  const long long orig = s << l;
  const size_t nn = (size_t)n * n;
  float *sK0 = smem;                        // W_R(s-1)^T, later W_R(s+1)^T, k-major
  float *sK1 = sK0 + kMaxN * kPB;           // W_L(s+1)^T, k-major
  float *sY = sK1 + kMaxN * kPB;            // y_{s-1}, y_{s+1}: [2][d][n]
  const float *W = a.Wb + (size_t)a.p.off[l] * nn;
  const int tr = threadIdx.x >> 4, tc = threadIdx.x & 15;
  stage_kmajor(sK0, hasM ? W + (size_t)(s - 1) * nn : nullptr, n);
  stage_kmajor(sK1, hasP ? W + (size_t)s * nn : nullptr, n);
  if (d > 0)
    for (int e = threadIdx.x; e < 2 * n * d; e += blockDim.x) {
      const int side = e / (n * d), rem = e - side * n * d, q = rem / d, c = rem - q * d;
      const bool have = side == 0 ? hasM : hasP;
      const long long blk = side == 0 ? s - 1 : s + 1;
      sY[(side * d + c) * n + q] = have ? ldcg(a.Y + (size_t)(blk << l) * n * d + rem) : 0.0f;
    }
  __syncthreads();
  if (factor) {
    float acc[4][4] = {};
    if (hasM) tile_acc_kmajor(acc, sK0, sK0, n, tr, tc);
    if (hasP) tile_acc_kmajor(acc, sK1, sK1, n, tr, tc);
    float *Dg = a.Ld + (size_t)orig * nn;
    const double *Ag = a.A_diag + (size_t)orig * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * tr + i, c = 4 * tc + j;
        if (r < n && c <= r) {
          const float base = (l == 0) ? 0.5f * ((float)ldcg(Ag + r * n + c) + (float)ldcg(Ag + c * n + r))
                                      : ldcg(Dg + r * n + c);
          Dg[r * n + c] = base - acc[i][j];
        }
      }
  }
  if (d > 0) {
    const size_t boff = (size_t)orig * n * d;
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int r = e / d, c = e - r * d;
      float acc;
      if (l == 0 && a.B64) acc = (float)ldcg(a.B64 + boff + e);
      else if (l == 0 && a.Bt) acc = ldcg(a.Bt + boff + e);
      else acc = ldcg(a.Y + boff + e);
      const float *ym = sY + (size_t)c * n, *yp = sY + (size_t)(d + c) * n;
      for (int q = 0; q < n; ++q) acc = fmaf(-sK0[q * kPB + r], ym[q], fmaf(-sK1[q * kPB + r], yp[q], acc));
      a.Y[boff + e] = acc;
    }
  }
  if (factor && hasE) {
    __syncthreads();
    stage_kmajor(sK0, W + (size_t)(s + 1) * nn, n);
    __syncthreads();
    float acc[4][4] = {};
    tile_acc_kmajor(acc, sK0, sK1, n, tr, tc);
    float *En = a.Wb + ((size_t)a.p.off[l + 1] + (size_t)k) * nn;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = 4 * tr + i, c = 4 * tc + j;
        if (r < n && c < n) En[r * n + c] = -acc[i][j];
      }
  }
  __syncthreads();
}

// FP64 / generic phase B.  Its outputs -- the lower triangle of S_ss, the
// n x d RHS update and the n x n coupling S_{s+2,s} -- may be split over
// `nparts` CTAs, each taking a contiguous share of each; every entry is
// formed by the same operations whatever the split.
template <typename T>
__device__ void phaseB(const Args<T> &a, int l, long long k, bool factor, T *smem, int part = 0, int nparts = 1) {
  if constexpr (std::is_same<T, float>::value) {
    if (blockDim.x == kThreads && nparts == 1) {
      phaseB_f32(a, l, k, factor, smem);
      return;
    }
  }
  const int n = a.p.n, ld = ldstride(n), d = a.d;
  const long long Nl = a.p.Nl[l];
  const long long s = 2 * k;
  const bool hasM = (s >= 2), hasP = (s + 1 < Nl), hasE = (s + 2 < Nl);
  const long long orig = s << l;
  const size_t nn = (size_t)n * n;
  const int ntri = n * (n + 1) / 2;
  const int t0 = (int)((long long)part * ntri / nparts), t1 = (int)((long long)(part + 1) * ntri / nparts);
  const int b0 = (int)((long long)part * n * d / nparts), b1 = (int)((long long)(part + 1) * n * d / nparts);
  const int e0 = (int)((long long)part * n * n / nparts), e1 = (int)((long long)(part + 1) * n * n / nparts);
  T *sW0 = smem;                      // W_R(s-1)^T, later W_R(s+1)^T
  T *sW1 = sW0 + (size_t)n * ld;      // W_L(s+1)^T
  T *sY = sW1 + (size_t)n * ld;       // y_{s-1}, y_{s+1} as d vectors each
  const T *W = a.Wb + (size_t)a.p.off[l] * nn;
  if (hasM) stage_rows(sW0, ld, W + (size_t)(s - 1) * nn, n);
  if (hasP) stage_rows(sW1, ld, W + (size_t)s * nn, n);
  if (d > 0 && b1 > b0) {
    if (hasM) stage_cols(sY, ld, a.Y + (size_t)((s - 1) << l) * n * d, n, d);
    if (hasP) stage_cols(sY + (size_t)d * ld, ld, a.Y + (size_t)((s + 1) << l) * n * d, n, d);
  }
  __syncthreads();
  if (factor) {
    // diagonal update, lower triangle
    T *Dg = a.Ld + (size_t)orig * nn;
    const double *Ag = a.A_diag + (size_t)orig * nn;
    for (int t = t0 + threadIdx.x; t < t1; t += blockDim.x) {
      int r, c;
      tri_index(t, r, c);
      T acc;
      if (l == 0) acc = T(0.5) * ((T)ldcg(Ag + r * n + c) + (T)ldcg(Ag + c * n + r));
      else acc = ldcg(Dg + r * n + c);
      if (hasM) {
        const T *wr = sW0 + r * ld, *wc = sW0 + c * ld;
        for (int q = 0; q < n; ++q) acc = fma(-wr[q], wc[q], acc);
      }
      if (hasP) {
        const T *wr = sW1 + r * ld, *wc = sW1 + c * ld;
        for (int q = 0; q < n; ++q) acc = fma(-wr[q], wc[q], acc);
      }
      Dg[r * n + c] = acc;
    }
  }
  if (d > 0) {
    const size_t boff = (size_t)orig * n * d;
    for (int e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
      const int r = e / d, c = e - r * d;
      T acc;
      if (l == 0 && a.B64) acc = (T)ldcg(a.B64 + boff + e);
      else if (l == 0 && a.Bt) acc = ldcg(a.Bt + boff + e);
      else acc = ldcg(a.Y + boff + e);
      if (hasM) {
        const T *wr = sW0 + r * ld, *y = sY + (size_t)c * ld;
        for (int q = 0; q < n; ++q) acc = fma(-wr[q], y[q], acc);
      }
      if (hasP) {
        const T *wr = sW1 + r * ld, *y = sY + (size_t)(d + c) * ld;
        for (int q = 0; q < n; ++q) acc = fma(-wr[q], y[q], acc);
      }
      a.Y[boff + e] = acc;
    }
  }
  if (factor && hasE && e1 > e0) {
    __syncthreads();
    stage_rows(sW0, ld, W + (size_t)(s + 1) * nn, n);
    __syncthreads();
    T *En = a.Wb + ((size_t)a.p.off[l + 1] + (size_t)k) * nn;
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
      const int r = e / n, c = e - r * n;
      const T *wr = sW0 + r * ld, *wc = sW1 + c * ld;
      T acc = T(0);
      for (int q = 0; q < n; ++q) acc = fma(-wr[q], wc[q], acc);
      En[e] = acc;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Serial top sweep: the recursion stops at the first level with at most N_*
// blocks (Sec. 3.3: below the crossover N_* the serial block-Cholesky sweep
// is used) and the M blocks of that level are factored by Algorithm 1 with
// K = 1 and solved by Algorithm 2 with K = 1, in FP64 by one CTA:
//   D_j' = D_j - C_{j-1} C_{j-1}^T,  L_j = chol(D_j'),  C_j = E_j L_j^{-T},
//   y_j = L_j^{-1} (b_j - C_{j-1} y_{j-1}),  x_j = L_j^{-T} (y_j - C_j^T x_{j+1}),
// with E_j = A_{j+1,j} of that level.  Ltop holds L_j at j n^2, C_j at
// (kNStarMax + j) n^2 and y_j / x_j at 2 kNStarMax n^2 + j n d (doubles).
// Shared memory: (2 n + d) ldstride(n) doubles.
// ---------------------------------------------------------------------------
constexpr int kNStarMax = 64;  // largest N_* (top blocks of the serial sweep)

template <typename T>
__device__ bool top_sweep(const Args<T> &a, bool factor, double *smem, int *s_flag) {
  const int n = a.p.n, ld = ldstride(n), d = a.d, L = a.p.L;
  const int M = (int)a.p.Nl[L];
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  double *sL = smem;                     // L_j (lower, reciprocal diagonal)
  double *sC = sL + (size_t)n * ld;      // rows of E_j, then of C_j
  double *sB = sC + (size_t)n * ld;      // d vectors
  double *LC = a.Ltop + (size_t)kNStarMax * nn;
  double *Ys = a.Ltop + (size_t)2 * kNStarMax * nn;
  const T *E = (L == 0) ? nullptr : a.Wb + (size_t)a.p.off[L] * nn;
  for (int j = 0; j < M; ++j) {
    const long long orig = (long long)j << L;
    if (factor) {
      if (L == 0) stage_sym_lower(sL, ld, a.A_diag + orig * nn, n);
      else stage_lower(sL, ld, a.Ld + orig * nn, n);
      __syncthreads();
      if (j > 0) {  // D_j -= C_{j-1} C_{j-1}^T (lower triangle)
        const double *Cp = LC + (size_t)(j - 1) * nn;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
          const int r = e / n, c = e - r * n;
          if (c > r) continue;
          double acc = 0.0;
          for (int k = 0; k < n; ++k) acc = fma(ldcg(Cp + (size_t)r * n + k), ldcg(Cp + (size_t)c * n + k), acc);
          sL[r * ld + c] -= acc;
        }
        __syncthreads();
      }
      if (chol_staged(sL, ld, n, s_flag)) {
        if (threadIdx.x == 0) set_status(a.st, kStNotSPD, L, orig);
        __syncthreads();
        return false;
      }
      double *Lj = a.Ltop + (size_t)j * nn;
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        Lj[e] = (c <= r) ? sL[r * ld + c] : 0.0;
      }
      if (j + 1 < M) {  // C_j = E_j L_j^{-T}: row r of C_j solves L_j c = E_j[r]^T
        if (L == 0) stage_row_range(sC, ld, a.A_sub + (size_t)j * nn, n, 0, n);
        else stage_row_range(sC, ld, E + (size_t)j * nn, n, 0, n);
        __syncthreads();
        trsv_fwd_cta(sL, ld, n, sC, n);
        __syncthreads();
        double *Cj = LC + (size_t)j * nn;
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) Cj[e] = sC[(e / n) * ld + e % n];
      }
    } else {
      stage_lower(sL, ld, a.Ltop + (size_t)j * nn, n);
    }
    if (d > 0) {
      const size_t bo = (size_t)orig * nd;
      if (L == 0 && a.B64) stage_cols(sB, ld, a.B64 + bo, n, d);
      else if (L == 0 && a.Bt) stage_cols(sB, ld, a.Bt + bo, n, d);
      else stage_cols(sB, ld, a.Y + bo, n, d);
      __syncthreads();
      if (j > 0) {  // b_j -= C_{j-1} y_{j-1}
        const double *Cp = LC + (size_t)(j - 1) * nn, *yp = Ys + (size_t)(j - 1) * nd;
        for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
          const int c = e / n, i = e - c * n;
          double acc = 0.0;
          for (int k = 0; k < n; ++k) acc = fma(ldcg(Cp + (size_t)i * n + k), ldcg(yp + (size_t)k * d + c), acc);
          sB[c * ld + i] -= acc;
        }
        __syncthreads();
      }
      trsv_fwd_cta(sL, ld, n, sB, d);
      __syncthreads();
      double *yj = Ys + (size_t)j * nd;
      for (int e = threadIdx.x; e < n * d; e += blockDim.x) yj[e] = sB[(e % d) * ld + e / d];
    }
    __syncthreads();
  }
  if (d > 0) {
    for (int j = M - 1; j >= 0; --j) {  // x_j = L_j^{-T} (y_j - C_j^T x_{j+1})
      const long long orig = (long long)j << L;
      stage_lower(sL, ld, a.Ltop + (size_t)j * nn, n);
      double *yj = Ys + (size_t)j * nd;
      for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
        const int c = e / n, i = e - c * n;
        double v = ldcg(yj + (size_t)i * d + c);
        if (j + 1 < M) {
          const double *Cj = LC + (size_t)j * nn, *xn = Ys + (size_t)(j + 1) * nd;
          for (int k = 0; k < n; ++k) v = fma(-ldcg(Cj + (size_t)k * n + i), ldcg(xn + (size_t)k * d + c), v);
        }
        sB[c * ld + i] = v;
      }
      __syncthreads();
      trsv_bwd_cta(sL, ld, n, sB, d);
      __syncthreads();
      for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
        const int i = e / d, c = e - i * d;
        const double x = sB[c * ld + i];
        yj[e] = x;
        a.Y[(size_t)orig * nd + e] = (T)x;
        if (a.X64) {
          double *xo = a.X64 + (size_t)orig * nd + e;
          *xo = a.x_accumulate ? *xo + x : x;
        }
      }
      __syncthreads();
    }
  }
  return true;
}

// ---------------------------------------------------------------------------
// Top block (the base case of Algorithms 4 and 7 with N_* = 1), always FP64;
// a top level of several blocks (N_* > 1) goes to the serial sweep.
// ---------------------------------------------------------------------------
template <typename T>
__device__ bool top_block(const Args<T> &a, bool factor, double *smem, int *s_flag) {
  if (a.p.Nl[a.p.L] > 1) return top_sweep(a, factor, smem, s_flag);
  const int n = a.p.n, ld = ldstride(n), d = a.d, L = a.p.L;
  double *sL = smem;
  double *sB = sL + (size_t)n * ld;
  if (factor) {
    if (L == 0) stage_sym_lower(sL, ld, a.A_diag, n);
    else stage_lower(sL, ld, a.Ld, n);
  } else {
    stage_lower(sL, ld, a.Ltop, n);
  }
  if (d > 0) {
    if (L == 0 && a.B64) stage_cols(sB, ld, a.B64, n, d);
    else if (L == 0 && a.Bt) stage_cols(sB, ld, a.Bt, n, d);
    else stage_cols(sB, ld, a.Y, n, d);
  }
  __syncthreads();
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
    {
      const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int v = warp; v < d; v += nw) {
        trsv_fwd_warp<double, 1>(sL, ld, n, sB + (size_t)v * ld, 1);
        __syncwarp();
        trsv_bwd_warp<double, 1>(sL, ld, n, sB + (size_t)v * ld, 1);
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
      const int i = e / d, c = e - i * d;
      const double x = sB[c * ld + i];
      a.Y[e] = (T)x;
      if (a.X64) a.X64[e] = a.x_accumulate ? a.X64[e] + x : x;
    }
  }
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Downward pass at level l, eliminated position j = 2m+1 (Algorithms 6, 2):
//   x_j = L_j^{-T} (y_j - W_L x_{j-1} - W_R x_{j+1}).
// ---------------------------------------------------------------------------
template <typename T>
__device__ void phaseC(const Args<T> &a, int l, long long j, T *smem) {
  const int n = a.p.n, ld = ldstride(n), d = a.d;
  const long long Nl = a.p.Nl[l];
  const bool hasR = (j + 1 < Nl);
  const long long orig = j << l;
  const size_t nn = (size_t)n * n, nd = (size_t)n * d;
  T *sL = smem;
  T *sT = sL + (size_t)n * ld;          // t vectors (d)
  T *sXm = sT + (size_t)d * ld;         // x_{j-1}
  T *sXp = sXm + (size_t)d * ld;        // x_{j+1}
  stage_lower(sL, ld, a.Ld + (size_t)orig * nn, n);
  stage_cols(sXm, ld, a.Y + (size_t)((j - 1) << l) * nd, n, d);
  if (hasR) stage_cols(sXp, ld, a.Y + (size_t)((j + 1) << l) * nd, n, d);
  __syncthreads();
  const T *W = a.Wb + (size_t)a.p.off[l] * nn;
  const T *WL = W + (size_t)(j - 1) * nn;   // W_L^T: WL[c][q] = W_L[q][c]
  const T *WR = W + (size_t)j * nn;
  const T *Yj = a.Y + (size_t)orig * nd;
  // t[q][c] = y[q][c] - sum_p W_L[q][p] x_{j-1}[p][c] - sum_p W_R[q][p] x_{j+1}[p][c];
  // the W reads are issued 8 at a time ahead of their FMAs (L2 latency)
  for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
    const int c = e / n, q = e - c * n;
    T acc = ldcg(Yj + (size_t)q * d + c);
    for (int side = 0; side < (hasR ? 2 : 1); ++side) {
      const T *Wq = (side == 0 ? WL : WR) + q;
      const T *x = (side == 0 ? sXm : sXp) + (size_t)c * ld;
      int p = 0;
      for (; p + 8 <= n; p += 8) {
        T w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) w[u] = ldcg(Wq + (size_t)(p + u) * n);
#pragma unroll
        for (int u = 0; u < 8; ++u) acc = fma(-w[u], x[p + u], acc);
      }
      for (; p < n; ++p) acc = fma(-ldcg(Wq + (size_t)p * n), x[p], acc);
    }
    sT[c * ld + q] = acc;
  }
  __syncthreads();
  if (!kStoreInverse<T>) {
    trsv_bwd_cta(sL, ld, n, sT, d);
    __syncthreads();
  }
  T *Yo = a.Y + (size_t)orig * nd;
  for (int e = threadIdx.x; e < n * d; e += blockDim.x) {
    const int i = e / d, c = e - i * d;
    T x;
    if (kStoreInverse<T>) {  // x = L^{-T} t with the stored inverse
      const T *t = sT + c * ld;
      T acc = T(0);
      for (int k = i; k < n; ++k) acc = fma(sL[k * ld + i], t[k], acc);
      x = acc;
    } else {
      x = sT[c * ld + i];
    }
    Yo[e] = x;
    if (a.X64) {
      double *xo = a.X64 + (size_t)orig * nd + e;
      *xo = a.x_accumulate ? *xo + (double)x : (double)x;
    }
  }
  __syncthreads();
}

}  // namespace bdss
