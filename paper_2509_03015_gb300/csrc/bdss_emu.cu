// FP64-accurate residual R = B - A X of the mixed-precision refinement on the
// tcgen05 tensor cores, for the tiled path (64 < n <= 256, d <= 16).
//
// Representation.  An operator row (block row i, row r) is the 3n entries
// [A_{i,i-1}[r][:], sym(A_ii)[r][:], A_{i+1,i}[:][r]] with one exponent E
// (max |a| < 2^E).  Each entry becomes the 59-bit integer q = round(a 2^(59-E))
// written as ten signed base-64 digits, q = sum_p d_p 64^(9-p) with
// d_p in [-32, 32]; every digit is exact in BF16.  A column c of X gets one
// exponent F over all blocks and the same cut.  Then
//   sum_k a_k x_k = 2^(E+F-118) sum_t 64^(18-t) ACC_t,
//   ACC_t = sum_{p+q=t} sum_k d_p(a_k) d_q(x_k),
// where at most ten pairs meet on a diagonal t and K <= 3 x 256, so
// |ACC_t| <= 10 x 768 x 32 x 32 < 2^23: every partial sum is an integer below
// 2^24 and the FP32 accumulation of the tensor cores is exact whatever its
// order.  The 19 diagonal sums are combined in 64-bit integers and FP64.  The
// only error is the truncation of a and x to 59 bits below the row / column
// maximum, so the residual is as accurate as an FP64 product in the normwise
// sense of the backward error ||B - A X|| / (||A|| ||X||).
//
// Products.  One tcgen05.mma (kind::f16, BF16 in, FP32 accumulate) per A
// slice p and K step of 16 covers all ten X slices at once: the B operand
// stacks X's slices q = 0..9 (16 rows each, N = 160), and the D columns start
// at 16 p, so the result for slice pair (p, q) lands on TMEM columns
// 16 (p + q) .. + 15, the accumulator of diagonal p + q (304 columns).
//
// Kernel roles (one persistent CTA per SM, 192 threads): warp 0 issues the
// TMA loads of the slices into a ring of shared-memory stages, warp 1 issues
// the MMAs, warps 2-5 read the accumulators (one TMEM lane quarter each),
// form R and the norms, and clear the accumulators for the next tile.  Every
// wait is bounded; a timed-out wait sets BDSS_ERR_TIMEOUT, the roles stop,
// loads and MMAs still in flight are waited out (bounded) and TMEM is freed.
#include "bdss_emu.h"
#include "bdss_tc.cuh"

namespace bdss {

namespace {

constexpr int kS = kEmuSlices;
constexpr int kFrac = 59;                 // fraction bits of the fixed-point digits
constexpr int kDiag = 2 * kS - 1;         // accumulators (diagonals p + q)
constexpr int kM = 128;                   // output rows of a tile (TMEM lanes)
constexpr int kN = kS * kEmuDp;           // 160: X slices stacked as the B operand
constexpr int kRowsPerCta = 8;            // operator rows per slicing CTA
constexpr int kAStages = 8;
constexpr int kXStages = 2;
constexpr int kATile = kM * kEmuKc * 2;   // 16384 bytes
constexpr int kXTile = kN * kEmuKc * 2;   // 20480 bytes
constexpr int kEmuThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr size_t kResidualSmem = (size_t)kAStages * kATile + (size_t)kXStages * kXTile + 1024;

// q = round(v 2^(59 - E)) from the bit fields of v (integer operations only;
// |v| < 2^E gives |q| < 2^59).  Zero and subnormal inputs give 0.
__device__ __forceinline__ long long emu_fixed(double v, int E) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = ex - 1075 + kFrac - E;
  long long q;
  if (sh >= 0) q = m << (sh > 6 ? 6 : sh);
  else if (sh > -63) q = (m + (1LL << (-sh - 1))) >> (-sh);
  else q = 0;
  return b < 0 ? -q : q;
}

// Signed base-64 digits of q (|q| < 2^59): q = sum_p d[p] 64^(9-p) with
// d[p] in [-32, 31] for p >= 1 and |d[0]| <= 32.  With u = q + 32 sum_p 64^p
// every digit of u in plain base 64 is d[p] + 32 (the bias absorbs the
// borrows), so the digits come without a carry chain: the biased digit p is
// (u >> 6 (9 - p)) & 63, and the top one u >> 54 (at most 64).
constexpr long long kEmuBias = 32LL * 18300341342965825LL;  // 32 (64^10 - 1) / 63
__device__ __forceinline__ int emu_biased_digit(unsigned long long u, int p) {
  return p == 0 ? (int)(u >> 54) : (int)((u >> (6 * (kS - 1 - p))) & 63);
}

// BF16 bits of the integer b - 32 for a biased digit 0 <= b <= 64: 2^23 + b
// is exact in FP32, subtracting 2^23 + 32 leaves b - 32 exactly, and
// |b - 32| <= 32 needs at most 6 significant bits, so the upper half of its
// FP32 pattern is its BF16 pattern.
__device__ __forceinline__ unsigned emu_bf16_biased(int b) {
  const float f = __int_as_float(0x4B000000 + b) - 8388640.0f;
  return __float_as_uint(f) >> 16;
}

// Ten digit planes of four consecutive entries: writes 8 bytes (four BF16)
// per plane at dst + p * plane_stride (elements).
__device__ __forceinline__ void emu_store_quad(const double (&v)[4], int E, unsigned short *dst,
                                               size_t plane_stride) {
  unsigned long long u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) u[j] = (unsigned long long)(emu_fixed(v[j], E) + kEmuBias);
#pragma unroll
  for (int p = 0; p < kS; ++p) {
    const unsigned lo = emu_bf16_biased(emu_biased_digit(u[0], p)) | (emu_bf16_biased(emu_biased_digit(u[1], p)) << 16);
    const unsigned hi = emu_bf16_biased(emu_biased_digit(u[2], p)) | (emu_bf16_biased(emu_biased_digit(u[3], p)) << 16);
    *reinterpret_cast<uint2 *>(dst + (size_t)p * plane_stride) = make_uint2(lo, hi);
  }
}

// Exponent E with max |x| < 2^E from the bits of max |x| (a zero maximum:
// every digit is zero, any E works).
__device__ __forceinline__ int emu_exp(unsigned long long maxbits) {
  const int ex = (int)((maxbits >> 52) & 0x7FF);
  return ex == 0 ? -1022 : ex - 1022;
}

// ---------------------------------------------------------------------------
// Operator slices: CTA (block row i, rows r0 .. r0 + kRowsPerCta - 1).
// Aslc[((i S + p) n + r) 3np + g np + k] = digit p of entry k of block g of
// operator row (i, r); g = 0: A_{i,i-1}, 1: sym(A_ii), 2: A_{i,i+1} =
// A_{i+1,i}^T; zero for absent blocks and k >= n.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_emu_slice_operator(long long N, int n, int np, const double *A_diag,
                                                            const double *A_sub, unsigned short *Aslc, int *Aexp,
                                                            DevStatus *st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *T = reinterpret_cast<double *>(smem_raw);  // [3][kRowsPerCta][n]
  __shared__ int sE[kRowsPerCta];
  __shared__ float sNorm[8];
  const int groups = (n + kRowsPerCta - 1) / kRowsPerCta;
  const long long i = blockIdx.x / groups;
  const int r0 = (int)(blockIdx.x % groups) * kRowsPerCta;
  const int R = min(kRowsPerCta, n - r0);
  const size_t nn = (size_t)n * n;
  const bool hasL = i > 0, hasR = i + 1 < N;
  double *T0 = T, *T1 = T + (size_t)kRowsPerCta * n, *T2 = T + (size_t)2 * kRowsPerCta * n;
  // rows of A_{i,i-1} and A_ii (unrolled so that several loads are in flight)
#pragma unroll 4
  for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
    const int rr = e / n, k = e - rr * n;
    T0[e] = hasL ? __ldg(A_sub + (size_t)(i - 1) * nn + (size_t)(r0 + rr) * n + k) : 0.0;
    T1[e] = __ldg(A_diag + (size_t)i * nn + (size_t)(r0 + rr) * n + k);
  }
  __syncthreads();
  // columns r0 .. r0 + R - 1 of A_ii (symmetrise) and of A_{i+1,i}
#pragma unroll 4
  for (int e = threadIdx.x; e < R * n; e += blockDim.x) {
    const int k = e / R, rr = e - k * R;
    const double at = __ldg(A_diag + (size_t)i * nn + (size_t)k * n + r0 + rr);
    T1[rr * n + k] = 0.5 * (T1[rr * n + k] + at);
    T2[rr * n + k] = hasR ? __ldg(A_sub + (size_t)i * nn + (size_t)k * n + r0 + rr) : 0.0;
  }
  __syncthreads();
  // row exponents and ||A||_inf row sums (FP32 from the bit fields)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float best = 0.0f;
  for (int rr = warp; rr < R; rr += 8) {
    unsigned long long mx = 0;
    float sum = 0.0f;
    for (int g = 0; g < 3; ++g)
      for (int k = lane; k < n; k += 32) {
        const double v = T[(size_t)g * kRowsPerCta * n + (size_t)rr * n + k];
        const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7FFFFFFFFFFFFFFFULL;
        mx = b > mx ? b : mx;
        sum += abs_f32_bits(v);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
      mx = m2 > mx ? m2 : mx;
      sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (lane == 0) {
      sE[rr] = emu_exp(mx);
      Aexp[(size_t)i * n + r0 + rr] = emu_exp(mx);
    }
    best = fmaxf(best, sum);
  }
  if (lane == 0) sNorm[warp] = best;
  __syncthreads();
  if (threadIdx.x == 0 && st) {
    float m = 0.0f;
    for (int w = 0; w < 8; ++w) m = fmaxf(m, sNorm[w]);
    atomicMax(&st->nrm[2], (unsigned long long)__double_as_longlong((double)m));
  }
  // digits: consecutive threads take consecutive quads of k of one (row,
  // block); np is a multiple of 64, so a quad never straddles two blocks
  const int K3 = 3 * np, Q3 = K3 / 4;
  for (int e = threadIdx.x; e < R * Q3; e += blockDim.x) {
    const int rr = e / Q3, kk = 4 * (e - rr * Q3), g = kk / np, k = kk - g * np;
    const double *src = T + (size_t)g * kRowsPerCta * n + (size_t)rr * n;
    double v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = (k + j < n) ? src[k + j] : 0.0;
    emu_store_quad(v, sE[rr], Aslc + ((size_t)i * kS * n + r0 + rr) * K3 + kk, (size_t)n * K3);
  }
}

// max |X[:, c]| as FP64 bit patterns (xmax zeroed by the caller).
__global__ void __launch_bounds__(256) k_emu_xmax(long long rows, int d, const double *X, unsigned long long *xmax) {
  __shared__ unsigned long long sm[256];
  const int c = threadIdx.x % kEmuDp, rg = threadIdx.x / kEmuDp;
  unsigned long long mx = 0;
  if (c < d)
    for (long long r = (long long)blockIdx.x * 16 + rg; r < rows; r += (long long)gridDim.x * 16) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(__ldg(X + r * d + c)) & 0x7FFFFFFFFFFFFFFFULL;
      mx = b > mx ? b : mx;
    }
  sm[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x < kEmuDp && threadIdx.x < d) {
    unsigned long long m = 0;
    for (int g = 0; g < 16; ++g) m = sm[g * kEmuDp + threadIdx.x] > m ? sm[g * kEmuDp + threadIdx.x] : m;
    atomicMax(xmax + threadIdx.x, m);
  }
}

// X slices, one CTA per block j: Xslc[((j S + q) 16 + c) np + k] = digit q of
// X_j[k][c] with column exponent F_c; zero for c >= d or k >= n.
__global__ void __launch_bounds__(256) k_emu_slice_x(long long N, int n, int np, int d, const double *X,
                                                     const unsigned long long *xmax, int *xexp,
                                                     unsigned short *Xslc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *sX = reinterpret_cast<double *>(smem_raw);  // n x d
  __shared__ int sF[kEmuDp];
  const long long j = blockIdx.x;
  if (threadIdx.x < kEmuDp) {
    sF[threadIdx.x] = threadIdx.x < d ? emu_exp(xmax[threadIdx.x]) : 0;
    if (j == 0) xexp[threadIdx.x] = sF[threadIdx.x];
  }
  for (int e = threadIdx.x; e < n * d; e += blockDim.x) sX[e] = __ldg(X + (size_t)j * n * d + e);
  __syncthreads();
  const int nq = np / 4;
  for (int e = threadIdx.x; e < kEmuDp * nq; e += blockDim.x) {
    const int c = e / nq, k = 4 * (e - c * nq);
    double v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) v[t] = (c < d && k + t < n) ? sX[(k + t) * d + c] : 0.0;
    emu_store_quad(v, sF[c], Xslc + ((size_t)j * kS * kEmuDp + c) * np + k, (size_t)kEmuDp * np);
  }
}

// ---------------------------------------------------------------------------
// The tensor-core residual.
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool emu_try(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait (the limit counts from the first failed poll) that also gives
// up when another role has aborted (abort != null; the drains at the end
// pass null and wait for their loads and MMAs whatever happened).
__device__ __forceinline__ bool emu_wait(uint64_t *bar, uint32_t parity, long long timeout_ns, volatile int *abort) {
  long long ts = 0;
  for (uint32_t it = 0;; ++it) {
    if (emu_try(bar, parity)) return true;
    if ((it & 63) == 63) {
      if (abort && *abort) return false;
      const long long now = global_ns();
      if (ts == 0) ts = now;
      else if (now - ts > timeout_ns) return false;
    }
  }
}

__device__ __forceinline__ void emu_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void emu_mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, 1, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc)
      : "memory");
}

// D = FP32, A = B = BF16, both K-major, M x N.
__host__ __device__ constexpr uint32_t emu_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  const uint32_t z = 0;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

struct EmuKArgs {
  long long N;
  int n, np, d;
  const int *Aexp, *xexp;
  const double *X, *B;
  float *R32;
  double *R64;
  DevStatus *st;
  long long timeout_ns;
};

__global__ void __launch_bounds__(kEmuThreads, 1)
    k_emu_residual(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapX,
                   const __grid_constant__ EmuKArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t a_full[kAStages], a_empty[kAStages], x_full[kXStages], x_empty[kXStages];
  __shared__ uint64_t acc_full, acc_empty, drain;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int sF[kEmuDp];
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~(uintptr_t)1023);
  unsigned char *Ast = base;                                  // kAStages x 16 KB
  unsigned char *Xst = base + (size_t)kAStages * kATile;      // kXStages x 20 KB
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, np = a.np, d = a.d;
  const long long N = a.N;
  const int MT = (n + kM - 1) / kM, kchunks = np / kEmuKc;
  const long long tiles = N * MT;
  volatile int *abort = &s_abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kAStages; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < kXStages; ++s) {
      mbar_init(&x_full[s], 1);
      mbar_init(&x_empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 128);
    mbar_init(&drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < kEmuDp) sF[threadIdx.x] = a.xexp[threadIdx.x];
  if (warp == 1) tmem_alloc(&s_tmem, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  auto fail = [&]() {
    *abort = 1;
    set_status(a.st, kStTimeout, -1, -1);
  };

  if (warp == 0) {
    // ---- TMA producer -------------------------------------------------------
    if (lane == 0) {
      int as = 0, xs = 0;
      uint32_t aph = 0, xph = 0;
      for (long long t = blockIdx.x; t < tiles && !*abort; t += gridDim.x) {
        const long long i = t / MT;
        const int m = (int)(t % MT);
        for (int g = 0; g < 3 && !*abort; ++g) {
          if ((g == 0 && i == 0) || (g == 2 && i == N - 1)) continue;
          for (int kk = 0; kk < kchunks; ++kk) {
            if (!emu_wait(&x_empty[xs], xph ^ 1, a.timeout_ns, abort)) { fail(); break; }
            mbar_expect_tx(&x_full[xs], kXTile);
            tma_load_2d(Xst + (size_t)xs * kXTile, &mapX, kk * kEmuKc, (int)((i - 1 + g) * kS * kEmuDp),
                        &x_full[xs]);
            if (++xs == kXStages) { xs = 0; xph ^= 1; }
            for (int p = 0; p < kS; ++p) {
              if (!emu_wait(&a_empty[as], aph ^ 1, a.timeout_ns, abort)) { fail(); break; }
              mbar_expect_tx(&a_full[as], kATile);
              tma_load_2d(Ast + (size_t)as * kATile, &mapA, g * np + kk * kEmuKc,
                          (int)((i * kS + p) * n + m * kM), &a_full[as]);
              if (++as == kAStages) { as = 0; aph ^= 1; }
            }
            if (*abort) break;
          }
        }
      }
      // wait out the loads still in flight (each stage's last armed phase)
      for (int s = 0; s < kAStages; ++s) {
        const uint32_t ph = (s < as) ? aph : (aph ^ 1);
        emu_wait(&a_full[s], ph, a.timeout_ns, nullptr);
      }
      for (int s = 0; s < kXStages; ++s) {
        const uint32_t ph = (s < xs) ? xph : (xph ^ 1);
        emu_wait(&x_full[s], ph, a.timeout_ns, nullptr);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = emu_idesc(kM, kN);
      int as = 0, xs = 0;
      uint32_t aph = 0, xph = 0, eph = 0;
      for (long long t = blockIdx.x; t < tiles && !*abort; t += gridDim.x) {
        const long long i = t / MT;
        if (!emu_wait(&acc_empty, eph, a.timeout_ns, abort)) { fail(); break; }
        eph ^= 1;
        tc_fence_after();
        for (int g = 0; g < 3 && !*abort; ++g) {
          if ((g == 0 && i == 0) || (g == 2 && i == N - 1)) continue;
          for (int kk = 0; kk < kchunks; ++kk) {
            if (!emu_wait(&x_full[xs], xph, a.timeout_ns, abort)) { fail(); break; }
            const unsigned char *xb = Xst + (size_t)xs * kXTile;
            for (int p = 0; p < kS; ++p) {
              if (!emu_wait(&a_full[as], aph, a.timeout_ns, abort)) { fail(); break; }
              tc_fence_after();
              const unsigned char *ab = Ast + (size_t)as * kATile;
#pragma unroll
              for (int ks = 0; ks < kEmuKc / 16; ++ks)
                emu_mma_bf16(tmem + (uint32_t)(p * kEmuDp), tc_desc_sw128(ab, ks * 32), tc_desc_sw128(xb, ks * 32),
                             idesc);
              tc_commit(&a_empty[as]);
              if (++as == kAStages) { as = 0; aph ^= 1; }
            }
            tc_commit(&x_empty[xs]);
            if (++xs == kXStages) { xs = 0; xph ^= 1; }
            if (*abort) break;
          }
        }
        tc_commit(&acc_full);
      }
      // every MMA issued has completed before TMEM is released
      tc_commit(&drain);
      emu_wait(&drain, 0, a.timeout_ns, nullptr);
    }
  } else {
    // ---- epilogue: warps 2..5, TMEM lane quarter warp % 4 ---------------------
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    const int row = 32 * quarter + lane;
    auto clear = [&]() {
      for (int t = 0; t < kDiag; ++t) tmem_zero16(lane_base + (uint32_t)(t * kEmuDp));
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      emu_arrive(&acc_empty);
    };
    clear();
    uint32_t fph = 0;
    double maxR = 0.0, maxX = 0.0;
    for (long long t = blockIdx.x; t < tiles; t += gridDim.x) {
      const long long i = t / MT;
      const int m = (int)(t % MT);
      // warp-uniform wait: lane 0 polls, the others then observe the phase
      int ok = 0;
      if (lane == 0) ok = emu_wait(&acc_full, fph, a.timeout_ns, abort) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      if (lane != 0) emu_try(&acc_full, fph);
      fph ^= 1;
      tc_fence_after();
      // v[c] = sum_t 64^(18 - t) ACC_t[c], in three integer groups
      double v[kEmuDp];
      {
        long long G[kEmuDp];
#pragma unroll
        for (int c = 0; c < kEmuDp; ++c) G[c] = 0;
        for (int t = 0; t < kDiag; ++t) {
          uint32_t r[16];
          tmem_ld16(lane_base + (uint32_t)(t * kEmuDp), r);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int c = 0; c < kEmuDp; ++c) G[c] = G[c] * 64 + (long long)__float2int_rn(__uint_as_float(r[c]));
          if (t == 6 || t == 13 || t == kDiag - 1) {
            const double w = t == 6 ? 4722366482869645213696.0 /* 2^72 */ : t == 13 ? 1073741824.0 /* 2^30 */ : 1.0;
#pragma unroll
            for (int c = 0; c < kEmuDp; ++c) {
              v[c] = (t == 6) ? (double)G[c] * w : fma((double)G[c], w, v[c]);
              G[c] = 0;
            }
          }
        }
      }
      const int r = m * kM + row;
      if (r < n) {
        const int Ea = a.Aexp[(size_t)i * n + r];
        const size_t o = ((size_t)i * n + r) * d;
        double rs = 0.0, xs = 0.0;
#pragma unroll
        for (int c = 0; c < kEmuDp; ++c) {
          if (c < d) {
            // an Inf or NaN in the operator row or in column c of X (its
            // maximum's exponent field is all ones: E = 1025) poisons the entry,
            // as an FP64 product would
            const double ax = (Ea > 1024 || sF[c] > 1024) ? __longlong_as_double(0x7FF8000000000000LL)
                                                          : scalbn(v[c], Ea + sF[c] - 2 * kFrac);
            const double res = __ldg(a.B + o + c) - ax;
            if (a.R32) a.R32[o + c] = (float)res;
            if (a.R64) a.R64[o + c] = res;
            rs += fabs(res);
            xs += fabs(__ldg(a.X + o + c));
          }
        }
        // a NaN anywhere (e.g. an FP32 solve that overflowed) must reach the
        // host's backward-error test: keep it instead of fmax dropping it
        maxR = (rs > maxR || rs != rs) ? rs : maxR;
        maxX = (xs > maxX || xs != xs) ? xs : maxX;
      }
      tc_fence_before();
      clear();
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double r2 = __shfl_xor_sync(0xffffffffu, maxR, o), x2 = __shfl_xor_sync(0xffffffffu, maxX, o);
      maxR = (r2 > maxR || r2 != r2) ? r2 : maxR;
      maxX = (x2 > maxX || x2 != x2) ? x2 : maxX;
    }
    if (lane == 0) {
      atomicMax(&a.st->nrm[0], (unsigned long long)__double_as_longlong(maxR));
      atomicMax(&a.st->nrm[1], (unsigned long long)__double_as_longlong(maxX));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

cudaError_t encode_fn(EncodeTiledFn *out) {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !p) return cudaErrorNotSupported;
    fn = (EncodeTiledFn)p;
  }
  *out = fn;
  return cudaSuccess;
}

cudaError_t encode_bf16_2d(CUtensorMap *out, void *base, unsigned long long cols, unsigned long long rows,
                           unsigned box_cols, unsigned box_rows) {
  EncodeTiledFn fn = nullptr;
  const cudaError_t e = encode_fn(&fn);
  if (e != cudaSuccess) return e;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {box_cols, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// ===========================================================================
// FP64-accurate Schur products of the tiled FP64 factorisation on the tensor
// cores (the separator update of Algorithm 3, 64 < n <= 256).
//
// At level l the stored coupling blocks M_b (b = 0 .. N_l - 2; row m of M_b is
// column m of the coupling solve W, so D -= M M^T) are cut row by row in the
// same fixed-point digits as the operator rows of the residual: exponent
// E_b[m] with max_k |M_b[m][k]| < 2^E and ten planes
// Wslc[((b S + p) n + m) np + k], zero for k >= n.  Separator s = 2k needs
//   D_s     = D - M_{s-1} M_{s-1}^T - M_s M_s^T   (lower triangle),
//   E_{l+1} = - M_{s+1} M_s^T                     (slot k of level l + 1),
// computed over 128 x 16 output tiles.  Each product M_a M_b^T of a tile is
// one accumulation round: per K chunk of 64 the B operand is the ten slices
// of rows c0 .. c0 + 15 of M_b (one 3-D TMA box, N = 160 rows) and the A
// operand slice p of rows m0 .. m0 + 127 of M_a, written at TMEM column 16 p,
// so slice pair (p, q) lands on the accumulator of diagonal p + q as in the
// residual.  With K <= 256, |ACC_t| <= 10 x 256 x 32 x 32 < 2^22: every sum is
// exact.  The epilogue scales a round by 2^(E_a[r] + E_b[c] - 118) and adds
// the rounds of a tile in FP64; the only error is the 59-bit cut of the
// inputs, below an FP64 product's rounding in the normwise sense.
// ===========================================================================
constexpr int kSchurN = 16;      // output columns of a tile
constexpr int kSchurRounds = 2;  // products of one tile at most
constexpr int kSchurAStages = 10;  // A slabs in flight (one round of ten slices)

// Digit formats of the Schur engine.  Ten signed base-64 digits (59 bits)
// for K up to 256 (the n > 64 path); eight signed base-256 digits (60 bits)
// for K = 64 (n <= 64): |ACC_t| <= 8 x 64 x 128 x 128 = 2^23 stays exact in
// FP32, and 15 diagonals x 16 columns leave room for two accumulators in the
// 512 TMEM columns, so that a round's epilogue runs under the next round's
// products.  Diagonal groups of the int64 combination: t <= kG0 (shift kSh0),
// t <= kG1 (shift kSh1), the rest (shift 0).
template <int kSl> struct EmuDigits;
template <> struct EmuDigits<10> {
  static constexpr int kBits = 6, kFrac = 59, kDg = 19, kG0 = 6, kG1 = 13, kSh0 = 72, kSh1 = 30, kBuf = 1;
  static constexpr unsigned long long kBias = 32ULL * 18300341342965825ULL;  // 32 (64^10 - 1) / 63
};
template <> struct EmuDigits<8> {
  static constexpr int kBits = 8, kFrac = 60, kDg = 15, kG0 = 4, kG1 = 9, kSh0 = 80, kSh1 = 40, kBuf = 2;
  static constexpr unsigned long long kBias = 0x8080808080808080ULL;  // 128 (256^8 - 1) / 255
};

// q = round(v 2^(F - E)) as in emu_fixed, for the format's F.
template <int kSl>
__device__ __forceinline__ long long emu_fixed_t(double v, int E) {
  const long long b = __double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);
  if (ex == 0 || ex == 0x7FF) return 0;
  const long long m = (b & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;
  const int sh = ex - 1075 + EmuDigits<kSl>::kFrac - E;
  long long q;
  constexpr int cap = EmuDigits<kSl>::kFrac - 53;  // |v| < 2^E keeps sh <= cap
  if (sh >= 0) q = m << (sh > cap ? cap : sh);
  else if (sh > -63) q = (m + (1LL << (-sh - 1))) >> (-sh);
  else q = 0;
  return b < 0 ? -q : q;
}

// kSl digit planes of four consecutive entries (the biased digits of
// u = q + bias, each d + B/2 with B the base, as in emu_store_quad).
template <int kSl>
__device__ __forceinline__ void emu_store_quad_t(const double (&v)[4], int E, unsigned short *dst,
                                                 size_t plane_stride) {
  constexpr int B = EmuDigits<kSl>::kBits;
  constexpr unsigned long long mask = (1ULL << B) - 1;
  constexpr float off = 8388608.0f + (float)(1 << (B - 1));
  unsigned long long u[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) u[j] = (unsigned long long)emu_fixed_t<kSl>(v[j], E) + EmuDigits<kSl>::kBias;
#pragma unroll
  for (int p = 0; p < kSl; ++p) {
    unsigned h[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int dg = p == 0 ? (int)(u[j] >> (B * (kSl - 1))) : (int)((u[j] >> (B * (kSl - 1 - p))) & mask);
      h[j] = __float_as_uint(__int_as_float(0x4B000000 + dg) - off) >> 16;
    }
    *reinterpret_cast<uint2 *>(dst + (size_t)p * plane_stride) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
  }
}

// One warp per row b n + m of the level's stored blocks.
template <int kSl>
__global__ void __launch_bounds__(256) k_emu_slice_w(long long rows, int n, int np, const double *W,
                                                     unsigned short *Wslc, int *Wexp) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long row = (long long)blockIdx.x * 8 + warp;
  if (row >= rows) return;
  const long long b = row / n;
  const int m = (int)(row - b * n);
  const double *src = W + (size_t)row * n;
  double v[2][4];
  unsigned long long mx = 0;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int k = 4 * (lane + 32 * i) + t;
      v[i][t] = k < n ? __ldg(src + k) : 0.0;
      // |v| as bits: ordered like the values, a NaN above every finite value
      const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(v[i][t]));
      mx = bits > mx ? bits : mx;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = y > mx ? y : mx;
  }
  const int E = emu_exp(mx);
  if (lane == 0) Wexp[row] = E;
  unsigned short *dst = Wslc + ((size_t)b * kSl * n + m) * np;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int k = 4 * (lane + 32 * i);
    if (k < np) emu_store_quad_t<kSl>(v[i], E, dst + k, (size_t)n * np);
  }
}

// An accumulator entry: an exact integer |x| < 2^22 held in FP32.  Adding
// 1.5 * 2^23 puts it in the binade of unit spacing, so its bits minus those
// of 1.5 * 2^23 are x (integer pipe only).
__device__ __forceinline__ int emu_acc_int(uint32_t bits) {
  return __float_as_int(__uint_as_float(bits) + 12582912.0f) - 0x4B400000;
}

// V 2^E rounded once to FP64 (round to nearest even), built from the bits of
// the 128-bit integer: the leading one sets the exponent, the next 52 bits the
// fraction.  Results outside the normal range take the FP64 path.
__device__ __forceinline__ double emu_i128_to_double(__int128 V, int E) {
  if (V == 0) return 0.0;
  const bool neg = V < 0;
  unsigned __int128 m = neg ? (unsigned __int128)(-V) : (unsigned __int128)V;
  const unsigned long long hi0 = (unsigned long long)(m >> 64), lo0 = (unsigned long long)m;
  const int lz = hi0 ? __clzll((long long)hi0) : 64 + __clzll((long long)lo0);
  m <<= lz;  // leading one at bit 127
  unsigned long long top = (unsigned long long)(m >> 75);  // 53 bits
  const unsigned __int128 rem = m & ((((unsigned __int128)1) << 75) - 1);
  const unsigned __int128 half = ((unsigned __int128)1) << 74;
  if (rem > half || (rem == half && (top & 1ULL))) ++top;
  int e2 = 127 - lz + E;
  if (top >> 53) {
    top >>= 1;
    ++e2;
  }
  const int be = e2 + 1023;
  if (be <= 0 || be >= 2047)
    return scalbn(ldexp((double)(long long)(V >> 64), 64) + (double)(unsigned long long)V, E);
  const unsigned long long bits =
      ((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (top & ((1ULL << 52) - 1));
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

struct EmuSchurArgs {
  long long Nl;          // positions of level l
  int n, np, l;
  const int *Wexp;       // (N_l - 1) x n row exponents of the level's stored blocks
  const double *A_diag;  // level 0: the separators' D (symmetrised)
  double *Ld;            // D blocks (slot s << l)
  double *En;            // E blocks of level l + 1 (slot k)
  DevStatus *st;
  long long timeout_ns;
};

// Column tiles of row tile mt inside D's lower part (c0 < (mt + 1) 128).
__host__ __device__ inline int schur_d_cols(int n, int mt) {
  const int CT = (n + kSchurN - 1) / kSchurN, lim = (mt + 1) * kM / kSchurN;
  return CT < lim ? CT : lim;
}
__host__ __device__ inline int schur_tiles_per_sep(int n) {
  const int MT = (n + kM - 1) / kM, CT = (n + kSchurN - 1) / kSchurN;
  int t = MT * CT;
  for (int mt = 0; mt < MT; ++mt) t += schur_d_cols(n, mt);
  return t;
}

// Output tile u of the level: separator k, a D tile (lower set) or an E tile,
// and its rounds (stored blocks of the A and B operands).
struct SchurTile {
  long long k, ra0, ra1, rb0, rb1;  // stored blocks of the A and B operands of rounds 0, 1
  int isD, mt, ct, nr;
  // scalar fields and selects, so that the tile stays in registers
  __device__ long long a_of(int r) const { return r == 0 ? ra0 : ra1; }
  __device__ long long b_of(int r) const { return r == 0 ? rb0 : rb1; }
};
__device__ __forceinline__ SchurTile schur_tile(long long u, long long Nl, int n) {
  SchurTile T;
  const int per = schur_tiles_per_sep(n);
  const int MT = (n + kM - 1) / kM, CT = (n + kSchurN - 1) / kSchurN;
  T.k = u / per;
  int r = (int)(u - T.k * per);
  const long long s = 2 * T.k;
  T.isD = 0;
  T.mt = 0;
  T.ct = 0;
  T.nr = 0;
  T.ra0 = T.ra1 = T.rb0 = T.rb1 = 0;
  for (int mt = 0; mt < MT; ++mt) {
    const int c = schur_d_cols(n, mt);
    if (r < c) {
      T.isD = 1;
      T.mt = mt;
      T.ct = r;
      break;
    }
    r -= c;
  }
  if (T.isD) {
    const bool hasM = s >= 2, hasP = s + 1 < Nl;
    // round 0: the left neighbour's block if present, else the right one's
    T.ra0 = T.rb0 = hasM ? s - 1 : s;
    T.ra1 = T.rb1 = s;
    T.nr = (int)hasM + (int)hasP;
  } else {
    T.mt = r / CT;
    T.ct = r - T.mt * CT;
    if (s + 2 < Nl) {
      T.ra0 = s + 1;
      T.rb0 = s;
      T.nr = 1;
    }
  }
  return T;
}

// Roles as in the residual kernel: warp 0 TMA, warp 1 MMA, warps 2-5 the
// epilogue of one TMEM lane quarter each.  Every wait is bounded.
template <int kSl>
__global__ void __launch_bounds__(kEmuThreads, 1)
    k_emu_schur(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const __grid_constant__ EmuSchurArgs a) {
  using Fm = EmuDigits<kSl>;
  constexpr int kNs = kSl * kSchurN;           // B rows: the kSl slices of 16 columns stacked (MMA N)
  constexpr int kBTile = kNs * kEmuKc * 2;     // bytes of one B stage
  constexpr int kAccCols = Fm::kDg * kSchurN;  // TMEM columns of one accumulator
  constexpr int kNB = Fm::kBuf;                // accumulators (rounds in flight)
  constexpr int kAS = kSchurAStages;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t a_full[kAS], a_empty[kAS], b_full[kXStages], b_empty[kXStages];
  __shared__ uint64_t acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  unsigned char *base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  unsigned char *Ast = base;                         // kAS x 16 KB
  unsigned char *Bst = base + (size_t)kAS * kATile;  // kXStages x kBTile
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, kchunks = a.np / kEmuKc;
  const long long tiles = ((a.Nl + 1) / 2) * schur_tiles_per_sep(n);
  volatile int *abort = &s_abort;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kAS; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < kXStages; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    mbar_init(&drain, 1);
    s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&s_tmem, kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  auto fail = [&]() {
    *abort = 1;
    set_status(a.st, kStTimeout, -1, -1);
  };

  if (warp == 0) {
    // ---- TMA producer -------------------------------------------------------
    if (lane == 0) {
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      for (long long u = blockIdx.x; u < tiles && !*abort; u += gridDim.x) {
        const SchurTile T = schur_tile(u, a.Nl, n);
        for (int r = 0; r < T.nr && !*abort; ++r)
          for (int kk = 0; kk < kchunks; ++kk) {
            if (!emu_wait(&b_empty[bs], bph ^ 1, a.timeout_ns, abort)) { fail(); break; }
            mbar_expect_tx(&b_full[bs], kBTile);
            tma_load_3d(Bst + (size_t)bs * kBTile, &mapB, kk * kEmuKc, T.ct * kSchurN, (int)(T.b_of(r) * kSl),
                        &b_full[bs]);
            if (++bs == kXStages) { bs = 0; bph ^= 1; }
            for (int p = 0; p < kSl; ++p) {
              if (!emu_wait(&a_empty[as], aph ^ 1, a.timeout_ns, abort)) { fail(); break; }
              mbar_expect_tx(&a_full[as], kATile);
              tma_load_2d(Ast + (size_t)as * kATile, &mapA, kk * kEmuKc, (int)((T.a_of(r) * kSl + p) * n + T.mt * kM),
                          &a_full[as]);
              if (++as == kAS) { as = 0; aph ^= 1; }
            }
            if (*abort) break;
          }
      }
      for (int s = 0; s < kAS; ++s) {
        const uint32_t ph = (s < as) ? aph : (aph ^ 1);
        emu_wait(&a_full[s], ph, a.timeout_ns, nullptr);
      }
      for (int s = 0; s < kXStages; ++s) {
        const uint32_t ph = (s < bs) ? bph : (bph ^ 1);
        emu_wait(&b_full[s], ph, a.timeout_ns, nullptr);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ------------------------------------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = emu_idesc(kM, kNs);
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      long long i = 0;  // rounds so far: accumulator i % kNB
      for (long long u = blockIdx.x; u < tiles && !*abort; u += gridDim.x) {
        const SchurTile T = schur_tile(u, a.Nl, n);
        for (int r = 0; r < T.nr && !*abort; ++r) {
          const int ab = (int)(i % kNB);
          if (!emu_wait(&acc_empty[ab], (uint32_t)((i / kNB) & 1), a.timeout_ns, abort)) { fail(); break; }
          tc_fence_after();
          const uint32_t dacc = tmem + (uint32_t)(ab * kAccCols);
          for (int kk = 0; kk < kchunks; ++kk) {
            if (!emu_wait(&b_full[bs], bph, a.timeout_ns, abort)) { fail(); break; }
            const unsigned char *bb = Bst + (size_t)bs * kBTile;
            for (int p = 0; p < kSl; ++p) {
              if (!emu_wait(&a_full[as], aph, a.timeout_ns, abort)) { fail(); break; }
              tc_fence_after();
              const unsigned char *abuf = Ast + (size_t)as * kATile;
#pragma unroll
              for (int ks = 0; ks < kEmuKc / 16; ++ks)
                emu_mma_bf16(dacc + (uint32_t)(p * kSchurN), tc_desc_sw128(abuf, ks * 32), tc_desc_sw128(bb, ks * 32),
                             idesc);
              tc_commit(&a_empty[as]);
              if (++as == kAS) { as = 0; aph ^= 1; }
            }
            tc_commit(&b_empty[bs]);
            if (++bs == kXStages) { bs = 0; bph ^= 1; }
            if (*abort) break;
          }
          tc_commit(&acc_full[ab]);
          ++i;
        }
      }
      tc_commit(&drain);
      emu_wait(&drain, 0, a.timeout_ns, nullptr);
    }
  } else {
    // ---- epilogue: warps 2..5, TMEM lane quarter warp % 4 ---------------------
    const int quarter = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    auto clear = [&](int b) {
      for (int t = 0; t < Fm::kDg; ++t) tmem_zero16(lane_base + (uint32_t)(b * kAccCols + t * kSchurN));
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      emu_arrive(&acc_empty[b]);
    };
    for (int b = 0; b < kNB; ++b) clear(b);
    long long i = 0;  // rounds so far: accumulator i % kNB
    const size_t nn = (size_t)n * n;
    bool stop = false;
    for (long long u = blockIdx.x; u < tiles && !stop; u += gridDim.x) {
      const SchurTile T = schur_tile(u, a.Nl, n);
      if (T.nr == 0) continue;
      const int row = T.mt * kM + 32 * quarter + lane;
      double acc[kSchurN];
#pragma unroll
      for (int c = 0; c < kSchurN; ++c) acc[c] = 0.0;
      for (int r = 0; r < T.nr; ++r) {
        const int ab = (int)(i % kNB);
        const uint32_t fpar = (uint32_t)((i / kNB) & 1);
        int ok = 0;
        if (lane == 0) ok = emu_wait(&acc_full[ab], fpar, a.timeout_ns, abort) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
          if (lane == 0) fail();
          stop = true;
          break;
        }
        if (lane != 0) emu_try(&acc_full[ab], fpar);
        ++i;
        tc_fence_after();
        // the diagonals, combined exactly on the integer pipe: V = sum_t
        // ACC_t B^(kDg - 1 - t) in three int64 groups, then one 128-bit
        // integer (|V| < 2^126: a sum of K products of F-bit numbers, K <= 256
        // for F = 59, K = 64 for F = 60); the FP64 pipe (64 cycles per warp
        // instruction on this GPU) is left to one add per entry
        __int128 V[kSchurN];
        {
          long long G[kSchurN];
#pragma unroll
          for (int c = 0; c < kSchurN; ++c) G[c] = 0;
          for (int t = 0; t < Fm::kDg; ++t) {
            uint32_t rr[16];
            tmem_ld16(lane_base + (uint32_t)(ab * kAccCols + t * kSchurN), rr);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int c = 0; c < kSchurN; ++c) {
              // |ACC| < 2^22 (ten digits) takes the integer trick; up to 2^23 a conversion
              const int x = (kSl == 10) ? emu_acc_int(rr[c]) : __float2int_rn(__uint_as_float(rr[c]));
              G[c] = G[c] * (1LL << Fm::kBits) + (long long)x;
            }
            if (t == Fm::kG0 || t == Fm::kG1 || t == Fm::kDg - 1) {
              const int sh = t == Fm::kG0 ? Fm::kSh0 : t == Fm::kG1 ? Fm::kSh1 : 0;
#pragma unroll
              for (int c = 0; c < kSchurN; ++c) {
                const __int128 g = (__int128)G[c] << sh;
                V[c] = (t == Fm::kG0) ? g : V[c] + g;
                G[c] = 0;
              }
            }
          }
        }
        tc_fence_before();
        clear(ab);
        const int Ea = row < n ? __ldg(a.Wexp + (size_t)T.a_of(r) * n + row) : 0;
#pragma unroll
        for (int c = 0; c < kSchurN; ++c) {
          const int col = T.ct * kSchurN + c;
          const int Eb = col < n ? __ldg(a.Wexp + (size_t)T.b_of(r) * n + col) : 0;
          // an Inf or NaN in either row (exponent field all ones: E = 1025)
          // poisons the entry, as an FP64 product would
          acc[c] += (Ea > 1024 || Eb > 1024) ? __longlong_as_double(0x7FF8000000000000LL)
                                             : emu_i128_to_double(V[c], Ea + Eb - 2 * Fm::kFrac);
        }
      }
      if (stop || row >= n) continue;
      const long long s = 2 * T.k;
      if (T.isD) {
        const long long orig = s << a.l;
        double *Dg = a.Ld + (size_t)orig * nn + (size_t)row * n;
        const double *Ag = a.A_diag + (size_t)orig * nn;
#pragma unroll
        for (int c = 0; c < kSchurN; ++c) {
          const int col = T.ct * kSchurN + c;
          if (col < n && col <= row) {
            const double b0 = a.l == 0 ? 0.5 * (__ldg(Ag + (size_t)row * n + col) + __ldg(Ag + (size_t)col * n + row))
                                       : Dg[col];
            Dg[col] = b0 - acc[c];
          }
        }
      } else {
        double *Eg = a.En + (size_t)T.k * nn + (size_t)row * n;
#pragma unroll
        for (int c = 0; c < kSchurN; ++c) {
          const int col = T.ct * kSchurN + c;
          if (col < n) Eg[col] = -acc[c];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

cudaError_t encode_bf16_3d(CUtensorMap *out, void *base, unsigned long long cols, unsigned long long rows,
                           unsigned long long planes, unsigned box_cols, unsigned box_rows, unsigned box_planes) {
  EncodeTiledFn fn = nullptr;
  const cudaError_t e = encode_fn(&fn);
  if (e != cudaSuccess) return e;
  const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t strides[2] = {(cuuint64_t)cols * 2, (cuuint64_t)cols * rows * 2};
  const cuuint32_t box[3] = {box_cols, box_rows, box_planes};
  const cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}


}  // namespace

size_t emu_aslc_bytes(long long N, int n) { return (size_t)N * kS * n * 3 * emu_np(n) * 2; }
size_t emu_xslc_bytes(long long N, int n) { return (size_t)N * kS * kEmuDp * emu_np(n) * 2; }

cudaError_t emu_make_maps(EmuBuffers &b, long long N, int n) {
  const int np = emu_np(n);
  cudaError_t e = encode_bf16_2d(&b.maps[0], b.Aslc, (unsigned long long)3 * np, (unsigned long long)N * kS * n,
                                 kEmuKc, kM);
  if (e == cudaSuccess)
    e = encode_bf16_2d(&b.maps[1], b.Xslc, (unsigned long long)np, (unsigned long long)N * kS * kEmuDp, kEmuKc, kN);
  return e;
}

cudaError_t emu_configure() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const void *kernels[] = {(const void *)k_emu_residual, (const void *)k_emu_slice_operator,
                           (const void *)k_emu_slice_x, (const void *)k_emu_schur<10>,
                           (const void *)k_emu_schur<8>};
  for (const void *k : kernels) {
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  }
  if (e == cudaSuccess && kResidualSmem > (size_t)optin) e = cudaErrorInvalidConfiguration;
  return e;
}

cudaError_t launch_emu_slice_operator(long long N, int n, const double *A_diag, const double *A_sub,
                                      const EmuBuffers &b, DevStatus *st, cudaStream_t s) {
  const int groups = (n + kRowsPerCta - 1) / kRowsPerCta;
  const long long grid = N * groups;
  const size_t sm = (size_t)3 * kRowsPerCta * n * sizeof(double);
  k_emu_slice_operator<<<(unsigned)grid, 256, sm, s>>>(N, n, emu_np(n), A_diag, A_sub, b.Aslc, b.Aexp, st);
  return cudaGetLastError();
}

cudaError_t launch_emu_residual(long long N, int n, int d, const double *X, const double *B, float *R32,
                                double *R64, const EmuBuffers &b, DevStatus *st, long long timeout_ns, int sms,
                                cudaStream_t s) {
  if (d < 1 || d > kEmuDp) return cudaErrorInvalidValue;
  const int np = emu_np(n);
  cudaError_t e = cudaMemsetAsync(b.xmax, 0, kEmuDp * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const long long rows = N * n;
  long long gx = (rows + 15) / 16;
  if (gx > 4 * (long long)sms) gx = 4 * (long long)sms;
  k_emu_xmax<<<(unsigned)gx, 256, 0, s>>>(rows, d, X, b.xmax);
  k_emu_slice_x<<<(unsigned)N, 256, (size_t)n * d * sizeof(double), s>>>(N, n, np, d, X, b.xmax, b.xexp, b.Xslc);
  EmuKArgs k;
  k.N = N;
  k.n = n;
  k.np = np;
  k.d = d;
  k.Aexp = b.Aexp;
  k.xexp = b.xexp;
  k.X = X;
  k.B = B;
  k.R32 = R32;
  k.R64 = R64;
  k.st = st;
  k.timeout_ns = timeout_ns;
  const long long tiles = N * ((n + kM - 1) / kM);
  const int grid = (int)(tiles < sms ? tiles : sms);
  k_emu_residual<<<grid, kEmuThreads, kResidualSmem, s>>>(b.maps[0], b.maps[1], k);
  return cudaGetLastError();
}

size_t emu_wslc_bytes(long long nW, int n) { return (size_t)nW * kS * n * emu_np(n) * 2; }

// Digits of the Schur engine: eight base-256 digits when the whole K = n fits
// one chunk of 64 (two accumulators in TMEM), else ten base-64 digits.
static int schur_slices(int n) { return emu_np(n) == kEmuKc ? 8 : 10; }

template <int kSl>
static size_t schur_smem() {
  return (size_t)kSchurAStages * kATile + (size_t)kXStages * kSl * kSchurN * kEmuKc * 2 + 1024;
}

cudaError_t launch_emu_slice_w(long long nW, int n, const double *W, unsigned short *Wslc, int *Wexp,
                               cudaStream_t s) {
  if (n > 256) return cudaErrorInvalidValue;
  const long long rows = nW * n;
  if (rows <= 0) return cudaSuccess;
  const unsigned grid = (unsigned)((rows + 7) / 8);
  if (schur_slices(n) == 8) k_emu_slice_w<8><<<grid, 256, 0, s>>>(rows, n, emu_np(n), W, Wslc, Wexp);
  else k_emu_slice_w<10><<<grid, 256, 0, s>>>(rows, n, emu_np(n), W, Wslc, Wexp);
  return cudaGetLastError();
}

template <int kSl>
static cudaError_t launch_emu_schur_t(long long Nl, int n, int l, const unsigned short *Wslc, const int *Wexp,
                                      const double *A_diag, double *Ld, double *En, DevStatus *st,
                                      long long timeout_ns, int sms, cudaStream_t s) {
  const int np = emu_np(n);
  const long long nW = Nl - 1;
  CUtensorMap mapA, mapB;
  cudaError_t e = encode_bf16_2d(&mapA, (void *)Wslc, (unsigned long long)np, (unsigned long long)(nW * kSl * n),
                                 kEmuKc, kM);
  if (e == cudaSuccess)
    e = encode_bf16_3d(&mapB, (void *)Wslc, (unsigned long long)np, (unsigned long long)n,
                       (unsigned long long)(nW * kSl), kEmuKc, kSchurN, kSl);
  if (e != cudaSuccess) return e;
  EmuSchurArgs k;
  k.Nl = Nl;
  k.n = n;
  k.np = np;
  k.l = l;
  k.Wexp = Wexp;
  k.A_diag = A_diag;
  k.Ld = Ld;
  k.En = En;
  k.st = st;
  k.timeout_ns = timeout_ns;
  const long long tiles = ((Nl + 1) / 2) * schur_tiles_per_sep(n);
  const int grid = (int)(tiles < sms ? tiles : sms);
  k_emu_schur<kSl><<<grid, kEmuThreads, schur_smem<kSl>(), s>>>(mapA, mapB, k);
  return cudaGetLastError();
}

cudaError_t launch_emu_schur(long long Nl, int n, int l, const unsigned short *Wslc, const int *Wexp,
                             const double *A_diag, double *Ld, double *En, DevStatus *st, long long timeout_ns,
                             int sms, cudaStream_t s) {
  if (Nl < 2 || n > 256) return cudaErrorInvalidValue;
  if (schur_slices(n) == 8)
    return launch_emu_schur_t<8>(Nl, n, l, Wslc, Wexp, A_diag, Ld, En, st, timeout_ns, sms, s);
  return launch_emu_schur_t<10>(Nl, n, l, Wslc, Wexp, A_diag, Ld, En, st, timeout_ns, sms, s);
}

}  // namespace bdss
