// Tensor-core Schur-update tiles for sm_103a: TMA (cp.async.bulk.tensor)
// loads of W^T rows into 128B-swizzled shared memory, an in-place split of
// every FP32 element into a TF32 high part and its remainder (3xTF32:
// a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi), tcgen05.mma kind::tf32 with the
// 128 x 128 FP32 accumulator in tensor memory (TMEM), tcgen05.ld epilogue.
//
// C[m][n] = sum_k A[m][k] B[n][k]: both operands K-major (rows of W^T are
// K-contiguous), exactly the layout of the products W^T W in Algorithm 3.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "bdss_device.cuh"

namespace bdss {

constexpr int kTcM = 128;          // rows of the output tile (TMEM lanes)
constexpr int kTcN = 128;          // columns of the output tile (TMEM columns)
constexpr int kTcK = 32;           // K elements per staged chunk (128 bytes of FP32)
constexpr int kTcSlab = kTcM * 128;  // bytes of one 128-row x 128-byte slab
// shared memory of a tile task: 4 slabs (A hi, A lo, B hi, B lo), 1 KB of
// alignment slack and 16 KB of guard after the slabs
constexpr size_t kTcSmemBytes = 4 * kTcSlab + 1024 + 16384;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ---- mbarrier --------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bounded wait for the phase with the given parity.  Returns false when the
// limit is reached (the caller records a timeout).
// The clock is read only once the phase is late (after 64 failed polls): a
// wait that succeeds at once, the common case, costs no timer read.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long timeout_ns) {
  long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 63) {
      const long long now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > timeout_ns) return false;
    }
  }
}

// CTA-uniform bounded wait (all threads call it): thread 0 polls with the
// time limit and broadcasts the outcome through shared memory, so every
// thread takes the same branch afterwards; on success each thread then
// observes the completed phase itself (its wait returns at once), which makes
// the asynchronous writes of that phase visible to it.
__device__ __forceinline__ bool mbar_wait_cta(uint64_t *bar, uint32_t parity, long long timeout_ns, int *s_ok) {
  if (threadIdx.x == 0) *s_ok = mbar_wait(bar, parity, timeout_ns) ? 1 : 0;
  __syncthreads();
  const bool ok = *s_ok != 0;
  if (ok && threadIdx.x != 0) mbar_wait(bar, parity, timeout_ns);
  __syncthreads();  // *s_ok is read by all before thread 0 may write it again
  return ok;
}

// ---- TMA -------------------------------------------------------------------
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}

// ---- tcgen05 ----------------------------------------------------------------
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, rows of 128
// bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t tc_desc_sw128(const void *slab, int byte_offset) {
  const uint32_t addr = smem_u32(slab) + (uint32_t)byte_offset;
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);         // start address
  d |= (uint64_t)(16 >> 4) << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor: D = FP32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Allocate `ncols` TMEM columns (warp-wide, warp 0); the address lands in *slot.
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-CTA state of the tensor-core tile engine.
struct TcState {
  unsigned char *slab;   // 1024-aligned: A hi | A lo | B hi | B lo
  uint64_t *bar_tma;     // TMA completion
  uint64_t *bar_mma;     // MMA completion
  int *s_ok;             // shared word of mbar_wait_cta
  uint32_t tmem;         // TMEM base address (128 columns)
  uint32_t ph_tma, ph_mma;
  bool tma_pending;      // a TMA load or an MMA batch was issued and its
  bool mma_pending;      // completion has not been observed (CTA-uniform)
};

// Split the staged FP32 values of a slab in place into TF32 hi (rounded to
// the nearest TF32) and write the remainder x - hi to `lo` at the same byte
// position (the swizzled layout is element-position preserving).
__device__ __forceinline__ void tc_split_slab(unsigned char *hi, unsigned char *lo) {
  float4 *h = reinterpret_cast<float4 *>(hi);
  float4 *l = reinterpret_cast<float4 *>(lo);
  for (int i = threadIdx.x; i < kTcSlab / 16; i += blockDim.x) {
    float4 x = h[i], a, b;
    const float *xs = reinterpret_cast<const float *>(&x);
    float *as = reinterpret_cast<float *>(&a);
    float *bs = reinterpret_cast<float *>(&b);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t u = __float_as_uint(xs[q]);
      const float top = __uint_as_float((u + 0x1000u) & 0xFFFFE000u);
      as[q] = top;
      bs[q] = xs[q] - top;
    }
    h[i] = a;
    l[i] = b;
  }
}

// Accumulate into TMEM: C (+)= A_rows(ra..ra+127, 0..K) * B_rows(rb.., 0..K)^T
// where the rows live in the 2-D tensor map (row coordinate = global row of
// the W^T buffer).  `first` clears the accumulator.  All threads call this.
__device__ __forceinline__ bool tc_accumulate(TcState &s, const CUtensorMap *map, int ra, int rb, int K, bool first,
                                              long long timeout_ns) {
  unsigned char *Ahi = s.slab, *Alo = s.slab + kTcSlab, *Bhi = s.slab + 2 * kTcSlab, *Blo = s.slab + 3 * kTcSlab;
  constexpr uint32_t idesc = tc_idesc_tf32(kTcM, kTcN);
  for (int k0 = 0; k0 < K; k0 += kTcK) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(s.bar_tma, 2 * kTcSlab);
      tma_load_2d(Ahi, map, k0, ra, s.bar_tma);
      tma_load_2d(Bhi, map, k0, rb, s.bar_tma);
    }
    s.tma_pending = true;
    if (!mbar_wait_cta(s.bar_tma, s.ph_tma, timeout_ns, s.s_ok)) return false;
    s.tma_pending = false;
    s.ph_tma ^= 1;
    tc_split_slab(Ahi, Alo);
    tc_split_slab(Bhi, Blo);
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc_fence_after();
#pragma unroll
      for (int kk = 0; kk < kTcK / 8; ++kk) {
        const int off = kk * 32;  // 8 TF32 = 32 bytes along K inside the swizzle atom
        const uint32_t acc0 = (first && k0 == 0 && kk == 0) ? 0u : 1u;
        tc_mma_tf32(s.tmem, tc_desc_sw128(Ahi, off), tc_desc_sw128(Bhi, off), idesc, acc0);
        tc_mma_tf32(s.tmem, tc_desc_sw128(Ahi, off), tc_desc_sw128(Blo, off), idesc, 1u);
        tc_mma_tf32(s.tmem, tc_desc_sw128(Alo, off), tc_desc_sw128(Bhi, off), idesc, 1u);
      }
      tc_commit(s.bar_mma);
    }
    s.mma_pending = true;
    if (!mbar_wait_cta(s.bar_mma, s.ph_mma, timeout_ns, s.s_ok)) return false;
    s.mma_pending = false;
    s.ph_mma ^= 1;
  }
  return true;
}

// Read this thread's row of the accumulator: warp w holds TMEM lanes
// 32 (w % 4) .. + 31 and columns 64 (w / 4) .. + 63.  row = 32 (w % 4) + lane.
__device__ __forceinline__ void tc_read_row(const TcState &s, float (&v)[64], int &row, int &col0) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  row = 32 * (w & 3) + lane;
  col0 = 64 * (w >> 2);
  tc_fence_after();
  const uint32_t base = s.tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)col0;
  float a[32], b[32];
  tmem_ld32(base, a);
  tmem_ld32(base + 32, b);
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    v[i] = a[i];
    v[32 + i] = b[i];
  }
}

// Set up mbarriers (in static shared memory, `bars` = 3 words: the two
// barriers and the flag word of mbar_wait_cta, so that other phases reusing
// the dynamic shared memory cannot clobber them) and TMEM (warp 0
// allocates); call with all threads.
__device__ __forceinline__ void tc_begin(TcState &s, unsigned char *smem_base, uint64_t *bars, uint32_t *tmem_slot) {
  // aligned by pointer arithmetic, which keeps the slab reads of the split
  // shared-memory accesses (an integer round trip makes them generic)
  s.slab = smem_base + ((1024u - (smem_u32(smem_base) & 1023u)) & 1023u);
  s.bar_tma = bars;
  s.bar_mma = bars + 1;
  s.s_ok = reinterpret_cast<int *>(bars + 2);
  s.tma_pending = false;
  s.mma_pending = false;
  if (threadIdx.x == 0) {
    mbar_init(s.bar_tma, 1);
    mbar_init(s.bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < 32) tmem_alloc(tmem_slot, 128);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  s.tmem = *tmem_slot;
  s.ph_tma = 0;
  s.ph_mma = 0;
}

// Release TMEM (all threads call it).  After a timed-out wait, first wait
// again, with the same kind of limit, for the load or MMA batch still in
// flight, so that nothing writes the shared memory or TMEM being released;
// TMEM is freed whether or not that second wait completes.
__device__ __forceinline__ void tc_end(TcState &s, long long timeout_ns) {
  if (s.tma_pending && mbar_wait_cta(s.bar_tma, s.ph_tma, timeout_ns, s.s_ok)) s.tma_pending = false;
  if (s.mma_pending && mbar_wait_cta(s.bar_mma, s.ph_mma, timeout_ns, s.s_ok)) s.mma_pending = false;
  tc_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tmem_dealloc(s.tmem, 128);
}

}  // namespace bdss
