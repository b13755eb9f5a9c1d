// C ABI of the solver (include/bdss.h): handle and workspace ownership,
// argument checks, the level plan, launches and the mixed-precision
// refinement loop.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <vector>

#include "../../include/bdss.h"
#include "bdss_chunk.h"
#include "bdss_emu.h"
#include "bdss_launch.h"
#include "bdss_kalman.h"
#include "bdss_krylov.h"
#include "bdss_small.h"

using namespace bdss;

struct bdss_ctx {
  int64_t N = 0;
  int n = 0;
  int d_max = 0;
  bdss_precision prec = BDSS_FP64;
  cudaStream_t stream = nullptr;
  Plan plan{};
  int sms = 0;
  int bps = 0;          // resident CTAs per SM of the persistent kernel
  int bps_tc = 0;       // the same for the tiled path's tensor-core kernel (TF32 factor)
  size_t smem = 0;      // dynamic shared memory per CTA
  // workspace
  bool large = false;   // 64 < n <= 256: tiled path
  void *Ld = nullptr;   // N n n  (T)
  void *Wb = nullptr;   // coupling slots (T)
  void *Eb = nullptr;   // large path: couplings of levels >= 1 (T)
  int tf32 = 0;         // TF32 mode on the large path: tensor-core Schur tiles
  CUtensorMap *d_tmap = nullptr;  // TMA map of Wb (device copy)
  double *Ltop = nullptr;
  void *Li = nullptr;    // large mixed path: L^{-1} of the eliminated blocks (N n n, FP32)
  float *Yt = nullptr;   // large mixed path: y of the eliminated blocks in solve passes (N n d_max)
  float *Ltinv = nullptr;  // large mixed path: float(L_top) and its inverse (2 n n)
  float *Y32 = nullptr;  // mixed: working RHS / correction (N n d_max)
  float *R32 = nullptr;  // mixed: FP32 residual (N n d_max)
  double *partial = nullptr;  // log-det partial sums
  DevStatus *dst = nullptr;
  DevStatus *hst = nullptr;   // pinned
  // state
  bool factored = false;
  const double *A_diag = nullptr;  // remembered for the FP64 residual (mixed)
  const double *A_sub = nullptr;
  double normA = 0.0;
  bool norm_valid = false;
  // options
  long long timeout_ns = 10000000000LL;
  int persistent = 1;
  int max_refine = 10;
  double target = 1e-14;
  int krylov = 1;        // 0: plain refinement only; 1: CG when it stalls; 2: CG from the start
  int max_krylov = 300;  // CG iterations per cycle
  // mixed: preconditioned-CG refinement vectors (N n d_max each) and scalars,
  // allocated on first use
  double *kr_R = nullptr, *kr_Z = nullptr, *kr_P = nullptr, *kr_Q = nullptr;
  double *kr_part = nullptr, *kr_sc = nullptr;
  int last_plain = 0, last_cg = 0;  // refinement steps of the last solve
  // mixed precision: shifted factorisation when an FP32 pivot fails
  int nstar = 1;            // crossover N_*: top levels of up to nstar blocks are swept serially
  int shift_on = 1;
  double shift_used = 0.0;   // relative diagonal shift of the stored factors
  double *Ashift = nullptr;  // shifted copy of A_diag (allocated on first use)
  // mixed precision, tiled path: the FP64-accurate residual on the tensor
  // cores (sliced operator built once per factorisation)
  EmuBuffers emu{};
  CUtensorMap emu_maps[2];
  int emu_ready = 0;     // buffers allocated and maps encoded
  int emu_on = 0;        // option: use them
  // FP64 tiled path: Schur products on the tensor cores (digit slices of W)
  unsigned short *Wslc = nullptr;  // (N - 1) x S x n x np BF16
  int *Wexp = nullptr;             // (N - 1) x n row exponents
  int schur_emu_ready = 0;
  int schur_emu_on = 0;
  // large mixed path: streamed solve passes (maps over Li and Wb)
  CorrMaps corr_maps[3];  // split factors P = 1, 2, 4
  int corr_max_split = 1;
  int corr_ok = 0;
  // TF32 mode: the pipelined 3xTF32 Schur tiles read W through this map
  CUtensorMap ts_map_w;
  int ts_ok = 0;
  bool emu_sliced = false;
  int skip_barrier = 0;
  // one-cluster path for short systems (FP64, n <= 32, d_max <= 16)
  int small_opt = -1;            // -1: by size, 0: off, 1: whenever available
  int small_cluster = 0;         // CTAs of its cluster (0: unavailable)
  size_t small_smem = 0;         // its shared memory per CTA
  DevStatus *hst_dev = nullptr;  // device-visible address of hst
  // stats of the last call
  int64_t launches = 0;
  int64_t barriers = 0;
  int trace_count = 0;               // barrier stamps of the last persistent launch
  long long trace[kTraceSlots] = {};
  // per-kernel-class device times (BDSS_OPT_KERNEL_TIMING): pairs of events
  // recorded on the handle's stream around launches, harvested after the
  // stream is synchronised
  int ktiming = 0;
  int kt_cls = BDSS_KT_FACTOR;       // class of the launches being issued
  std::vector<cudaEvent_t> kt_ev;    // event pool (pairs)
  std::vector<int> kt_pair_cls, kt_pair_n;
  int kt_used = 0;                   // pairs recorded since the last harvest
  double kt_ms[BDSS_KT_CLASSES] = {};
  int64_t kt_n[BDSS_KT_CLASSES] = {};
  // guard bands after every workspace buffer (checked with the debug option)
  struct Guard { void *base; size_t bytes; };
  std::vector<Guard> guards;
  int debug_guards = 0;
};

// Workspace guard bands: kGuardBytes of kGuardByte after each buffer.
static constexpr size_t kGuardBytes = 256;
static constexpr unsigned char kGuardByte = 0xA5;

// Test hook: the k-th allocation of each following bdss_create fails (0 = off).
static std::atomic<int> g_fail_alloc{0};
static thread_local int t_alloc_count = 0;

static bool inject_alloc_failure() {
  const int k = g_fail_alloc.load();
  return k > 0 && ++t_alloc_count == k;
}

// Device workspace with a guard band after it.
static bool ws_alloc(bdss_ctx *h, void **p, size_t bytes) {
  *p = nullptr;
  if (inject_alloc_failure()) return false;
  if (cudaMalloc(p, bytes + kGuardBytes) != cudaSuccess) {
    *p = nullptr;
    return false;
  }
  h->guards.push_back({*p, bytes});
  return cudaMemset(static_cast<char *>(*p) + bytes, kGuardByte, kGuardBytes) == cudaSuccess;
}

// All guard bands intact?  (Synchronous copies; debug option only.)
static bool guards_intact(const bdss_ctx *h) {
  unsigned char buf[kGuardBytes];
  for (const auto &g : h->guards) {
    if (cudaMemcpy(buf, static_cast<const char *>(g.base) + g.bytes, kGuardBytes, cudaMemcpyDeviceToHost) !=
        cudaSuccess)
      return false;
    for (size_t i = 0; i < kGuardBytes; ++i)
      if (buf[i] != kGuardByte) return false;
  }
  return true;
}

static constexpr int kLogdetGrid = 256;

// Last CUDA runtime error met by a bdss_* call on this host thread.
static thread_local cudaError_t g_last_cuda_error = cudaSuccess;

static bdss_status cuda_fail(cudaError_t e) {
  g_last_cuda_error = e;
  return BDSS_ERR_CUDA;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// ---- per-kernel-class timing ------------------------------------------------
static constexpr int kKtPairs = 256;

// Add the elapsed times of the recorded pairs to their classes (the events
// have completed once the stream is synchronised; the wait on the last one
// covers a harvest forced by a full pool).
static void kt_harvest(bdss_ctx *h) {
  if (h->kt_used == 0) return;
  cudaEventSynchronize(h->kt_ev[2 * (h->kt_used - 1) + 1]);
  for (int i = 0; i < h->kt_used; ++i) {
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->kt_ev[2 * i], h->kt_ev[2 * i + 1]) == cudaSuccess) {
      h->kt_ms[h->kt_pair_cls[i]] += ms;
      h->kt_n[h->kt_pair_cls[i]] += h->kt_pair_n[i];
    }
  }
  cudaGetLastError();
  h->kt_used = 0;
}

static void kt_reset(bdss_ctx *h) {
  h->kt_used = 0;
  for (int c = 0; c < BDSS_KT_CLASSES; ++c) {
    h->kt_ms[c] = 0.0;
    h->kt_n[c] = 0;
  }
}

// Open a timed group of launches of class `cls` (no-op unless timing is on).
static void kt_begin(bdss_ctx *h, int cls) {
  if (!h->ktiming) return;
  if (h->kt_used == kKtPairs) kt_harvest(h);
  h->kt_pair_cls[h->kt_used] = cls;
  cudaEventRecord(h->kt_ev[2 * h->kt_used], h->stream);
}

// Close the group opened by kt_begin; it held `launches` kernel launches.
static void kt_end(bdss_ctx *h, int launches) {
  if (!h->ktiming) return;
  cudaEventRecord(h->kt_ev[2 * h->kt_used + 1], h->stream);
  h->kt_pair_n[h->kt_used] = launches;
  ++h->kt_used;
}

static bool is_mixed(const bdss_ctx *h) { return h->prec != BDSS_FP64; }

// Level sizes N_{l+1} = ceil(N_l / 2) down to one block (their coupling
// regions are laid out for every level); the reduction stops at the first
// level with at most nstar blocks, which the top sweep then factors.
static void make_plan(Plan &p, int64_t N, int n, int nstar = 1) {
  memset(&p, 0, sizeof(p));
  p.N = N;
  p.n = n;
  p.Nl[0] = N;
  p.off[0] = 0;
  int l = 0, stop = -1;
  while (p.Nl[l] > 1) {
    if (stop < 0 && p.Nl[l] <= nstar) stop = l;
    p.Nl[l + 1] = (p.Nl[l] + 1) / 2;
    p.off[l + 1] = p.off[l] + (p.Nl[l] - 1);
    ++l;
  }
  p.L = stop >= 0 ? stop : l;
}

static int grid_for(const bdss_ctx *h, long long items) {
  long long g = (long long)h->bps * h->sms;
  if (items < g) g = items;
  return (int)(g < 1 ? 1 : g);
}

// Read the device status word (synchronises the handle's stream).
static bdss_status finish(bdss_ctx *h, bdss_info *info) {
  cudaError_t e = cudaMemcpyAsync(h->hst, h->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  kt_harvest(h);
  const int st = h->hst->status;
  if (h->hst->trace[0] != 0) {  // a launch with grid barriers: keep its stamps
    int c = 0;
    while (c < kTraceSlots && h->hst->trace[c] != 0) ++c;
    memcpy(h->trace, h->hst->trace, sizeof(h->trace));
    h->trace_count = c;
  }
  if (info && st == BDSS_ERR_NOT_SPD) {
    info->level = h->hst->level;
    info->block = h->hst->block;
  }
  if (h->debug_guards && !guards_intact(h)) return BDSS_ERR_GUARD;
  return (bdss_status)st;
}

static cudaError_t reset_status(bdss_ctx *h) {
  return cudaMemsetAsync(h->dst, 0, sizeof(DevStatus), h->stream);
}

// The one-cluster path: on request, or by size.  Its time grows with the
// blocks each CTA eliminates in turn at level 0 and with each block's pivot
// chain (n columns), while the persistent grid spreads level 0 over every SM:
// measured on GB300 (d = 1) the cluster is faster up to N = 128 at n = 4 and
// 8, N = 64 at n = 12, N = 32-64 at n = 16, and never from n = 24.  The rule
// n <= 16, N <= 8 C and N n <= 64 C (C = the cluster's CTAs) keeps it to
// that range.  It runs in place of the persistent launch only (not with
// per-level launches, the slice products or the barrier test hook).
constexpr int kSmallAutoMaxN = 16;
constexpr int kSmallAutoPerCta = 8;
constexpr int kSmallAutoWorkPerCta = 64;
static bool use_small(const bdss_ctx *h) {
  if (is_mixed(h) || h->small_cluster < 2 || !h->persistent || h->skip_barrier || h->schur_emu_on) return false;
  if (h->small_opt >= 0) return h->small_opt == 1;
  const int64_t C = h->small_cluster;
  return h->n <= kSmallAutoMaxN && h->N <= kSmallAutoPerCta * C && h->N * h->n <= kSmallAutoWorkPerCta * C;
}

static cudaError_t run_small(bdss_ctx *h, const Args<double> &a, bool factor, bool rhs) {
  h->launches += 1;
  kt_begin(h, h->kt_cls);
  const cudaError_t e =
      launch_small(a, factor ? 1 : 0, rhs ? 1 : 0, h->small_cluster, h->small_smem, h->hst_dev, h->stream);
  kt_end(h, 1);
  return e;
}

// Outcome of a one-cluster launch, which cleared the device status itself
// and wrote status, level, block and its barrier stamps into hst at its end.
static bdss_status finish_small(bdss_ctx *h, bdss_info *info) {
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  kt_harvest(h);
  const volatile DevStatus *hs = h->hst;
  int c = 0;
  while (c < kTraceSlots && hs->trace[c] != 0) {
    h->trace[c] = hs->trace[c];
    ++c;
  }
  h->trace_count = c;
  const int st = hs->status;
  if (info && st == BDSS_ERR_NOT_SPD) {
    info->level = hs->level;
    info->block = hs->block;
  }
  if (h->debug_guards && !guards_intact(h)) return BDSS_ERR_GUARD;
  return (bdss_status)st;
}

template <typename T>
static Args<T> base_args(bdss_ctx *h) {
  Args<T> a;
  memset(&a, 0, sizeof(a));
  a.p = h->plan;
  a.Ld = (T *)h->Ld;
  a.Wb = (T *)h->Wb;
  a.Eb = (T *)h->Eb;
  a.Ltop = h->Ltop;
  a.st = h->dst;
  a.timeout_ns = h->timeout_ns;
  a.skip_barrier = h->skip_barrier;
  a.capacity = h->bps * h->sms;
  a.tf32 = h->tf32;
  a.tmap_w = h->d_tmap;
  a.Li = (T *)h->Li;
  a.Ltinv = (T *)h->Ltinv;
  return a;
}

// Separator update of level l on the tensor cores (FP64 factorisation):
// slice the level's stored couplings, form D and the next level's E, then the
// separators' RHS tiles (when the pass carries right-hand sides) on the ALU.
static cudaError_t schur_emu_level(bdss_ctx *h, const Args<double> &b, int l) {
  const Plan &p = h->plan;
  const long long Nl = p.Nl[l];
  const size_t nn = (size_t)p.n * p.n;
  kt_begin(h, BDSS_KT_SLICE);
  cudaError_t e = launch_emu_slice_w(Nl - 1, p.n, b.Wb + (size_t)p.off[l] * nn, h->Wslc, h->Wexp, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (e != cudaSuccess) return e;
  // the next level's couplings: Eb on the tiled path, region l + 1 of Wb for n <= 64
  double *En = (h->large ? b.Eb : b.Wb) + (size_t)p.off[l + 1] * nn;
  kt_begin(h, BDSS_KT_SCHUR_TC);
  e = launch_emu_schur(Nl, p.n, l, h->Wslc, h->Wexp, b.A_diag, b.Ld, En, h->dst, h->timeout_ns, h->sms, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (e != cudaSuccess || b.d == 0) return e;
  kt_begin(h, h->kt_cls);
  if (h->large) {
    e = launch_large_sub<double>(b, l, kSubBRhsOnly, 1,
                                 grid_for(h, large_sub_tasks(p, l, kSubBRhsOnly, 1, b.d, 8, 0, 0)), h->smem,
                                 h->stream);
  } else {  // phase B without the factor work is the separators' RHS update
    const int cap = h->bps * h->sms;
    e = launch_phaseB<double>(b, l, 0, grid_for(h, ((Nl + 1) / 2) * parts_B<double>(p, l, false, cap)), h->smem,
                              h->stream);
  }
  kt_end(h, 1);
  h->launches += 1;
  return e;
}

// FP64 factorisation for n <= 64 with the Schur products on the tensor
// cores: per level phase A (Cholesky, coupling and RHS substitutions), the
// slice products, the separators' RHS update; then the top block and the
// downward pass, one launch each.
static cudaError_t run_levels_emu_small(bdss_ctx *h, const Args<double> &a, bool rhs) {
  const Plan &p = h->plan;
  const int cap = h->bps * h->sms;
  Args<double> b = a;
  if (!rhs) b.d = 0;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < p.L && e == cudaSuccess; ++l) {
    const long long nElim = p.Nl[l] / 2;
    kt_begin(h, h->kt_cls);
    e = launch_phaseA<double>(b, l, 1, grid_for(h, nElim * parts_A<double>(p, l, true, cap)), h->smem, h->stream);
    kt_end(h, 1);
    h->launches += 1;
    if (e == cudaSuccess) e = schur_emu_level(h, b, l);
  }
  kt_begin(h, h->kt_cls);
  if (e == cudaSuccess) e = launch_top<double>(b, 1, h->smem, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (rhs)
    for (int l = p.L - 1; l >= 0 && e == cudaSuccess; --l) {
      kt_begin(h, h->kt_cls);
      e = launch_phaseC<double>(b, l, grid_for(h, p.Nl[l] / 2), h->smem, h->stream);
      kt_end(h, 1);
      h->launches += 1;
    }
  return e;
}

// Solve pass of the large mixed path with the stored inverses, streamed: per
// level the upward products (A2, B), the top block, then per level the
// downward products (C), one launch each.
static cudaError_t run_corr_passes(bdss_ctx *h, const Args<float> &b) {
  const Plan &p = h->plan;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < p.L && e == cudaSuccess; ++l)
    for (int sub = kSubA2; sub <= kSubB && e == cudaSuccess; ++sub) {
      kt_begin(h, h->kt_cls);
      e = launch_large_corr(h->corr_maps, h->corr_max_split, b, l, sub, h->sms, h->stream);
      kt_end(h, 1);
      h->launches += 1;
    }
  kt_begin(h, h->kt_cls);
  if (e == cudaSuccess) e = launch_large_top<float>(b, 0, h->smem, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  for (int l = p.L - 1; l >= 0 && e == cudaSuccess; --l) {
    kt_begin(h, h->kt_cls);
    if (corr_split(p.n, p.Nl[l] / 2, h->sms, h->corr_max_split) > 1) {
      // few blocks: t = y - W x, then x = L^{-T} t, each block split over SMs
      e = launch_large_corr(h->corr_maps, h->corr_max_split, b, l, kSubC1, h->sms, h->stream);
      if (e == cudaSuccess) e = launch_large_corr(h->corr_maps, h->corr_max_split, b, l, kSubC2, h->sms, h->stream);
      h->launches += 1;
    } else {
      e = launch_large_corr(h->corr_maps, h->corr_max_split, b, l, kSubC, h->sms, h->stream);
    }
    kt_end(h, 1);
    h->launches += 1;
  }
  return e;
}

// Separator update of level l in the TF32 mode: the D and E tiles on the
// pipelined tensor-core kernel, then the separators' RHS tiles on the ALU.
static cudaError_t schur_tf32_level(bdss_ctx *h, const Args<float> &b, int l) {
  const Plan &p = h->plan;
  kt_begin(h, BDSS_KT_SCHUR_TC);
  cudaError_t e = launch_tf32_schur(h->ts_map_w, b, l, h->sms, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (e != cudaSuccess || b.d == 0) return e;
  kt_begin(h, h->kt_cls);
  // b_s -= W^T y of the neighbours: the streamed product of the solve passes
  // (the factor pass keeps y in Y), else the RHS tiles
  if (h->corr_ok && b.d <= kCorrMaxD)
    e = launch_large_corr(h->corr_maps, h->corr_max_split, b, l, kSubB, h->sms, h->stream);
  else
    e = launch_large_sub<float>(b, l, kSubBRhsOnly, 1,
                                grid_for(h, large_sub_tasks(p, l, kSubBRhsOnly, 1, b.d, 4, 0, 0)), h->smem, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  return e;
}

// One factor and/or RHS pass over all levels, persistent or per level.
// Large-block path: three tile sub-phases per level (see bdss_large.cu).
template <typename T>
static cudaError_t run_levels_large(bdss_ctx *h, const Args<T> &a, bool factor, bool rhs) {
  const Plan &p = h->plan;
  const int esz = (int)sizeof(T);
  // The TF32 factorisation runs sub-phase by sub-phase even in persistent
  // mode: a kernel holding tcgen05 code gets one CTA per SM, so only the
  // Schur-update tiles use that kernel and the Cholesky / substitution tasks
  // keep the two-CTA FP32 kernel.
  const bool tc_factor = sizeof(T) == 4 && h->tf32 && factor;
  // FP64 factorisation with the Schur products on the tensor cores: sub-phase
  // by sub-phase as well (the slicing and the product kernels are launches
  // of their own)
  const bool emu_factor = sizeof(T) == 8 && factor && h->schur_emu_on;
  const int inv = a.Li ? 1 : 0;
  Args<T> b = a;
  if (!rhs) b.d = 0;
  // solve passes with the stored inverses keep y of the eliminated blocks in Yt
  b.Yt = (!factor && inv) ? (T *)h->Yt : nullptr;
  if constexpr (sizeof(T) == 4) {
    if (!factor && rhs && inv && h->corr_ok && b.d <= kCorrMaxD) return run_corr_passes(h, b);
  }
  if (h->persistent && !tc_factor && !emu_factor) {
    long long most = 1;
    for (int l = 0; l < p.L; ++l)
      for (int sub = 0; sub < 4; ++sub) {
        const long long t = large_sub_tasks(p, l, sub, factor ? 1 : 0, rhs ? a.d : 0, esz, h->tf32, inv);
        if (t > most) most = t;
      }
    h->launches += 1;
    h->barriers += 1 + (factor ? 3 : 2) * p.L + ((rhs && p.L > 0) ? p.L : 0);
    kt_begin(h, h->kt_cls);
    const cudaError_t e = launch_large_persistent<T>(b, factor ? 1 : 0, rhs ? 1 : 0, grid_for(h, most), h->smem,
                                                     h->stream);
    kt_end(h, 1);
    return e;
  }
  const int f = factor ? 1 : 0;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < p.L && e == cudaSuccess; ++l)
    for (int sub = factor ? 0 : 1; sub < 3 && e == cudaSuccess; ++sub) {
      if constexpr (sizeof(T) == 8) {
        if (emu_factor && sub == 2) {
          e = schur_emu_level(h, b, l);
          continue;
        }
      } else {
        if (tc_factor && sub == 2 && h->ts_ok) {
          e = schur_tf32_level(h, b, l);
          continue;
        }
      }
      kt_begin(h, (tc_factor && sub == 2) ? BDSS_KT_SCHUR_TC : h->kt_cls);
      e = launch_large_sub<T>(b, l, sub, f, grid_for(h, large_sub_tasks(p, l, sub, f, b.d, esz, h->tf32, inv)),
                              h->smem, h->stream);
      kt_end(h, 1);
      h->launches += 1;
    }
  kt_begin(h, h->kt_cls);
  if (e == cudaSuccess) e = launch_large_top<T>(b, f, h->smem, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (rhs)
    for (int l = p.L - 1; l >= 0 && e == cudaSuccess; --l) {
      kt_begin(h, h->kt_cls);
      e = launch_large_sub<T>(b, l, 3, 0, grid_for(h, large_sub_tasks(p, l, 3, 0, b.d, esz, 0, inv)), h->smem,
                              h->stream);
      kt_end(h, 1);
      h->launches += 1;
    }
  return e;
}

template <typename T>
static cudaError_t run_levels(bdss_ctx *h, const Args<T> &a, bool factor, bool rhs) {
  const Plan &p = h->plan;
  if (h->large) return run_levels_large<T>(h, a, factor, rhs);
  if constexpr (sizeof(T) == 8) {
    if (factor && h->schur_emu_on) return run_levels_emu_small(h, a, rhs);
  }
  const int cap = h->bps * h->sms;
  if (h->persistent) {
    long long most = 1;  // tasks of the busiest step
    for (int l = 0; l < p.L; ++l) {
      most = std::max(most, (p.Nl[l] / 2) * parts_A<T>(p, l, factor, cap));
      most = std::max(most, ((p.Nl[l] + 1) / 2) * parts_B<T>(p, l, factor, cap));
    }
    const int grid = grid_for(h, most);
    h->launches += 1;
    int bars = 1 + 2 * p.L;  // the spread-rank barrier, then two per level
    if (rhs && p.L > 0) bars += 1 + (p.L - 1);
    h->barriers += bars;
    kt_begin(h, h->kt_cls);
    const cudaError_t e = launch_persistent<T>(a, factor ? 1 : 0, rhs ? 1 : 0, grid, h->smem, h->stream);
    kt_end(h, 1);
    return e;
  }
  Args<T> b = a;
  if (!rhs) b.d = 0;
  cudaError_t e = cudaSuccess;
  kt_begin(h, h->kt_cls);  // the per-level launches of one pass as one group
  const int64_t launches0 = h->launches;
  for (int l = 0; l < p.L && e == cudaSuccess; ++l) {
    const long long nElim = p.Nl[l] / 2, nSep = (p.Nl[l] + 1) / 2;
    e = launch_phaseA<T>(b, l, factor ? 1 : 0, grid_for(h, nElim * parts_A<T>(p, l, factor, cap)), h->smem,
                         h->stream);
    if (e == cudaSuccess)
      e = launch_phaseB<T>(b, l, factor ? 1 : 0, grid_for(h, nSep * parts_B<T>(p, l, factor, cap)), h->smem,
                           h->stream);
    h->launches += 2;
  }
  if (e == cudaSuccess) e = launch_top<T>(b, factor ? 1 : 0, h->smem, h->stream);
  h->launches += 1;
  if (rhs)
    for (int l = p.L - 1; l >= 0 && e == cudaSuccess; --l) {
      e = launch_phaseC<T>(b, l, grid_for(h, p.Nl[l] / 2), h->smem, h->stream);
      h->launches += 1;
    }
  kt_end(h, (int)(h->launches - launches0));
  return e;
}

extern "C" {

const char *bdss_status_string(bdss_status s) {
  switch (s) {
    case BDSS_OK: return "ok";
    case BDSS_ERR_INVALID_ARG: return "invalid argument";
    case BDSS_ERR_NOT_SPD: return "matrix not SPD (non-positive or non-finite pivot)";
    case BDSS_ERR_NOT_FACTORED: return "not factored";
    case BDSS_ERR_ALLOC: return "allocation failed";
    case BDSS_ERR_CUDA: return "CUDA runtime error";
    case BDSS_ERR_TIMEOUT: return "device wait timed out";
    case BDSS_ERR_NO_CONVERGENCE: return "refinement did not converge";
    case BDSS_ERR_UNSUPPORTED: return "unsupported size or mode";
    case BDSS_ERR_GUARD: return "a workspace guard band was overwritten";
  }
  return "unknown status";
}

bdss_status bdss_destroy(bdss_handle h) {
  if (!h) return BDSS_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  cudaFree(h->Ld);
  cudaFree(h->Wb);
  cudaFree(h->Eb);
  cudaFree(h->d_tmap);
  cudaFree(h->Ltop);
  cudaFree(h->emu.Aslc);
  cudaFree(h->emu.Aexp);
  cudaFree(h->emu.Xslc);
  cudaFree(h->emu.xexp);
  cudaFree(h->emu.xmax);
  cudaFree(h->Wslc);
  cudaFree(h->Wexp);
  cudaFree(h->Li);
  cudaFree(h->Yt);
  cudaFree(h->Ltinv);
  cudaFree(h->Y32);
  cudaFree(h->R32);
  cudaFree(h->partial);
  cudaFree(h->Ashift);
  cudaFree(h->kr_R);
  cudaFree(h->kr_Z);
  cudaFree(h->kr_P);
  cudaFree(h->kr_Q);
  cudaFree(h->kr_part);
  cudaFree(h->kr_sc);
  cudaFree(h->dst);
  if (h->hst) cudaFreeHost(h->hst);
  for (cudaEvent_t ev : h->kt_ev) cudaEventDestroy(ev);
  delete h;
  return BDSS_OK;
}

bdss_status bdss_create(bdss_handle *out, int64_t N, int32_t n, int32_t d_max, bdss_precision prec,
                        void *cuda_stream) {
  if (!out) return BDSS_ERR_INVALID_ARG;
  *out = nullptr;
  if (N < 1 || n < 1 || d_max < 1 || d_max > 64) return BDSS_ERR_INVALID_ARG;
  if (prec != BDSS_FP64 && prec != BDSS_FP32_IR && prec != BDSS_TF32_IR) return BDSS_ERR_INVALID_ARG;
  if (n > kMaxNLarge) return BDSS_ERR_UNSUPPORTED;
  if (N > ((int64_t)1 << (kMaxLevels - 2))) return BDSS_ERR_UNSUPPORTED;
  bdss_ctx *h = new (std::nothrow) bdss_ctx();
  if (!h) return BDSS_ERR_ALLOC;
  h->N = N;
  h->n = n;
  h->d_max = d_max;
  h->prec = prec;
  h->stream = (cudaStream_t)cuda_stream;
  make_plan(h->plan, N, n);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev);
  int smem_optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) { bdss_destroy(h); return cuda_fail(e); }
  const size_t esz = is_mixed(h) ? sizeof(float) : sizeof(double);
  h->large = n > kMaxN;
  size_t need;
  if (h->large) need = is_mixed(h) ? smem_bytes_large<float>(n, d_max) : smem_bytes_large<double>(n, d_max);
  else need = is_mixed(h) ? smem_bytes<float>(n, d_max) : smem_bytes<double>(n, d_max);
  if (need > (size_t)smem_optin) { bdss_destroy(h); return BDSS_ERR_UNSUPPORTED; }
  if (h->large) {
    e = configure<double>(1, 1, &h->smem, &h->bps);  // raises every kernel's shared-memory limit
    if (e == cudaSuccess)
      e = is_mixed(h) ? configure_large<float>(n, d_max, &h->smem, &h->bps, &h->bps_tc)
                      : configure_large<double>(n, d_max, &h->smem, &h->bps, &h->bps_tc);
  } else {
    e = is_mixed(h) ? configure<float>(n, d_max, &h->smem, &h->bps) : configure<double>(n, d_max, &h->smem, &h->bps);
  }
  if (e == cudaSuccess && !h->large) h->bps_tc = h->bps;
  if (e != cudaSuccess || h->bps < 1 || h->bps_tc < 1) {
    bdss_destroy(h);
    return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidConfiguration);
  }
  const size_t nn = (size_t)n * n;
  const size_t slots = (size_t)(h->plan.off[h->plan.L] > 0 ? h->plan.off[h->plan.L] : 1);
  t_alloc_count = 0;
  bool ok = ws_alloc(h, &h->Ld, (size_t)N * nn * esz);
  ok = ok && ws_alloc(h, &h->Wb, slots * nn * esz);
  if (h->large) ok = ok && ws_alloc(h, &h->Eb, slots * nn * esz);
  // the top factors: one block, or (blocks up to n = 64) the L_j, C_j and
  // y_j of a serial top sweep of up to kNStarMax blocks
  const size_t top_words = h->large ? nn : (size_t)kNStarMax * (2 * nn + (size_t)n * d_max);
  ok = ok && ws_alloc(h, (void **)&h->Ltop, top_words * sizeof(double));
  ok = ok && ws_alloc(h, (void **)&h->partial, kLogdetGrid * sizeof(double));
  ok = ok && ws_alloc(h, (void **)&h->dst, sizeof(DevStatus));
  ok = ok && !inject_alloc_failure() && cudaMallocHost((void **)&h->hst, sizeof(DevStatus)) == cudaSuccess;
  if (ok && h->large && prec == BDSS_TF32_IR && n % 4 == 0) {
    // tensor-core Schur tiles read W^T rows of Wb through TMA
    CUtensorMap map;
    cudaError_t em = make_w_tensor_map(&map, (const float *)h->Wb, (long long)slots * n, n);
    ok = em == cudaSuccess && ws_alloc(h, (void **)&h->d_tmap, sizeof(CUtensorMap)) &&
         cudaMemcpy(h->d_tmap, &map, sizeof(CUtensorMap), cudaMemcpyHostToDevice) == cudaSuccess;
    h->tf32 = ok ? 1 : 0;
    if (ok) {
      h->ts_map_w = map;
      h->ts_ok = 1;
    }
  }
  if (ok && is_mixed(h)) {
    const size_t nd = (size_t)N * n * d_max;
    ok = ws_alloc(h, (void **)&h->Y32, nd * sizeof(float));
    ok = ok && ws_alloc(h, (void **)&h->R32, nd * sizeof(float));
    if (h->large) {  // inverse factors and the y buffer of the solve passes
      ok = ok && ws_alloc(h, &h->Li, (size_t)N * nn * sizeof(float));
      ok = ok && ws_alloc(h, (void **)&h->Yt, nd * sizeof(float));
      ok = ok && ws_alloc(h, (void **)&h->Ltinv, 2 * nn * sizeof(float));
      if (ok && n % 4 == 0 && d_max <= 16 && corr_smem_bytes(n) <= (size_t)smem_optin) {
        const float *Lif = (const float *)h->Li, *Wbf = (const float *)h->Wb;
        const long long rl = N * n, rw = (long long)slots * n;
        CorrMaps &m0 = h->corr_maps[0];
        h->corr_ok = make_f32_map(&m0.rowsLi, Lif, rl, n, n) == cudaSuccess &&
                     make_f32_map(&m0.rowsW, Wbf, rw, n, n) == cudaSuccess;
        m0.colsLi = m0.rowsLi;  // P = 1: the column products use bulk copies
        m0.colsW = m0.rowsW;
        if (h->corr_ok && n % 32 == 0) {
          bool split = true;
          for (int i = 1; i <= 2 && split; ++i) {
            const int R = n >> i;
            CorrMaps &m = h->corr_maps[i];
            split = make_f32_map_box(&m.rowsLi, Lif, rl, n, 32, R, true) == cudaSuccess &&
                    make_f32_map_box(&m.rowsW, Wbf, rw, n, 32, R, true) == cudaSuccess &&
                    make_f32_map_box(&m.colsLi, Lif, rl, n, R, 32, false) == cudaSuccess &&
                    make_f32_map_box(&m.colsW, Wbf, rw, n, R, 32, false) == cudaSuccess;
            if (split) h->corr_max_split = 1 << i;
          }
        }
      }
    }
    if (ok && h->large && d_max <= kEmuDp) {  // the tensor-core FP64 residual
      ok = ws_alloc(h, (void **)&h->emu.Aslc, emu_aslc_bytes(N, n));
      ok = ok && ws_alloc(h, (void **)&h->emu.Aexp, (size_t)N * n * sizeof(int));
      ok = ok && ws_alloc(h, (void **)&h->emu.Xslc, emu_xslc_bytes(N, n));
      ok = ok && ws_alloc(h, (void **)&h->emu.xexp, kEmuDp * sizeof(int));
      ok = ok && ws_alloc(h, (void **)&h->emu.xmax, kEmuDp * sizeof(unsigned long long));
      if (ok) {
        h->emu.maps = h->emu_maps;
        const cudaError_t em = emu_make_maps(h->emu, N, n);
        const cudaError_t ec = em == cudaSuccess ? emu_configure() : em;
        if (ec != cudaSuccess) {
          bdss_destroy(h);
          return cuda_fail(ec);
        }
        h->emu_ready = 1;
        h->emu_on = 1;
      }
    }
  }
  if (ok && prec == BDSS_FP64 && N > 1 && (h->large || n >= 32)) {  // Schur products on the tensor cores
    ok = ws_alloc(h, (void **)&h->Wslc, emu_wslc_bytes(N - 1, n));
    ok = ok && ws_alloc(h, (void **)&h->Wexp, (size_t)(N - 1) * n * sizeof(int));
    if (ok) {
      const cudaError_t ec = emu_configure();
      if (ec != cudaSuccess) {
        bdss_destroy(h);
        return cuda_fail(ec);
      }
      h->schur_emu_ready = 1;
      // on by default for the tiled path; for n <= 64 the slice products do
      // not yet beat the FP64 pipe (half of each 128-row tile is padding),
      // so there the option opts in
      h->schur_emu_on = h->large ? 1 : 0;
    }
  }
  if (!ok) {
    cudaGetLastError();  // clear the allocation error
    bdss_destroy(h);
    return BDSS_ERR_ALLOC;
  }
  memset(h->hst, 0, sizeof(DevStatus));
  if (prec == BDSS_FP64 && !h->large && n <= kSmallMaxN && d_max <= kSmallMaxD) {
    // the one-cluster path writes its outcome straight into hst
    void *dp = nullptr;
    int c = 0;
    const size_t sm = small_smem_bytes(n, d_max);
    if (cudaHostGetDevicePointer(&dp, h->hst, 0) == cudaSuccess && dp &&
        small_cluster_size(sm, &c) == cudaSuccess && c >= 2) {
      h->small_cluster = c;
      h->small_smem = sm;
      h->hst_dev = (DevStatus *)dp;
    }
    cudaGetLastError();  // the path is optional: no error of the call
  }
  *out = h;
  return BDSS_OK;
}

bdss_status bdss_set_option(bdss_handle h, bdss_option key, int64_t value) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  switch (key) {
    case BDSS_OPT_TIMEOUT_MS:
      if (value < 1 || value > 600000) return BDSS_ERR_INVALID_ARG;
      h->timeout_ns = value * 1000000LL;
      return BDSS_OK;
    case BDSS_OPT_PERSISTENT:
      if (value != 0 && value != 1) return BDSS_ERR_INVALID_ARG;
      h->persistent = (int)value;
      return BDSS_OK;
    case BDSS_OPT_MAX_REFINE:
      if (value < 0 || value > 100) return BDSS_ERR_INVALID_ARG;
      h->max_refine = (int)value;
      return BDSS_OK;
    case BDSS_OPT_TARGET_BERR_E18:
      if (value < 1) return BDSS_ERR_INVALID_ARG;
      h->target = (double)value * 1e-18;
      return BDSS_OK;
    case BDSS_OPT_DEBUG_SKIP_ARRIVE:
      if (value < 0) return BDSS_ERR_INVALID_ARG;
      h->skip_barrier = (int)value;
      return BDSS_OK;
    case BDSS_OPT_DEBUG_GUARDS:
      if (value != 0 && value != 1) return BDSS_ERR_INVALID_ARG;
      h->debug_guards = (int)value;
      return BDSS_OK;
    case BDSS_OPT_REFINE_KRYLOV:
      if (value < 0 || value > 2) return BDSS_ERR_INVALID_ARG;
      h->krylov = (int)value;
      return BDSS_OK;
    case BDSS_OPT_MAX_KRYLOV_ITERS:
      if (value < 1 || value > 100000) return BDSS_ERR_INVALID_ARG;
      h->max_krylov = (int)value;
      return BDSS_OK;
    case BDSS_OPT_NSTAR: {
      if (value < 1 || value > kNStarMax) return BDSS_ERR_INVALID_ARG;
      // the serial sweep stages two blocks and the vectors in FP64
      const size_t need = ((size_t)(2 * h->n + h->d_max) * ldstride(h->n) + 8) * sizeof(double);
      if (value > 1 && (h->large || is_mixed(h) || need > h->smem)) return BDSS_ERR_UNSUPPORTED;
      h->nstar = (int)value;
      make_plan(h->plan, h->N, h->n, h->nstar);
      h->factored = false;
      return BDSS_OK;
    }
    case BDSS_OPT_SMALL_CLUSTER:
      if (value < -1 || value > 1) return BDSS_ERR_INVALID_ARG;
      if (value == 1 && h->small_cluster < 2) return BDSS_ERR_UNSUPPORTED;
      h->small_opt = (int)value;
      return BDSS_OK;
    case BDSS_OPT_SHIFT:
      if (value != 0 && value != 1) return BDSS_ERR_INVALID_ARG;
      h->shift_on = (int)value;
      return BDSS_OK;
    case BDSS_OPT_SCHUR_EMU:
      if (value != 0 && value != 1) return BDSS_ERR_INVALID_ARG;
      if (value && !h->schur_emu_ready) return BDSS_ERR_UNSUPPORTED;
      h->schur_emu_on = (int)value;
      return BDSS_OK;
    case BDSS_OPT_RESIDUAL_EMU:
      if (value != 0 && value != 1) return BDSS_ERR_INVALID_ARG;
      if (value && !h->emu_ready) return BDSS_ERR_UNSUPPORTED;
      h->emu_on = (int)value;
      h->norm_valid = false;  // the two residual paths form ||A||_inf alike, but afresh
      return BDSS_OK;
    case BDSS_OPT_KERNEL_TIMING:
      if (value != 0 && value != 1) return BDSS_ERR_INVALID_ARG;
      if (value && h->kt_ev.empty()) {
        h->kt_ev.assign(2 * kKtPairs, nullptr);
        for (auto &ev : h->kt_ev)
          if (cudaEventCreate(&ev) != cudaSuccess) {
            const cudaError_t err = cudaGetLastError();
            for (auto &e2 : h->kt_ev)
              if (e2) cudaEventDestroy(e2);
            h->kt_ev.clear();
            return cuda_fail(err);
          }
        h->kt_pair_cls.assign(kKtPairs, 0);
        h->kt_pair_n.assign(kKtPairs, 0);
      }
      h->ktiming = (int)value;
      kt_reset(h);
      return BDSS_OK;
    case BDSS_OPT_DEBUG_CORRUPT_GUARD: {
      // test hook: overwrite one byte of buffer `value`'s guard band from the host
      if (value < 1 || value > (int64_t)h->guards.size()) return BDSS_ERR_INVALID_ARG;
      const auto &g = h->guards[(size_t)value - 1];
      if (cudaMemset(static_cast<char *>(g.base) + g.bytes, 0, 1) != cudaSuccess) return cuda_fail(cudaGetLastError());
      return BDSS_OK;
    }
  }
  return BDSS_ERR_INVALID_ARG;
}

// Can the device read p in place?  Device and managed memory; page-locked
// host memory mapped at the same address (unified addressing); other host
// memory only where the device reads pageable memory.
static bool device_readable(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
    case cudaMemoryTypeManaged:
      return true;
    case cudaMemoryTypeHost:
      return at.devicePointer == p;
    default: {
      int dev = 0, pageable = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      return pageable != 0;
    }
  }
}

static bool device_memory(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static bdss_status check_factor_args(bdss_ctx *h, const double *A_diag, const double *A_sub) {
  if (!A_diag || !aligned16(A_diag) || !device_readable(A_diag)) return BDSS_ERR_INVALID_ARG;
  if (h->N > 1 && (!A_sub || !aligned16(A_sub) || !device_readable(A_sub))) return BDSS_ERR_INVALID_ARG;
  return BDSS_OK;
}

static bdss_status check_solve_args(bdss_ctx *h, const double *B, double *X, int d) {
  if (!B || !X || !aligned16(B) || !aligned16(X)) return BDSS_ERR_INVALID_ARG;
  if (d < 1 || d > h->d_max) return BDSS_ERR_INVALID_ARG;
  if (!device_readable(B) || !device_memory(X)) return BDSS_ERR_INVALID_ARG;
  return BDSS_OK;
}

static void info_init(bdss_info *info) {
  if (!info) return;
  info->level = -1;
  info->block = -1;
  info->iters = 0;
  info->reserved = 0;
  info->backward_err = -1.0;
}

// Factor (and, if B != NULL, the first solve) -- both precisions.
static bdss_status factor_impl(bdss_ctx *h, const double *A_diag, const double *A_sub, const double *B, double *X,
                               int d, bdss_info *info) {
  h->factored = false;
  h->launches = 0;
  h->barriers = 0;
  kt_reset(h);
  h->kt_cls = BDSS_KT_FACTOR;
  const bool rhs = (B != nullptr);
  const bool small = use_small(h);
  cudaError_t e = small ? cudaSuccess : reset_status(h);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!is_mixed(h)) {
    Args<double> a = base_args<double>(h);
    a.A_diag = A_diag;
    a.A_sub = A_sub;
    if (rhs) {
      a.d = d;
      a.B64 = B;
      a.Y = X;
    }
    e = small ? run_small(h, a, true, rhs) : run_levels<double>(h, a, true, rhs);
  } else {
    Args<float> a = base_args<float>(h);
    a.A_diag = A_diag;
    a.A_sub = A_sub;
    if (rhs) {
      a.d = d;
      a.B64 = B;
      a.Y = h->Y32;
      a.X64 = X;
      a.x_accumulate = 0;
    }
    e = run_levels<float>(h, a, true, rhs);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  bdss_status st = small ? finish_small(h, info) : finish(h, info);
  h->shift_used = 0.0;
  if (st == BDSS_ERR_NOT_SPD && is_mixed(h) && h->shift_on) {
    // kappa(A) u_32 near or above one: an FP32 pivot failed.  Factor
    // A + sigma diag(A) instead (Higham and Pranesh's shifted low-precision
    // Cholesky), sigma = 2^-20 (about 8 u_32) growing 16x per failure up to
    // 2^-4; the FP64 CG refinement on the unshifted A, preconditioned by these
    // factors, absorbs the shift.
    if (!h->Ashift) {
      t_alloc_count = 0;
      if (!ws_alloc(h, (void **)&h->Ashift, (size_t)h->N * h->n * h->n * sizeof(double))) {
        cudaGetLastError();
        h->Ashift = nullptr;
        return BDSS_ERR_ALLOC;
      }
    }
    for (double sigma = 0x1p-20; sigma <= 0x1p-4 && st == BDSS_ERR_NOT_SPD; sigma *= 16.0) {
      e = reset_status(h);
      if (e == cudaSuccess) e = launch_shift_diag(h->N, h->n, A_diag, sigma, h->Ashift, h->sms, h->stream);
      h->launches += 1;
      Args<float> a = base_args<float>(h);
      a.A_diag = h->Ashift;
      a.A_sub = A_sub;
      if (rhs) {
        a.d = d;
        a.B64 = B;
        a.Y = h->Y32;
        a.X64 = X;
        a.x_accumulate = 0;
      }
      if (e == cudaSuccess) e = run_levels<float>(h, a, true, rhs);
      if (e != cudaSuccess) return cuda_fail(e);
      st = finish(h, info);
      if (st == BDSS_OK) h->shift_used = sigma;
    }
    if (st == BDSS_OK && info) {
      info->level = -1;
      info->block = -1;
    }
  }
  if (st != BDSS_OK) return st;
  h->norm_valid = false;  // ||A||_inf comes with the first residual
  h->emu_sliced = false;  // the sliced operator is rebuilt from the new A
  h->A_diag = A_diag;
  h->A_sub = A_sub;
  h->factored = true;
  return BDSS_OK;
}

// Mixed precision: X already holds the FP32 solve; refine with FP64 residuals.
// Backward error ||B - A X||_inf / (||A||_inf ||X||_inf) of the current X from
// the FP64 residual kernel, which also leaves the residual in R32 (FP32) for a
// plain correction and forms ||A||_inf on its first call.
// Slice the operator for the tensor-core residual if this factorisation has
// not been sliced yet; forms ||A||_inf into the status word (reset before).
static cudaError_t emu_slice_if_needed(bdss_ctx *h) {
  if (h->emu_sliced) return cudaSuccess;
  kt_begin(h, BDSS_KT_SLICE);
  const cudaError_t e = launch_emu_slice_operator(h->N, h->n, h->A_diag, h->A_sub, h->emu, h->dst, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (e == cudaSuccess) h->emu_sliced = true;
  return e;
}

static bool use_emu(const bdss_ctx *h, int d) { return h->emu_on && d <= kEmuDp; }

static bdss_status residual_berr(bdss_ctx *h, const double *B, const double *X, int d, double *berr) {
  cudaError_t e = reset_status(h);
  const bool emu = use_emu(h, d);
  int with_norm = h->norm_valid ? 0 : 1;
  if (emu && (!h->emu_sliced || !h->norm_valid)) {
    h->emu_sliced = false;
    if (e == cudaSuccess) e = emu_slice_if_needed(h);  // its ||A||_inf lands in nrm[2]
    with_norm = 1;
  } else if (emu) {
    with_norm = 0;
  }
  kt_begin(h, BDSS_KT_RESIDUAL);
  if (e == cudaSuccess && emu)
    e = launch_emu_residual(h->N, h->n, d, X, B, h->R32, nullptr, h->emu, h->dst, h->timeout_ns, h->sms, h->stream);
  else if (e == cudaSuccess)
    e = h->large ? launch_residual_rows(h->N, h->n, d, h->A_diag, h->A_sub, X, B, h->R32, h->dst, with_norm,
                                        (int)std::min<long long>(h->N, 2LL * h->sms), h->stream)
                 : launch_residual(h->N, h->n, d, h->A_diag, h->A_sub, X, B, h->R32, h->dst, with_norm,
                                   grid_for(h, h->N) * 2, h->stream);
  kt_end(h, 1);
  h->launches += 1;
  if (e != cudaSuccess) return cuda_fail(e);
  bdss_status st = finish(h, nullptr);
  if (st != BDSS_OK) return st;
  if (with_norm) {
    uint64_t bits = h->hst->nrm[2];
    memcpy(&h->normA, &bits, sizeof(double));
    h->norm_valid = true;
  }
  double rn, xn;
  uint64_t b0 = h->hst->nrm[0], b1 = h->hst->nrm[1];
  memcpy(&rn, &b0, sizeof(double));
  memcpy(&xn, &b1, sizeof(double));
  const double den = h->normA * xn;
  *berr = den > 0 ? rn / den : (rn == 0 ? 0.0 : INFINITY);
  return BDSS_OK;
}

// The CG vectors and scalars, allocated on the first CG refinement of the
// handle (allocations counted per call for the allocation-failure hook).
static bdss_status krylov_alloc(bdss_ctx *h) {
  const size_t vec = (size_t)h->N * h->n * h->d_max * sizeof(double);
  t_alloc_count = 0;
  double **bufs[4] = {&h->kr_R, &h->kr_Z, &h->kr_P, &h->kr_Q};
  for (double **b : bufs)
    if (!*b && !ws_alloc(h, (void **)b, vec)) return BDSS_ERR_ALLOC;
  if (!h->kr_part && !ws_alloc(h, (void **)&h->kr_part, kPartWords * sizeof(double))) return BDSS_ERR_ALLOC;
  if (!h->kr_sc && !ws_alloc(h, (void **)&h->kr_sc, kScWords * sizeof(double))) return BDSS_ERR_ALLOC;
  return BDSS_OK;
}

// z = M^-1 r: the FP32 substitutions on the stored factors, FP64 in and out.
static bdss_status apply_precond(bdss_ctx *h, int d) {
  cudaError_t e = reset_status(h);
  Args<float> a = base_args<float>(h);
  a.d = d;
  a.B64 = h->kr_R;
  a.Y = h->Y32;
  a.X64 = h->kr_Z;
  a.x_accumulate = 0;
  h->kt_cls = BDSS_KT_KRYLOV;
  if (e == cudaSuccess) e = run_levels<float>(h, a, false, true);
  if (e != cudaSuccess) return cuda_fail(e);
  return finish(h, nullptr);
}

// One cycle of preconditioned CG on A dX = B - A X from the current X, which
// is updated in place.  Stops when the recursively updated residual meets half
// the target backward error, when it has not halved its best value for
// kCgStall iterations, or after max_krylov iterations.
static bdss_status krylov_cycle(bdss_ctx *h, const double *B, double *X, int d) {
  constexpr int kCgStall = 50;
  const long long rows = h->N * h->n;
  const int gD = col_dots_grid(rows, d), gU = pcg_update_grid(rows);
  cudaStream_t s = h->stream;
  double *R = h->kr_R, *Z = h->kr_Z, *P = h->kr_P, *Q = h->kr_Q, *part = h->kr_part, *sc = h->kr_sc;
  kt_begin(h, BDSS_KT_KRYLOV);
  cudaError_t e = launch_btd_apply(h->N, h->n, d, h->A_diag, h->A_sub, X, B, R, h->sms, s);  // r = B - A X
  kt_end(h, 1);
  h->launches += 1;
  if (e != cudaSuccess) return cuda_fail(e);
  bdss_status st = apply_precond(h, d);
  if (st != BDSS_OK) return st;
  kt_begin(h, BDSS_KT_KRYLOV);
  e = launch_col_dots(rows, d, Z, R, nullptr, nullptr, part, gD, s);
  if (e == cudaSuccess) e = launch_pcg_scalars(gD, d, part, kPcgStart, sc, s);
  if (e == cudaSuccess) e = launch_pcg_direction(rows, d, sc, Z, P, 1, h->sms, s);
  kt_end(h, 3);
  h->launches += 3;
  if (e != cudaSuccess) return cuda_fail(e);
  double best = INFINITY;
  int since_best = 0;
  for (int k = 0; k < h->max_krylov; ++k) {
    kt_begin(h, BDSS_KT_KRYLOV);
    e = launch_btd_apply(h->N, h->n, d, h->A_diag, h->A_sub, P, nullptr, Q, h->sms, s);  // q = A p
    if (e == cudaSuccess) e = launch_col_dots(rows, d, P, Q, nullptr, nullptr, part, gD, s);
    if (e == cudaSuccess) e = launch_pcg_scalars(gD, d, part, kPcgAlpha, sc, s);
    if (e == cudaSuccess) e = launch_pcg_update(rows, d, sc, P, Q, X, R, part, gU, s);
    if (e == cudaSuccess) e = launch_pcg_scalars(gU, d, part, kPcgNorms, sc, s);
    double nrm[2] = {0.0, 0.0};
    kt_end(h, 5);
    if (e == cudaSuccess) e = cudaMemcpyAsync(nrm, sc + kScNorm, sizeof(nrm), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    kt_harvest(h);
    h->launches += 5;
    if (e != cudaSuccess) return cuda_fail(e);
    ++h->last_cg;
    const double den = h->normA * nrm[1];
    const double est = den > 0 ? nrm[0] / den : (nrm[0] == 0 ? 0.0 : INFINITY);
    if (!(est < INFINITY) || est <= 0.5 * h->target) break;
    if (est < 0.5 * best) {
      best = est;
      since_best = 0;
    } else if (++since_best >= kCgStall) {
      break;
    }
    st = apply_precond(h, d);  // z = M^-1 r
    if (st != BDSS_OK) return st;
    kt_begin(h, BDSS_KT_KRYLOV);
    e = launch_col_dots(rows, d, Z, R, Z, Q, part, gD, s);
    if (e == cudaSuccess) e = launch_pcg_scalars(gD, d, part, kPcgBeta, sc, s);
    if (e == cudaSuccess) e = launch_pcg_direction(rows, d, sc, Z, P, 0, h->sms, s);
    kt_end(h, 3);
    h->launches += 3;
    if (e != cudaSuccess) return cuda_fail(e);
  }
  return BDSS_OK;
}

// Mixed precision: refine X (the FP32 solution, stored in FP64) until its
// backward error meets the target.  Plain refinement first (X += M^-1 r with
// the FP32 residual, at most max_refine steps); when that stalls -- kappa(A)
// u_32 near or above one -- or runs out of steps, or from the start (option),
// cycles of FP64 CG preconditioned by M.  max_refine = 0 means no correction
// of either kind.
static bdss_status refine(bdss_ctx *h, const double *B, double *X, int d, bdss_info *info) {
  constexpr int kMaxCgCycles = 4;
  double prev = INFINITY, berr = -1.0;
  int cycles = 0;
  bdss_status result = BDSS_ERR_NO_CONVERGENCE;
  h->last_plain = 0;
  h->last_cg = 0;
  for (int it = 0;; ++it) {
    bdss_status st = residual_berr(h, B, X, d, &berr);
    if (st != BDSS_OK) return st;
    if (berr <= h->target) { result = BDSS_OK; break; }
    const bool stalled = it > 0 && !(berr < 0.5 * prev);
    const bool plain_done = stalled || it >= h->max_refine;
    // shifted factors are no accurate solver of A: CG from the first correction
    const bool cg = cycles > 0 || h->krylov == 2 || (h->krylov == 1 && (plain_done || h->shift_used > 0));
    if (!cg) {
      if (plain_done) break;
      prev = berr;
      // correction: solve A dX = r in FP32, X += dX (FP64), fused in the downward pass
      cudaError_t e = reset_status(h);
      Args<float> a = base_args<float>(h);
      a.d = d;
      a.Bt = h->R32;
      a.Y = h->Y32;
      a.X64 = X;
      a.x_accumulate = 1;
      h->kt_cls = BDSS_KT_CORRECTION;
      if (e == cudaSuccess) e = run_levels<float>(h, a, false, true);
      if (e != cudaSuccess) return cuda_fail(e);
      st = finish(h, nullptr);
      if (st != BDSS_OK) return st;
      ++h->last_plain;
      continue;
    }
    if (h->max_refine == 0 || cycles >= kMaxCgCycles || (cycles > 0 && stalled)) break;
    prev = berr;
    st = krylov_alloc(h);
    if (st == BDSS_OK) st = krylov_cycle(h, B, X, d);
    if (st != BDSS_OK) return st;
    ++cycles;
  }
  if (info) {
    info->iters = h->last_plain + h->last_cg;
    info->backward_err = berr;
  }
  return result;
}

bdss_status bdss_factor(bdss_handle h, const double *A_diag, const double *A_sub, bdss_info *info) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  info_init(info);
  bdss_status st = check_factor_args(h, A_diag, A_sub);
  if (st != BDSS_OK) return st;
  return factor_impl(h, A_diag, A_sub, nullptr, nullptr, 0, info);
}

bdss_status bdss_solve(bdss_handle h, const double *B, double *X, int32_t d, bdss_info *info) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  info_init(info);
  bdss_status st = check_solve_args(h, B, X, d);
  if (st != BDSS_OK) return st;
  if (!h->factored) return BDSS_ERR_NOT_FACTORED;
  h->launches = 0;
  h->barriers = 0;
  kt_reset(h);
  h->kt_cls = BDSS_KT_SOLVE;
  const bool small = use_small(h);
  cudaError_t e = small ? cudaSuccess : reset_status(h);
  if (e != cudaSuccess) return cuda_fail(e);
  if (!is_mixed(h)) {
    Args<double> a = base_args<double>(h);
    a.d = d;
    a.B64 = B;
    a.Y = X;
    e = small ? run_small(h, a, false, true) : run_levels<double>(h, a, false, true);
    if (e != cudaSuccess) return cuda_fail(e);
    return small ? finish_small(h, info) : finish(h, info);
  }
  if (X == B) return BDSS_ERR_INVALID_ARG;  // the residual needs B after X is written
  Args<float> a = base_args<float>(h);
  a.d = d;
  a.B64 = B;
  a.Y = h->Y32;
  a.X64 = X;
  a.x_accumulate = 0;
  e = run_levels<float>(h, a, false, true);
  if (e != cudaSuccess) return cuda_fail(e);
  st = finish(h, info);
  if (st != BDSS_OK) return st;
  return refine(h, B, X, d, info);
}

bdss_status bdss_factor_solve(bdss_handle h, const double *A_diag, const double *A_sub, const double *B, double *X,
                              int32_t d, bdss_info *info) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  info_init(info);
  bdss_status st = check_factor_args(h, A_diag, A_sub);
  if (st == BDSS_OK) st = check_solve_args(h, B, X, d);
  if (st != BDSS_OK) return st;
  if (is_mixed(h) && X == B) return BDSS_ERR_INVALID_ARG;
  st = factor_impl(h, A_diag, A_sub, B, X, d, info);
  if (st != BDSS_OK || !is_mixed(h)) return st;
  return refine(h, B, X, d, info);
}

bdss_status bdss_logdet(bdss_handle h, double *out) {
  if (!h || !out) return BDSS_ERR_INVALID_ARG;
  if (!h->factored) return BDSS_ERR_NOT_FACTORED;
  const long long total = h->N * h->n;
  int grid = (int)((total + kThreads - 1) / kThreads);
  if (grid > kLogdetGrid) grid = kLogdetGrid;
  cudaError_t e = is_mixed(h)
                      ? launch_logdet<float>(h->N, h->n, h->plan.L, (const float *)h->Ld, h->Ltop, h->partial, grid,
                                             h->stream)
                      : launch_logdet<double>(h->N, h->n, h->plan.L, (const double *)h->Ld, h->Ltop, h->partial,
                                              grid, h->stream);
  double part[kLogdetGrid];
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(part, h->partial, grid * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  double s = 0.0;
  for (int i = 0; i < grid; ++i) s += part[i];
  *out = s;
  return BDSS_OK;
}

bdss_status bdss_adjoint_grads(bdss_handle h, const double *Lambda, const double *X, int32_t d, double *dA_diag,
                               double *dA_sub) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  if (!Lambda || !X || !dA_diag || !aligned16(Lambda) || !aligned16(X) || !aligned16(dA_diag))
    return BDSS_ERR_INVALID_ARG;
  if (h->N > 1 && (!dA_sub || !aligned16(dA_sub))) return BDSS_ERR_INVALID_ARG;
  if (d < 1 || d > h->d_max) return BDSS_ERR_INVALID_ARG;
  cudaError_t e = launch_adjoint_grads(h->N, h->n, d, Lambda, X, dA_diag, dA_sub, grid_for(h, h->N) * 2, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return BDSS_OK;
}

bdss_status bdss_kalman_assemble(int64_t N, int32_t n, int32_t m, int32_t rinv_diagonal,
                                 const double *G, const double *H, const double *Qinv,
                                 const double *Rinv, const double *z, const double *zeta,
                                 double *A_diag, double *A_sub, double *B, void *cuda_stream) {
  if (N < 1 || n < 1 || m < 1 || (rinv_diagonal != 0 && rinv_diagonal != 1)) return BDSS_ERR_INVALID_ARG;
  if (n > kMaxNLarge || m > 4096 || N > kalman_max_steps(n, m)) return BDSS_ERR_UNSUPPORTED;
  auto ok_in = [](const void *p) { return p && aligned16(p) && device_memory(p); };
  if (!ok_in(G) || !ok_in(H) || !ok_in(Qinv) || !ok_in(Rinv) || !ok_in(A_diag)) return BDSS_ERR_INVALID_ARG;
  if (N > 1 && !ok_in(A_sub)) return BDSS_ERR_INVALID_ARG;
  if (B && (!ok_in(B) || !ok_in(z))) return BDSS_ERR_INVALID_ARG;
  if (B && zeta && !ok_in(zeta)) return BDSS_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  KalmanArgs a{};
  a.N = N;
  a.n = n;
  a.m = m;
  a.rinv_diag = rinv_diagonal;
  a.G = G;
  a.H = H;
  a.Qinv = Qinv;
  a.Rinv = Rinv;
  a.z = B ? z : nullptr;
  a.zeta = B ? zeta : nullptr;
  a.A_diag = A_diag;
  a.A_sub = N > 1 ? A_sub : nullptr;
  a.B = B;
  const size_t words = (size_t)N * ((size_t)m * n + m + n);
  void *ws = nullptr;
  t_alloc_count = 0;
  if (inject_alloc_failure() || cudaMallocAsync(&ws, words * sizeof(double), s) != cudaSuccess) {
    cudaGetLastError();
    return BDSS_ERR_ALLOC;
  }
  a.U = static_cast<double *>(ws);
  a.v = a.U + (size_t)N * m * n;
  a.w = a.v + (size_t)N * m;
  cudaError_t e = launch_kalman_assemble(a, s);
  cudaError_t f = cudaFreeAsync(ws, s);
  if (e == cudaSuccess) e = f;
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  return BDSS_OK;
}

bdss_status bdss_tc_selftest(double *max_rel_err) {
  if (!max_rel_err) return BDSS_ERR_INVALID_ARG;
  int st = 0;
  cudaError_t e = run_tc_selftest(max_rel_err, &st);
  if (e != cudaSuccess) return cuda_fail(e);
  return (bdss_status)st;
}

bdss_status bdss_debug_fail_alloc(int32_t k) {
  if (k < 0) return BDSS_ERR_INVALID_ARG;
  g_fail_alloc.store(k);
  return BDSS_OK;
}

bdss_status bdss_factor_shift(bdss_handle h, double *sigma) {
  if (!h || !sigma) return BDSS_ERR_INVALID_ARG;
  *sigma = h->shift_used;
  return BDSS_OK;
}

bdss_status bdss_last_refine_stats(bdss_handle h, int32_t *plain_steps, int32_t *cg_iters) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  if (plain_steps) *plain_steps = h->last_plain;
  if (cg_iters) *cg_iters = h->last_cg;
  return BDSS_OK;
}

bdss_status bdss_get_launch_config(bdss_handle h, int32_t *ctas_per_sm, int32_t *sm_count, int64_t *smem_bytes) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  if (ctas_per_sm) *ctas_per_sm = h->bps;
  if (sm_count) *sm_count = h->sms;
  if (smem_bytes) *smem_bytes = (int64_t)h->smem;
  return BDSS_OK;
}

bdss_status bdss_last_trace(bdss_handle h, int64_t *release_ns, int32_t capacity, int32_t *count) {
  if (!h || capacity < 0 || (capacity > 0 && !release_ns)) return BDSS_ERR_INVALID_ARG;
  const int c = std::min(h->trace_count, (int)capacity);
  for (int i = 0; i < c; ++i) release_ns[i] = h->trace[i];
  if (count) *count = h->trace_count;
  return BDSS_OK;
}

// Stream-ordered temporary of the partitioned-solve entry points (counted
// by the allocation-failure hook).
static bool tmp_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  if (inject_alloc_failure() || cudaMallocAsync(p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

static bool opt_block_ok(const double *p) { return !p || (aligned16(p) && device_readable(p)); }

bdss_status bdss_chunk_reduce(bdss_handle h, const double *A_diag, const double *A_sub, const double *A_left,
                              const double *A_right, const double *B, int32_t d, double *S, double *b_hat,
                              bdss_info *info) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  info_init(info);
  if (is_mixed(h)) return BDSS_ERR_UNSUPPORTED;
  bdss_status st = check_factor_args(h, A_diag, A_sub);
  if (st != BDSS_OK) return st;
  if (!B || !aligned16(B) || !device_readable(B) || d < 1 || d > h->d_max) return BDSS_ERR_INVALID_ARG;
  if (!S || !b_hat || !aligned16(S) || !aligned16(b_hat) || !device_memory(S) || !device_memory(b_hat))
    return BDSS_ERR_INVALID_ARG;
  if (!opt_block_ok(A_left) || !opt_block_ok(A_right)) return BDSS_ERR_INVALID_ARG;
  st = factor_impl(h, A_diag, A_sub, nullptr, nullptr, 0, info);
  if (st != BDSS_OK) return st;
  const long long N = h->N;
  const int n = h->n, dc = std::min(n, h->d_max);
  const size_t nn = (size_t)n * n;
  cudaStream_t s = h->stream;
  double *Z = nullptr, *Zs = nullptr;
  const size_t words = (size_t)N * n * std::max(dc, (int)d);
  t_alloc_count = 0;
  if (!tmp_alloc((void **)&Z, words * sizeof(double), s) || !tmp_alloc((void **)&Zs, words * sizeof(double), s)) {
    if (Z) cudaFreeAsync(Z, s);
    return BDSS_ERR_ALLOC;
  }
  cudaError_t e = cudaMemsetAsync(S, 0, 3 * nn * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b_hat, 0, (size_t)2 * n * d * sizeof(double), s);
  const double *last = nullptr;
  // y = A_I^{-1} B, then b_hat = [A_left^T y_first, A_right y_last]
  if (e == cudaSuccess) {
    st = bdss_solve(h, B, Zs, d, nullptr);
    if (st != BDSS_OK) e = cudaErrorUnknown;
  }
  last = Zs + (size_t)(N - 1) * n * d;
  if (e == cudaSuccess && A_left) e = launch_chunk_product(n, d, A_left, 1, Zs, b_hat, d, 0, s);
  if (e == cudaSuccess && A_right) e = launch_chunk_product(n, d, A_right, 0, last, b_hat + (size_t)n * d, d, 0, s);
  // the couplings, dc columns at a time:
  //   S_LL = A_left^T (A_I^{-1})_{first,first} A_left, S_RL = A_right (A_I^{-1})_{last,first} A_left,
  //   S_RR = A_right (A_I^{-1})_{last,last} A_right^T
  for (int c0 = 0; c0 < n && e == cudaSuccess && st == BDSS_OK; c0 += dc) {
    const int m = std::min(dc, n - c0);
    const double *zl = Zs + (size_t)(N - 1) * n * m;
    if (A_left) {
      e = launch_chunk_rhs(N, n, m, 0, A_left, 0, c0, Z, s);
      if (e == cudaSuccess) st = bdss_solve(h, Z, Zs, m, nullptr);
      if (e == cudaSuccess && st == BDSS_OK) e = launch_chunk_product(n, m, A_left, 1, Zs, S, n, c0, s);
      if (e == cudaSuccess && st == BDSS_OK && A_right)
        e = launch_chunk_product(n, m, A_right, 0, zl, S + 2 * nn, n, c0, s);
    }
    if (A_right && e == cudaSuccess && st == BDSS_OK) {
      e = launch_chunk_rhs(N, n, m, (int)(N - 1), A_right, 1, c0, Z, s);
      if (e == cudaSuccess) st = bdss_solve(h, Z, Zs, m, nullptr);
      if (e == cudaSuccess && st == BDSS_OK) e = launch_chunk_product(n, m, A_right, 0, zl, S + nn, n, c0, s);
    }
  }
  cudaFreeAsync(Z, s);
  cudaFreeAsync(Zs, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (st != BDSS_OK) return st;
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e);
  return BDSS_OK;
}

bdss_status bdss_chunk_backsolve(bdss_handle h, const double *B, const double *A_left, const double *A_right,
                                 const double *x_left, const double *x_right, int32_t d, double *X) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  if (is_mixed(h)) return BDSS_ERR_UNSUPPORTED;
  bdss_status st = check_solve_args(h, B, X, d);
  if (st != BDSS_OK) return st;
  if (!opt_block_ok(A_left) || !opt_block_ok(A_right)) return BDSS_ERR_INVALID_ARG;
  if ((A_left && !opt_block_ok(x_left)) || (A_right && !opt_block_ok(x_right)) || (A_left && !x_left) ||
      (A_right && !x_right))
    return BDSS_ERR_INVALID_ARG;
  if (!h->factored) return BDSS_ERR_NOT_FACTORED;
  cudaStream_t s = h->stream;
  double *Bp = nullptr;
  t_alloc_count = 0;
  if (!tmp_alloc((void **)&Bp, (size_t)h->N * h->n * d * sizeof(double), s)) return BDSS_ERR_ALLOC;
  cudaError_t e = launch_chunk_fix_rhs(h->N, h->n, d, B, A_left, A_right, x_left, x_right, Bp, s);
  if (e == cudaSuccess) st = bdss_solve(h, Bp, X, d, nullptr);
  cudaFreeAsync(Bp, s);
  const cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e);
  if (st != BDSS_OK) return st;
  if (e2 != cudaSuccess) return cuda_fail(e2);
  return BDSS_OK;
}

bdss_status bdss_residual(bdss_handle h, const double *B, const double *X, int32_t d, double *R) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  if (!B || !X || !R || !aligned16(B) || !aligned16(X) || !aligned16(R)) return BDSS_ERR_INVALID_ARG;
  if (d < 1 || d > h->d_max) return BDSS_ERR_INVALID_ARG;
  if (!device_readable(B) || !device_readable(X) || !device_memory(R)) return BDSS_ERR_INVALID_ARG;
  if (!h->factored) return BDSS_ERR_NOT_FACTORED;
  cudaError_t e = reset_status(h);
  if (use_emu(h, d)) {
    if (e == cudaSuccess) e = emu_slice_if_needed(h);
    if (e == cudaSuccess)
      e = launch_emu_residual(h->N, h->n, d, X, B, nullptr, R, h->emu, h->dst, h->timeout_ns, h->sms, h->stream);
  } else if (e == cudaSuccess) {
    e = launch_btd_apply(h->N, h->n, d, h->A_diag, h->A_sub, X, B, R, h->sms, h->stream);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  return finish(h, nullptr);
}

bdss_status bdss_last_kernel_times(bdss_handle h, double *ms, int64_t *launches, int32_t classes) {
  if (!h || classes < 0 || (classes > 0 && !ms)) return BDSS_ERR_INVALID_ARG;
  const int c = std::min((int)classes, (int)BDSS_KT_CLASSES);
  for (int i = 0; i < c; ++i) {
    ms[i] = h->kt_ms[i];
    if (launches) launches[i] = h->kt_n[i];
  }
  return BDSS_OK;
}

const char *bdss_last_cuda_error(void) { return cudaGetErrorString(g_last_cuda_error); }

bdss_status bdss_last_launch_stats(bdss_handle h, int64_t *kernel_launches, int64_t *grid_barriers) {
  if (!h) return BDSS_ERR_INVALID_ARG;
  if (kernel_launches) *kernel_launches = h->launches;
  if (grid_barriers) *grid_barriers = h->barriers;
  return BDSS_OK;
}

}  // extern "C"
