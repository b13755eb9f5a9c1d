// Batched solver: K independent SPD block-tridiagonal systems of uneven N_k
// and n_k, factored and solved (FP64) in ONE launch driven by a device work
// queue over (instance, stage, item range) tasks -- the batch notation
// {A^(k)} of Sec. 3.2 carried across all levels of Algorithms 4 and 7.
//
// Stages of instance k (L_k levels): A(0), B(0), A(1), B(1), ..., A(L-1),
// B(L-1), top, C(L-1), ..., C(0).  Stage s of an instance may start once
// stage s-1 of the same instance has completed all its items; instances do
// not wait on one another.  Tasks are stored stage-major (every instance's
// stage 0, then every instance's stage 1, ...), and CTAs take them from an
// atomic counter in that order, so every task's prerequisites were taken
// earlier by CTAs that are running: the queue always makes progress without
// co-residency of the grid.  Every wait is still bounded in time.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "../../include/bdss.h"
#include "bdss_launch.h"

using namespace bdss;

namespace {

struct Task {
  int inst;
  int stage;
  long long first;  // first item of the stage in this task
  int count;        // items in this task
  int need;         // items of stage-1 that must be complete (0 for stage 0)
};

struct BatchArgs {
  Args<double> *args;     // per instance
  const Task *tasks;
  long long ntasks;
  unsigned long long *next;
  unsigned int *done;     // per (instance, stage) completed items
  const int *stage_off;   // per instance offset into done
  const int *nstages;     // per instance stage count
  unsigned long long *t0, *t1;  // per instance first-start / last-end (globaltimer, ns)
  long long timeout_ns;
};

__device__ __forceinline__ unsigned ld_acq(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__global__ void __launch_bounds__(kThreads) k_batched(const __grid_constant__ BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_flag, s_ok;
  __shared__ long long s_task;
  double *smem = reinterpret_cast<double *>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) s_task = (long long)atomicAdd(b.next, 1ull);
    __syncthreads();
    const long long t = s_task;
    if (t >= b.ntasks) return;
    const Task tk = b.tasks[t];
    const Args<double> &a = b.args[tk.inst];
    unsigned *done = b.done + b.stage_off[tk.inst];
    if (threadIdx.x == 0) {
      int ok = 1;
      if (tk.stage > 0) {
        const long long t_begin = global_ns();
        unsigned long long spins = 0;
        const unsigned long long cap = 1000000ull + (unsigned long long)(b.timeout_ns / 16);
        while (ld_acq(done + tk.stage - 1) < (unsigned)tk.need) {
          if (ld_relaxed_i32(&a.st->status) != 0) { ok = 0; break; }
          ++spins;
          if ((spins & 31) == 0 && (global_ns() - t_begin > b.timeout_ns || spins > cap)) {
            set_status(a.st, kStTimeout, -1, -1);
            ok = 0;
            break;
          }
          __nanosleep(32);
        }
        __threadfence();
      } else {
        atomicMin(b.t0 + tk.inst, (unsigned long long)global_ns());
      }
      if (ld_relaxed_i32(&a.st->status) != 0) ok = 0;
      s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
      const int L = a.p.L;
      const int st = tk.stage;
      for (long long it = tk.first; it < tk.first + tk.count; ++it) {
        if (st < 2 * L) {
          const int l = st >> 1;
          if ((st & 1) == 0) {
            if (!phaseA(a, l, 2 * it + 1, true, smem, &s_flag)) break;
          } else {
            phaseB(a, l, it, true, smem);
          }
        } else if (st == 2 * L) {
          top_block(a, true, smem, &s_flag);
        } else {
          const int l = L - 1 - (st - 2 * L - 1);
          phaseC(a, l, 2 * it + 1, smem);
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(done + tk.stage, (unsigned)tk.count);
      if (tk.stage == b.nstages[tk.inst] - 1) atomicMax(b.t1 + tk.inst, (unsigned long long)global_ns());
    }
  }
}

long long stage_items(long long N, int L, int s) {
  auto Nl = [&](int l) { return ((N - 1) >> l) + 1; };
  if (s < 2 * L) return (s & 1) == 0 ? Nl(s >> 1) / 2 : (Nl(s >> 1) + 1) / 2;
  if (s == 2 * L) return 1;
  return Nl(L - 1 - (s - 2 * L - 1)) / 2;
}

void plan_of(Plan &p, int64_t N, int n) {
  memset(&p, 0, sizeof(p));
  p.N = N;
  p.n = n;
  p.Nl[0] = N;
  int l = 0;
  while (p.Nl[l] > 1) {
    p.Nl[l + 1] = (p.Nl[l] + 1) / 2;
    p.off[l + 1] = p.off[l] + (p.Nl[l] - 1);
    ++l;
  }
  p.L = l;
}

// Autotuner table: (n_max, d) -> (threads per CTA, items per task).
std::mutex g_tune_mutex;
std::map<std::pair<int, int>, std::pair<int, int>> g_tune_table;

}  // namespace

struct bdss_batch_ctx {
  int K = 0, d = 0, n_max = 0;
  cudaStream_t stream = nullptr;
  std::vector<int64_t> N;
  std::vector<int> n;
  std::vector<Args<double>> host_args;
  // device memory
  Args<double> *d_args = nullptr;
  Task *d_tasks = nullptr;
  unsigned long long *d_next = nullptr;
  unsigned int *d_done = nullptr;
  int *d_stage_off = nullptr, *d_nstages = nullptr;
  unsigned long long *d_t = nullptr;  // t0[K], t1[K]
  DevStatus *d_status = nullptr;      // K
  std::vector<void *> ws;             // per-instance workspace blocks
  int total_stages = 0;
  long long ntasks = 0;
  int threads = 128, items = 1;
  size_t smem = 0;
  int grid = 0;
  bool inputs_set = false;
  cudaGraphExec_t graph = nullptr;
  long long timeout_ns = 10000000000LL;
  DevStatus *h_status = nullptr;       // pinned, K
  unsigned long long *h_t = nullptr;   // pinned, 2K
};

// Queue order.  The instances with the most work (N n^3, the top
// 1/kBatchGroups) form one stage-major sequence; the others form a second
// sequence of groups of ascending work, each group stage-major (within a
// stage, larger instances first).  The two sequences are merged in
// proportion to their work, so the large instances advance through the
// whole launch (their thin last stages end together with the rest), while
// the small ones complete early instead of all instances finishing together
// at the end of a fully stage-major queue.  Tasks never wait on a later
// position of the queue, so every wait ends.
constexpr int kBatchGroups = 8;

static bdss_status batch_build_tasks(bdss_batch_ctx *b) {
  std::vector<int> order(b->K);
  for (int k = 0; k < b->K; ++k) order[k] = k;
  auto work = [&](int k) { return (double)b->N[k] * b->n[k] * b->n[k] * b->n[k]; };
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work(x) < work(y); });
  std::vector<int> nst(b->K), off(b->K);
  int acc = 0;
  for (int k = 0; k < b->K; ++k) {
    nst[k] = 3 * b->host_args[k].p.L + 1;
    off[k] = acc;
    acc += nst[k];
  }
  b->total_stages = acc;
  // stage-major tasks of a group, with their work (items x n^3)
  auto emit = [&](std::vector<int> grp, std::vector<Task> &out, std::vector<double> &w) {
    std::stable_sort(grp.begin(), grp.end(), [&](int x, int y) { return work(x) > work(y); });
    int maxst = 0;
    for (int k : grp) maxst = std::max(maxst, nst[k]);
    for (int s = 0; s < maxst; ++s)
      for (int k : grp) {
        if (s >= nst[k]) continue;
        const int L = b->host_args[k].p.L;
        const long long items = stage_items(b->N[k], L, s);
        const int need = s > 0 ? (int)stage_items(b->N[k], L, s - 1) : 0;
        for (long long f = 0; f < items; f += b->items) {
          Task t;
          t.inst = k;
          t.stage = s;
          t.first = f;
          t.count = (int)std::min<long long>(b->items, items - f);
          t.need = need;
          out.push_back(t);
          w.push_back((double)t.count * b->n[k] * b->n[k] * b->n[k]);
        }
      }
  };
  const int G = std::min(kBatchGroups, b->K);
  const size_t cut = (size_t)b->K * (G - 1) / G;  // instances [cut, K) form the large sequence
  std::vector<Task> big, small;
  std::vector<double> wbig, wsmall;
  emit(std::vector<int>(order.begin() + cut, order.end()), big, wbig);
  for (int g = 0; g < G - 1; ++g)
    emit(std::vector<int>(order.begin() + (size_t)b->K * g / G, order.begin() + (size_t)b->K * (g + 1) / G), small,
         wsmall);
  double tb = 0, ts = 0;
  for (double x : wbig) tb += x;
  for (double x : wsmall) ts += x;
  std::vector<Task> tasks;
  tasks.reserve(big.size() + small.size());
  size_t ib = 0, is = 0;
  double cb = 0, cs = 0;
  while (ib < big.size() || is < small.size()) {
    const bool take_big = is >= small.size() || (ib < big.size() && cb / (tb > 0 ? tb : 1) <= cs / (ts > 0 ? ts : 1));
    if (take_big) {
      cb += wbig[ib];
      tasks.push_back(big[ib++]);
    } else {
      cs += wsmall[is];
      tasks.push_back(small[is++]);
    }
  }
  b->ntasks = (long long)tasks.size();
  cudaFree(b->d_tasks);
  b->d_tasks = nullptr;
  if (cudaMalloc(&b->d_tasks, tasks.size() * sizeof(Task)) != cudaSuccess) return BDSS_ERR_ALLOC;
  cudaError_t e = cudaMemcpy(b->d_tasks, tasks.data(), tasks.size() * sizeof(Task), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !b->d_stage_off) {
    if (cudaMalloc(&b->d_stage_off, b->K * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_nstages, b->K * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_done, (size_t)acc * sizeof(unsigned)) != cudaSuccess)
      return BDSS_ERR_ALLOC;
  }
  if (e == cudaSuccess) e = cudaMemcpy(b->d_stage_off, off.data(), b->K * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_nstages, nst.data(), b->K * sizeof(int), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? BDSS_OK : BDSS_ERR_CUDA;
}

static bdss_status batch_configure(bdss_batch_ctx *b, int threads, int items) {
  if (threads < b->n_max || threads > kThreads || threads % 32) return BDSS_ERR_INVALID_ARG;
  b->threads = threads;
  b->items = items;
  size_t sm = 0;
  int bps = 0;
  cudaError_t e = configure<double>(b->n_max, b->d, &sm, &bps);  // raises the smem limits
  if (e != cudaSuccess) return BDSS_ERR_CUDA;
  // raise the limit once to the device maximum (minus static shared memory),
  // so that batches of different sizes never lower it under one another
  int occ = 0, dev = 0, sms = 0, optin = 0;
  cudaFuncAttributes fa;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, (const void *)k_batched);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void *)k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batched, threads, sm);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || occ < 1) return BDSS_ERR_CUDA;
  b->smem = sm;
  b->grid = occ * sms;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return batch_build_tasks(b);
}

static cudaError_t batch_enqueue(bdss_batch_ctx *b) {
  BatchArgs a;
  a.args = b->d_args;
  a.tasks = b->d_tasks;
  a.ntasks = b->ntasks;
  a.next = b->d_next;
  a.done = b->d_done;
  a.stage_off = b->d_stage_off;
  a.nstages = b->d_nstages;
  a.t0 = b->d_t;
  a.t1 = b->d_t + b->K;
  a.timeout_ns = b->timeout_ns;
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, (size_t)b->total_stages * sizeof(unsigned), b->stream);
  if (e == cudaSuccess)
    e = cudaMemset2DAsync(b->d_status, sizeof(DevStatus), 0, kStatusCoreBytes, (size_t)b->K, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_t, 0xff, (size_t)b->K * sizeof(unsigned long long), b->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(b->d_t + b->K, 0, (size_t)b->K * sizeof(unsigned long long), b->stream);
  if (e != cudaSuccess) return e;
  k_batched<<<b->grid, b->threads, b->smem, b->stream>>>(a);
  return cudaGetLastError();
}

extern "C" {

bdss_status bdss_batch_destroy(bdss_batch b) {
  if (!b) return BDSS_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (void *p : b->ws) cudaFree(p);
  cudaFree(b->d_args);
  cudaFree(b->d_tasks);
  cudaFree(b->d_next);
  cudaFree(b->d_done);
  cudaFree(b->d_stage_off);
  cudaFree(b->d_nstages);
  cudaFree(b->d_t);
  cudaFree(b->d_status);
  if (b->h_status) cudaFreeHost(b->h_status);
  if (b->h_t) cudaFreeHost(b->h_t);
  delete b;
  return BDSS_OK;
}

bdss_status bdss_batch_create(bdss_batch *out, int32_t K, const int64_t *N_k, const int32_t *n_k, int32_t d,
                              void *cuda_stream) {
  if (!out) return BDSS_ERR_INVALID_ARG;
  *out = nullptr;
  if (K < 1 || !N_k || !n_k || d < 1 || d > 64) return BDSS_ERR_INVALID_ARG;
  int n_max = 0;
  for (int k = 0; k < K; ++k) {
    if (N_k[k] < 1 || n_k[k] < 1) return BDSS_ERR_INVALID_ARG;
    if (n_k[k] > kMaxN || N_k[k] > ((int64_t)1 << (kMaxLevels - 2))) return BDSS_ERR_UNSUPPORTED;
    n_max = std::max(n_max, (int)n_k[k]);
  }
  bdss_batch_ctx *b = new (std::nothrow) bdss_batch_ctx();
  if (!b) return BDSS_ERR_ALLOC;
  b->K = K;
  b->d = d;
  b->n_max = n_max;
  b->stream = (cudaStream_t)cuda_stream;
  b->N.assign(N_k, N_k + K);
  b->n.assign(n_k, n_k + K);
  b->host_args.resize(K);
  bool ok = cudaMalloc(&b->d_status, (size_t)K * sizeof(DevStatus)) == cudaSuccess;
  for (int k = 0; ok && k < K; ++k) {
    Args<double> &a = b->host_args[k];
    memset(&a, 0, sizeof(a));
    plan_of(a.p, N_k[k], n_k[k]);
    const size_t nn = (size_t)n_k[k] * n_k[k];
    const size_t slots = (size_t)std::max<long long>(a.p.off[a.p.L], 1);
    const size_t bytes = ((size_t)N_k[k] + slots + 1) * nn * sizeof(double);
    void *p = nullptr;
    ok = cudaMalloc(&p, bytes) == cudaSuccess;
    if (!ok) break;
    b->ws.push_back(p);
    a.Ld = (double *)p;
    a.Wb = a.Ld + (size_t)N_k[k] * nn;
    a.Ltop = a.Wb + slots * nn;
    a.d = d;
    a.st = b->d_status + k;
    a.timeout_ns = b->timeout_ns;
  }
  ok = ok && cudaMalloc(&b->d_args, (size_t)K * sizeof(Args<double>)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_next, sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&b->d_t, (size_t)2 * K * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_status, (size_t)K * sizeof(DevStatus)) == cudaSuccess;
  ok = ok && cudaMallocHost(&b->h_t, (size_t)2 * K * sizeof(unsigned long long)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    bdss_batch_destroy(b);
    return BDSS_ERR_ALLOC;
  }
  // configuration: the tuned one for (n_max, d) if the autotuner has run
  int threads = n_max <= 32 ? 64 : 128, items = 1;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_table.find({n_max, d});
    if (it != g_tune_table.end()) {
      threads = it->second.first;
      items = it->second.second;
    }
  }
  bdss_status st = batch_configure(b, threads, items);
  if (st != BDSS_OK) {
    bdss_batch_destroy(b);
    return st;
  }
  *out = b;
  return BDSS_OK;
}

bdss_status bdss_batch_set_inputs(bdss_batch b, const double *const *A_diag_k, const double *const *A_sub_k,
                                  const double *const *B_k, double *const *X_k) {
  if (!b || !A_diag_k || !A_sub_k || !B_k || !X_k) return BDSS_ERR_INVALID_ARG;
  for (int k = 0; k < b->K; ++k) {
    const bool needs_sub = b->N[k] > 1;
    if (!A_diag_k[k] || !B_k[k] || !X_k[k] || (needs_sub && !A_sub_k[k])) return BDSS_ERR_INVALID_ARG;
    if ((((uintptr_t)A_diag_k[k] | (uintptr_t)B_k[k] | (uintptr_t)X_k[k] |
          (uintptr_t)(needs_sub ? A_sub_k[k] : nullptr)) & 15u) != 0)
      return BDSS_ERR_INVALID_ARG;
    Args<double> &a = b->host_args[k];
    a.A_diag = A_diag_k[k];
    a.A_sub = needs_sub ? A_sub_k[k] : nullptr;
    a.B64 = B_k[k];
    a.Y = X_k[k];
  }
  cudaError_t e = cudaMemcpyAsync(b->d_args, b->host_args.data(), (size_t)b->K * sizeof(Args<double>),
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return BDSS_ERR_CUDA;
  b->inputs_set = true;
  return BDSS_OK;
}

bdss_status bdss_batch_launch(bdss_batch b, int32_t use_graph) {
  if (!b) return BDSS_ERR_INVALID_ARG;
  if (!b->inputs_set) return BDSS_ERR_NOT_FACTORED;
  cudaError_t e;
  if (!use_graph) {
    e = batch_enqueue(b);
    return e == cudaSuccess ? BDSS_OK : BDSS_ERR_CUDA;
  }
  if (!b->graph) {
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return BDSS_ERR_CUDA;
    cudaStream_t saved = b->stream;
    b->stream = cap;
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = batch_enqueue(b);
      e = cudaStreamEndCapture(cap, &g);
      if (e == cudaSuccess) e = e2;
    }
    b->stream = saved;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) {
      b->graph = nullptr;
      return BDSS_ERR_CUDA;
    }
  }
  e = cudaGraphLaunch(b->graph, b->stream);
  return e == cudaSuccess ? BDSS_OK : BDSS_ERR_CUDA;
}

bdss_status bdss_batch_wait(bdss_batch b, bdss_info *info_k, double *latency_us_k) {
  if (!b) return BDSS_ERR_INVALID_ARG;
  cudaError_t e = cudaMemcpy2DAsync(b->h_status, sizeof(DevStatus), b->d_status, sizeof(DevStatus), kStatusCoreBytes,
                                    (size_t)b->K, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->h_t, b->d_t, (size_t)2 * b->K * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                        b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return BDSS_ERR_CUDA;
  unsigned long long t_start = ~0ull;  // first task start of the launch
  for (int k = 0; k < b->K; ++k) t_start = std::min(t_start, b->h_t[k]);
  bdss_status worst = BDSS_OK;
  for (int k = 0; k < b->K; ++k) {
    const int st = b->h_status[k].status;
    if (info_k) {
      info_k[k].level = st == BDSS_ERR_NOT_SPD ? b->h_status[k].level : -1;
      info_k[k].block = st == BDSS_ERR_NOT_SPD ? b->h_status[k].block : -1;
      info_k[k].iters = 0;
      info_k[k].reserved = st;
      info_k[k].backward_err = -1.0;
    }
    if (latency_us_k) {
      const unsigned long long t1 = b->h_t[b->K + k];
      latency_us_k[k] = (t1 >= t_start && t_start != ~0ull) ? (double)(t1 - t_start) * 1e-3 : -1.0;
    }
    if (st != BDSS_OK && worst == BDSS_OK) worst = (bdss_status)st;
  }
  return worst;
}

bdss_status bdss_batch_autotune(bdss_batch b, int32_t reps, int32_t *threads_out, int32_t *items_out) {
  if (!b || reps < 1) return BDSS_ERR_INVALID_ARG;
  if (!b->inputs_set) return BDSS_ERR_NOT_FACTORED;
  const int cand_t[] = {32, 64, 128, 256};
  const int cand_i[] = {1, 2, 4};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return BDSS_ERR_CUDA;
  float best = 1e30f;
  int bt = b->threads, bi = b->items;
  for (int t : cand_t) {
    if (t < b->n_max) continue;
    for (int it : cand_i) {
      if (batch_configure(b, t, it) != BDSS_OK) continue;
      if (batch_enqueue(b) != cudaSuccess) continue;  // warm-up
      cudaEventRecord(e0, b->stream);
      for (int r = 0; r < reps; ++r) batch_enqueue(b);
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bt = t;
        bi = it;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  bdss_status st = batch_configure(b, bt, bi);
  if (st != BDSS_OK) return st;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_table[{b->n_max, b->d}] = {bt, bi};
  }
  if (threads_out) *threads_out = bt;
  if (items_out) *items_out = bi;
  return BDSS_OK;
}

bdss_status bdss_factor_solve_batched(int32_t K, const int64_t *N_k, const int32_t *n_k, int32_t d,
                                      const double *const *A_diag_k, const double *const *A_sub_k,
                                      const double *const *B_k, double *const *X_k, void *cuda_stream,
                                      bdss_info *info_k) {
  bdss_batch b = nullptr;
  bdss_status st = bdss_batch_create(&b, K, N_k, n_k, d, cuda_stream);
  if (st != BDSS_OK) return st;
  st = bdss_batch_set_inputs(b, A_diag_k, A_sub_k, B_k, X_k);
  if (st == BDSS_OK) st = bdss_batch_launch(b, 0);
  if (st == BDSS_OK) st = bdss_batch_wait(b, info_k, nullptr);
  bdss_batch_destroy(b);
  return st;
}

}  // extern "C"
