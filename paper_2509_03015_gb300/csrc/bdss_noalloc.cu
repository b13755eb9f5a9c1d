// bdss_factor_solve_noalloc: FP64 factor + solve of one system whose whole
// workspace lives in a fixed, file-scope device array instead of memory the
// library allocates.
//
// Who needs it: callers that must not allocate device memory once they are
// running -- a real-time control loop (MPC, estimation) where cudaMalloc /
// cudaFree may synchronise the device and take unbounded time, or a plugin
// inside a host application whose own allocator owns all device memory and
// forbids allocations by libraries.  Such callers pass their inputs and
// outputs and get the same result as bdss_create + bdss_factor_solve.
//
// The price: kScratchBytes of device memory are reserved on every GPU that
// loads this library, from load until process exit, whether or not the entry
// point is used.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/bdss.h"
#include "bdss_launch.h"

using namespace bdss;

namespace {

constexpr size_t kScratchBytes = BDSS_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The shared scratch: status word, factors, coupling slots, top factor.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device.  In host code `g_scratch` names a
// host-side stand-in, never the device memory, so it is only ever used via
// cudaGetSymbolAddress.
static void *g_scratch_dev[kMaxDevices];
static bool g_ready[kMaxDevices];
static std::mutex g_setup_mutex;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Once per device, with that device current: look up the array's device
// address and raise the kernels' shared-memory limits.
cudaError_t setup_device(int dev, void **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_ready[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
    g_ready[dev] = true;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

void make_plan_noalloc(Plan &p, int64_t N, int n) {
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

}  // namespace

extern "C" bdss_status bdss_factor_solve_noalloc(int64_t N, int32_t n, int32_t d, const double *A_diag,
                                                 const double *A_sub, const double *B, double *X,
                                                 void *cuda_stream, bdss_info *info) {
  if (info) {
    info->level = -1;
    info->block = -1;
    info->iters = 0;
    info->reserved = 0;
    info->backward_err = -1.0;
  }
  if (N < 1 || n < 1 || n > kMaxN || d < 1 || d > 64) return BDSS_ERR_INVALID_ARG;
  if (N > ((int64_t)1 << (kMaxLevels - 2))) return BDSS_ERR_INVALID_ARG;
  if (!A_diag || !B || !X || (N > 1 && !A_sub)) return BDSS_ERR_INVALID_ARG;
  if ((((uintptr_t)A_diag | (uintptr_t)A_sub | (uintptr_t)B | (uintptr_t)X) & 15u) != 0)
    return BDSS_ERR_INVALID_ARG;
  Plan plan;
  make_plan_noalloc(plan, N, n);
  const size_t nn = (size_t)n * n;
  const size_t slots = (size_t)plan.off[plan.L];
  const size_t b_status = align256(sizeof(DevStatus));
  const size_t b_Ld = align256((size_t)N * nn * sizeof(double));
  const size_t b_Wb = align256((slots > 0 ? slots : 1) * nn * sizeof(double));
  const size_t b_top = align256(nn * sizeof(double));
  if (b_status + b_Ld + b_Wb + b_top > kScratchBytes) return BDSS_ERR_UNSUPPORTED;  // beyond the fixed scratch

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BDSS_ERR_CUDA;
  void *base = nullptr;
  e = setup_device(dev, &base);
  if (e != cudaSuccess) return BDSS_ERR_CUDA;
  size_t smem = 0;
  int bps = 0, sms = 0;
  e = configure<double>(n, d, &smem, &bps);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess || bps < 1) return BDSS_ERR_CUDA;

  unsigned char *p = (unsigned char *)base;
  DevStatus *st = (DevStatus *)p;
  Args<double> a;
  memset(&a, 0, sizeof(a));
  a.p = plan;
  a.A_diag = A_diag;
  a.A_sub = A_sub;
  a.Ld = (double *)(p + b_status);
  a.Wb = (double *)(p + b_status + b_Ld);
  a.Ltop = (double *)(p + b_status + b_Ld + b_Wb);
  a.d = d;
  a.B64 = B;
  a.Y = X;
  a.st = st;
  a.timeout_ns = 10000000000LL;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the status word and barrier counters must start at zero; the rest of the
  // scratch is written before it is read
  e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  long long grid = (long long)bps * sms;
  if ((N + 1) / 2 < grid) grid = (N + 1) / 2;
  if (grid < 1) grid = 1;
  if (e == cudaSuccess) e = launch_persistent<double>(a, 1, 1, (int)grid, smem, s);
  DevStatus h;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return BDSS_ERR_CUDA;
  if (h.status == BDSS_ERR_NOT_SPD && info) {
    info->level = h.level;
    info->block = h.block;
  }
  return (bdss_status)h.status;
}
