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

// Per-device set-up: the device address of g_scratch (in host code
// `g_scratch` names a host-side stand-in, never the device memory, so it is
// only ever used via cudaGetSymbolAddress), the SM count and the opt-in
// shared-memory limit.
struct DeviceSetup {
  void *scratch = nullptr;
  int sms = 0;
  int smem_optin = 0;
  bool ready = false;
};
static DeviceSetup g_dev[kMaxDevices];
static std::mutex g_setup_mutex;

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Once per device, with that device current: look up the array's device
// address and the device's limits, and raise the kernels' shared-memory
// limits, so that later calls make no attribute calls.
cudaError_t setup_device(int dev, DeviceSetup *out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup &g = g_dev[dev];
  if (!g.ready) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = raise_smem_limits();
    if (e != cudaSuccess) return e;
    g.scratch = p;
    g.ready = true;
  }
  *out = g;
  return cudaSuccess;
}

// Can the device read p in place (device, managed or mapped page-locked
// memory, or any host memory where the device reads pageable memory)?  With
// `write`, only device and managed memory qualify.
bool device_accessible(const void *p, bool write) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return true;
  if (write) return false;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer == p;
  int dev = 0, pageable = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return pageable != 0;
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
  if (N < 1 || n < 1 || d < 1 || d > 64) return BDSS_ERR_INVALID_ARG;
  // blocks up to n = 64 only (the shared-memory path); longer horizons than
  // the level plan holds are beyond the scratch anyway
  if (n > kMaxN || N > ((int64_t)1 << (kMaxLevels - 2))) return BDSS_ERR_UNSUPPORTED;
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
  DeviceSetup g;
  e = setup_device(dev, &g);
  if (e != cudaSuccess) return BDSS_ERR_CUDA;
  if (!device_accessible(A_diag, false) || !device_accessible(B, false) || !device_accessible(X, true) ||
      (N > 1 && !device_accessible(A_sub, false)))
    return BDSS_ERR_INVALID_ARG;
  if (smem_bytes<double>(n, d) > (size_t)g.smem_optin) return BDSS_ERR_UNSUPPORTED;
  size_t smem = 0;
  int bps = 0;
  e = occupancy<double>(n, d, &smem, &bps);
  if (e != cudaSuccess || bps < 1) return BDSS_ERR_CUDA;

  unsigned char *p = (unsigned char *)g.scratch;
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
  // as bdss_create: tail levels with fewer blocks than resident CTAs split
  // each block's work over several CTAs (same arithmetic, same result)
  a.capacity = bps * g.sms;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the status word and barrier counters must start at zero; the rest of the
  // scratch is written before it is read
  e = cudaMemsetAsync(st, 0, sizeof(DevStatus), s);
  long long most = 1;  // tasks of the busiest step, as bdss_factor_solve sizes its grid
  for (int l = 0; l < plan.L; ++l) {
    const long long tA = (plan.Nl[l] / 2) * parts_A<double>(plan, l, true, a.capacity);
    const long long tB = ((plan.Nl[l] + 1) / 2) * parts_B<double>(plan, l, true, a.capacity);
    if (tA > most) most = tA;
    if (tB > most) most = tB;
  }
  const long long grid = most < a.capacity ? most : a.capacity;
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
