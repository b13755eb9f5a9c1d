// Host-side declarations of the Kalman-smoother assembly (Sec. 4.2), internal
// to the library.
#pragma once
#include <cuda_runtime.h>

namespace bdss {

// Normal equations assembled on the device.  U (N m n), v (N m), w (N n) are
// workspace; B == nullptr skips the right-hand side; rinv_diag: Rinv holds
// only the diagonals (N x m) of diagonal observation precisions.
struct KalmanArgs {
  long long N;
  int n, m, rinv_diag;
  const double *G, *H, *Qinv, *Rinv, *z, *zeta;
  double *A_diag, *A_sub, *B;
  double *U, *v, *w;
};
cudaError_t launch_kalman_assemble(const KalmanArgs &a, cudaStream_t s);
long long kalman_max_steps(int n, int m);  // largest N whose grids fit one launch

}  // namespace bdss
