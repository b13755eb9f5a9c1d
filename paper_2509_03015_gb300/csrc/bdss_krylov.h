// Host-side declarations of the preconditioned-CG refinement kernels,
// internal to the library.
#pragma once
#include <cuda_runtime.h>

namespace bdss {

constexpr int kKrylovMaxD = 64;     // right-hand-side columns (= the handle's d_max limit)
constexpr int kKrylovGrid = 1024;   // CTAs of the reduction kernels (partial buffers)
// Scalar block: rho, alpha, beta per column, then ||R||_inf and ||X||_inf.
constexpr int kScRho = 0, kScAlpha = kKrylovMaxD, kScBeta = 2 * kKrylovMaxD, kScNorm = 3 * kKrylovMaxD;
constexpr int kScWords = 3 * kKrylovMaxD + 2;
// partial sums: [kKrylovGrid][2][kKrylovMaxD], then maxima [kKrylovGrid][2]
constexpr size_t kPartWords = (size_t)kKrylovGrid * 2 * kKrylovMaxD + (size_t)kKrylovGrid * 2;

// what k_pcg_scalars forms from the partial sums
enum PcgStep { kPcgStart = 0, kPcgAlpha = 1, kPcgBeta = 2, kPcgNorms = 3 };

cudaError_t launch_btd_apply(long long N, int n, int d, const double *A_diag, const double *A_sub, const double *P,
                             const double *B, double *out, int sms, cudaStream_t s);
int col_dots_grid(long long rows, int d);
cudaError_t launch_col_dots(long long rows, int d, const double *x1, const double *y1, const double *x2,
                            const double *y2, double *part, int grid, cudaStream_t s);
int pcg_update_grid(long long rows);
cudaError_t launch_pcg_update(long long rows, int d, const double *sc, const double *P, const double *Q, double *X,
                              double *R, double *part, int grid, cudaStream_t s);
cudaError_t launch_pcg_scalars(int nparts, int d, const double *part, int step, double *sc, cudaStream_t s);
// out = A_diag with the diagonal scaled by (1 + sigma): the shifted FP32 factorisation.
cudaError_t launch_shift_diag(long long N, int n, const double *A_diag, double sigma, double *out, int sms,
                              cudaStream_t s);
cudaError_t launch_pcg_direction(long long rows, int d, const double *sc, const double *Z, double *P, int init,
                                 int sms, cudaStream_t s);

}  // namespace bdss
