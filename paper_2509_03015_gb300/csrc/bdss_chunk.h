// Launchers of the partitioned-solve kernels (internal to the library).
#pragma once
#include <cuda_runtime.h>

namespace bdss {

cudaError_t launch_chunk_rhs(long long Nb, int n, int dc, int blk, const double *M, int trans, int c0, double *Z,
                             cudaStream_t s);
cudaError_t launch_chunk_product(int n, int m, const double *P, int trans, const double *Q, double *C, int ldc,
                                 int c0, cudaStream_t s);
cudaError_t launch_chunk_fix_rhs(long long Nb, int n, int d, const double *B, const double *A_left,
                                 const double *A_right, const double *x_left, const double *x_right, double *Bp,
                                 cudaStream_t s);

}  // namespace bdss
