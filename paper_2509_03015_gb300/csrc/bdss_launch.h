// Host-side declarations of the kernel launchers (internal to the library).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "bdss_device.cuh"

namespace bdss {

template <typename T> size_t smem_bytes(int n, int d);
// configure = raise_smem_limits (every kernel's dynamic shared-memory limit
// to the device's opt-in maximum) + occupancy (shared memory per CTA and
// resident CTAs per SM of the persistent kernel for (n, d)).
template <typename T> cudaError_t configure(int n, int d, size_t *smem, int *blocks_per_sm);
cudaError_t raise_smem_limits();
template <typename T> cudaError_t occupancy(int n, int d, size_t *smem, int *blocks_per_sm);
template <typename T>
cudaError_t launch_persistent(const Args<T> &a, int factor, int rhs, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_phaseA(const Args<T> &a, int l, int factor, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_phaseB(const Args<T> &a, int l, int factor, int grid, size_t smem, cudaStream_t s);
template <typename T> cudaError_t launch_top(const Args<T> &a, int factor, size_t smem, cudaStream_t s);
template <typename T> cudaError_t launch_phaseC(const Args<T> &a, int l, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_logdet(long long N, int n, int Ltop_level, const T *Ld, const double *Ltop, double *partial, int grid,
                          cudaStream_t s);
cudaError_t launch_residual(long long N, int n, int d, const double *A_diag, const double *A_sub, const double *X,
                            const double *B, float *R32, DevStatus *st, int with_norm, int grid, cudaStream_t s);
cudaError_t launch_adjoint_grads(long long N, int n, int d, const double *Lam, const double *X, double *dA_diag,
                                 double *dA_sub, int grid, cudaStream_t s);

// large-block path (64 < n <= 256)
constexpr int kMaxNLarge = 256;
template <typename T> size_t smem_bytes_large(int n, int d);
template <typename T>
cudaError_t configure_large(int n, int d, size_t *smem, int *blocks_per_sm, int *blocks_per_sm_tc);
template <typename T>
cudaError_t launch_large_persistent(const Args<T> &a, int factor, int rhs, int grid, size_t smem, cudaStream_t s);
template <typename T>
cudaError_t launch_large_sub(const Args<T> &a, int l, int sub, int factor, int grid, size_t smem, cudaStream_t s);
template <typename T> cudaError_t launch_large_top(const Args<T> &a, int factor, size_t smem, cudaStream_t s);
// Tasks of sub-phase `sub` at level l; inv = the pass uses the stored
// inverses (FP32 tiled path).
// Sub-phases of a level of the large path (bdss_large.cu): A1 Cholesky per
// eliminated block, A2 forward substitution, B separator (Schur) update,
// C downward back-substitution.
constexpr int kSubA1 = 0, kSubA2 = 1, kSubB = 2, kSubC = 3;

// Streamed solve passes of the large FP32 path with the stored inverses
// (n % 4 == 0, d <= 16): sub-phases kSubA2 (1), kSubB (2), kSubC (3) of level
// l as one launch each (bdss_large.cu).
constexpr int kCorrMaxD = 16;  // right-hand-side columns of one streamed pass
size_t corr_smem_bytes(int n);
cudaError_t make_f32_map(CUtensorMap *out, const float *base, long long rows, int n, int box_rows);
cudaError_t make_f32_map_box(CUtensorMap *out, const float *base, long long rows, int n, int box_cols,
                             int box_rows, bool swizzle);
// The maps of one split factor P of the streamed passes: boxes of 32 columns x
// n/P rows (row products, swizzled) and n/P columns x 32 rows (column
// products) over Li and Wb.
struct CorrMaps {
  CUtensorMap rowsLi, rowsW, colsLi, colsW;
};
// maps[0]: P = 1 (rows maps over Li and Wb with boxes of n rows), maps[1]:
// P = 2, maps[2]: P = 4; max_split bounds P (the maps that exist).
int corr_split(int n, long long tasks, int sms, int max_split);
cudaError_t launch_large_corr(const CorrMaps *maps, int max_split, const Args<float> &a, int l, int sub, int sms,
                              cudaStream_t s);
// Sub-phases of the split downward pass (levels of few blocks): C1 forms
// t = y_j - W x of the neighbours in place in Yt, C2 x_j = L_j^{-T} t.
constexpr int kSubC1 = 5, kSubC2 = 6;

// TF32 Schur products of level l on the tensor cores (pipelined, warp roles):
// a map over Wb (boxes of 128 rows x 32 columns).
cudaError_t launch_tf32_schur(const CUtensorMap &mapW, const Args<float> &a, int l, int sms, cudaStream_t s);

// Sub-phase code of the large path: the separators' RHS tiles alone (their D
// and E tiles ran elsewhere, e.g. on the tensor cores).
constexpr int kSubBRhsOnly = 4;
long long large_sub_tasks(const Plan &p, int l, int sub, int factor, int d, int esz, int tf32, int inv);
cudaError_t make_w_tensor_map(CUtensorMap *out, const float *Wb, long long rows, int n);
cudaError_t run_tc_selftest(double *max_err, int *status);
cudaError_t launch_residual_rows(long long N, int n, int d, const double *A_diag, const double *A_sub,
                                 const double *X, const double *B, float *R32, DevStatus *st, int with_norm,
                                 int grid, cudaStream_t s);

}  // namespace bdss
