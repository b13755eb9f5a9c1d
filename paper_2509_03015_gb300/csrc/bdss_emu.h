// FP64-accurate block-tridiagonal residual R = B - A X on the tcgen05 tensor
// cores (internal to the library).  A and X are cut into signed base-64
// digits ("slices") held exactly in BF16; every slice product is an integer
// and every sum of them stays below 2^24, so the FP32 tensor-core
// accumulation is exact and the only error is the 59-bit truncation of the
// inputs (see bdss_emu.cu).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "bdss_device.cuh"

namespace bdss {

constexpr int kEmuSlices = 10;  // digits per value: 5 + 6 x 9 = 59 bits below the row / column maximum
constexpr int kEmuDp = 16;      // right-hand-side columns of one product (d <= 16)
constexpr int kEmuKc = 64;      // K elements per staged chunk (128 bytes of BF16)

// Padded block width of the sliced layouts (multiple of the K chunk).
inline int emu_np(int n) { return (n + kEmuKc - 1) / kEmuKc * kEmuKc; }

// Device buffers of the emulated residual for one handle.
struct EmuBuffers {
  unsigned short *Aslc;  // N x S x n x 3 np BF16: digits of the operator rows
  int *Aexp;             // N x n: exponent E of each operator row (max |a| < 2^E)
  unsigned short *Xslc;  // N x S x 16 x np BF16: digits of X (per block, column, row)
  int *xexp;             // 16: exponent of each column of X
  unsigned long long *xmax;  // 16: bits of max |X[:, c]|
  CUtensorMap *maps;     // host copies: [0] operator slices, [1] X slices
};

size_t emu_aslc_bytes(long long N, int n);
size_t emu_xslc_bytes(long long N, int n);
// Encode the two TMA maps (host memory) for the buffers.
cudaError_t emu_make_maps(EmuBuffers &b, long long N, int n);
cudaError_t emu_configure();
// Slice the operator (once per factorisation); with st != null also forms
// ||A||_inf (FP32 row sums, only scaling the stop test) into st->nrm[2].
cudaError_t launch_emu_slice_operator(long long N, int n, const double *A_diag, const double *A_sub,
                                      const EmuBuffers &b, DevStatus *st, cudaStream_t s);
// R = B - A X: R32 (FP32) and/or R64 (FP64) outputs (either may be null);
// ||R||_inf, ||X||_inf into st->nrm[0], st->nrm[1].  d <= 16.
cudaError_t launch_emu_residual(long long N, int n, int d, const double *X, const double *B, float *R32,
                                double *R64, const EmuBuffers &b, DevStatus *st, long long timeout_ns, int sms,
                                cudaStream_t s);

// Schur products of the tiled FP64 factorisation on the tensor cores (see
// bdss_emu.cu): the level's N_l - 1 stored coupling blocks W (n x n each) are
// sliced into Wslc / Wexp, then the separators' D (lower, in Ld at slot s << l;
// level 0 reads sym(A_diag)) and the next level's E (En, slot k) are formed.
size_t emu_wslc_bytes(long long nW, int n);
cudaError_t launch_emu_slice_w(long long nW, int n, const double *W, unsigned short *Wslc, int *Wexp,
                               cudaStream_t s);
cudaError_t launch_emu_schur(long long Nl, int n, int l, const unsigned short *Wslc, const int *Wexp,
                             const double *A_diag, double *Ld, double *En, DevStatus *st, long long timeout_ns,
                             int sms, cudaStream_t s);

}  // namespace bdss
