// Host-side declarations of the one-cluster path for short systems of small
// blocks (bdss_small.cu; internal to the library): FP64, n <= kSmallMaxN,
// d <= kSmallMaxD, the whole call in one launch of a single thread-block
// cluster of up to 16 CTAs with cluster barriers between the phases.
// small_cluster_size finds the largest supported cluster (16, 8, 4 or 2 CTAs;
// 0: none) for `smem` bytes per CTA; `out` is a device-visible address of the
// page-locked status copy the kernel writes at its end.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "bdss_device.cuh"

namespace bdss {

constexpr int kSmallThreads = 128;
constexpr int kSmallMaxN = 32;
constexpr int kSmallMaxD = 16;
size_t small_smem_bytes(int n, int d);
cudaError_t small_cluster_size(size_t smem, int *cluster);
cudaError_t launch_small(const Args<double> &a, int factor, int rhs, int cluster, size_t smem, DevStatus *out,
                         cudaStream_t s);

}  // namespace bdss
