// Batched FP32 tensor-product operator apply (spmm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace igm {

// y_b = (Y2 (x) X1 + Z2 (x) W1) x_b for b < nrhs (W1, Z2 may be null), 1D bands
// [n][2p+1]; x, y [nrhs][ld] FP32 with n*n <= ld.  grid: persistent CTAs.
cudaError_t launch_spmm32(int n, int p, int nrhs, const float* X1, const float* W1,
                          const float* Y2, const float* Z2, const float* x, float* y, long ld,
                          int grid, cudaStream_t st);
size_t spmm32_smem(int n, int p);

}  // namespace igm
