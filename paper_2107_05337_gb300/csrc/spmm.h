// Batched FP32 tensor-product operator apply (spmm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

namespace igm {

// The four 1D factors of y = (Y2 (x) X1 + Z2 (x) W1) x as combinations of the
// bands of M1 and K1: X1 = xm M1 + xk K1, W1 = wm M1 + wk K1, and so on.
struct SpmmCoef {
  float xm, xk, wm, wk, ym, yk, zm, zk;
};

// y_b for b < nrhs; M1, K1 the 1D interior bands [n][2p+1] (entry o of row i
// couples column i - p + o), FP32 in device memory; x, y [nrhs][ld] FP32 with
// n*n <= ld, any alignment.  grid: persistent CTAs, one per SM.  smem_max: the
// device's opt-in shared memory per block; cudaErrorInvalidValue when the
// grid does not fit (spmm32_slots == 0) or p is outside [2, 8].
cudaError_t launch_spmm32(int n, int p, int nrhs, const float* M1, const float* K1, SpmmCoef cf,
                          const float* x, float* y, long ld, int grid, size_t smem_max,
                          cudaStream_t st);
// copy ring depth the kernel would use for an n x n grid (0: does not fit)
int spmm32_slots(int n, int p, size_t smem_max);
// The row-strip form for grids the persistent layouts do not hold: strips of
// spmm32_strip_rows(n, p, smem_max) grid rows (0: does not fit either), a grid
// of strips x column groups sized from the SM count `sms`.
cudaError_t launch_spmm32_strip(int n, int p, int nrhs, const float* M1, const float* K1,
                                SpmmCoef cf, const float* x, float* y, long ld, int sms,
                                size_t smem_max, cudaStream_t st);
int spmm32_strip_rows(int n, int p, size_t smem_max);
// The launch plan of the row-strip form for nrhs columns on a device with sms
// SMs: out[5] = {strip rows SR (0: does not fit), threads per CTA, dynamic
// shared bytes, strips (grid x), column groups (grid y)}.  Host code only.
void spmm32_strip_plan(int n, int p, int nrhs, int sms, size_t smem_max, int* out);
// The launch plan of the curved form: out[6] = {tile rows, tile columns,
// staged rows, staged columns, tiles (grid x), column groups (grid y)}; its
// dynamic shared memory is two stages of staged rows x columns float4.
void spmm32_curved_plan(int n, int p, int nrhs, int sms, int* out);
// The curved map: assembled stencils in FP32, coefficient q of point i at
// Mq[q N + i] (q = (dy + p)(2p + 1) + dx + p, N = n*n; the [N][(2p+1)^2]
// stencil transposed), y_b = (cm M + ck K) x_b; Mq or Kq may be null (that
// term left out).  x, y [nrhs][ld], any alignment; p in [2, 8].
cudaError_t launch_spmm32_curved(int n, int p, int nrhs, const float* Mq, const float* Kq,
                                 float cm, float ck, const float* x, float* y, long ld, int sms,
                                 cudaStream_t st);
// The shared-memory plan for an n x n grid: out[7] = {grid-line cap of the
// layout (0: does not fit), ring depth, grid lines per thread J, padded x row
// stride, (tm, tk) row stride in pairs, (tm, tk) rows, dynamic shared bytes}.
// Returns 1 when the grid fits.  Host code only.
int spmm32_layout(int n, int p, size_t smem_max, int* out);

}  // namespace igm
