// Batched FP32 operator apply on the affine map (a block of right-hand-side
// columns, e.g. time intervals): y_b = (Y2 (x) X1 + Z2 (x) W1) x_b with the
// 1D interior bands of half-width p (Sec. 2: M = M1 (x) M1, K = K1 (x) M1 +
// M1 (x) K1 on the unit square), by sum factorisation:
//   stage 1 (along xi):  tm = x X1^T, tk = x W1^T  (rows of the n x n grid)
//   stage 2 (along eta): y = Y2 tm + Z2 tk          (columns of the grid)
// Persistent CTAs loop over the columns; both stages run in shared memory
// with four outputs per thread and the stage-1 band rows in registers.
#include <cuda_runtime.h>

#include "device.cuh"
#include "spmm.h"

namespace igm {

namespace {

constexpr int kThreads = 256;

template <int W>
__global__ void __launch_bounds__(kThreads, 2) k_spmm32(int n, int nrhs, const float* X1,
                                                     const float* W1, const float* Y2,
                                                     const float* Z2, const float* x, float* y,
                                                     long ld) {
  constexpr int p = (W - 1) / 2;
  extern __shared__ __align__(16) float sm[];
  const int G = (n + 3) / 4;                 // groups of four along a grid row
  const int xs = ((4 * G + 2 * p + 3) / 4) * 4;   // padded x row (halo p each side)
  float* xsm = sm;                           // [n][xs]
  float* tm = xsm + (size_t)n * xs;          // [n + 2p][n] with zero halo rows
  float* tk = tm + (size_t)(n + 2 * p) * n;
  float* y2 = tk + (size_t)(n + 2 * p) * n;  // [n][W]
  float* z2 = y2 + (size_t)n * W;
  const bool haveK = W1 != nullptr;
  for (int i = threadIdx.x; i < n * W; i += blockDim.x) {
    y2[i] = Y2[i];
    z2[i] = Z2 ? Z2[i] : 0.0f;
  }
  // zero the x halo and the tm / tk halo rows once (never overwritten)
  for (int i = threadIdx.x; i < n * xs; i += blockDim.x) xsm[i] = 0.0f;
  for (int i = threadIdx.x; i < p * n; i += blockDim.x) {
    tm[i] = 0.0f;
    tk[i] = 0.0f;
    tm[(size_t)(n + p) * n + i] = 0.0f;
    tk[(size_t)(n + p) * n + i] = 0.0f;
  }
  // stage-1 assignment: group g of every row iy = r0, r0 + R1, ...
  const int R1 = blockDim.x / G;
  const int g = threadIdx.x % G, r0 = threadIdx.x / G;
  const bool on1 = r0 < R1;
  float a[4][W], k[4][W];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int ix = 4 * g + j;
#pragma unroll
    for (int o = 0; o < W; ++o) {
      a[j][o] = ix < n ? X1[(size_t)ix * W + o] : 0.0f;
      k[j][o] = (ix < n && haveK) ? W1[(size_t)ix * W + o] : 0.0f;
    }
  }
  // stage-2 assignment: column ix, row groups gy = c0, c0 + R2, ...
  const int R2 = blockDim.x / n;
  const int ix2 = threadIdx.x % n, c0 = threadIdx.x / n;
  const bool on2 = c0 < R2;
  for (int b = blockIdx.x; b < nrhs; b += gridDim.x) {
    const float* xb = x + (size_t)b * ld;
    float* yb = y + (size_t)b * ld;
    __syncthreads();  // the previous column's stage 2 is done with tm / tk
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
      const int iy = i / n, ix = i % n;
      xsm[(size_t)iy * xs + p + ix] = xb[i];
    }
    __syncthreads();
    if (on1) {
      for (int iy = r0; iy < n; iy += R1) {
        // x[iy][4g - p .. 4g + 3 + p] sits at xsm[iy][4g .. 4g + 3 + 2p]
        const float4* row = (const float4*)(xsm + (size_t)iy * xs + 4 * g);
        float v[((W + 3 + 3) / 4) * 4];
#pragma unroll
        for (int q = 0; q < (W + 3 + 3) / 4; ++q) {
          const float4 t = row[q];
          v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int ix = 4 * g + j;
          float sm_ = 0.0f, sk = 0.0f;
#pragma unroll
          for (int o = 0; o < W; ++o) {
            sm_ = fmaf(a[j][o], v[j + o], sm_);
            sk = fmaf(k[j][o], v[j + o], sk);
          }
          if (ix < n) {
            tm[(size_t)(iy + p) * n + ix] = sm_;
            tk[(size_t)(iy + p) * n + ix] = sk;
          }
        }
      }
    }
    __syncthreads();
    if (on2) {
      for (int gy = c0; 4 * gy < n; gy += R2) {
        float um[4 + W - 1], uk[4 + W - 1];
#pragma unroll
        for (int q = 0; q < 4 + W - 1; ++q) {
          const int r = 4 * gy + q;  // halo row index (iy + p - p)
          const bool in = r < n + 2 * p;
          um[q] = in ? tm[(size_t)r * n + ix2] : 0.0f;
          uk[q] = in ? tk[(size_t)r * n + ix2] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int iy = 4 * gy + j;
          if (iy >= n) break;
          float s = 0.0f;
#pragma unroll
          for (int o = 0; o < W; ++o) {
            s = fmaf(y2[iy * W + o], um[j + o], s);
            s = fmaf(z2[iy * W + o], uk[j + o], s);
          }
          yb[(size_t)iy * n + ix2] = s;
        }
      }
    }
  }
}

// The same operator with the columns streamed by cp.async.bulk through a ring
// of NB shared-memory buffers (column k + NB is in flight while column k is
// computed).  Needs ld % 4 == 0 (16-byte aligned columns).  A wait that does
// not complete within the bounded number of polls ends the CTA's work early.
constexpr int NB = 3;
template <int W>
__global__ void __launch_bounds__(kThreads, 2) k_spmm32_stream(int n, int nrhs, const float* X1,
                                                               const float* W1, const float* Y2,
                                                               const float* Z2, const float* x,
                                                               float* y, long ld) {
  constexpr int p = (W - 1) / 2;
  extern __shared__ __align__(128) float sm[];
  const int N = n * n;
  const int Np = (N + 3) & ~3;                       // 16-byte multiple
  float* xb = sm;                                    // [NB][Np]
  float* tm = xb + (size_t)NB * Np;                  // [n + 2p][n], zero halo rows
  float* tk = tm + (size_t)(n + 2 * p) * n;
  float* y2 = tk + (size_t)(n + 2 * p) * n;
  float* z2 = y2 + (size_t)n * W;
  // every region above holds an even number of floats: the barriers are 8-byte aligned
  uint64_t* bar = (uint64_t*)(z2 + (size_t)n * W);
  const bool haveK = W1 != nullptr;
  const int G = (n + 3) / 4;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NB; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  for (int i = threadIdx.x; i < n * W; i += blockDim.x) {
    y2[i] = Y2[i];
    z2[i] = Z2 ? Z2[i] : 0.0f;
  }
  for (int i = threadIdx.x; i < p * n; i += blockDim.x) {
    tm[i] = 0.0f;
    tk[i] = 0.0f;
    tm[(size_t)(n + p) * n + i] = 0.0f;
    tk[(size_t)(n + p) * n + i] = 0.0f;
  }
  __syncthreads();
  const int cnt = nrhs > (int)blockIdx.x ? (nrhs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const uint32_t bytes = (uint32_t)Np * 4u;
  if (threadIdx.x == 0)
    for (int k = 0; k < NB && k < cnt; ++k)
      bulk_load(xb + (size_t)k * Np, x + (size_t)(blockIdx.x + k * gridDim.x) * ld, bytes, &bar[k]);
  const int R1 = blockDim.x / G;
  const int g = threadIdx.x % G, r0 = threadIdx.x / G;
  const bool on1 = r0 < R1;
  float a[4][W], kk[4][W];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int ix = 4 * g + j;
#pragma unroll
    for (int o = 0; o < W; ++o) {
      a[j][o] = ix < n ? X1[(size_t)ix * W + o] : 0.0f;
      kk[j][o] = (ix < n && haveK) ? W1[(size_t)ix * W + o] : 0.0f;
    }
  }
  const int R2 = blockDim.x / n;
  const int ix2 = threadIdx.x % n, c0 = threadIdx.x / n;
  const bool on2 = c0 < R2;
  int done = cnt;
  for (int k = 0; k < cnt; ++k) {
    const int s = k % NB;
    const bool got = mbar_wait(&bar[s], (uint32_t)(k / NB) & 1u);
    if (__syncthreads_or(!got)) {
      done = k;
      break;
    }
    const float* xs = xb + (size_t)s * Np;
    float* yb = y + (size_t)(blockIdx.x + k * gridDim.x) * ld;
    if (on1) {
      for (int iy = r0; iy < n; iy += R1) {
        const float* row = xs + (size_t)iy * n;
        float v[W + 3];
#pragma unroll
        for (int q = 0; q < W + 3; ++q) {
          const int ix = 4 * g + q - p;
          const int ic = ix < 0 ? 0 : (ix >= n ? n - 1 : ix);  // in-bounds address always
          v[q] = (ix >= 0 && ix < n) ? row[ic] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int ix = 4 * g + j;
          float sm_ = 0.0f, sk = 0.0f;
#pragma unroll
          for (int o = 0; o < W; ++o) {
            sm_ = fmaf(a[j][o], v[j + o], sm_);
            sk = fmaf(kk[j][o], v[j + o], sk);
          }
          if (ix < n) {
            tm[(size_t)(iy + p) * n + ix] = sm_;
            tk[(size_t)(iy + p) * n + ix] = sk;
          }
        }
      }
    }
    __syncthreads();
    // buffer s is free: stream in column k + NB
    if (threadIdx.x == 0 && k + NB < cnt) {
      fence_proxy_async();
      bulk_load(xb + (size_t)s * Np, x + (size_t)(blockIdx.x + (k + NB) * gridDim.x) * ld, bytes,
                &bar[s]);
    }
    if (on2) {
      for (int gy = c0; 4 * gy < n; gy += R2) {
        float um[4 + W - 1], uk[4 + W - 1];
#pragma unroll
        for (int q = 0; q < 4 + W - 1; ++q) {
          const int r = 4 * gy + q;
          const bool in = r < n + 2 * p;
          um[q] = in ? tm[(size_t)r * n + ix2] : 0.0f;
          uk[q] = in ? tk[(size_t)r * n + ix2] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int iy = 4 * gy + j;
          if (iy >= n) break;
          float sacc = 0.0f;
#pragma unroll
          for (int o = 0; o < W; ++o) {
            sacc = fmaf(y2[iy * W + o], um[j + o], sacc);
            sacc = fmaf(z2[iy * W + o], uk[j + o], sacc);
          }
          yb[(size_t)iy * n + ix2] = sacc;
        }
      }
    }
    __syncthreads();
  }
  // after an early exit, drain the copies still in flight (bounded) before
  // the CTA's shared memory is released
  if (threadIdx.x == 0)
    for (int k = done; k < cnt && k < done + NB; ++k)
      mbar_wait(&bar[k % NB], (uint32_t)(k / NB) & 1u);
}

template <int W>
size_t stream_smem(int n) {
  const int p = (W - 1) / 2, N = n * n, Np = (N + 3) & ~3;
  return sizeof(float) * ((size_t)NB * Np + 2 * (size_t)(n + 2 * p) * n + 2 * (size_t)n * W) +
         8 * NB;
}

template <int W>
cudaError_t launch_w(int n, int nrhs, const float* X1, const float* W1, const float* Y2,
                     const float* Z2, const float* x, float* y, long ld, int grid, cudaStream_t st) {
  if (ld % 4 == 0) {
    const size_t smem = stream_smem<W>(n);
    cudaError_t e = cudaFuncSetAttribute(k_spmm32_stream<W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_spmm32_stream<W><<<grid, kThreads, smem, st>>>(n, nrhs, X1, W1, Y2, Z2, x, y, ld);
    return cudaGetLastError();
  }
  const int p = (W - 1) / 2;
  const int G = (n + 3) / 4;
  const int xs = ((4 * G + 2 * p + 3) / 4) * 4;
  const size_t smem = sizeof(float) * ((size_t)n * xs + 2 * (size_t)(n + 2 * p) * n + 2 * (size_t)n * W);
  cudaError_t e = cudaFuncSetAttribute(k_spmm32<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_spmm32<W><<<grid, kThreads, smem, st>>>(n, nrhs, X1, W1, Y2, Z2, x, y, ld);
  return cudaGetLastError();
}

}  // namespace

size_t spmm32_smem(int n, int p) {
  const int W = 2 * p + 1, G = (n + 3) / 4, xs = ((4 * G + 2 * p + 3) / 4) * 4;
  return sizeof(float) * ((size_t)n * xs + 2 * (size_t)(n + 2 * p) * n + 2 * (size_t)n * W);
}

cudaError_t launch_spmm32(int n, int p, int nrhs, const float* X1, const float* W1,
                          const float* Y2, const float* Z2, const float* x, float* y, long ld,
                          int grid, cudaStream_t st) {
  switch (p) {
    case 1: return launch_w<3>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    case 2: return launch_w<5>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    case 3: return launch_w<7>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    case 4: return launch_w<9>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    case 5: return launch_w<11>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    case 6: return launch_w<13>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    case 7: return launch_w<15>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
    default: return launch_w<17>(n, nrhs, X1, W1, Y2, Z2, x, y, ld, grid, st);
  }
}

}  // namespace igm
