// Learned coarse propagator Phi_c for MGRIT: a 3 x 3 convolutional network on
// the n x n grid of interior coefficients (zero padding = the homogeneous
// Dirichlet condition), BF16 weights and activations with FP32 accumulation:
//   x = u / s (s = max |u|),  h1 = g(K1 * x),  h2 = g(K2 * h1),  h3 = g(K3 * h2),
//   Phi_c(u) = s (x + K4 * h3),  g(z) = z (1 + erf(z / sqrt 2)) / 2 (GELU),
// K1: 1 -> C, K2, K3: C -> C, K4: C -> 1 channels, no biases; and the kernels
// of its training (back-propagation, Adam).  The C -> C layers, their input
// gradients and their weight gradients are implicit-GEMM products on the
// tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulators); the
// one-channel layers are FP32 FMA loops.  Pixel p = y n + x of an image (x,
// the xi index, fastest); the C-channel tensors are [image][pixel][channel].
#include <cuda_bf16.h>
#include <stdint.h>

#include "phic.h"

namespace igm {

namespace {

constexpr int KS = 3, NTAP = 9;

__device__ __forceinline__ float gelu(float z) {
  return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_deriv(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

// Offsets of tap t = 3a + b: (dy, dx) = (a - 1, b - 1).
__device__ __forceinline__ int tap_dy(int t) { return t / KS - 1; }
__device__ __forceinline__ int tap_dx(int t) { return t % KS - 1; }
// Pixel q = p + (dy, dx) of an n x n image, or -1 outside it (or p >= N).
__device__ __forceinline__ int neighbour(int p, int n, int t) {
  if (p >= n * n) return -1;
  const int y = p / n + tap_dy(t), x = p % n + tap_dx(t);
  return (y >= 0 && y < n && x >= 0 && x < n) ? y * n + x : -1;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// D = A B + D on one 16 x 8 tile, A 16 x 16 and B 16 x 8 in BF16 (the
// per-thread fragments of the PTX m16n8k16 layout).
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// BF16 copies of the master weights (layouts in PhicNet).
__global__ void k_phic_refresh(int C, const float* wall, int o1, int o2, int o3, int o4,
                               __nv_bfloat16* wf, __nv_bfloat16* wb, float* w1, float* w4) {
  const int tot = 2 * C * NTAP * C;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < tot + 2 * C * NTAP;
       i += gridDim.x * blockDim.x) {
    if (i < tot) {
      // i over (layer L, cout o, cin c, tap t) in the master layout
      const int t = i % NTAP, c = (i / NTAP) % C, o = (i / (NTAP * C)) % C, L = i / (NTAP * C * C);
      const __nv_bfloat16 v = __float2bfloat16(wall[(L == 0 ? o2 : o3) + i % (NTAP * C * C)]);
      wf[(((size_t)L * C + o) * NTAP + t) * C + c] = v;
      wb[(((size_t)L * C + c) * NTAP + (NTAP - 1 - t)) * C + o] = v;
    } else {
      const int k = i - tot;
      if (k < C * NTAP) {
        w1[k] = __bfloat162float(__float2bfloat16(wall[o1 + k]));   // [o][t]
      } else {
        const int q = k - C * NTAP, t = q / C, c = q % C;             // [t][c]
        w4[q] = __bfloat162float(__float2bfloat16(wall[o4 + c * NTAP + t]));
      }
    }
  }
}

// Layer 1 (1 -> C): z1 = K1 * x0, h1 = g(z1); one thread per pixel.
__global__ void k_phic_l1(int n, int C, const __nv_bfloat16* x0, const float* w1,
                          __nv_bfloat16* z1, __nv_bfloat16* h1) {
  const int N = n * n, b = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  float xv[NTAP];
#pragma unroll
  for (int t = 0; t < NTAP; ++t) {
    const int q = neighbour(p, n, t);
    xv[t] = q >= 0 ? __bfloat162float(x0[(size_t)b * N + q]) : 0.0f;
  }
  uint32_t* zo = z1 ? (uint32_t*)(z1 + ((size_t)b * N + p) * C) : nullptr;
  uint32_t* ho = (uint32_t*)(h1 + ((size_t)b * N + p) * C);
  for (int o = 0; o < C; o += 2) {
    float za = 0.0f, zb = 0.0f;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) {
      za = fmaf(w1[o * NTAP + t], xv[t], za);
      zb = fmaf(w1[(o + 1) * NTAP + t], xv[t], zb);
    }
    if (zo) zo[o / 2] = pack_bf16(za, zb);
    ho[o / 2] = pack_bf16(gelu(za), gelu(zb));
  }
}

// Layer 4 (C -> 1): z4 = K4 * h3 (FP32); one thread per pixel.
__global__ void k_phic_l4(int n, int C, const __nv_bfloat16* h3, const float* w4, float* z4) {
  const int N = n * n, b = blockIdx.y;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  float z = 0.0f;
  for (int t = 0; t < NTAP; ++t) {
    const int q = neighbour(p, n, t);
    if (q < 0) continue;
    const __nv_bfloat162* hq = (const __nv_bfloat162*)(h3 + ((size_t)b * N + q) * C);
    const float* wt = w4 + t * C;
    for (int c = 0; c < C; c += 2) {
      const float2 v = __bfloat1622float2(hq[c / 2]);
      z = fmaf(wt[c], v.x, z);
      z = fmaf(wt[c + 1], v.y, z);
    }
  }
  z4[(size_t)b * N + p] = z;
}

// One C -> C layer as an implicit GEMM on the tensor cores: out[p][o] =
// sum over taps t and channels c of W[o][t][c] in[p + d_t][c], W given as
// [cout][tap][cin] BF16.  Each warp computes 16 consecutive pixels of one
// image for all C outputs (C / 8 tiles of 16 x 8) over 9 C / 16 steps of K.
// Epilogue: BWD = 0: zout = z, hout = g(z) (the forward layer; zout may be
// null); BWD = 1: hout = z g'(zprev) (the gradient through the GELU of the
// layer below, zprev its pre-activation).
constexpr int kMidWarps = 4;
template <int C, bool BWD>
__global__ void __launch_bounds__(32 * kMidWarps) k_phic_mid(int n, const __nv_bfloat16* in,
                                                             const __nv_bfloat16* W,
                                                             const __nv_bfloat16* zprev,
                                                             __nv_bfloat16* zout,
                                                             __nv_bfloat16* hout) {
  constexpr int NT = C / 8, KB = C / 16;
  __shared__ __align__(16) __nv_bfloat16 ws[C * NTAP * C];
  const int N = n * n, b = blockIdx.y;
  for (int i = threadIdx.x; i < C * NTAP * C / 8; i += blockDim.x)
    reinterpret_cast<uint4*>(ws)[i] = reinterpret_cast<const uint4*>(W)[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int p0 = (blockIdx.x * kMidWarps + warp) * 16;
  if (p0 >= N) return;
  const __nv_bfloat16* img = in + (size_t)b * N * C;
  const int pa = p0 + g, pb = p0 + g + 8;
  float acc[NT][4];
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll 1
  for (int t = 0; t < NTAP; ++t) {
    const int qa = neighbour(pa, n, t), qb = neighbour(pb, n, t);
    const uint32_t* ra = (const uint32_t*)(img + (size_t)(qa < 0 ? 0 : qa) * C);
    const uint32_t* rb = (const uint32_t*)(img + (size_t)(qb < 0 ? 0 : qb) * C);
#pragma unroll
    for (int kb = 0; kb < KB; ++kb) {
      const int c0 = kb * 16 + 2 * tig;   // channel pair of this lane
      uint32_t a[4];
      a[0] = qa >= 0 ? ra[c0 / 2] : 0u;
      a[1] = qb >= 0 ? rb[c0 / 2] : 0u;
      a[2] = qa >= 0 ? ra[c0 / 2 + 4] : 0u;
      a[3] = qb >= 0 ? rb[c0 / 2 + 4] : 0u;
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        const uint32_t* wr = (const uint32_t*)(ws + ((size_t)(j * 8 + g) * NTAP + t) * C);
        mma_bf16(acc[j], a, wr[c0 / 2], wr[c0 / 2 + 4]);
      }
    }
  }
  // accumulator (row r, column 2 tig + e) of tile j: pixel p0 + r, channel j 8 + 2 tig + e
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int p = half ? pb : pa;
    if (p >= N) continue;
    const size_t base = ((size_t)b * N + p) * C;
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const int c = j * 8 + 2 * tig;
      const float z0 = acc[j][2 * half], z1 = acc[j][2 * half + 1];
      if (BWD) {
        const float2 zp = __bfloat1622float2(*(const __nv_bfloat162*)(zprev + base + c));
        *(uint32_t*)(hout + base + c) = pack_bf16(z0 * gelu_deriv(zp.x), z1 * gelu_deriv(zp.y));
      } else {
        if (zout) *(uint32_t*)(zout + base + c) = pack_bf16(z0, z1);
        *(uint32_t*)(hout + base + c) = pack_bf16(gelu(z0), gelu(z1));
      }
    }
  }
}

// Weight gradient of a C -> C layer on the tensor cores, one image and one
// tap per CTA: part[b][o][c][t] = sum over pixels p of gz[p][o] h[p + d_t][c]
// (a 32 x 32 product over K = the pixels).  The CTA's warps take interleaved
// 16-pixel steps of K; their partial tiles are summed in warp order.  part
// is laid out like a kernel of the master weights, [o][c][t] per image.
template <int C>
__global__ void __launch_bounds__(32 * kMidWarps) k_phic_wgrad(int n, const __nv_bfloat16* gz,
                                                               const __nv_bfloat16* h,
                                                               float* part, long part_ld) {
  constexpr int MT = C / 16, NT = C / 8;
  __shared__ float red[kMidWarps][C * C];
  const int N = n * n, b = blockIdx.y, t = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const __nv_bfloat16* G = gz + (size_t)b * N * C;
  const __nv_bfloat16* H = h + (size_t)b * N * C;
  float acc[MT][NT][4];
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int p0 = warp * 16; p0 < N; p0 += 16 * kMidWarps) {
    // the four pixels of this lane in the step: k = 2 tig, 2 tig + 1, 2 tig + 8, 2 tig + 9
    int pk[4], qk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      pk[e] = p0 + 2 * tig + (e & 1) + (e >> 1) * 8;
      qk[e] = neighbour(pk[e], n, t);
      if (pk[e] >= N) pk[e] = -1;
    }
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      // A = gz^T: row o = i 16 + g (+ 8), column k = pixel
      uint32_t a[4];
      const int oa = i * 16 + g, ob = oa + 8;
      auto ga = [&](int e, int o) { return pk[e] >= 0 ? G[(size_t)pk[e] * C + o] : zero; };
      a[0] = pack_raw(ga(0, oa), ga(1, oa));
      a[1] = pack_raw(ga(0, ob), ga(1, ob));
      a[2] = pack_raw(ga(2, oa), ga(3, oa));
      a[3] = pack_raw(ga(2, ob), ga(3, ob));
#pragma unroll
      for (int j = 0; j < NT; ++j) {
        // B = im2col(h): row k = pixel, column c = j 8 + g
        const int c = j * 8 + g;
        auto hb = [&](int e) { return qk[e] >= 0 ? H[(size_t)qk[e] * C + c] : zero; };
        mma_bf16(acc[i][j], a, pack_raw(hb(0), hb(1)), pack_raw(hb(2), hb(3)));
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MT; ++i)
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = i * 16 + g + (e >> 1) * 8, c = j * 8 + 2 * tig + (e & 1);
        red[warp][o * C + c] = acc[i][j][e];
      }
  __syncthreads();
  for (int k = threadIdx.x; k < C * C; k += blockDim.x) {
    float s = 0.0f;
    for (int w = 0; w < kMidWarps; ++w) s += red[w][k];
    part[(size_t)b * part_ld + (size_t)k * NTAP + t] = s;   // [o][c][t]
  }
}

// Back through layer 4 and the GELU of layer 3: gz3[q][c] = g'(z3[q][c]) sum
// over taps t of K4[c][t] gy[q - d_t]; one thread per pixel.
__global__ void k_phic_l4_back(int n, int C, const float* gy, const float* w4,
                               const __nv_bfloat16* z3, __nv_bfloat16* gz3) {
  const int N = n * n, b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  float gv[NTAP];
#pragma unroll
  for (int t = 0; t < NTAP; ++t) {
    const int s = neighbour(q, n, NTAP - 1 - t);   // the pixel q - d_t
    gv[t] = s >= 0 ? gy[(size_t)b * N + s] : 0.0f;
  }
  const size_t base = ((size_t)b * N + q) * C;
  for (int c = 0; c < C; c += 2) {
    float ga = 0.0f, gb = 0.0f;
#pragma unroll
    for (int t = 0; t < NTAP; ++t) {
      ga = fmaf(w4[t * C + c], gv[t], ga);
      gb = fmaf(w4[t * C + c + 1], gv[t], gb);
    }
    const float2 z = __bfloat1622float2(*(const __nv_bfloat162*)(z3 + base + c));
    *(uint32_t*)(gz3 + base + c) = pack_bf16(ga * gelu_deriv(z.x), gb * gelu_deriv(z.y));
  }
}

// Input gradient of the network (phic_grad): gx[q] = gy[q] (the skip
// connection) + sum over taps t and channels o of K1[o][t] gz1[q - d_t][o].
__global__ void k_phic_l1_back(int n, int C, const float* gy, const float* w1,
                               const __nv_bfloat16* gz1, float* gx) {
  const int N = n * n, b = blockIdx.y;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  float s = 0.0f;
  for (int t = 0; t < NTAP; ++t) {
    const int r = neighbour(q, n, NTAP - 1 - t);
    if (r < 0) continue;
    const __nv_bfloat162* gr = (const __nv_bfloat162*)(gz1 + ((size_t)b * N + r) * C);
    for (int o = 0; o < C; o += 2) {
      const float2 v = __bfloat1622float2(gr[o / 2]);
      s = fmaf(w1[o * NTAP + t], v.x, s);
      s = fmaf(w1[(o + 1) * NTAP + t], v.y, s);
    }
  }
  gx[(size_t)b * N + q] = gy[(size_t)b * N + q] + s;
}

// Weight gradients of the one-channel layers, one image and one tap per CTA
// (256 threads; per-thread sums over its pixels, then a CTA reduction in
// warp order):
//   L1 = 1: part[b][o][t] = sum_p gz1[p][o] x0[p + d_t]           (K1, [o][t])
//   L1 = 0: part[b][c][t] = sum_p gy[p] h3[p + d_t][c]            (K4, [c][t])
template <int C, bool L1>
__global__ void __launch_bounds__(256) k_phic_wgrad1(int n, const __nv_bfloat16* gz1,
                                                     const __nv_bfloat16* x0, const float* gy,
                                                     const __nv_bfloat16* h3, float* part,
                                                     long part_ld) {
  __shared__ float red[8][C];
  const int N = n * n, b = blockIdx.y, t = blockIdx.x;
  float acc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) acc[c] = 0.0f;
  for (int p = threadIdx.x; p < N; p += blockDim.x) {
    const int q = neighbour(p, n, t);
    if (q < 0) continue;
    if (L1) {
      const float xv = __bfloat162float(x0[(size_t)b * N + q]);
      const __nv_bfloat162* gr = (const __nv_bfloat162*)(gz1 + ((size_t)b * N + p) * C);
#pragma unroll
      for (int o = 0; o < C; o += 2) {
        const float2 v = __bfloat1622float2(gr[o / 2]);
        acc[o] = fmaf(v.x, xv, acc[o]);
        acc[o + 1] = fmaf(v.y, xv, acc[o + 1]);
      }
    } else {
      const float gv = gy[(size_t)b * N + p];
      const __nv_bfloat162* hr = (const __nv_bfloat162*)(h3 + ((size_t)b * N + q) * C);
#pragma unroll
      for (int c = 0; c < C; c += 2) {
        const float2 v = __bfloat1622float2(hr[c / 2]);
        acc[c] = fmaf(gv, v.x, acc[c]);
        acc[c + 1] = fmaf(gv, v.y, acc[c + 1]);
      }
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    float v = acc[c];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float s = 0.0f;
    for (int w = 0; w < 8; ++w) s += red[w][c];
    part[(size_t)b * part_ld + (size_t)c * NTAP + t] = s;
  }
}

// gw[k] = sum over images b of part[b][k], in image order.
__global__ void k_phic_sum_parts(int nb, int cnt, const float* part, float* gw) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= cnt) return;
  float s = 0.0f;
  for (int b = 0; b < nb; ++b) s += part[(size_t)b * cnt + k];
  gw[k] = s;
}

// Normalise: s[b] = max |u_b|, x0[b] = bf16(u_b / s) (0 where s = 0).
__global__ void k_phic_in(int N, const double* u, long ldu, __nv_bfloat16* x0, double* s) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const double* ub = u + (size_t)b * ldu;
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(ub[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
  const double inv = t > 0.0 ? 1.0 / t : 0.0;
  if (threadIdx.x == 0) s[b] = t;
  for (int i = threadIdx.x; i < N; i += blockDim.x)
    x0[(size_t)b * N + i] = __float2bfloat16((float)(ub[i] * inv));
}

// out_b = u_b + s_b * z4_b (+ add_b) (- sub_b): the network output (with its
// skip connection, in FP64), optionally with a vector added and one
// subtracted (the FAS terms).
__global__ void k_phic_out(int N, const double* u, long ldu, const float* z4, const double* s,
                           const double* add, long lda, const double* sub, long lds, double* out,
                           long ldo) {
  const int b = blockIdx.y;
  const double sb = s[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double v = u[(size_t)b * ldu + i] + sb * (double)z4[(size_t)b * N + i];
    if (add) v += add[(size_t)b * lda + i];
    if (sub) v -= sub[(size_t)b * lds + i];
    out[(size_t)b * ldo + i] = v;
  }
}

// Training pairs, normalised by each input's scale: X = U0 / s, Y = U1 / s (FP32).
__global__ void k_phic_pairs(int N, const double* U0, const double* U1, long ld, float* X,
                             float* Y) {
  __shared__ double red[32];
  const int b = blockIdx.x;
  const double* u = U0 + (size_t)b * ld;
  double m = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, fabs(u[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
  const double inv = t > 0.0 ? 1.0 / t : 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    X[(size_t)b * N + i] = (float)(u[i] * inv);
    Y[(size_t)b * N + i] = (float)(U1[(size_t)b * ld + i] * inv);
  }
}

// Gather a minibatch: xf[k] = X[idx[k]], x0[k] = bf16(xf[k]), y[k] = Y[idx[k]].
__global__ void k_phic_gather(int N, int nb, const int* idx, const float* X, const float* Y,
                              float* xf, __nv_bfloat16* x0, float* y) {
  const int k = blockIdx.y;
  const size_t src = (size_t)idx[k] * N, dst = (size_t)k * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    xf[dst + i] = X[src + i];
    x0[dst + i] = __float2bfloat16(X[src + i]);
    y[dst + i] = Y[src + i];
  }
}

// Output gradient of the mean squared error: gy = (2 / (nb N)) (x + z4 - y),
// loss accumulated into *loss (atomic; the order does not matter for Adam).
__global__ void k_phic_lossgrad(int N, int nb, const float* xf, const float* z4, const float* y,
                                float* gy, float* loss) {
  const size_t tot = (size_t)nb * N;
  const float sc = 2.0f / (float)tot;
  float l = 0.0f;
  for (size_t i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
    const float d = xf[i] + z4[i] - y[i];
    gy[i] = sc * d;
    l += d * d;
  }
  for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, l / (float)tot);
}

// Adam step on FP32 master weights w with moments m, v (t = step number >= 1).
__global__ void k_adam(int cnt, float* w, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FAS coarse right-hand side (two levels, m fine steps per coarse step):
// tau_j = u_{jm} - w_j + r_j for j = 1..Nc, where w_j = Phi_c(u_{(j-1)m}) is
// already in tau_j and r_j (the C-point residual) in r_j.
__global__ void k_fas_tau(int N, int Nc, int m, const double* U, const double* r, double* tau) {
  const int j = blockIdx.y + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const size_t k = (size_t)j * N + i;
    tau[k] = U[(size_t)j * m * N + i] - tau[k] + r[k];
  }
}

// Correction for the C-points as the sweep's C-point correction expects it
// (it adds wc_j + r_j): wc_j = v_j - u_{jm} - r_j, j = 1..Nc.
__global__ void k_fas_corr(int N, int Nc, int m, const double* v, const double* U, const double* r,
                           double* wc) {
  const int j = blockIdx.y + 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const size_t k = (size_t)j * N + i;
    wc[k] = v[k] - U[(size_t)j * m * N + i] - r[k];
  }
}

dim3 pix_grid(int N, int nb) { return dim3((N + 127) / 128, nb); }
dim3 mid_grid(int N, int nb) { return dim3((N + 16 * kMidWarps - 1) / (16 * kMidWarps), nb); }

// The C -> C layers, by the hidden channel count (16 or 32).
template <bool BWD>
void launch_mid(int C, int n, int nb, const __nv_bfloat16* in, const __nv_bfloat16* W,
                const __nv_bfloat16* zprev, __nv_bfloat16* zout, __nv_bfloat16* hout,
                cudaStream_t st) {
  if (C == 32)
    k_phic_mid<32, BWD><<<mid_grid(n * n, nb), 32 * kMidWarps, 0, st>>>(n, in, W, zprev, zout, hout);
  else
    k_phic_mid<16, BWD><<<mid_grid(n * n, nb), 32 * kMidWarps, 0, st>>>(n, in, W, zprev, zout, hout);
}

// The network on nb normalised inputs w.x0 (keep: also the pre-activations).
void network(const PhicNet& net, int nb, PhicWork& w, bool keep, cudaStream_t st) {
  const int n = net.n, N = n * n, C = net.C;
  const size_t L = (size_t)C * NTAP * C;
  k_phic_l1<<<pix_grid(N, nb), 128, 0, st>>>(n, C, w.x0, net.w1, keep ? w.z[0] : nullptr, w.h[0]);
  launch_mid<false>(C, n, nb, w.h[0], net.wf, nullptr, keep ? w.z[1] : nullptr, w.h[1], st);
  launch_mid<false>(C, n, nb, w.h[1], net.wf + L, nullptr, keep ? w.z[2] : nullptr, w.h[2], st);
  k_phic_l4<<<pix_grid(N, nb), 128, 0, st>>>(n, C, w.h[2], net.w4, w.z4);
}

}  // namespace

cudaError_t phic_refresh(const PhicNet& net, cudaStream_t st) {
  const int C = net.C;
  const int tot = 2 * C * NTAP * C + 2 * C * NTAP;
  k_phic_refresh<<<(tot + 255) / 256, 256, 0, st>>>(C, net.wall, net.o[0], net.o[1], net.o[2],
                                                    net.o[3], net.wf, net.wb, net.w1, net.w4);
  return cudaGetLastError();
}

cudaError_t phic_forward(const PhicNet& net, int nb, const double* u, long ldu, const double* add,
                         long lda, const double* sub, long lds, double* out, long ldo,
                         PhicWork& w, cudaStream_t st) {
  const int N = net.n * net.n;
  k_phic_in<<<nb, 256, 0, st>>>(N, u, ldu, w.x0, w.s);
  network(net, nb, w, false, st);
  k_phic_out<<<dim3((N + 255) / 256, nb), 256, 0, st>>>(N, u, ldu, w.z4, w.s, add, lda, sub, lds,
                                                       out, ldo);
  return cudaGetLastError();
}

cudaError_t phic_fas_coarse(const PhicNet& net, int Nc, int m, const double* U, const double* r,
                            double* tau, double* v, double* wc, PhicWork& w, cudaStream_t st) {
  const int N = net.n * net.n;
  const dim3 g((N + 255) / 256, Nc);
  // w_j = Phi_c(u_{(j-1)m}) for all j at once, then tau_j
  cudaError_t e = phic_forward(net, Nc, U, (long)m * N, nullptr, 0, nullptr, 0, tau + N, N, w, st);
  if (e != cudaSuccess) return e;
  k_fas_tau<<<g, 256, 0, st>>>(N, Nc, m, U, r, tau);
  // v_0 = u_0; v_j = Phi_c(v_{j-1}) + tau_j in order
  e = cudaMemcpyAsync(v, U, sizeof(double) * N, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return e;
  for (int j = 1; j <= Nc; ++j) {
    e = phic_forward(net, 1, v + (size_t)(j - 1) * N, N, tau + (size_t)j * N, N, nullptr, 0,
                     v + (size_t)j * N, N, w, st);
    if (e != cudaSuccess) return e;
  }
  k_fas_corr<<<g, 256, 0, st>>>(N, Nc, m, v, U, r, wc);
  return cudaGetLastError();
}

cudaError_t phic_prepare_pairs(int n, int np, const double* U0, const double* U1, long ld,
                               float* X, float* Y, cudaStream_t st) {
  k_phic_pairs<<<np, 256, 0, st>>>(n * n, U0, U1, ld, X, Y);
  return cudaGetLastError();
}

cudaError_t phic_backprop(const PhicNet& net, PhicTrain& t, int nb, const int* idx, float* loss,
                          bool input_grad, cudaStream_t st) {
  const int n = net.n, N = n * n, C = net.C;
  const size_t L = (size_t)C * NTAP * C;
  PhicWork& w = t.work;
  k_phic_gather<<<dim3((N + 255) / 256, nb), 256, 0, st>>>(N, nb, idx, t.X, t.Y, t.xf, w.x0, t.y);
  network(net, nb, w, true, st);
  k_phic_lossgrad<<<64, 256, 0, st>>>(N, nb, t.xf, w.z4, t.y, t.gy, loss);
  // back through layer 4 (weights and input), then the two C -> C layers
  const dim3 tg(NTAP, nb);
  float* P = t.part;
  const long cnt = net.count;
  if (C == 32) k_phic_wgrad1<32, false><<<tg, 256, 0, st>>>(n, nullptr, nullptr, t.gy, w.h[2], P + net.o[3], cnt);
  else k_phic_wgrad1<16, false><<<tg, 256, 0, st>>>(n, nullptr, nullptr, t.gy, w.h[2], P + net.o[3], cnt);
  k_phic_l4_back<<<pix_grid(N, nb), 128, 0, st>>>(n, C, t.gy, net.w4, w.z[2], t.gz[2]);
  for (int l = 2; l >= 1; --l) {
    // weight gradient of layer l + 1 (K2 or K3) from gz_l and its input h_{l-1}
    if (C == 32) k_phic_wgrad<32><<<tg, 32 * kMidWarps, 0, st>>>(n, t.gz[l], w.h[l - 1], P + net.o[l], cnt);
    else k_phic_wgrad<16><<<tg, 32 * kMidWarps, 0, st>>>(n, t.gz[l], w.h[l - 1], P + net.o[l], cnt);
    // gradient through it and through the GELU below: gz_{l-1}
    launch_mid<true>(C, n, nb, t.gz[l], net.wb + (size_t)(l - 1) * L, w.z[l - 1], nullptr,
                     t.gz[l - 1], st);
  }
  if (C == 32) k_phic_wgrad1<32, true><<<tg, 256, 0, st>>>(n, t.gz[0], w.x0, nullptr, nullptr, P + net.o[0], cnt);
  else k_phic_wgrad1<16, true><<<tg, 256, 0, st>>>(n, t.gz[0], w.x0, nullptr, nullptr, P + net.o[0], cnt);
  k_phic_sum_parts<<<(net.count + 255) / 256, 256, 0, st>>>(nb, net.count, P, t.gw);
  if (input_grad) k_phic_l1_back<<<pix_grid(N, nb), 128, 0, st>>>(n, C, t.gy, net.w1, t.gz[0], t.gx);
  return cudaGetLastError();
}

cudaError_t phic_adam(PhicNet& net, PhicTrain& t, int step, float lr, cudaStream_t st) {
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)(step + 1)), c2 = 1.0f - powf(b2, (float)(step + 1));
  k_adam<<<(net.count + 255) / 256, 256, 0, st>>>(net.count, net.wall, t.gw, t.m, t.v, lr, b1, b2,
                                                  1e-8f, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return phic_refresh(net, st);
}

}  // namespace igm
