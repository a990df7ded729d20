// Learned coarse propagator Phi_c for MGRIT: a 5 x 5 convolutional network on
// the n x n grid of interior coefficients (zero padding = the homogeneous
// Dirichlet condition), BF16 weights and activations with FP32 accumulation:
//   x = u / s (s = max |u|),  Phi_c(u) = u + s * K3 * tanh(K2 * tanh(K1 * x)),
// and the kernels of its training (back-propagation, Adam).  Every tensor is
// [image][channel][row][column] with row-major n x n planes.
#include <cuda_bf16.h>
#include <stdint.h>

#include "phic.h"

namespace igm {

namespace {

constexpr int KS = 5, HALO = 2, TILE = 16, TW = TILE + 2 * HALO;
constexpr int kMaxC = kPhicMaxC;  // max channels of one layer (inputs and outputs)

template <typename T>
__device__ __forceinline__ float ld_as_float(const T* p, size_t i);
template <>
__device__ __forceinline__ float ld_as_float<float>(const float* p, size_t i) { return p[i]; }
template <>
__device__ __forceinline__ float ld_as_float<__nv_bfloat16>(const __nv_bfloat16* p, size_t i) {
  return __bfloat162float(p[i]);
}

// out[b][o] = sum_c w[o][c] * in[b][c] (5 x 5 'same' correlation), one
// 16 x 16 output tile of one image per CTA (256 threads).  Epilogue:
//   EPI_TANH:  out = bf16(tanh(z))
//   EPI_F32:   out = z (FP32)
//   EPI_DTANH: out = z * (1 - a^2) with a = act[b][o] (BF16 activations of
//              the forward pass; FP32 output: the gradient through tanh)
enum { EPI_TANH = 0, EPI_F32 = 1, EPI_DTANH = 2 };
template <typename TI, int EPI>
__global__ void __launch_bounds__(TILE * TILE) k_conv5(int n, int cin, int cout, const TI* in,
                                                       const float* w, void* out,
                                                       const __nv_bfloat16* act) {
  __shared__ float tile[kMaxC][TW][TW];
  __shared__ float ws[kMaxC * kMaxC * KS * KS];
  const int b = blockIdx.z;
  const int ty0 = blockIdx.y * TILE, tx0 = blockIdx.x * TILE;
  const size_t plane = (size_t)n * n;
  for (int i = threadIdx.x; i < cout * cin * KS * KS; i += blockDim.x) ws[i] = w[i];
  for (int i = threadIdx.x; i < cin * TW * TW; i += blockDim.x) {
    const int c = i / (TW * TW), r = (i / TW) % TW, q = i % TW;
    const int y = ty0 + r - HALO, x = tx0 + q - HALO;
    tile[c][r][q] = (y >= 0 && y < n && x >= 0 && x < n)
                        ? ld_as_float(in, ((size_t)b * cin + c) * plane + (size_t)y * n + x)
                        : 0.0f;
  }
  __syncthreads();
  const int ly = threadIdx.x / TILE, lx = threadIdx.x % TILE;
  const int y = ty0 + ly, x = tx0 + lx;
  if (y >= n || x >= n) return;
  for (int o = 0; o < cout; ++o) {
    float z = 0.0f;
    for (int c = 0; c < cin; ++c) {
      const float* wk = ws + (o * cin + c) * KS * KS;
#pragma unroll
      for (int a = 0; a < KS; ++a)
#pragma unroll
        for (int q = 0; q < KS; ++q) z = fmaf(wk[a * KS + q], tile[c][ly + a][lx + q], z);
    }
    const size_t idx = ((size_t)b * cout + o) * plane + (size_t)y * n + x;
    if (EPI == EPI_TANH) {
      ((__nv_bfloat16*)out)[idx] = __float2bfloat16(tanhf(z));
    } else if (EPI == EPI_F32) {
      ((float*)out)[idx] = z;
    } else {
      const float a = __bfloat162float(act[idx]);
      ((float*)out)[idx] = z * (1.0f - a * a);
    }
  }
}

// Weight gradient gw[o][c][a][q] = sum_b sum_{y,x} g[b][o][y][x] *
// in[b][c][y+a-2][x+q-2]; one CTA per (o, c, a, q), a CTA-wide reduction.
template <typename TI>
__global__ void k_wgrad5(int n, int nb, int cin, int cout, const float* g, const TI* in, float* gw) {
  __shared__ float red[32];
  const int k = blockIdx.x;
  const int q = k % KS, a = (k / KS) % KS, c = (k / (KS * KS)) % cin, o = k / (KS * KS * cin);
  const size_t plane = (size_t)n * n;
  float s = 0.0f;
  const long tot = (long)nb * n * n;
  for (long i = threadIdx.x; i < tot; i += blockDim.x) {
    const int b = (int)(i / plane), p = (int)(i % plane), y = p / n, x = p % n;
    const int yy = y + a - HALO, xx = x + q - HALO;
    if (yy < 0 || yy >= n || xx < 0 || xx >= n) continue;
    s = fmaf(g[((size_t)b * cout + o) * plane + p],
             ld_as_float(in, ((size_t)b * cin + c) * plane + (size_t)yy * n + xx), s);
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    gw[k] = t;
  }
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
  for (int i = threadIdx.x; i < N; i += blockDim.x) x0[(size_t)b * N + i] = __float2bfloat16((float)(ub[i] * inv));
}

// out_b = u_b + s_b * z3_b (+ add_b) (- sub_b): the network output, optionally
// with a vector added and one subtracted (the FAS terms), in FP64.
__global__ void k_phic_out(int N, const double* u, long ldu, const float* z3, const double* s,
                           const double* add, long lda, const double* sub, long lds, double* out,
                           long ldo) {
  const int b = blockIdx.y;
  const double sb = s[b];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    double v = u[(size_t)b * ldu + i] + sb * (double)z3[(size_t)b * N + i];
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

// Output gradient of the mean squared error: g = (2 / (nb N)) (x + z3 - y),
// loss accumulated into *loss (atomic; the order does not matter for Adam).
__global__ void k_phic_lossgrad(int N, int nb, const float* xf, const float* z3, const float* y,
                                float* g, float* loss) {
  const size_t tot = (size_t)nb * N;
  const float sc = 2.0f / (float)tot;
  float l = 0.0f;
  for (size_t i = blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += gridDim.x * blockDim.x) {
    const float d = xf[i] + z3[i] - y[i];
    g[i] = sc * d;
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

// Flipped, channel-transposed copy of a kernel (for the input gradient):
// wf[c][o][a][q] = w[o][c][4-a][4-q].
__global__ void k_flip(int cin, int cout, const float* w, float* wf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cin * cout * KS * KS) return;
  const int q = i % KS, a = (i / KS) % KS, c = (i / (KS * KS)) % cin, o = i / (KS * KS * cin);
  wf[((c * cout + o) * KS + (KS - 1 - a)) * KS + (KS - 1 - q)] = w[i];
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

dim3 conv_grid(int n, int nb) { return dim3((n + TILE - 1) / TILE, (n + TILE - 1) / TILE, nb); }

}  // namespace

cudaError_t phic_forward(const PhicNet& net, int nb, const double* u, long ldu, const double* add,
                         long lda, const double* sub, long lds, double* out, long ldo,
                         PhicWork& w, cudaStream_t st) {
  const int n = net.n, N = n * n, C = net.C;
  k_phic_in<<<nb, 256, 0, st>>>(N, u, ldu, w.x0, w.s);
  k_conv5<__nv_bfloat16, EPI_TANH><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, 1, C, w.x0, net.w1, w.a1, nullptr);
  k_conv5<__nv_bfloat16, EPI_TANH><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, C, C, w.a1, net.w2, w.a2, nullptr);
  k_conv5<__nv_bfloat16, EPI_F32><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, C, 1, w.a2, net.w3, w.z3, nullptr);
  k_phic_out<<<dim3((N + 255) / 256, nb), 256, 0, st>>>(N, u, ldu, w.z3, w.s, add, lda, sub, lds, out, ldo);
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

cudaError_t phic_train_step(PhicNet& net, PhicTrain& t, int nb, const int* idx, int step, float lr,
                            cudaStream_t st) {
  const int n = net.n, N = n * n, C = net.C;
  PhicWork& w = t.work;
  k_phic_gather<<<dim3((N + 255) / 256, nb), 256, 0, st>>>(N, nb, idx, t.X, t.Y, t.xf, w.x0, t.y);
  // forward
  k_conv5<__nv_bfloat16, EPI_TANH><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, 1, C, w.x0, net.w1, w.a1, nullptr);
  k_conv5<__nv_bfloat16, EPI_TANH><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, C, C, w.a1, net.w2, w.a2, nullptr);
  k_conv5<__nv_bfloat16, EPI_F32><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, C, 1, w.a2, net.w3, w.z3, nullptr);
  k_phic_lossgrad<<<64, 256, 0, st>>>(N, nb, t.xf, w.z3, t.y, t.g3, t.loss + step);
  // backward
  k_flip<<<(C * KS * KS + 255) / 256, 256, 0, st>>>(C, 1, net.w3, t.wf3);
  k_flip<<<(C * C * KS * KS + 255) / 256, 256, 0, st>>>(C, C, net.w2, t.wf2);
  k_wgrad5<__nv_bfloat16><<<C * KS * KS, 256, 0, st>>>(n, nb, C, 1, t.g3, w.a2, t.gw + net.o3);
  k_conv5<float, EPI_DTANH><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, 1, C, t.g3, t.wf3, t.g2, w.a2);
  k_wgrad5<__nv_bfloat16><<<C * C * KS * KS, 256, 0, st>>>(n, nb, C, C, t.g2, w.a1, t.gw + net.o2);
  k_conv5<float, EPI_DTANH><<<conv_grid(n, nb), TILE * TILE, 0, st>>>(n, C, C, t.g2, t.wf2, t.g1, w.a1);
  k_wgrad5<__nv_bfloat16><<<C * KS * KS, 256, 0, st>>>(n, nb, 1, C, t.g1, w.x0, t.gw + net.o1);
  // Adam on all weights at once (w1, w2, w3 are contiguous in net.wall)
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)(step + 1)), c2 = 1.0f - powf(b2, (float)(step + 1));
  k_adam<<<(net.count + 255) / 256, 256, 0, st>>>(net.count, net.wall, t.gw, t.m, t.v, lr, b1, b2,
                                                  1e-8f, c1, c2);
  return cudaGetLastError();
}

}  // namespace igm
