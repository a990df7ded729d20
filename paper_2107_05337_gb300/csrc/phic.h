// Device data and kernel launchers of the learned coarse propagator (phic.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace igm {

constexpr int kPhicMaxC = 8;  // max channels of the hidden layers

// Network weights (FP32, used by the BF16 kernels after conversion of the
// activations): wall = [w1 (C x 1 x 25) | w2 (C x C x 25) | w3 (1 x C x 25)].
struct PhicNet {
  int n = 0, C = 0, count = 0;
  int o1 = 0, o2 = 0, o3 = 0;
  float* wall = nullptr;
  float *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
};

// Per-batch activations: x0 [nb][N] BF16, a1, a2 [nb][C][N] BF16, z3 [nb][N] FP32, s [nb].
struct PhicWork {
  int cap = 0;
  __nv_bfloat16 *x0 = nullptr, *a1 = nullptr, *a2 = nullptr;
  float* z3 = nullptr;
  double* s = nullptr;
};

// Training state: normalised pairs X, Y (FP32); the batch inputs xf and targets y,
// gradients g1, g2 ([nb][C][N]) and g3 ([nb][N]); flipped kernels; weight
// gradient gw, Adam moments m, v; per-step losses.
struct PhicTrain {
  int np = 0;
  float *X = nullptr, *Y = nullptr;
  float *xf = nullptr, *y = nullptr, *g1 = nullptr, *g2 = nullptr, *g3 = nullptr;
  float *wf2 = nullptr, *wf3 = nullptr;
  float *gw = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  PhicWork work;
};

// out_b = Phi_c(u_b) (+ add_b) (- sub_b) for nb vectors of N = n*n (FP64,
// row strides ldu, lda, lds, ldo); w must hold nb images.
cudaError_t phic_forward(const PhicNet& net, int nb, const double* u, long ldu, const double* add,
                         long lda, const double* sub, long lds, double* out, long ldo,
                         PhicWork& w, cudaStream_t st);
// FAS coarse level of two-level MGRIT with Phi_c (Nc coarse steps of m fine
// steps; U [Nl+1][N] the fine iterate, r [Nc+1][N] the C-point residuals at
// rows 1..Nc): tau, v [Nc+1][N] scratch; writes wc [Nc+1][N] (rows 1..Nc) =
// v_j - u_{jm} - r_j.  w must hold Nc images.
cudaError_t phic_fas_coarse(const PhicNet& net, int Nc, int m, const double* U, const double* r,
                            double* tau, double* v, double* wc, PhicWork& w, cudaStream_t st);
cudaError_t phic_prepare_pairs(int n, int np, const double* U0, const double* U1, long ld,
                               float* X, float* Y, cudaStream_t st);
// One Adam step on the minibatch idx[0..nb); loss of the step added to t.loss[step].
cudaError_t phic_train_step(PhicNet& net, PhicTrain& t, int nb, const int* idx, int step, float lr,
                            cudaStream_t st);

}  // namespace igm
