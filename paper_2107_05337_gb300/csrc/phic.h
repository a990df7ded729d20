// Device data and kernel launchers of the learned coarse propagator (phic.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace igm {

constexpr int kPhicLayers = 4;  // 3 x 3 convolutions: 1 -> C, C -> C, C -> C, C -> 1

// Network weights.  wall: the FP32 master copy [K1 (C,1,3,3) | K2 (C,C,3,3) |
// K3 (C,C,3,3) | K4 (1,C,3,3)] (tap t = 3a + b of kernel row a, column b).
// The BF16 copies the kernels read, refreshed from wall by phic_refresh:
// wf = K2, K3 as [cout][tap][cin] (the forward products); wb = the same
// kernels for the input gradient, [cin][8 - tap][cout]; w1 = K1 as
// [cout][tap] and w4 = K4 as [tap][cin], rounded to BF16 and held as FP32.
struct PhicNet {
  int n = 0, C = 0, count = 0;
  int o[kPhicLayers] = {0, 0, 0, 0};
  float* wall = nullptr;
  __nv_bfloat16* wf = nullptr;   // [2][C][9][C]
  __nv_bfloat16* wb = nullptr;   // [2][C][9][C]
  float* w1 = nullptr;           // [C][9]
  float* w4 = nullptr;           // [9][C]
};

// Activations of nb images: x0 [nb][N] BF16 (the normalised input), the
// pre-activations z1..z3 and the GELU outputs h1..h3 [nb][N][C] BF16
// (channel fastest), z4 [nb][N] FP32 (the network output), s [nb] (scales).
// The z's are kept for training only (nullptr for inference).
struct PhicWork {
  int cap = 0;
  __nv_bfloat16* x0 = nullptr;
  __nv_bfloat16 *z[3] = {nullptr, nullptr, nullptr}, *h[3] = {nullptr, nullptr, nullptr};
  float* z4 = nullptr;
  double* s = nullptr;
};

// Training state: normalised pairs X, Y (FP32); the batch inputs xf and targets
// y; the output gradient gy [nb][N] FP32; the pre-activation gradients gz1..gz3
// [nb][N][C] BF16; per-image partial weight gradients part [nb][count]; the
// weight gradient gw, Adam moments m, v; per-step losses; the input gradient
// gx [nb][N] (phic_grad only).
struct PhicTrain {
  int np = 0;
  float *X = nullptr, *Y = nullptr;
  float *xf = nullptr, *y = nullptr, *gy = nullptr;
  __nv_bfloat16* gz[3] = {nullptr, nullptr, nullptr};
  float *part = nullptr, *gw = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr, *gx = nullptr;
  PhicWork work;
};

// Refresh the BF16 weight copies from the FP32 master weights.
cudaError_t phic_refresh(const PhicNet& net, cudaStream_t st);
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
// Loss and weight gradient t.gw of the minibatch idx[0..nb) (loss of the step
// added to *loss); with input_grad also t.gx.
cudaError_t phic_backprop(const PhicNet& net, PhicTrain& t, int nb, const int* idx, float* loss,
                          bool input_grad, cudaStream_t st);
// One Adam step (t = step + 1) with the gradient in t.gw, then phic_refresh.
cudaError_t phic_adam(PhicNet& net, PhicTrain& t, int step, float lr, cudaStream_t st);

}  // namespace igm
