// Solver kernels instantiated for the FP64 form.
#include "kernels_impl.cuh"

namespace igm {

cudaError_t launch_pmg_solve_f64(const PmgD& P, int grid, long smem, cudaStream_t st,
                                 const double* b, double* x, long ld, int ncycles, int* cycles_out,
                                 int* status, char* garena) {
  k_pmg_solve<0><<<grid, kBlock, smem, st>>>(P, b, x, ld, ncycles, cycles_out, status, garena);
  return cudaGetLastError();
}

cudaError_t launch_ilut_apply_f64(const PmgD& P, int grid, long smem, cudaStream_t st,
                                  const double* r, double* z, long ld, char* garena, int* status) {
  k_ilut_apply<0><<<grid, kBlock, smem, st>>>(P, r, z, ld, garena, status);
  return cudaGetLastError();
}

cudaError_t launch_mgrit_sweep_f64(const SweepArgs& a, int grid, long smem, cudaStream_t st) {
  k_mgrit_sweep<0><<<grid, kBlock, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t set_smem_f64(long bytes) {
  cudaError_t e = cudaFuncSetAttribute((const void*)k_pmg_solve<0>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_ilut_apply<0>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_mgrit_sweep<0>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

// y = M x or y = K x in FP64 (iga_apply).
__global__ void __launch_bounds__(kBlock) k_apply_op(PmgD P, int which, const double* x,
                                                     double* y, long ld, double* scratch) {
  const double* xc = x + (size_t)blockIdx.x * ld;
  double* yc = y + (size_t)blockIdx.x * ld;
  double* tm = scratch + (size_t)blockIdx.x * 2 * P.N;
  double* tk = tm + P.N;
  if (P.affine) {
    if (which == 0)
      apply_A_affine<double>(P.n, P.p, P.bM64, (const double*)nullptr, P.bM64,
                             (const double*)nullptr, xc, (const double*)nullptr,
                             (const double*)nullptr, yc, tm, (double*)nullptr, (double*)nullptr);
    else
      apply_A_affine<double>(P.n, P.p, P.bM64, P.bK64, P.bK64, P.bM64, xc, (const double*)nullptr,
                             (const double*)nullptr, yc, tm, tk, (double*)nullptr);
  } else {
    apply_stencil<double>(P.n, P.w, which == 0 ? P.sM64 : P.sA64, xc, (const double*)nullptr,
                          (const double*)nullptr, yc, (double*)nullptr);
  }
}

// Failure-detection self-test: the same bounded wait the record ring uses, on
// a barrier that nothing completes; the kernel then returns normally.
__global__ void k_wait_selftest(long spins, int* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  const bool got = mbar_wait(&bar, 0u, spins);
  if (!got && threadIdx.x == 0) atomicMin(status, ST_TIMEOUT);
}

cudaError_t launch_wait_selftest(long spins, int* status, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(spins, status);
  return cudaGetLastError();
}

cudaError_t launch_apply_op(const PmgD& P, int which, int nrhs, const double* x, double* y, long ld,
                            double* scratch, cudaStream_t st) {
  k_apply_op<<<nrhs, kBlock, 0, st>>>(P, which, x, y, ld, scratch);
  return cudaGetLastError();
}

}  // namespace igm
