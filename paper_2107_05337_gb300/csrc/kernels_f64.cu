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

cudaError_t launch_mgrit_level_f64(const SweepArgs& a, int grid, long smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mgrit_sweep<0>, a);
}

cudaError_t launch_mgrit_batch_f64(const BatchMember* mem, BatchState* st, int nmem,
                                   unsigned long long* ctl, int grid, long smem, cudaStream_t s) {
  k_mgrit_batch<0><<<grid, kBlock, smem, s>>>(mem, st, nmem, ctl);
  return cudaGetLastError();
}

int mgrit_sweep_max_resident_f64(long smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mgrit_sweep<0>, kBlock,
                                                    (size_t)smem) != cudaSuccess)
    return 0;
  return per * sms;
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
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_mgrit_batch<0>,
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

// Failure-detection self-test of the grid barrier of the fused level visits:
// two barriers; with hold, CTA 0 does not arrive at the first one.
__global__ void k_barrier_selftest(long long cycles, int hold, unsigned* gbar, int* status) {
  if (!grid_barrier(gbar, (int)gridDim.x, cycles, status, hold && blockIdx.x == 0)) return;
  grid_barrier(gbar, (int)gridDim.x, cycles, status, false);
}

cudaError_t launch_barrier_selftest(int nctas, long long cycles, int hold, unsigned* gbar,
                                    int* status, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(32);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_barrier_selftest, cycles, hold, gbar, status);
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
