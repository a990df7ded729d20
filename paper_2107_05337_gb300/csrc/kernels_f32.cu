// Solver kernels instantiated for the mixed (FP32 smoothing, FP64 refinement) form.
#include "kernels_impl.cuh"

namespace igm {

cudaError_t launch_pmg_solve_f32(const PmgD& P, int grid, long smem, cudaStream_t st,
                                 const double* b, double* x, long ld, int ncycles, int* cycles_out,
                                 int* status, char* garena) {
  k_pmg_solve<1><<<grid, kBlock, smem, st>>>(P, b, x, ld, ncycles, cycles_out, status, garena);
  return cudaGetLastError();
}

cudaError_t launch_ilut_apply_f32(const PmgD& P, int grid, long smem, cudaStream_t st,
                                  const double* r, double* z, long ld, char* garena, int* status) {
  k_ilut_apply<1><<<grid, kBlock, smem, st>>>(P, r, z, ld, garena, status);
  return cudaGetLastError();
}

cudaError_t launch_mgrit_sweep_f32(const SweepArgs& a, int grid, long smem, cudaStream_t st) {
  k_mgrit_sweep<1><<<grid, kBlock, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_mgrit_level_f32(const SweepArgs& a, int grid, long smem, cudaStream_t st) {
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
  return cudaLaunchKernelEx(&cfg, k_mgrit_sweep<1>, a);
}

cudaError_t launch_mgrit_batch_f32(const BatchMember* mem, BatchState* st, int nmem,
                                   unsigned long long* ctl, int grid, long smem, cudaStream_t s) {
  k_mgrit_batch<1><<<grid, kBlock, smem, s>>>(mem, st, nmem, ctl);
  return cudaGetLastError();
}

int mgrit_sweep_max_resident_f32(long smem) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_mgrit_sweep<1>, kBlock,
                                                    (size_t)smem) != cudaSuccess)
    return 0;
  return per * sms;
}

cudaError_t set_smem_f32(long bytes) {
  cudaError_t e = cudaFuncSetAttribute((const void*)k_pmg_solve<1>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_ilut_apply<1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_mgrit_sweep<1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute((const void*)k_mgrit_batch<1>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

}  // namespace igm
