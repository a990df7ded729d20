// Kernel launch interface between the host code (capi.cu) and the kernel
// translation units (kernels_f32.cu: mixed form, kernels_f64.cu: FP64 form).
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace igm {

// MGRIT sweep modes (Sec. 3): F-relaxation, C-relaxation, F-relaxation plus
// C-point residual and injection, coarse correction plus F-relaxation (ideal
// interpolation), sequential stepping on the coarsest level, and the C-point
// residual alone.
enum : int { MODE_F = 0, MODE_C = 1, MODE_FR = 2, MODE_CF = 3, MODE_SEQ = 4, MODE_R = 5,
             MODE_FUSED = 6 /* profile records of a fused level visit */ };

struct SweepArgs {
  PmgD P;
  int mode, m, Nl, nint;
  double* W;              // [Nl+1][N]: the part of u each step's solve produces
  const double* g;        // [Nl+1][N] right-hand side g^(l) (nullptr on the fine level)
  const double* Wc;       // next level's W and g (correction)
  const double* gc;
  double* gnext;          // next level's g, written by the residual
  double* norms;          // [nint] ||r_j||^2 (fine level) or nullptr
  const double* fhat;     // fine level source profile or nullptr
  const double* fcoef;    // device [Nt+1] time factors
  double dt0;
  double theta;           // theta-scheme weight of the source: theta c(t_n) + (1-theta) c(t_{n-1})
  double* scratch;        // per CTA: 2 N doubles (rhs, residual iterate)
  char* garena;
  int ncycles;
  unsigned long long* counters;  // [0] solves, [1] cycles
  int* status;
  // fused level visit (one cooperative launch): the modes run in this order
  // with a bounded grid barrier between consecutive ones; nmodes = 0: `mode` alone
  int nmodes;
  int modes[3];
  unsigned* gbar;         // [0] arrivals, [1] generation, [2] abort; zeroed before the launch
  long long bar_cycles;   // bound of one barrier wait in SM clocks
};

// ---------------------------------------------------------------------------
// Device-scheduled batch of MGRIT solves (one persistent launch for many
// independent problems).  Each member's run is a program of phases: A0 (the
// first fine-level part), then B (coarse levels and the fine correction) and
// A (a later fine-level part) repeated; every A-part ends with the stopping
// test.  A phase is `grid` tasks (one per interval) of one sweep mode on one
// level, the zeroing of a level's iterate, or the test.  Persistent CTAs
// claim tasks of the members' current phases; the CTA that completes a
// phase's last task moves the member to its next phase.
// ---------------------------------------------------------------------------
enum : int { BOP_SWEEP = 0, BOP_ZERO = 1, BOP_TEST = 2 };
constexpr int kBatchHist = 256;   // residual norms kept per member

struct BatchPhase {
  int level, mode, grid, op;
};

struct BatchMember {
  const SweepArgs* lv;     // [levels] arguments of every level's sweeps
  const BatchPhase* prog;  // [nA0 + nB + nA]: A0, then B, then A
  int nA0, nB, nA;
  int nint0;               // fine-level C-intervals: entries of norms
  const double* norms;     // [nint0] ||r_j||^2 written by the fine-level residual phase
  double tol;
  int max_iter;
};

struct BatchState {
  unsigned long long word;   // (phase << 32) | next task of the phase
  int done;                  // tasks of the current phase completed
  int it;                    // coarse corrections done
  int finished;
  int nhist;
  unsigned long long t_end;  // globaltimer (ns) at the end of the member's run
  double hist[kBatchHist];
};

// Run the batch: nmem members (in the order of `mem`, which is also the order
// in which idle CTAs look for work), `grid` persistent CTAs with `smem` bytes
// of dynamic shared memory.  ctl: [0] progress count, [1] abort flag, [2]
// start time (globaltimer ns); zeroed by the caller.  A CTA that finds no
// work for kWaitCycles SM clocks while no task anywhere completes raises the
// abort flag and every CTA returns.
cudaError_t launch_mgrit_batch(int prec, const BatchMember* mem, BatchState* st, int nmem,
                               unsigned long long* ctl, int grid, long smem, cudaStream_t st_);
cudaError_t launch_mgrit_batch_f32(const BatchMember*, BatchState*, int, unsigned long long*, int,
                                   long, cudaStream_t);
cudaError_t launch_mgrit_batch_f64(const BatchMember*, BatchState*, int, unsigned long long*, int,
                                   long, cudaStream_t);

// prec: 0 = FP64 form, 1 = mixed form.  Each returns cudaGetLastError().
cudaError_t launch_pmg_solve(int prec, const PmgD& P, int grid, long smem, cudaStream_t st,
                             const double* b, double* x, long ld, int ncycles, int* cycles_out,
                             int* status, char* garena);
cudaError_t launch_ilut_apply(int prec, const PmgD& P, int grid, long smem, cudaStream_t st,
                              const double* r, double* z, long ld, char* garena, int* status);
cudaError_t launch_mgrit_sweep(int prec, const SweepArgs& a, int grid, long smem, cudaStream_t st);
// The same kernel launched cooperatively (all CTAs resident at once), for a
// fused level visit (a.nmodes > 1).
cudaError_t launch_mgrit_level(int prec, const SweepArgs& a, int grid, long smem, cudaStream_t st);
// CTAs of the sweep kernel that can be resident at once on the current device
// with `smem` bytes of dynamic shared memory (0 on error).
int mgrit_sweep_max_resident(int prec, long smem);
// Failure-detection self-test of the grid barrier: nctas CTAs (cooperative
// launch) pass two barriers; with hold, CTA 0 never arrives at the first, so
// every CTA's wait runs out after `cycles` SM clocks and records ST_TIMEOUT.
cudaError_t launch_barrier_selftest(int nctas, long long cycles, int hold, unsigned* gbar,
                                    int* status, cudaStream_t st);
cudaError_t launch_apply_op(const PmgD& P, int which, int nrhs, const double* x, double* y, long ld,
                            double* scratch, cudaStream_t st);
// One CTA waits (bounded by `spins` polls) on an mbarrier that no copy or
// arrival will ever complete, and records ST_TIMEOUT in *status.
cudaError_t launch_wait_selftest(long spins, int* status, cudaStream_t st);
// Allow up to `bytes` of dynamic shared memory for the solve kernels.
cudaError_t set_solver_smem(long bytes);

// per-precision entry points (kernels_f32.cu / kernels_f64.cu)
cudaError_t launch_pmg_solve_f32(const PmgD&, int, long, cudaStream_t, const double*, double*, long,
                                 int, int*, int*, char*);
cudaError_t launch_pmg_solve_f64(const PmgD&, int, long, cudaStream_t, const double*, double*, long,
                                 int, int*, int*, char*);
cudaError_t launch_ilut_apply_f32(const PmgD&, int, long, cudaStream_t, const double*, double*, long,
                                  char*, int*);
cudaError_t launch_ilut_apply_f64(const PmgD&, int, long, cudaStream_t, const double*, double*, long,
                                  char*, int*);
cudaError_t launch_mgrit_sweep_f32(const SweepArgs&, int, long, cudaStream_t);
cudaError_t launch_mgrit_sweep_f64(const SweepArgs&, int, long, cudaStream_t);
cudaError_t launch_mgrit_level_f32(const SweepArgs&, int, long, cudaStream_t);
cudaError_t launch_mgrit_level_f64(const SweepArgs&, int, long, cudaStream_t);
int mgrit_sweep_max_resident_f32(long smem);
int mgrit_sweep_max_resident_f64(long smem);
cudaError_t set_smem_f32(long bytes);
cudaError_t set_smem_f64(long bytes);

}  // namespace igm
