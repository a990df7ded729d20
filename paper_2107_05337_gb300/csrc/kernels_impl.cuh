// Kernel templates of the solver, instantiated per precision in
// kernels_f32.cu (mixed form) and kernels_f64.cu (FP64 form).
#pragma once
#include <type_traits>

#include "kernels.h"
#include "solver.cuh"

namespace igm {

// Dynamic shared memory: [record ring][mbarriers] then the CTA's arena when it
// fits; otherwise the arena is this CTA's slice of the global scratch.
__device__ __forceinline__ char* cta_setup(const PmgD& P, char* garena, Pipe& pp,
                                           int slot = -1) {
  extern __shared__ __align__(128) char dyn_smem[];
  pp.ring = dyn_smem;
  pp.bar = (uint64_t*)(dyn_smem + (size_t)P.nstage * P.slot_bytes);
  pp.nstage = P.nstage;
  pp.slot = P.slot_bytes;
  pipe_init(pp);
  if (slot < 0) slot = (int)blockIdx.x;
  return P.arena_smem ? dyn_smem + P.ring_bytes : garena + (size_t)slot * P.arena_bytes;
}

template <int PREC>
__global__ void __launch_bounds__(kBlock) k_pmg_solve(PmgD P, const double* b, double* x, long ld,
                                                      int ncycles, int* cycles_out, int* status,
                                                      char* garena) {
  __shared__ double red[32];
  Pipe pp;
  char* arena = cta_setup(P, garena, pp);
  const double* bc = b + (size_t)blockIdx.x * ld;
  double* xc = x + (size_t)blockIdx.x * ld;
  const int c = pmg_solve<PREC>(P, pp, bc, xc, arena, red, ncycles, status);
  if (threadIdx.x == 0 && cycles_out) cycles_out[blockIdx.x] = c;
}

template <int PREC>
__global__ void __launch_bounds__(kBlock) k_ilut_apply(PmgD P, const double* r, double* z, long ld,
                                                       char* garena, int* status) {
  using T = typename std::conditional<PREC == 0, double, float>::type;
  Pipe pp;
  char* arena = cta_setup(P, garena, pp);
  const double* rc = r + (size_t)blockIdx.x * ld;
  double* zc = z + (size_t)blockIdx.x * ld;
  T* A = (T*)arena;
  T* t = A + P.o_t;
  IGM_FOR_CTA(i, P.N) t[i] = (T)rc[i];
  __syncthreads();
  ilut_apply<T>(P, pp, t, status);
  IGM_FOR_CTA(i, P.N) zc[i] = (double)t[i];
}

// One backward-Euler step into point n of the level (Sec. 3: the step
// u_n = Phi_l(u_{n-1}) + g_n with Phi_l = (M + kappa dt_l K)^{-1} M), or the
// C-point residual r = Phi_l(u_{n-1}) + g_n - u_n injected into g^(l+1)_{j+1}.
template <int PREC>
__device__ __forceinline__ void mgrit_step(const SweepArgs& a, Pipe& pp, char* arena, double* red,
                                           int n, bool residual, int j) {
  const PmgD& P = a.P;
  const int N = P.N;
  double* rhs = a.scratch + (size_t)j * 2 * N;
  double* xr = rhs + N;
  double* tm = (PREC == 0) ? (double*)arena + P.o_u : (double*)((float*)arena + P.o_d);
  const double* u = a.W + (size_t)(n - 1) * N;
  const double* ug = a.g ? a.g + (size_t)(n - 1) * N : nullptr;
  const double scale =
      a.fhat ? a.dt0 * (a.theta * a.fcoef[n] + (1.0 - a.theta) * a.fcoef[n - 1]) : 0.0;
  {
    PhaseClock pc(P.trace);
    build_rhs(P, u, ug, scale, a.fhat, rhs, tm);
    pc.stop(6);
  }
  double* Wn = a.W + (size_t)n * N;
  double* x = Wn;
  if (residual) {
    IGM_FOR_CTA(i, N) xr[i] = Wn[i];
    __syncthreads();
    x = xr;
  }
  const int cyc = pmg_solve<PREC>(P, pp, rhs, x, arena, red, a.ncycles, a.status);
  if (threadIdx.x == 0 && a.counters) {
    atomicAdd(&a.counters[0], 1ull);
    atomicAdd(&a.counters[1], (unsigned long long)cyc);
  }
  if (residual) {
    double* gout = a.gnext + (size_t)(j + 1) * N;
    double s = 0.0;
    IGM_FOR_CTA(i, N) {
      const double r = xr[i] - Wn[i];
      gout[i] = r;
      s += r * r;
    }
    s = block_sum(s, red);
    if (a.norms && threadIdx.x == 0) a.norms[j] = s;
  }
}

// Bounded barrier over all CTAs of a cooperatively launched kernel (the
// phases of one MGRIT level visit, Sec. 3).  gb[0] counts arrivals, gb[1] is
// the generation, gb[2] an abort flag; the host zeroes them before the
// launch.  Thread 0 of each CTA arrives, then waits (suspended for short
// periods, at most `cycles` SM clocks) for the generation to change; a CTA
// that gives up records ST_TIMEOUT and raises the abort flag, so that the
// others stop waiting as well.  hold: this CTA does not arrive (the
// failure-detection self-test).  Returns false on a timeout (CTA-uniform).
__device__ inline bool grid_barrier(unsigned* gb, int nctas, long long cycles, int* status,
                                    bool hold) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    s_ok = 1;
    volatile unsigned* vgb = gb;
    const unsigned gen = vgb[1];
    __threadfence();  // this CTA's writes before its arrival
    bool released = false;
    if (!hold && atomicAdd(gb, 1u) == (unsigned)nctas - 1) {
      atomicExch(gb, 0u);
      __threadfence();
      atomicAdd(gb + 1, 1u);
      released = true;
    }
    if (!released) {
      const long long t0 = clock64();
      while (vgb[1] == gen) {
        if (vgb[2] != 0u || clock64() - t0 > cycles) {
          atomicExch(gb + 2, 1u);
          if (status) atomicMin(status, ST_TIMEOUT);
          s_ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();  // the other CTAs' writes before this CTA goes on
  }
  __syncthreads();
  return s_ok != 0;
}

// The work of CTA j in one sweep mode.  Every mode is a run of consecutive
// steps n0..n1 of one interval, the last of which may be the C-point
// residual.  When m does not divide N_l, CTA j = nint owns the partial last
// interval (steps nint*m + 1 .. N_l, all F-points) in the F-relaxation modes
// and has nothing to do in the C-point modes.
template <int PREC>
__device__ __forceinline__ void sweep_mode(const SweepArgs& a, Pipe& pp, char* arena, double* red,
                                           int mode, int j) {
  const int m = a.m, N = a.P.N;
  const bool tail = j == a.nint;
  if (tail && (mode == MODE_C || mode == MODE_R)) return;
  int n0 = j * m + 1, n1 = tail ? a.Nl : j * m + m - 1;
  bool resid = false;
  switch (mode) {
    case MODE_C: n0 = n1 = (j + 1) * m; break;
    case MODE_R: n0 = n1 = (j + 1) * m; resid = true; break;
    case MODE_FR:
      if (!tail) {
        n1 = (j + 1) * m;
        resid = true;
      }
      break;
    case MODE_SEQ: n0 = 1; n1 = a.Nl; break;
    case MODE_CF:
      // u_{jm} += u^(l+1)_j at the C-point this CTA starts from; when the
      // level ends on a C-point, the last CTA also corrects it (read by no
      // F-relaxation)
      if (j >= 1) {
        double* w = a.W + (size_t)(j * m) * N;
        const double* wc = a.Wc + (size_t)j * N;
        const double* gc = a.gc + (size_t)j * N;
        IGM_FOR_CTA(i, N) w[i] += wc[i] + gc[i];
      }
      if (j == a.nint - 1 && a.Nl == a.nint * m) {
        double* w = a.W + (size_t)a.Nl * N;
        const double* wc = a.Wc + (size_t)a.nint * N;
        const double* gc = a.gc + (size_t)a.nint * N;
        IGM_FOR_CTA(i, N) w[i] += wc[i] + gc[i];
      }
      __syncthreads();
      break;
    default: break;  // MODE_F
  }
  for (int n = n0; n <= n1; ++n) mgrit_step<PREC>(a, pp, arena, red, n, resid && n == n1, j);
}

// One CTA per interval j of the level (or one CTA for the sequential coarsest
// level), running one sweep mode; or, launched cooperatively with
// a.nmodes > 1, the modes of one level visit in turn (F, C, F + residual:
// Sec. 3's FCF relaxation and C-point residual) with a grid barrier between
// them, so that a level visit is one launch.
template <int PREC>
__global__ void __launch_bounds__(kBlock) k_mgrit_sweep(SweepArgs a) {
  __shared__ double red[32];
  Pipe pp;
  char* arena = cta_setup(a.P, a.garena, pp);
  if (a.nmodes <= 0) {
    sweep_mode<PREC>(a, pp, arena, red, a.mode, (int)blockIdx.x);
    return;
  }
  for (int q = 0; q < a.nmodes; ++q) {
    if (q > 0 && !grid_barrier(a.gbar, (int)gridDim.x, a.bar_cycles, a.status, false)) return;
    sweep_mode<PREC>(a, pp, arena, red, a.modes[q], (int)blockIdx.x);
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Phase pc of a member's program: A0, then B, A, B, A, ...
__device__ __forceinline__ BatchPhase phase_at(const BatchMember& M, int pc) {
  if (pc < M.nA0) return M.prog[pc];
  return M.prog[M.nA0 + (pc - M.nA0) % (M.nB + M.nA)];
}

// Persistent CTAs of a device-scheduled batch of MGRIT solves.  Thread 0
// looks for work: for each unfinished member in order it reads the member's
// (phase, next task) word and claims the task by compare-and-swap while the
// phase has tasks left.  The CTA runs the task (a sweep of one interval, a
// slice of zeroing, or nothing for the stopping test); the CTA that completes
// the last task of a phase advances the member: after the stopping test it
// records the residual norm and either ends the member's run or counts the
// coarse correction that follows.  No task waits for another: a CTA without
// work polls (sleeping briefly) and gives up after kWaitCycles clocks in
// which no task completed anywhere.
template <int PREC>
__global__ void __launch_bounds__(kBlock) k_mgrit_batch(const BatchMember* mem, BatchState* st,
                                                        int nmem, unsigned long long* ctl) {
  __shared__ double red[32];
  __shared__ int s_m, s_pc, s_task;
  volatile unsigned long long* vctl = ctl;
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&ctl[2], 0ull, global_ns());
  long long idle_since = -1;
  unsigned long long seen = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      s_m = -1;
      bool alive = false;
      for (int i = 0; i < nmem && s_m < 0; ++i) {
        if (*(volatile int*)&st[i].finished) continue;
        alive = true;
        unsigned long long w = *(volatile unsigned long long*)&st[i].word;
        for (;;) {
          const int pc = (int)(w >> 32), tk = (int)(w & 0xffffffffull);
          if (tk >= phase_at(mem[i], pc).grid) break;
          const unsigned long long old = atomicCAS(&st[i].word, w, w + 1ull);
          if (old == w) {
            s_m = i;
            s_pc = pc;
            s_task = tk;
            break;
          }
          w = old;
        }
      }
      if (s_m >= 0) {
        idle_since = -1;
        __threadfence();  // the results of the member's earlier phases
      } else if (!alive || vctl[1] != 0ull) {
        s_m = -2;
      } else {
        const unsigned long long pr = vctl[0];
        const long long now = clock64();
        if (idle_since < 0 || pr != seen) {
          seen = pr;
          idle_since = now;
        } else if (now - idle_since > kWaitCycles) {
          atomicExch(&ctl[1], 1ull);
          s_m = -2;
        }
        if (s_m == -1) __nanosleep(500);
      }
    }
    __syncthreads();
    const int mi = s_m, pc = s_pc, task = s_task;
    __syncthreads();
    if (mi == -2) return;
    if (mi < 0) continue;
    const BatchMember& M = mem[mi];
    const BatchPhase ph = phase_at(M, pc);
    if (ph.op == BOP_SWEEP) {
      const SweepArgs& a = M.lv[ph.level];
      Pipe pp;
      char* arena = cta_setup(a.P, a.garena, pp, task);
      sweep_mode<PREC>(a, pp, arena, red, ph.mode, task);
    } else if (ph.op == BOP_ZERO) {
      const SweepArgs& a = M.lv[ph.level];
      const size_t N = (size_t)a.P.N;
      for (int row = task; row <= a.Nl; row += ph.grid) {
        double* w = a.W + (size_t)row * N;
        for (size_t i = threadIdx.x; i < N; i += blockDim.x) w[i] = 0.0;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // this task's results before its completion is counted
      BatchState& S = st[mi];
      if (atomicAdd(&S.done, 1) + 1 == ph.grid) {
        bool finish = false;
        if (ph.op == BOP_TEST) {
          double rr = 0.0;
          for (int j = 0; j < M.nint0; ++j) rr += M.norms[j];
          const double rho = sqrt(rr);
          if (S.nhist < kBatchHist) S.hist[S.nhist] = rho;
          const double rho0 = S.nhist == 0 ? rho : S.hist[0];
          S.nhist += 1;
          finish = !(rho == rho) || rho == 0.0 || rho <= M.tol * rho0 || S.it >= M.max_iter;
          if (!finish) S.it += 1;
        }
        S.done = 0;
        __threadfence();
        if (finish) {
          S.t_end = global_ns();
          __threadfence();
          atomicExch(&S.finished, 1);
        } else {
          atomicExch(&S.word, (unsigned long long)(pc + 1) << 32);
        }
      }
      atomicAdd(&ctl[0], 1ull);
    }
    __syncthreads();
  }
}

}  // namespace igm
