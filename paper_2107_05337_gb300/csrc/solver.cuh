// The spatial solve (Sec. 4 p-multigrid cycle, repeated to a tolerance) and
// the MGRIT time step (Sec. 3) as CTA-wide device functions.
#pragma once
#include "device.cuh"

namespace igm {

__device__ __forceinline__ void record_status(int* status, int code) {
  if (status && threadIdx.x == 0) atomicMin(status, code);
}

// FP64 residual out = (b - A x) * oscale (out may be float: the mixed form's
// r32); returns ||(b - A x) * nscale||_2^2 computed in FP64.
template <typename O>
__device__ double residual64(const PmgD& P, const double* b, const double* x, O* out, double* tm,
                             double* tk, double* red, double oscale = 1.0, double nscale = 1.0) {
  if (P.affine)
    return apply_A_affine<double>(P.n, P.p, P.bM64, P.bK64, P.bA64, P.bcM64, x,
                                  (const double*)nullptr, b, out, tm, tk, red, oscale, nscale);
  return apply_stencil<double>(P.n, P.w, P.sA64, x, (const double*)nullptr, b, out, red, oscale,
                               nscale);
}

// t = b - A x in the smoothing precision (no norm).
template <typename T>
__device__ void residualT(const PmgD& P, const T* b, const T* x, T* t, T* tm, T* tk);

template <>
__device__ inline void residualT<float>(const PmgD& P, const float* b, const float* x, float* t, float* tm,
                                 float* tk) {
  if (P.affine)
    apply_A_affine<float>(P.n, P.p, P.bM32, P.bK32, P.bA32, P.bcM32, x, (const float*)nullptr, b, t,
                          tm, tk, (double*)nullptr);
  else
    apply_stencil<float>(P.n, P.w, P.sA32, x, (const float*)nullptr, b, t, (double*)nullptr);
}

template <>
__device__ inline void residualT<double>(const PmgD& P, const double* b, const double* x, double* t,
                                  double* tm, double* tk) {
  residual64<double>(P, b, x, t, tm, tk, (double*)nullptr);
}

template <typename T> struct Prec;
template <> struct Prec<float> {
  __device__ static const float* Pv(const PmgD& P) { return P.Pval32; }
  __device__ static const float* PTv(const PmgD& P) { return P.PTval32; }
  __device__ static const float* Pb(const PmgD& P) { return P.Pb32; }
  __device__ static const float* PTb(const PmgD& P) { return P.PTb32; }
  __device__ static const float* MpL(const PmgD& P) { return P.MpL32; }
  __device__ static const float* M1L(const PmgD& P) { return P.M1L32; }
  __device__ static const float* HA(const HLevelD& H) { return H.A32; }
};
template <> struct Prec<double> {
  __device__ static const double* Pv(const PmgD& P) { return P.Pval64; }
  __device__ static const double* PTv(const PmgD& P) { return P.PTval64; }
  __device__ static const double* Pb(const PmgD& P) { return P.Pb64; }
  __device__ static const double* PTb(const PmgD& P) { return P.PTb64; }
  __device__ static const double* MpL(const PmgD& P) { return P.MpL64; }
  __device__ static const double* M1L(const PmgD& P) { return P.M1L64; }
  __device__ static const double* HA(const HLevelD& H) { return H.A64; }
};

// v <- U^{-1} L^{-1} v (the ILUT smoother S = (LU)^{-1} applied to v, Sec. 4).
// The factor records are in the handle's smoothing precision T.  When the
// arena is in global memory and shared memory has room, both sweeps run on a
// staged shared-memory copy of v.
template <typename T>
__device__ bool ilut_apply(const PmgD& P, Pipe& pp, T* v, int* status) {
  extern __shared__ __align__(128) char dyn_smem[];
  PhaseClock pc(P.trace);
  char* scr = dyn_smem + P.o_sweep;
  T* w = v;
  if (P.o_vstage >= 0) {
    w = (T*)(dyn_smem + P.o_vstage);
    IGM_FOR_CTA(i, P.N) w[i] = v[i];
    __syncthreads();
  }
  bool ok;
  if (P.sweep_team == 256)
    ok = wave_sweep<T, false, 256>(P.n, P.Lrec, pp, w, scr, status, P.trace) &&
         wave_sweep<T, true, 256>(P.n, P.Urec, pp, w, scr, status, P.trace);
  else
    ok = wave_sweep<T, false, kSweepTeam>(P.n, P.Lrec, pp, w, scr, status, P.trace) &&
         wave_sweep<T, true, kSweepTeam>(P.n, P.Urec, pp, w, scr, status, P.trace);
  if (P.o_vstage >= 0) {
    IGM_FOR_CTA(i, P.N) v[i] = w[i];
    __syncthreads();
  }
  pc.stop(2);
  return ok;
}

// x_k = A_k^{-1} b_k on the coarsest h-level with the FP64 inverse.
template <typename T>
__device__ void coarse_solve(int Nc, const double* Cinv, const T* b, T* x) {
  for_group_rows(Nc, [&](int r, bool act, int gl) {
    double s = 0.0;
    if (act)
      for (int j = gl; j < Nc; j += kGroup) s += Cinv[(size_t)r * Nc + j] * (double)b[j];
    s = group_sum(s);
    if (act && gl == 0) x[r] = (T)s;
  });
  __syncthreads();
}

// One W-cycle of h-multigrid at p = 1 (Sec. 4, Fig. 5), interpreting the
// host-generated op list.  h-level 0 holds b_0 = restricted residual and
// x_0 = 0 on entry and the coarse correction on exit.
template <typename T>
__device__ bool wcycle(const PmgD& P, Pipe& pp, T* A, int* status) {
  for (int o = 0; o < P.nops; ++o) {
    const int op = P.ops[o] & 0xff, k = P.ops[o] >> 8;
    const HLevelD& H = P.h[k];
    T* xk = A + H.ox;
    T* bk = A + H.ob;
    T* tk = A + H.ot;
    switch (op) {
      case W_GS: {
        PhaseClock pc(P.trace);
        const bool ok = gs_sweep<T>(H.n, H.G, pp, bk, xk, tk, status, P.trace);
        pc.stop(7);
        if (!ok) return false;
        break;
      }
      case W_RESTRICT:
        residual9<T>(H.n, Prec<T>::HA(H), bk, xk, tk);
        restrict_bilinear<T>(H.n, tk, A + P.h[k + 1].ob, A + P.h[k + 1].ox);
        break;
      case W_COARSE:
        coarse_solve<T>(H.n * H.n, P.Cinv, bk, xk);
        break;
      case W_PROLONG:
        prolong_bilinear<T>(H.n, A + P.h[k + 1].ox, xk);
        break;
    }
  }
  return true;
}

// r_1 = (M_1^L)^{-1} P^T t into r1 (Sec. 4, step 2).
template <typename T>
__device__ void restrict_p1_to(const PmgD& P, const T* t, T* A, T* r1) {
  if (P.tp)
    transfer_tp<T, false>(P.n, P.n1, P.wP, P.PTis, Prec<T>::PTb(P), Prec<T>::M1L(P), t, A + P.o_tr,
                          r1);
  else
    csr_scaled<T, false>(P.N1, P.PTptr, P.PTcol, Prec<T>::PTv(P), Prec<T>::M1L(P), t, r1);
}

// r_1 into h-level 0's b, and x_0 = 0.
template <typename T>
__device__ void restrict_p1(const PmgD& P, const T* t, T* A) {
  const HLevelD& H0 = P.h[0];
  restrict_p1_to<T>(P, t, A, A + H0.ob);
  IGM_FOR_CTA(i, P.N1) A[H0.ox + i] = 0;
  __syncthreads();
}

// x += (M_p^L)^{-1} P e_1 (Sec. 4, step 4).
template <typename T>
__device__ void prolong_p1_from(const PmgD& P, T* x, T* A, const T* e1) {
  if (P.tp)
    transfer_tp<T, true>(P.n1, P.n, P.wP, P.Pjs, Prec<T>::Pb(P), Prec<T>::MpL(P), e1, A + P.o_tr,
                         x);
  else
    csr_scaled<T, true>(P.N, P.Pptr, P.Pcol, Prec<T>::Pv(P), Prec<T>::MpL(P), e1, x);
}

// with e_1 = h-level 0's x
template <typename T>
__device__ void prolong_p1(const PmgD& P, T* x, T* A) {
  prolong_p1_from<T>(P, x, A, A + P.h[0].ox);
}

// Steps 2-4 of the mixed form's cycle with the W-cycle in FP64 (hmg64): the
// FP32 restriction into the order-1 buffer, then h-level 0's b (FP64) from
// it and x_0 = 0, the FP64 W-cycle, and the FP32 prolongation of its result.
__device__ inline bool coarse_correction_fp64(const PmgD& P, Pipe& pp, const float* t, float* x,
                                              float* A, int* status) {
  const HLevelD& H0 = P.h[0];
  double* A64 = (double*)A;
  float* c1 = A + P.o_c1;
  {
    PhaseClock pc(P.trace);
    restrict_p1_to<float>(P, t, A, c1);
    IGM_FOR_CTA(i, P.N1) {
      A64[H0.ob + i] = (double)c1[i];
      A64[H0.ox + i] = 0.0;
    }
    __syncthreads();
    pc.stop(3);
  }
  {
    PhaseClock pc(P.trace);
    const bool ok = wcycle<double>(P, pp, A64, status);
    pc.stop(4);
    if (!ok) return false;
  }
  {
    PhaseClock pc(P.trace);
    IGM_FOR_CTA(i, P.N1) c1[i] = (float)A64[H0.ox + i];
    __syncthreads();
    prolong_p1_from<float>(P, x, A, c1);
    pc.stop(5);
  }
  return true;
}

// One p-multigrid cycle (Sec. 4, steps 1-5) on A x = b in precision T.
// t: scratch of N; on entry t may already hold b - A x (t_is_residual).
// x_is_zero: x = 0 on entry (the first pre-smoothing then needs no product).
// Returns false if a record wait timed out (the solve is abandoned).
template <typename T>
__device__ bool pmg_cycle(const PmgD& P, Pipe& pp, const T* b, T* x, T* A, bool t_is_residual,
                          bool x_is_zero, int* status) {
  const int N = P.N;
  T* t = A + P.o_t;
  T* tm = A + P.o_u;
  T* tk = tm + N;
  for (int s = 0; s < P.nu1; ++s) {
    const bool zero = x_is_zero && s == 0;
    if (zero) {
      IGM_FOR_CTA(i, N) t[i] = b[i];
      __syncthreads();
    } else if (!(s == 0 && t_is_residual)) {
      PhaseClock pc(P.trace);
      residualT<T>(P, b, x, t, tm, tk);
      pc.stop(1);
    }
    if (!ilut_apply<T>(P, pp, t, status)) return false;
    IGM_FOR_CTA(i, N) x[i] = zero ? t[i] : x[i] + t[i];
    __syncthreads();
  }
  if (P.nu1 == 0 && x_is_zero) {
    IGM_FOR_CTA(i, N) x[i] = 0;
    __syncthreads();
  }
  // step 2: r_1 = (M_1^L)^{-1} P^T (b - A x)
  {
    PhaseClock pc(P.trace);
    residualT<T>(P, b, x, t, tm, tk);
    pc.stop(1);
  }
  if (sizeof(T) == 4 && P.hmg64) {
    // steps 2-4 with the W-cycle in FP64
    if (!coarse_correction_fp64(P, pp, (const float*)t, (float*)x, (float*)A, status)) return false;
  } else {
  {
    PhaseClock pc(P.trace);
    restrict_p1<T>(P, t, A);
    pc.stop(3);
  }
  // step 3: one W-cycle of h-multigrid on A_1 e_1 = r_1
  {
    PhaseClock pc(P.trace);
    const bool ok = wcycle<T>(P, pp, A, status);
    pc.stop(4);
    if (!ok) return false;
  }
  // step 4: x += (M_p^L)^{-1} P e_1
  {
    PhaseClock pc(P.trace);
    prolong_p1<T>(P, x, A);
    pc.stop(5);
  }
  }
  // step 5: post-smoothing
  for (int s = 0; s < P.nu2; ++s) {
    {
      PhaseClock pc(P.trace);
      residualT<T>(P, b, x, t, tm, tk);
      pc.stop(1);
    }
    if (!ilut_apply<T>(P, pp, t, status)) return false;
    IGM_FOR_CTA(i, N) x[i] += t[i];
    __syncthreads();
  }
  return true;
}

// Conjugate gradients with the preconditioner D^-1 = diag(A)^-1 on A x = b
// in FP64 (the comparison solver of Sec. 5), warm start x, on the FP64
// arena: r at o_t; p, q and the operator's two temporaries at o_u.
// ncycles > 0: exactly ncycles iterations; else iterate until
// ||b - A x|| <= tol ||b|| or max_cycles.  Returns the iterations done.
__device__ inline int cg_solve(const PmgD& P, const double* b, double* x, double* A, double* red,
                               double nb2, double sc, int ncycles, int* status) {
  const int N = P.N;
  double* r = A + P.o_t;
  double* pv = A + P.o_u;
  double* q = pv + N;
  double* tm = q + N;
  double* tk = tm + N;
  // r, p, q are carried scaled by the power of two sc (alpha and beta do
  // not depend on it); x is updated with alpha p / sc
  const double isc = 1.0 / sc;
  const double tol2 = P.tol * P.tol * nb2;
  double rr = residual64<double>(P, b, x, r, tm, tk, red, sc, sc);
  if (ncycles == 0 && rr <= tol2) return 0;
  double rz = 0.0;
  IGM_FOR_CTA(i, N) {
    const double z = P.dinv64[i] * r[i];
    pv[i] = z;
    rz += r[i] * z;
  }
  rz = block_sum(rz, red);
  int it = 0;
  while (true) {
    if (P.affine)
      apply_A_affine<double>(P.n, P.p, P.bM64, P.bK64, P.bA64, P.bcM64, pv, (const double*)nullptr,
                             (const double*)nullptr, q, tm, tk, (double*)nullptr);
    else
      apply_stencil<double>(P.n, P.w, P.sA64, pv, (const double*)nullptr, (const double*)nullptr,
                            q, (double*)nullptr);
    double pq = 0.0;
    IGM_FOR_CTA(i, N) pq += pv[i] * q[i];
    pq = block_sum(pq, red);
    const double alpha = rz / pq;
    double rr2 = 0.0, rz2 = 0.0;
    IGM_FOR_CTA(i, N) {
      x[i] += alpha * pv[i] * isc;
      const double ri = r[i] - alpha * q[i];
      r[i] = ri;
      rr2 += ri * ri;
      rz2 += ri * P.dinv64[i] * ri;
    }
    rr2 = block_sum(rr2, red);
    rz2 = block_sum(rz2, red);
    ++it;
    if (!(rr2 == rr2)) { record_status(status, ST_NUMERIC); break; }
    if (ncycles > 0) {
      if (it >= ncycles) break;
    } else {
      if (rr2 <= tol2) break;
      if (it >= P.max_cycles) { record_status(status, ST_NOT_CONVERGED); break; }
    }
    const double beta = rz2 / rz;
    rz = rz2;
    IGM_FOR_CTA(i, N) pv[i] = P.dinv64[i] * r[i] + beta * pv[i];
    __syncthreads();
  }
  return it;
}

// Spatial solve of A x = b (b, x FP64 in global memory), warm start x.
// ncycles > 0: exactly ncycles cycles; else cycle until
// ||b - A x|| <= tol ||b|| (checked before each cycle) or max_cycles.
// PREC 0 (FP64 form): one cycle = one p-multigrid cycle in FP64.
// PREC 1 (mixed form): one cycle = FP64 residual r, then `inner` FP32
// p-multigrid cycles on A d = r from d = 0, then x += d (iterative
// refinement).  Returns the number of cycles.
template <int PREC>
__device__ int pmg_solve(const PmgD& P, Pipe& pp, const double* b, double* x, char* arena,
                         double* red, int ncycles, int* status) {
  const int N = P.N;
  // power of two sc with max |b| sc in [1/2, 1): norms are taken of scaled
  // vectors and the mixed form's FP32 residual is b - A x scaled by sc, so
  // tiny right-hand sides (decayed solutions) neither underflow in FP32 nor
  // in the squared norms; the scaling is exact, results are unchanged
  double bmax = 0.0;
  IGM_FOR_CTA(i, N) bmax = fmax(bmax, fabs(b[i]));
  bmax = block_max(bmax, red);
  if (bmax == 0.0) {
    IGM_FOR_CTA(i, N) x[i] = 0.0;
    __syncthreads();
    return 0;
  }
  int ex;
  frexp(bmax, &ex);
  const double sc = ldexp(1.0, -ex), isc = ldexp(1.0, ex);
  double nb2 = 0.0;
  IGM_FOR_CTA(i, N) nb2 += (b[i] * sc) * (b[i] * sc);
  nb2 = block_sum(nb2, red);
  if (PREC == 0 && P.solver == 1)
    return cg_solve(P, b, x, (double*)arena, red, nb2, sc, ncycles, status);
  const double tol2 = P.tol * P.tol * nb2;
  int cyc = 0;
  if (PREC == 0) {
    double* A = (double*)arena;
    double* t = A + P.o_t;
    double* tm = A + P.o_u;
    double* tk = tm + N;
    while (true) {
      PhaseClock pc(P.trace);
      const double rr = residual64<double>(P, b, x, t, tm, tk, red, 1.0, sc);
      pc.stop(0);
      if (!(rr == rr)) { record_status(status, ST_NUMERIC); break; }
      if (ncycles > 0) {
        if (cyc >= ncycles) break;
      } else {
        if (rr <= tol2) break;
        if (cyc >= P.max_cycles) { record_status(status, ST_NOT_CONVERGED); break; }
      }
      if (!pmg_cycle<double>(P, pp, b, x, A, true, false, status)) break;
      ++cyc;
    }
  } else {
    float* A = (float*)arena;
    float* r = A + P.o_r;
    float* d = A + P.o_d;
    double* tm64 = (double*)(A + P.o_d);
    double* tk64 = tm64 + N;
    while (true) {
      if (ncycles > 0 && cyc >= ncycles) break;
      PhaseClock pc(P.trace);
      const double rr = residual64<float>(P, b, x, r, tm64, tk64, red, sc, sc);
      pc.stop(0);
      if (!(rr == rr)) { record_status(status, ST_NUMERIC); break; }
      if (ncycles == 0) {
        if (rr <= tol2) break;
        if (cyc >= P.max_cycles) { record_status(status, ST_NOT_CONVERGED); break; }
      }
      bool ok = true;
      for (int k = 0; k < P.inner && ok; ++k)
        ok = pmg_cycle<float>(P, pp, r, d, A, false, k == 0, status);
      if (!ok) break;
      IGM_FOR_CTA(i, N) x[i] += (double)d[i] * isc;
      __syncthreads();
      ++cyc;
    }
  }
  return cyc;
}

// out = R (u + ug) + scale * fhat in FP64 with R = M - expl K (the
// right-hand side of one theta-scheme step, Sec. 2 Eq. (los) and Sec. 3:
// R u^{n-1} + dt f; R = M for backward Euler).  tm: 2 N doubles scratch.
__device__ inline void build_rhs(const PmgD& P, const double* u, const double* ug, double scale,
                          const double* fhat, double* out, double* tm) {
  if (P.expl != 0.0) {
    if (P.affine)
      apply_A_affine<double>(P.n, P.p, P.bM64, P.bK64, P.bR64, P.bcR64, u, ug,
                             (const double*)nullptr, out, tm, tm + P.N, (double*)nullptr);
    else
      apply_stencil<double>(P.n, P.w, P.sR64, u, ug, (const double*)nullptr, out, (double*)nullptr);
  } else if (P.affine) {
    apply_A_affine<double>(P.n, P.p, P.bM64, (const double*)nullptr, P.bM64,
                           (const double*)nullptr, u, ug, (const double*)nullptr, out, tm,
                           (double*)nullptr, (double*)nullptr);
  } else {
    apply_stencil<double>(P.n, P.w, P.sM64, u, ug, (const double*)nullptr, out, (double*)nullptr);
  }
  if (fhat && scale != 0.0) {
    IGM_FOR_CTA(i, P.N) out[i] += scale * fhat[i];
    __syncthreads();
  }
}

}  // namespace igm
