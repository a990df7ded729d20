// Device building blocks of the p-multigrid cycle (Sec. 4) and the MGRIT
// time step (Sec. 3).  Execution model: one CTA owns one right-hand side
// (one time interval of an MGRIT sweep, or one column of a pmg_vcycle call)
// and runs the whole spatial solve for it with CTA-wide barriers only.  The
// CTA's working vectors live in an "arena" that is dynamic shared memory when
// it fits and a per-CTA slice of global memory (L2-resident) otherwise; all
// routines take generic pointers, so the same code serves both.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace igm {

constexpr int kBlock = 512;       // threads per CTA of the solve kernels
constexpr int kGroup = 4;         // lanes cooperating on one matrix row
constexpr int kMaxH = 8;          // max h-multigrid levels at p = 1
constexpr int kMaxStage = 4;      // max depth of the record ring
constexpr int kRowBars = 16;      // grid-row completion barriers of the wavefront sweeps
constexpr long kSpinLimit = 1L << 26;  // bounded mbarrier polls (~1 s), then IGM_ERR_TIMEOUT

enum WOp : int { W_GS = 0, W_RESTRICT = 1, W_COARSE = 2, W_PROLONG = 3 };

// device status codes (the igm_status values)
enum : int { ST_OK = 0, ST_NOT_CONVERGED = -4, ST_TIMEOUT = -5, ST_NUMERIC = -6 };

// Gauss--Seidel coefficients per unknown, in this order.
enum GsCoef : int { G_SW = 0, G_S, G_SE, G_E, G_NW, G_N, G_NE, G_ALPHA, G_INVC, G_NCOEF };

// Block-row records of one triangular factor (or of Gauss--Seidel rows),
// streamed into shared memory: record k is grid row k (L, Gauss--Seidel) or
// n-1-k (U); the factor layout is described at RecLayout.
struct RecSet {
  const char* recs;        // record k at recs + k * bytes (every record padded to `bytes`)
  int bytes;
};

struct HLevelD {
  int n;                       // unknowns per direction (N_k = n*n)
  const double* A64;           // 9-point stencil [N_k][9], (dy+1)*3 + (dx+1)
  const float* A32;
  RecSet G;                    // Gauss--Seidel row records in the smoothing precision:
                               // per grid row, coefficient q of unknown r = lane*E + e at
                               // (q*E + e)*32 + lane (q: GsCoef, E = ceil(n/32))
  int ox, ob, ot;              // arena element offsets of x_k, b_k, t_k
};

// Everything one spatial solve needs, by value as a kernel parameter.
struct PmgD {
  int p, n, N, w, affine;
  double c;                    // A = M + c K
  // affine operator: 1D interior bands [n][2p+1]; bA = M1 + c K1, bcM = c M1
  const double *bM64, *bK64, *bA64, *bcM64;
  const float *bM32, *bK32, *bA32, *bcM32;
  // explicit part of a theta-scheme step, R = M - expl K (expl = (1-theta)
  // kappa dt; 0 for backward Euler): affine y-bands bR = M1 - expl K1,
  // bcR = -expl M1; curved stencil sR
  double expl;
  const double *bR64, *bcR64, *sR64;
  // spatial solver: 0 p-multigrid, 1 diagonally preconditioned CG (dinv = 1 / diag A)
  int solver;
  const double* dinv64;
  // curved operator: stencils [N][(2p+1)^2]
  const double *sA64, *sM64;
  const float* sA32;
  // ILUT factors as block-row records in the smoothing precision
  RecSet Lrec, Urec;
  int nstage, slot_bytes;      // record ring: nstage slots of slot_bytes
  // L2 transfers between order p and order 1 (Sec. 4, Eq. (prolongation))
  int N1, n1, wP, tp;          // tp: tensor-product transfers with 1D bands of width wP
  const int *Pptr, *Pcol, *PTptr, *PTcol;        // curved: CSR of P and P^T
  const double *Pval64, *PTval64, *MpL64, *M1L64;
  const float *Pval32, *PTval32, *MpL32, *M1L32;
  const int *Pjs, *PTis;                          // affine: band starts of P1 [n], P1^T [n1]
  const double *Pb64, *PTb64;                     // affine: bands [n][wP], [n1][wP]
  const float *Pb32, *PTb32;
  // h-multigrid at p = 1
  int nh;
  HLevelD h[kMaxH];
  const double* Cinv;          // coarsest operator inverse [Nc][Nc], FP64
  int nops;
  int ops[160];                // W-cycle program: op | (level << 8)
  // options
  unsigned long long* trace;   // per-phase SM clocks (IGM_PH_*) or nullptr
  int precision;               // 0 FP64, 1 mixed
  int inner, nu1, nu2, max_cycles;
  double tol;
  // arena layout (element offsets in the smoothing precision)
  int o_r, o_d, o_t, o_u, o_tr;  // o_tr: transfer temporary
  // mixed form with the p = 1 W-cycle in FP64 (hmg64 = 1): the h-level
  // offsets ox, ob, ot are in doubles from the arena's start, the GS records
  // and the W-cycle run in FP64, and o_c1 (floats) holds the order-1
  // vector between the FP32 transfers and the FP64 W-cycle
  int hmg64, o_c1;
  long arena_bytes;
  // dynamic shared memory: [record ring: nstage * slot_bytes][mbarriers: ring slots
  // (kMaxStage), sweep row completion (kRowBars)]
  // [ILUT sweep teams' scratch at o_sweep][staged copy of the vector being
  // swept at o_vstage, when the arena is in global memory and it fits]
  // followed by the arena (at ring_bytes) when arena_smem
  long ring_bytes;
  int arena_smem;
  int o_sweep, o_vstage;       // byte offsets; o_vstage < 0: no staged copy
  int sweep_team;              // threads per ILUT sweep team: 128 or 256
};

// ---------------------------------------------------------------------------
// asynchronous bulk copies (TMA, 1D) into shared memory with mbarriers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
               ::"r"(smem_u32(b)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(b)) : "memory");
}
// Non-blocking probe of the phase with the given parity (test_wait never
// suspends the thread; the records are normally complete long before use).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: false after `limit` unsuccessful polls (the caller then
// records IGM_ERR_TIMEOUT and abandons the solve instead of hanging).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, long limit = kSpinLimit) {
  for (long k = 0; k < limit; ++k)
    if (mbar_try_wait(b, parity)) return true;
  return false;
}

constexpr long long kWaitCycles = 1LL << 31;  // ~1 s of SM clocks: bound of a sleeping wait

// Wait for the phase of the given parity with the thread suspended in
// hardware between checks (mbarrier.try_wait with a suspend-time hint), so a
// waiting warp takes no issue slots.  Gives up after kWaitCycles SM clocks or
// once *abort_flag is set; returns false then.
__device__ __forceinline__ bool mbar_sleep_wait(uint64_t* b, uint32_t parity, const int* abort_flag) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok) : "r"(smem_u32(b)), "r"(parity), "r"(20000u) : "memory");
    if (ok) return true;
    if ((abort_flag && *(const volatile int*)abort_flag) || clock64() - t0 > kWaitCycles) return false;
  }
}
// Wait for the phase of the given parity by polling (test_wait); reacts
// faster than a suspended wait but takes issue slots, so it is meant for the
// one waiter whose turn comes next.  Gives up after kSpinLimit polls or once
// *abort_flag is set (checked every 256 polls); returns false then.
__device__ __forceinline__ bool mbar_spin_wait(uint64_t* b, uint32_t parity, const int* abort_flag) {
  for (long k = 0; k < kSpinLimit; ++k) {
    if (mbar_try_wait(b, parity)) return true;
    if ((k & 255) == 255 && abort_flag && *(const volatile int*)abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// Per-CTA state of the record ring: the expected parity of every stage.
struct Pipe {
  char* ring;
  uint64_t* bar;      // ring slot barriers [kMaxStage]
  uint64_t* rowbar;   // grid-row completion barriers of the sweeps [kRowBars]
  int nstage, slot;
  uint32_t phase;     // bit s: parity of the next phase of ring slot s
  uint32_t rowphase;  // bit b: parity of the next phase of row barrier b
  bool dead;      // set (CTA-uniformly) after a wait timed out: no further copies
};

// Initialise the ring's and the sweeps' mbarriers (whole CTA; once per kernel).
__device__ __forceinline__ void pipe_init(Pipe& pp) {
  pp.rowbar = pp.bar + kMaxStage;
  if (threadIdx.x == 0) {
    for (int s = 0; s < pp.nstage; ++s) mbar_init(&pp.bar[s], 1);
    for (int b = 0; b < kRowBars; ++b) mbar_init(&pp.rowbar[b], 1);
    fence_mbar_init();
  }
  pp.phase = 0;
  pp.rowphase = 0;
  pp.dead = false;
  __syncthreads();
}

// Phase timing (thread 0 of each CTA; the phase ends with a CTA barrier).
struct PhaseClock {
  unsigned long long* acc;
  long long t0;
  __device__ __forceinline__ PhaseClock(unsigned long long* a) : acc(a), t0(0) {
    if (acc && threadIdx.x == 0) t0 = clock64();
  }
  __device__ __forceinline__ void stop(int phase) {
    if (acc && threadIdx.x == 0) atomicAdd(&acc[phase], (unsigned long long)(clock64() - t0));
  }
};

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T group_sum(T s) {
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

// Sum of one double per thread over the CTA, returned to every thread.
// Fixed reduction order for a fixed blockDim (deterministic).
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  const int nw = blockDim.x >> 5;
  for (int k = 0; k < nw; ++k) s += red[k];
  __syncthreads();
  return s;
}

// Maximum of one non-negative double per thread over the CTA, returned to
// every thread.
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double m = 0.0;
  const int nw = blockDim.x >> 5;
  for (int k = 0; k < nw; ++k) m = fmax(m, red[k]);
  __syncthreads();
  return m;
}

// Strided CTA loop whose trip count is the same for every thread; the bound
// test is a predicate inside the body.  (A loop whose trip count differs
// between the lanes of a warp needs a reconvergence point and makes the next
// CTA barrier several times more expensive on this GPU.)
#define IGM_FOR_CTA(i, lim)                                                          \
  for (int i##_b = 0, i##_n = (lim); i##_b < i##_n; i##_b += (int)blockDim.x)        \
    if (const int i = i##_b + (int)threadIdx.x; i < i##_n)

// Warp-uniform loop over rows with kGroup lanes per row: every lane of every
// warp runs the same number of passes, so the group shuffles inside f are
// always executed by the full warp.  f(row, active, lane_in_group).
template <typename F>
__device__ __forceinline__ void for_group_rows(int nrows, F&& f) {
  const int gl = threadIdx.x % kGroup;
  const int per = blockDim.x / kGroup;
  const int wrow = (int)(threadIdx.x & ~31u) / kGroup;  // first row of this warp in a pass
  for (int r0 = 0; r0 < nrows; r0 += per) {
    if (r0 + wrow >= nrows) break;  // the whole warp is past the last row
    const int r = r0 + (int)threadIdx.x / kGroup;
    f(r, r < nrows, gl);
  }
}

// ---------------------------------------------------------------------------
// operator application: affine sum factorisation and curved stencils
// ---------------------------------------------------------------------------
// Source vector: x[i] (+ x2[i] when x2 != nullptr).
template <typename T, typename S>
__device__ __forceinline__ T src(const S* x, const S* x2, int i) {
  T v = (T)x[i];
  if (x2) v += (T)x2[i];
  return v;
}

// Sum factorisation on the affine map (A = M1 (x) M1 + c (K1 (x) M1 + M1 (x) K1)):
//   stage 1 (along xi):  tm = (I (x) bM) x,  tk = (I (x) bK) x
//   stage 2 (along eta): y  = (bA (x) I) tm + (bcM (x) I) tk
// With bM = M1, bK = K1, bA = M1 + c K1, bcM = c M1 this is A; with
// bK = bcM = nullptr and bA = M1 it is the mass matrix.  Bands are [n][W],
// W = 2p+1, zero outside the grid.  Each thread owns one band row (held in
// registers: W is a template parameter) and walks the other grid direction.
// If b != nullptr, out = b - y and, when red != nullptr, the CTA-wide sum of
// out^2 is returned; else out = y.
template <typename T, int W, typename S>
__device__ void sf_stage1_w(int n, const T* bM, const T* bK, const S* x, const S* x2, T* tm, T* tk) {
  constexpr int p = (W - 1) / 2;
  const int R = blockDim.x / n;
  const bool on = (int)threadIdx.x < R * n;
  const int ix = on ? threadIdx.x % n : 0, g = threadIdx.x / n;
  T m[W], k[W];
  int jx[W];
#pragma unroll
  for (int o = 0; o < W; ++o) {
    m[o] = bM[(size_t)ix * W + o];
    k[o] = bK ? bK[(size_t)ix * W + o] : (T)0;
    const int j = ix + o - p;
    jx[o] = j < 0 ? 0 : (j >= n ? n - 1 : j);   // coefficient is 0 outside the grid
  }
  const int iters = (n + R - 1) / R;  // the same for every thread
  for (int t = 0; t < iters; ++t) {
    const int iy = g + t * R;
    if (!on || iy >= n) continue;
    const int row0 = iy * n;
    T sm = 0, sk = 0;
#pragma unroll
    for (int o = 0; o < W; ++o) {
      const T xv = src<T>(x, x2, row0 + jx[o]);
      sm += m[o] * xv;
      sk += k[o] * xv;
    }
    tm[row0 + ix] = sm;
    if (tk) tk[row0 + ix] = sk;
  }
}

// With b: out = (b - y) * oscale and the return value is sum ((b - y) *
// nscale)^2 (power-of-two scales keep FP32 copies and squared norms of tiny
// residuals in range without changing any rounding).
template <typename T, int W, typename B, typename O>
__device__ double sf_stage2_w(int n, const T* bA, const T* bcM, const T* tm, const T* tk,
                              const B* b, O* out, double oscale = 1.0, double nscale = 1.0) {
  constexpr int p = (W - 1) / 2;
  const int R = blockDim.x / n;
  double acc = 0.0;
  const bool on = (int)threadIdx.x < R * n;
  const int iy = on ? threadIdx.x % n : 0, g = threadIdx.x / n;
  T a[W], cm[W];
  int jy[W];
#pragma unroll
  for (int o = 0; o < W; ++o) {
    a[o] = bA[(size_t)iy * W + o];
    cm[o] = bcM ? bcM[(size_t)iy * W + o] : (T)0;
    const int j = iy + o - p;
    jy[o] = (j < 0 ? 0 : (j >= n ? n - 1 : j)) * n;
  }
  const int iters = (n + R - 1) / R;
  for (int t = 0; t < iters; ++t) {
    const int ix = g + t * R;
    if (!on || ix >= n) continue;
    T y = 0;
#pragma unroll
    for (int o = 0; o < W; ++o) {
      y += a[o] * tm[jy[o] + ix];
      if (bcM) y += cm[o] * tk[jy[o] + ix];
    }
    const int i = iy * n + ix;
    if (b) {
      const T r = (T)b[i] - y;
      out[i] = (O)((double)r * oscale);
      const double rs = (double)r * nscale;
      acc += rs * rs;
    } else {
      out[i] = (O)y;
    }
  }
  return acc;
}

template <typename T, int W, typename S, typename B, typename O>
__device__ double apply_A_affine_w(int n, const T* bM, const T* bK, const T* bA, const T* bcM,
                                   const S* x, const S* x2, const B* b, O* out, T* tm, T* tk,
                                   double* red, double oscale = 1.0, double nscale = 1.0) {
  sf_stage1_w<T, W>(n, bM, bK, x, x2, tm, tk);
  __syncthreads();
  const double acc = sf_stage2_w<T, W>(n, bA, bcM, tm, tk, b, out, oscale, nscale);
  if (b && red) return block_sum(acc, red);
  __syncthreads();
  return 0.0;
}

template <typename T, typename S, typename B, typename O>
__device__ double apply_A_affine(int n, int p, const T* bM, const T* bK, const T* bA,
                                 const T* bcM, const S* x, const S* x2, const B* b, O* out, T* tm,
                                 T* tk, double* red, double oscale = 1.0,
                                 double nscale = 1.0) {
  switch (p) {
    case 2: return apply_A_affine_w<T, 5>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
    case 3: return apply_A_affine_w<T, 7>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
    case 4: return apply_A_affine_w<T, 9>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
    case 5: return apply_A_affine_w<T, 11>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
    case 6: return apply_A_affine_w<T, 13>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
    case 7: return apply_A_affine_w<T, 15>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
    default: return apply_A_affine_w<T, 17>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red, oscale, nscale);
  }
}

// Curved: y = A x from the (2p+1)^2 stencil; same out/b convention.
template <typename T, typename S, typename B, typename O>
__device__ double apply_stencil(int n, int w, const T* sA, const S* x, const S* x2, const B* b,
                                O* out, double* red, double oscale = 1.0, double nscale = 1.0) {
  const int W = 2 * w + 1, N = n * n;
  double acc = 0.0;
  IGM_FOR_CTA(i, N) {
    const int ix = i % n, iy = i / n;
    const T* a = sA + (size_t)i * W * W;
    T y = 0;
    for (int dy = -w; dy <= w; ++dy) {
      const int jy = iy + dy;
      if (jy < 0 || jy >= n) continue;
      for (int dx = -w; dx <= w; ++dx) {
        const int jx = ix + dx;
        if (jx < 0 || jx >= n) continue;
        y += a[(dy + w) * W + (dx + w)] * src<T>(x, x2, jx + n * jy);
      }
    }
    if (b) {
      const T r = (T)b[i] - y;
      out[i] = (O)((double)r * oscale);
      const double rs = (double)r * nscale;
      acc += rs * rs;
    } else {
      out[i] = (O)y;
    }
  }
  if (b && red) return block_sum(acc, red);
  __syncthreads();
  return 0.0;
}

// ---------------------------------------------------------------------------
// block-row triangular sweeps (ILUT factors) and Gauss--Seidel
// ---------------------------------------------------------------------------
// Byte offsets inside a factor record (must match the host packing in
// capi.cu).  Record of grid row `by`: int header[4] = {KF, KN, by, 0}; the
// off-block entries coupling to grid rows two or more steps back in the sweep
// order ("far", KF per row) and to the grid row one step back ("near", KN
// per row) as T fv[KF][n], uint16 fi[KF][n], T nv[KN][n], uint16 ni[KN][n]:
// entry k of row r has value fv[k * n + r] and couples to unknown
// fi[k * n + r] of the swept vector (KF, KN = max entries per row, padding
// entries (0, 0)).  Then the dense inverse of the diagonal block in 16-byte
// chunks of V = 16/sizeof(T) columns: row r covers the chunks of columns
// [0, r] (lower) or [r - r % V, n) (upper), zero-padded; in row order these
// chunks form a flat list of rec_inv_row(n) chunks, of which lane l of a
// sweep team of `team` threads takes [l * S, (l + 1) * S), S = wave_steps.
// The record stores them lane-step-major: Vec inv[S][team] (step s of lane l
// at s * team + l, zero past the list), then int desc[S][team]: bits 0-7 the
// chunk index of the right-hand side t, bits 8-17 the partial-sum slot r + l
// of the row r the chunk belongs to, bit 31 set where the lane's piece of row
// r ends (0 past the list).  Every part 16-byte aligned.
template <typename T>
struct RecLayout {
  int o_fv, o_fi, o_nv, o_ni, o_inv, o_desc, bytes;
  __host__ __device__ RecLayout(int n, int KF, int KN, bool upper, int team) {
    const int S = wave_steps(n, upper, team);
    auto a16 = [](int b) { return (b + 15) & ~15; };
    o_fv = 16;
    o_fi = o_fv + a16((int)sizeof(T) * KF * n);
    o_nv = o_fi + a16(2 * KF * n);
    o_ni = o_nv + a16((int)sizeof(T) * KN * n);
    o_inv = o_ni + a16(2 * KN * n);
    o_desc = o_inv + 16 * S * team;
    bytes = o_desc + 4 * S * team;
  }
  // chunk offset of row r in the flat list (r = n gives its length)
  __host__ __device__ static int rec_inv_row(int r, int n, bool upper) {
    constexpr int V = 16 / (int)sizeof(T);
    const int nc = (n + V - 1) / V;  // chunks in a full row
    const int q = r / V, rem = r % V;
    if (!upper) return V * q * (q + 1) / 2 + rem * (q + 1);   // row i: floor(i/V)+1 chunks
    return V * (q * nc - q * (q - 1) / 2) + rem * (nc - q);   // row i: nc-floor(i/V) chunks
  }
  // steps (chunks per lane) of the diagonal-block product
  __host__ __device__ static int wave_steps(int n, bool upper, int team) {
    return (rec_inv_row(n, n, upper) + team - 1) / team;
  }
};

// Issue the bulk copy of record k of a set into ring slot s (one thread).
// Records have a fixed size so that no offset needs to be loaded here (a
// global load at this point would sit on every row's critical path).
__device__ __forceinline__ void pipe_issue(Pipe& pp, const RecSet& R, int k, int s) {
  bulk_load(pp.ring + (size_t)s * pp.slot, R.recs + (size_t)k * R.bytes, (uint32_t)R.bytes,
            &pp.bar[s]);
}

// ---------------------------------------------------------------------------
// wavefront block-row triangular sweeps
// ---------------------------------------------------------------------------
constexpr int kSweepTeam = 128;  // default threads per ILUT sweep team (4 warps, one per SM sub-partition)

// Scratch of a sweep in shared memory: int pieces[n] (per row r: first lane
// of its pieces | count << 16), then per team (kBlock / team of them) the
// grid row's right-hand side t (padded with zeros to whole 16-byte chunks)
// and the partial sums of the diagonal-block product (slot r + lane for the
// piece of row r that a lane computes), in elements of T.
__host__ __device__ inline int wave_tb(int n) { return (n + 16 + 3) & ~3; }
__host__ __device__ inline int wave_team_elems(int n, int team) {
  return wave_tb(n) + ((n + team + 3) & ~3);
}
__host__ __device__ inline int wave_scratch_bytes(int n, int es, int team) {
  return ((4 * n + 15) & ~15) + (kBlock / team) * wave_team_elems(n, team) * es;
}

// Barrier of the `nthreads` threads of sweep team `team` (named barrier
// team + 1); the _or form also returns the OR of a predicate over the team.
__device__ __forceinline__ void team_bar(int team, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(nthreads) : "memory");
}
__device__ __forceinline__ bool team_bar_or(int team, int nthreads, bool pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 q, %1, 0;\n bar.red.or.pred p, %2, %3, q;\n"
      " selp.s32 %0, 1, 0, p;\n}"
      : "=r"(r) : "r"((int)pred), "r"(team + 1), "r"(nthreads) : "memory");
  return r != 0;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }

// Completion of the sweep's grid rows: row j completes phase j / kRowBars
// (counted from the sweep's start) of row barrier j % kRowBars (arrival
// count 1).  A waiter waits on rows at most two steps back and starts a row
// only after its previous row (at most kBlock / 32 = 16 steps back) is
// complete, so with kRowBars >= 16 the parity of the awaited phase is
// unambiguous.

// Bounded wait until grid row j of the sweep is complete (j < 0: nothing to
// wait for), suspended in hardware or (spin) polling.  On failure the sweep
// is marked abandoned.
__device__ __forceinline__ bool wait_row(const Pipe& pp, int* abort_flag, int j, bool spin = false) {
  if (j < 0) return true;
  const int b = j % kRowBars;
  const uint32_t par = ((pp.rowphase >> b) ^ (uint32_t)(j / kRowBars)) & 1u;
  if (spin ? mbar_spin_wait(&pp.rowbar[b], par, abort_flag)
           : mbar_sleep_wait(&pp.rowbar[b], par, abort_flag))
    return true;
  *(volatile int*)abort_flag = 1;
  return false;
}

// acc += sum over e < K of val[e * n + r] * v[idx[e * n + r]] for one row r,
// in e order.  The entries are fetched in batches of B independent loads,
// then the B gathers, so that a warp keeps several shared-memory loads in
// flight instead of waiting on each entry in turn.
template <typename T>
__device__ __forceinline__ T couple(const T* val, const uint16_t* idx, int K, int n, int r,
                                    const T* v, T acc) {
  constexpr int B = 8;
  for (int e0 = 0; e0 < K; e0 += B) {
    T a[B];
    int c[B];
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int e = (e0 + j < K ? e0 + j : 0) * n + r;
      a[j] = val[e];
      c[j] = idx[e];
    }
    T y[B];
#pragma unroll
    for (int j = 0; j < B; ++j) y[j] = v[c[j]];
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (e0 + j < K) acc += a[j] * y[j];
  }
  return acc;
}

// Sum of p[l0 + j] for j < np in j order (np <= 8 in one batch of loads).
template <typename T>
__device__ __forceinline__ T sum_pieces(const T* p, int l0, int np) {
  T s = 0;
  for (int j0 = 0; j0 < np; j0 += 8) {
    T y[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) y[j] = p[l0 + (j0 + j < np ? j0 + j : 0)];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j0 + j < np) s += y[j];
  }
  return s;
}

// Block-row triangular sweep over the n grid rows of a record set (L: grid
// rows 0..n-1; U: n-1..0): per grid row, t = v_row - sum over the
// off-block entries of val * v[off], then v_row = inv(D_row) t with the dense
// inverse of the diagonal block (lower for L, upper for U).
//
// Wavefront schedule: the CTA's threads form NT = min(kBlock / TEAM, ring
// slots) teams of TEAM threads; team j takes the grid rows k = j, j + NT, ...
// of the sweep, row k's record arrives in ring slot k % S (S slots) and the
// team that completes row k streams in record k + S.  A team waits for its
// row's record, accumulates the couplings to rows at least two steps back as
// soon as those rows are complete, then the couplings to the row one step
// back, then applies the inverse (the flat chunk list of the packed inverse
// is cut into equal ranges, one per lane; the pieces of a row are summed in
// lane order) and signals the row's completion on a row barrier.  One thread
// per team waits (suspended in hardware) for records and rows and shares the
// outcome at a team barrier; every wait is bounded.  Returns false after a
// timeout (status gets ST_TIMEOUT; the copies in flight are drained).
template <typename T, bool UPPER, int TEAM>
__device__ bool wave_sweep(int n, const RecSet& R, Pipe& pp, T* v, char* scr, int* status,
                           unsigned long long* trace = nullptr) {
  __shared__ int s_abort, s_done;
  if (pp.dead) return false;
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  constexpr int NTM = kBlock / TEAM;
  const int S = pp.nstage;
  const int NT = S < NTM ? S : NTM;
  const int team = (int)threadIdx.x / TEAM, tl = (int)threadIdx.x % TEAM;
  const bool member = team < NT;
  const int TB = wave_tb(n);
  int* pieces = (int*)scr;
  T* tb = (T*)(scr + ((4 * n + 15) & ~15)) + (size_t)(member ? team : 0) * wave_team_elems(n, TEAM);
  T* part = tb + TB;
  auto C = [&](int r) { return RecLayout<T>::rec_inv_row(r, n, UPPER); };
  const int L = RecLayout<T>::wave_steps(n, UPPER, TEAM);
  IGM_FOR_CTA(r, n) {
    const int l0 = C(r) / L;
    pieces[r] = l0 | (((C(r + 1) - 1) / L - l0 + 1) << 16);
  }
  if (threadIdx.x == 0) {
    s_abort = 0;
    s_done = 0;
  }
  if (member)
    for (int i = n + tl; i < TB; i += TEAM) tb[i] = (T)0;
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_proxy_async();  // earlier generic accesses of the ring before the copies
    for (int k = 0; k < S && k < n; ++k) pipe_issue(pp, R, k, k);
  }
  unsigned long long t_wait = 0, t_off = 0, t_diag = 0;
  for (int k = team; member && k < n; k += NT) {
    const long long ta = (trace && threadIdx.x == 0) ? clock64() : 0;
    const int sl = k % S;
    const char* rec = pp.ring + (size_t)sl * pp.slot;
    bool ok = true;
    if (tl == 0) {
      ok = mbar_sleep_wait(&pp.bar[sl], ((pp.phase >> sl) ^ (uint32_t)(k / S)) & 1u, &s_abort);
      if (!ok) *(volatile int*)&s_abort = 1;
      // couplings to rows at least two steps back need rows <= k-2
      else if (((const int*)rec)[0] > 0) ok = wait_row(pp, &s_abort, k - 2);
    }
    if (team_bar_or(team, TEAM, !ok)) break;
    const long long t1 = (trace && threadIdx.x == 0) ? clock64() : 0;
    const int* hdr = (const int*)rec;
    const int KF = hdr[0], KN = hdr[1], by = hdr[2];
    const RecLayout<T> lay(n, KF, KN, UPPER, TEAM);
    const T* fv = (const T*)(rec + lay.o_fv);
    const uint16_t* fi = (const uint16_t*)(rec + lay.o_fi);
    const T* nv = (const T*)(rec + lay.o_nv);
    const uint16_t* ni = (const uint16_t*)(rec + lay.o_ni);
    T* vr = v + (size_t)by * n;
    for (int r = tl; r < n; r += TEAM) tb[r] = vr[r] - couple<T>(fv, fi, KF, n, r, v, (T)0);
    // couplings to the row one step back
    const long long tw = (trace && threadIdx.x == 0) ? clock64() : 0;
    if (tl == 0 && KN > 0) ok = wait_row(pp, &s_abort, k - 1, true);
    if (team_bar_or(team, TEAM, !ok)) break;
    const long long tw2 = (trace && threadIdx.x == 0) ? clock64() : 0;
    for (int r = tl; r < n; r += TEAM) tb[r] -= couple<T>(nv, ni, KN, n, r, v, (T)0);
    team_bar(team, TEAM);
    const long long t4 = (trace && threadIdx.x == 0) ? clock64() : 0;
    // diagonal block: partial products over this lane's chunk range, in
    // batches of DB steps (all loads of a batch issued before the products)
    {
      constexpr int DB = sizeof(T) == 4 ? 8 : 4;
      const Vec* inv = (const Vec*)(rec + lay.o_inv) + tl;
      const int* desc = (const int*)(rec + lay.o_desc) + tl;
      const Vec* tv = (const Vec*)tb;
      T s0 = 0, s1 = 0;
      for (int b0 = 0; b0 < L; b0 += DB) {
        int d[DB];
        Vec a[DB], x[DB];
#pragma unroll
        for (int jj = 0; jj < DB; ++jj) {
          const int st = b0 + jj < L ? b0 + jj : 0;
          d[jj] = b0 + jj < L ? desc[st * TEAM] : 0;
          a[jj] = inv[st * TEAM];
        }
#pragma unroll
        for (int jj = 0; jj < DB; ++jj) x[jj] = tv[d[jj] & 0xff];
#pragma unroll
        for (int jj = 0; jj < DB; ++jj) {
          if (b0 + jj < L) {
            if (sizeof(T) == 4) {
              const float4& af = reinterpret_cast<const float4&>(a[jj]);
              const float4& xf = reinterpret_cast<const float4&>(x[jj]);
              s0 += af.x * xf.x + af.y * xf.y;
              s1 += af.z * xf.z + af.w * xf.w;
            } else {
              const double2& ad = reinterpret_cast<const double2&>(a[jj]);
              const double2& xd = reinterpret_cast<const double2&>(x[jj]);
              s0 += ad.x * xd.x;
              s1 += ad.y * xd.y;
            }
            if (d[jj] < 0) {
              part[(d[jj] >> 8) & 0x3ff] = s0 + s1;
              s0 = 0;
              s1 = 0;
            }
          }
        }
      }
    }
    team_bar(team, TEAM);
    // v_row = sum of the pieces of each row, in lane order
    for (int r = tl; r < n; r += TEAM) {
      const int e = pieces[r];
      vr[r] = sum_pieces<T>(part + r, e & 0xffff, e >> 16);
    }
    if (team_bar_or(team, TEAM, tl == 0 && ld_volatile(&s_abort))) break;
    if (tl == 0) {
      mbar_arrive(&pp.rowbar[k % kRowBars]);  // release: this row's values are complete
      *(volatile int*)&s_done = k + 1;
      if (k + S < n) {
        fence_proxy_async();
        pipe_issue(pp, R, k + S, sl);
      }
    }
    if (trace && threadIdx.x == 0) {
      const long long te = clock64();
      t_wait += (unsigned long long)((t1 - ta) + (tw2 - tw));
      t_off += (unsigned long long)((tw - t1) + (t4 - tw2));
      t_diag += (unsigned long long)(te - t4);
    }
  }
  __syncthreads();
  const bool okall = ld_volatile(&s_abort) == 0;
  if (trace && threadIdx.x == 0) {
    atomicAdd(&trace[8], t_wait);
    atomicAdd(&trace[9], t_off);
    atomicAdd(&trace[10], t_diag);
  }
  if (!okall) {
    // records [0, min(n, D + S)) were issued (D rows complete); drain them
    if (threadIdx.x == 0) {
      const int D = ld_volatile(&s_done);
      for (int k = D; k < n && k < D + S; ++k)
        mbar_sleep_wait(&pp.bar[k % S], ((pp.phase >> (k % S)) ^ (uint32_t)(k / S)) & 1u, nullptr);
      if (status) atomicMin(status, ST_TIMEOUT);
    }
    __syncthreads();
    pp.dead = true;
    return false;
  }
  __syncthreads();
  // slot j completed one phase per row k = j, j + S, ... < n; row barrier b
  // one per row k = b, b + kRowBars, ... < n
  for (int j = 0; j < S; ++j)
    if (j < n && (((n - j + S - 1) / S) & 1)) pp.phase ^= 1u << j;
  for (int b = 0; b < kRowBars; ++b)
    if (b < n && (((n - b + kRowBars - 1) / kRowBars) & 1)) pp.rowphase ^= 1u << b;
  return true;
}

// One forward lexicographic Gauss--Seidel sweep on a 9-point operator (the
// smoother of the h-multigrid at p = 1, Sec. 4) in two passes.  Pass 1 (all
// threads): pre_i = b_i - (E, NW, N, NE couplings) x with the values before
// the sweep, i.e. the couplings to unknowns that come later in the
// lexicographic order.  Pass 2: the grid rows in order, warp w taking rows
// w, w + 16, ...; a warp loads its row's coefficients and pre and forms the
// products of the alphas its scan combines, waits for the preceding row (row
// barrier), forms t_r = pre_r - (SW, S, SE couplings) x with that row's new
// values, and solves the in-row recurrence
// x_r = alpha_r x_{r-1} + t_r / a_C,r (alpha = -a_W/a_C) as a warp-wide scan
// of affine maps, E consecutive unknowns per lane.  Row records hold
// coefficient q of unknown r = lane * E + e at (q * E + e) * 32 + lane.
// Returns false after a timeout (status gets ST_TIMEOUT).
template <typename T, int E>
__device__ bool gs_wave(int n, const RecSet& R, Pipe& pp, const T* b, T* x, T* pre, int* status,
                        unsigned long long* trace) {
  __shared__ int s_abort;
  const int N = n * n;
  auto coef = [&](int by, int r, int q) -> T {
    const T* cf = (const T*)(R.recs + (size_t)by * R.bytes);
    return cf[(q * E + r % E) * 32 + r / E];
  };
  PhaseClock p0(trace);
  IGM_FOR_CTA(i, N) {
    const int by = i / n, r = i % n;
    const bool hasE = r + 1 < n, hasW = r > 0, hasN = by + 1 < n;
    T s = 0;
    if (hasE) s += coef(by, r, G_E) * x[i + 1];
    if (hasN) {
      const int iN = i + n;
      if (hasW) s += coef(by, r, G_NW) * x[iN - 1];
      s += coef(by, r, G_N) * x[iN];
      if (hasE) s += coef(by, r, G_NE) * x[iN + 1];
    }
    pre[i] = b[i] - s;
  }
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();
  p0.stop(12);
  const int w = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31, NW = (int)blockDim.x >> 5;
  const int r0 = lane * E;
  unsigned long long t_wait = 0, t_row = 0;
  for (int by = w; by < n; by += NW) {
    const long long ta = (trace && threadIdx.x == 0) ? clock64() : 0;
    // everything that does not depend on the preceding row
    const T* cf = (const T*)(R.recs + (size_t)by * R.bytes);
    T cSW[E], cS[E], cSE[E], al[E], ic[E], pr[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int r = r0 + e;
      const bool in = r < n;
      auto c = [&](int q) { return in ? cf[(q * E + e) * 32 + lane] : (T)0; };
      cSW[e] = c(G_SW);
      cS[e] = c(G_S);
      cSE[e] = c(G_SE);
      al[e] = c(G_ALPHA);
      ic[e] = c(G_INVC);
      pr[e] = in ? pre[by * n + r] : (T)0;
    }
    // the lane's composed factor A = prod alpha and the value it has at each
    // level of the scan below depend on the coefficients only: formed before
    // the wait, off the chain through the preceding row
    T alpha[E];
    T A = 1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      alpha[e] = r0 + e < n ? al[e] : (T)0;
      if (r0 + e < n) A = alpha[e] * A;
    }
    T Al[5];
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      Al[o] = A;
      const T Ap = __shfl_up_sync(0xffffffffu, A, 1 << o);
      if (lane >= (1 << o)) A = A * Ap;
    }
    bool ok = true;
    // suspended until the row two back is complete, then polling for the
    // preceding one (at most one warp polls at a time)
    if (lane == 0 && by > 0) ok = wait_row(pp, &s_abort, by - 2) && wait_row(pp, &s_abort, by - 1, true);
    __syncwarp();  // lane 0's acquire of the preceding row, for the whole warp
    if (!__shfl_sync(0xffffffffu, ok, 0)) break;
    const long long tw = (trace && threadIdx.x == 0) ? clock64() : 0;
    T beta[E];
    T B = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      beta[e] = 0;
      const int r = r0 + e;
      if (r < n) {
        T t = pr[e];
        if (by > 0) {
          // neighbours outside the grid have coefficient 0: clamp their index
          const int iS = (by - 1) * n + r;
          const T xSW = x[r > 0 ? iS - 1 : iS], xS = x[iS], xSE = x[r + 1 < n ? iS + 1 : iS];
          const T sw = r > 0 ? cSW[e] : (T)0, se = r + 1 < n ? cSE[e] : (T)0;
          t -= (sw * xSW + cS[e] * xS) + se * xSE;
        }
        beta[e] = ic[e] * t;
        B = alpha[e] * B + beta[e];
      }
    }
    // inclusive scan of the lanes' affine maps x_out = A x_in + B (the A of
    // each level precomputed above)
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      const T Bp = __shfl_up_sync(0xffffffffu, B, 1 << o);
      if (lane >= (1 << o)) B = Al[o] * Bp + B;
    }
    T xin = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) xin = 0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int r = r0 + e;
      if (r < n) {
        xin = alpha[e] * xin + beta[e];
        x[by * n + r] = xin;
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&pp.rowbar[by % kRowBars]);  // release: the row is complete
    if (trace && threadIdx.x == 0) {
      const long long te = clock64();
      t_wait += (unsigned long long)(tw - ta);
      t_row += (unsigned long long)(te - tw);
    }
  }
  __syncthreads();
  const bool okall = ld_volatile(&s_abort) == 0;
  __syncthreads();
  if (trace && threadIdx.x == 0) {
    atomicAdd(&trace[11], t_wait);
    atomicAdd(&trace[13], t_row);
  }
  if (!okall) {
    if (threadIdx.x == 0 && status) atomicMin(status, ST_TIMEOUT);
    pp.dead = true;
    return false;
  }
  for (int bb = 0; bb < kRowBars; ++bb)
    if (bb < n && (((n - bb + kRowBars - 1) / kRowBars) & 1)) pp.rowphase ^= 1u << bb;
  return true;
}

// A Gauss--Seidel sweep (pre: scratch of n * n).
template <typename T>
__device__ bool gs_sweep(int n, const RecSet& R, Pipe& pp, const T* b, T* x, T* pre, int* status,
                         unsigned long long* trace = nullptr) {
  if (pp.dead) return false;
  if (n <= 32) return gs_wave<T, 1>(n, R, pp, b, x, pre, status, trace);
  if (n <= 64) return gs_wave<T, 2>(n, R, pp, b, x, pre, status, trace);
  if (n <= 128) return gs_wave<T, 4>(n, R, pp, b, x, pre, status, trace);
  return gs_wave<T, 8>(n, R, pp, b, x, pre, status, trace);
}

// Tensor-product transfer on the affine map, stage along xi then eta:
// out[jy][jx] (op)= (sum_ky band[jy][ky] sum_kx band[jx][kx] in[s(jy)+ky][s(jx)+kx]) / scale
// with in an nin x nin grid, out nout x nout, tmp nin x nout.
template <typename T, bool ADD>
__device__ void transfer_tp(int nin, int nout, int w, const int* start, const T* band,
                            const T* scale, const T* in, T* tmp, T* out) {
  IGM_FOR_CTA(i, nin * nout) {
    const int jx = i % nout, iy = i / nout;
    const T* bd = band + (size_t)jx * w;
    const T* src = in + (size_t)iy * nin + start[jx];
    T s = 0;
    for (int k = 0; k < w; ++k) s += bd[k] * src[k];
    tmp[i] = s;
  }
  __syncthreads();
  IGM_FOR_CTA(i, nout * nout) {
    const int jx = i % nout, jy = i / nout;
    const T* bd = band + (size_t)jy * w;
    const int s0 = start[jy];
    T s = 0;
    for (int k = 0; k < w; ++k) s += bd[k] * tmp[(size_t)(s0 + k) * nout + jx];
    const T v = s / scale[i];
    if (ADD) out[i] += v; else out[i] = v;
  }
  __syncthreads();
}

// t = b - A x on a 9-point operator.
template <typename T>
__device__ void residual9(int n, const T* A, const T* b, const T* x, T* t) {
  const int N = n * n;
  IGM_FOR_CTA(i, N) {
    const int ix = i % n, iy = i / n;
    const T* a = A + (size_t)i * 9;
    T y = 0;
    for (int dy = -1; dy <= 1; ++dy) {
      const int jy = iy + dy;
      if (jy < 0 || jy >= n) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int jx = ix + dx;
        if (jx < 0 || jx >= n) continue;
        y += a[(dy + 1) * 3 + (dx + 1)] * x[jx + n * jy];
      }
    }
    t[i] = b[i] - y;
  }
  __syncthreads();
}

// Bilinear restriction (transpose of the knot-insertion prolongation) from
// an nf x nf grid to nc = (nf-1)/2; also zeroes the coarse iterate.
template <typename T>
__device__ void restrict_bilinear(int nf, const T* t, T* bc, T* xc) {
  const int nc = (nf - 1) / 2, Nc = nc * nc;
  IGM_FOR_CTA(I, Nc) {
    const int cx = I % nc, cy = I / nc;
    T s = 0;
    for (int fy = 2 * cy; fy <= 2 * cy + 2; ++fy) {
      const T wy = (fy == 2 * cy + 1) ? (T)1 : (T)0.5;
      for (int fx = 2 * cx; fx <= 2 * cx + 2; ++fx) {
        const T wx = (fx == 2 * cx + 1) ? (T)1 : (T)0.5;
        s += wx * wy * t[fx + nf * fy];
      }
    }
    bc[I] = s;
    xc[I] = 0;
  }
  __syncthreads();
}

// x_f += P x_c (bilinear interpolation from nc to nf = 2 nc + 1).
template <typename T>
__device__ void prolong_bilinear(int nf, const T* xc, T* xf) {
  const int nc = (nf - 1) / 2, Nf = nf * nf;
  IGM_FOR_CTA(i, Nf) {
    const int fx = i % nf, fy = i / nf;
    // odd fine index 2c+1: coarse c with weight 1; even 2c: coarse c-1 and c with 1/2
    const bool ox = fx & 1, oy = fy & 1;
    const int cx0 = ox ? (fx - 1) / 2 : fx / 2 - 1, cx1 = fx / 2;
    const int cy0 = oy ? (fy - 1) / 2 : fy / 2 - 1, cy1 = fy / 2;
    const T wx0 = ox ? (T)1 : (T)0.5, wy0 = oy ? (T)1 : (T)0.5;
    const bool vx0 = cx0 >= 0 && cx0 < nc, vx1 = !ox && cx1 < nc;
    const bool vy0 = cy0 >= 0 && cy0 < nc, vy1 = !oy && cy1 < nc;
    T s = 0;
    if (vy0 && vx0) s += wx0 * wy0 * xc[cx0 + nc * cy0];
    if (vy0 && vx1) s += (T)0.5 * wy0 * xc[cx1 + nc * cy0];
    if (vy1 && vx0) s += wx0 * (T)0.5 * xc[cx0 + nc * cy1];
    if (vy1 && vx1) s += (T)0.25 * xc[cx1 + nc * cy1];
    xf[i] += s;
  }
  __syncthreads();
}

// CSR product with a row scale: out_i (op)= (sum_k val_k x_col_k) / scale_i.
template <typename T, bool ADD>
__device__ void csr_scaled(int rows, const int* ptr, const int* col, const T* val, const T* scale,
                           const T* x, T* out) {
  for_group_rows(rows, [&](int r, bool act, int gl) {
    T s = 0;
    if (act)
      for (int k = ptr[r] + gl; k < ptr[r + 1]; k += kGroup) s += val[k] * x[col[k]];
    s = group_sum(s);
    if (act && gl == 0) {
      const T v = s / scale[r];
      if (ADD) out[r] += v; else out[r] = v;
    }
  });
  __syncthreads();
}

}  // namespace igm
