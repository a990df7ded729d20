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
constexpr long kSpinLimit = 1L << 26;  // bounded mbarrier polls (~1 s), then IGM_ERR_TIMEOUT

enum WOp : int { W_GS = 0, W_RESTRICT = 1, W_COARSE = 2, W_PROLONG = 3 };

// device status codes (the igm_status values)
enum : int { ST_OK = 0, ST_NOT_CONVERGED = -4, ST_TIMEOUT = -5, ST_NUMERIC = -6 };

// Gauss--Seidel coefficients per unknown, in this order.
enum GsCoef : int { G_SW = 0, G_S, G_SE, G_E, G_NW, G_N, G_NE, G_ALPHA, G_INVC, G_NCOEF };

// Block-row records of one triangular factor (or of Gauss--Seidel rows),
// streamed into shared memory: record k is grid row k (L, Gauss--Seidel) or
// n-1-k (U); the layout is described at RecLayout.
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
  // curved operator: stencils [N][(2p+1)^2]
  const double *sA64, *sM64;
  const float* sA32;
  // ILUT factors as block-row records in the smoothing precision
  RecSet Lrec, Urec;
  int rec_lanes;               // lanes per row G of the factor records (4 or 8)
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
  int o_r, o_d, o_t, o_u, o_row, o_tr;  // o_tr: transfer temporary
  long arena_bytes;
  // dynamic shared memory: [record ring: nstage * slot_bytes][mbarriers: 8 * kMaxStage]
  // followed by the arena when arena_smem
  long ring_bytes;
  int arena_smem;
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

// Per-CTA state of the record ring: the expected parity of every stage.
struct Pipe {
  char* ring;
  uint64_t* bar;
  int nstage, slot;
  uint32_t phase;
  bool dead;      // set (CTA-uniformly) after a wait timed out: no further copies
};

// Initialise the ring's mbarriers (whole CTA; once per kernel).
__device__ __forceinline__ void pipe_init(Pipe& pp) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < pp.nstage; ++s) mbar_init(&pp.bar[s], 1);
    fence_mbar_init();
  }
  pp.phase = 0;
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

// As for_group_rows with G lanes per row (G a power of two <= 32).
template <int G, typename F>
__device__ __forceinline__ void for_rows_g(int nrows, F&& f) {
  const int gl = threadIdx.x % G;
  const int per = blockDim.x / G;
  const int wrow = (int)(threadIdx.x & ~31u) / G;
  for (int r0 = 0; r0 < nrows; r0 += per) {
    if (r0 + wrow >= nrows) break;
    const int r = r0 + (int)threadIdx.x / G;
    f(r, r < nrows, gl);
  }
}

template <int G, typename T>
__device__ __forceinline__ T group_sum_g(T s) {
#pragma unroll
  for (int o = 1; o < G; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
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

template <typename T, int W, typename B, typename O>
__device__ double sf_stage2_w(int n, const T* bA, const T* bcM, const T* tm, const T* tk,
                              const B* b, O* out) {
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
      out[i] = (O)r;
      acc += (double)r * (double)r;
    } else {
      out[i] = (O)y;
    }
  }
  return acc;
}

template <typename T, int W, typename S, typename B, typename O>
__device__ double apply_A_affine_w(int n, const T* bM, const T* bK, const T* bA, const T* bcM,
                                   const S* x, const S* x2, const B* b, O* out, T* tm, T* tk,
                                   double* red) {
  sf_stage1_w<T, W>(n, bM, bK, x, x2, tm, tk);
  __syncthreads();
  const double acc = sf_stage2_w<T, W>(n, bA, bcM, tm, tk, b, out);
  if (b && red) return block_sum(acc, red);
  __syncthreads();
  return 0.0;
}

template <typename T, typename S, typename B, typename O>
__device__ double apply_A_affine(int n, int p, const T* bM, const T* bK, const T* bA,
                                 const T* bcM, const S* x, const S* x2, const B* b, O* out, T* tm,
                                 T* tk, double* red) {
  switch (p) {
    case 2: return apply_A_affine_w<T, 5>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
    case 3: return apply_A_affine_w<T, 7>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
    case 4: return apply_A_affine_w<T, 9>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
    case 5: return apply_A_affine_w<T, 11>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
    case 6: return apply_A_affine_w<T, 13>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
    case 7: return apply_A_affine_w<T, 15>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
    default: return apply_A_affine_w<T, 17>(n, bM, bK, bA, bcM, x, x2, b, out, tm, tk, red);
  }
}

// Curved: y = A x from the (2p+1)^2 stencil; same out/b convention.
template <typename T, typename S, typename B, typename O>
__device__ double apply_stencil(int n, int w, const T* sA, const S* x, const S* x2, const B* b,
                                O* out, double* red) {
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
      out[i] = (O)r;
      acc += (double)r * (double)r;
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
__device__ __forceinline__ size_t lower_off(int i) { return (size_t)i * (i + 1) / 2; }
__device__ __forceinline__ size_t upper_off(int i, int n) {
  return (size_t)i * n - (size_t)i * (i - 1) / 2;
}

__device__ __forceinline__ int align16(int bytes) { return (bytes + 15) & ~15; }

// One off-block entry of a factor record: the value and the byte offset of
// the coupled unknown in the vector being solved.
template <typename T>
struct alignas(sizeof(T) == 4 ? 8 : 16) RecEntry {
  T val;
  int off;
};

// Byte offsets inside a factor record (must match the host packing in
// capi.cu).  Record of grid row `by` for G lanes per row: int header[4] =
// {KL, by, G, 0}; RecEntry ent[KL][n][G]: the off-block entries of the grid
// row's n rows, entry k of row r at ((k / G) * n + r) * G + k % G, KL =
// ceil(max entries per row / G), padding entries (0, 0); then the dense
// inverse of the diagonal block stored by rows in 16-byte chunks of
// V = 16/sizeof(T) columns: row r covers the chunks of columns [0, r]
// (lower) or [r - r % V, n) (upper), zero-padded, at chunk offset
// rec_inv_row(r).  Every part 16-byte aligned.
template <typename T>
struct RecLayout {
  int o_ent, o_inv, bytes;
  __host__ __device__ RecLayout(int n, int KL, int G, bool upper) {
    o_ent = 16;
    o_inv = o_ent + (((int)sizeof(RecEntry<T>) * KL * n * G + 15) & ~15);
    bytes = o_inv + 16 * rec_inv_row(n, n, upper);
  }
  // chunk offset of row r (r = n gives the total number of chunks)
  __host__ __device__ static int rec_inv_row(int r, int n, bool upper) {
    constexpr int V = 16 / (int)sizeof(T);
    const int nc = (n + V - 1) / V;  // chunks in a full row
    const int q = r / V, rem = r % V;
    if (!upper) return V * q * (q + 1) / 2 + rem * (q + 1);   // row i: floor(i/V)+1 chunks
    return V * (q * nc - q * (q - 1) / 2) + rem * (nc - q);   // row i: nc-floor(i/V) chunks
  }
};

// Issue the bulk copy of record k of a set into ring slot s (thread 0 only).
// Records have a fixed size so that no offset needs to be loaded here (a
// global load at this point would sit on every row's critical path).
__device__ __forceinline__ void pipe_issue(Pipe& pp, const RecSet& R, int k, int s) {
  bulk_load(pp.ring + (size_t)s * pp.slot, R.recs + (size_t)k * R.bytes, (uint32_t)R.bytes,
            &pp.bar[s]);
}

// Block-row triangular sweep v <- D^{-1}-weighted substitution over the n
// grid rows of a record set (L: grid rows 0..n-1; U: n-1..0).  Per grid row:
// phase 1 forms t_r = v_i - sum_k val_k v_{base+col_k} over the off-block
// entries in parallel (kGroup lanes per row); phase 2 writes
// v_row = inv(D_row) t (packed dense, lower for L, upper for U).  Record k+S
// is in flight while record k is used.  Returns false after a wait timeout.
template <typename T, bool UPPER, int G>
__device__ bool block_sweep(int n, const RecSet& R, Pipe& pp, T* v, T* row, int* status,
                            unsigned long long* trace = nullptr) {
  if (pp.dead) return false;
  const int S = pp.nstage < n ? pp.nstage : n;
  if (threadIdx.x == 0)
    for (int s = 0; s < S; ++s) pipe_issue(pp, R, s, s);
  // the vector loads of phase 2 read t up to the next 16-byte boundary past n
  if (threadIdx.x < 16 / sizeof(T)) row[n + threadIdx.x] = (T)0;
  for (int k = 0; k < n; ++k) {
    const int s = k % pp.nstage;
    PhaseClock pw(trace);
    // warp 0 observes the copy's completion (acquire); the barrier then
    // orders the record's contents before every thread's reads
    const bool got = threadIdx.x < 32 ? mbar_wait(&pp.bar[s], (pp.phase >> s) & 1u) : true;
    pp.phase ^= 1u << s;
    const bool timeout = __syncthreads_or(!got);
    pw.stop(8);
    if (timeout) {
      if (threadIdx.x == 0 && status) atomicMin(status, ST_TIMEOUT);
      // drain the copies still in flight (bounded) before giving up
      for (int j = k + 1; j < k + S && j < n; ++j) {
        const int sj = j % pp.nstage;
        if (threadIdx.x < 32) mbar_wait(&pp.bar[sj], (pp.phase >> sj) & 1u);
        pp.phase ^= 1u << sj;
      }
      pp.dead = true;
      return false;
    }
    const char* rec = pp.ring + (size_t)s * pp.slot;
    const int* hdr = (const int*)rec;
    const int KL = hdr[0], by = hdr[1];
    const RecLayout<T> lay(n, KL, G, UPPER);
    const RecEntry<T>* ent = (const RecEntry<T>*)(rec + lay.o_ent);
    const char* inv = rec + lay.o_inv;
    const char* vbytes = (const char*)v;
    PhaseClock p1(trace);
    // phase 1: t_r = v_i - sum over the row's off-block entries of val * v[off];
    // a warp covers 32/G rows x G lanes and reads 32 consecutive entries per
    // step; KL is the same for every lane (padding entries are (0, 0))
    for_rows_g<G>(n, [&](int r, bool act, int c) {
      const RecEntry<T>* ep = ent + (size_t)(act ? r : 0) * G + c;
      const int stride = n * G;
      T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      int u = 0;
      for (; u + 4 <= KL; u += 4) {
        const RecEntry<T> e0 = ep[(u + 0) * stride], e1 = ep[(u + 1) * stride];
        const RecEntry<T> e2 = ep[(u + 2) * stride], e3 = ep[(u + 3) * stride];
        s0 += e0.val * *(const T*)(vbytes + e0.off);
        s1 += e1.val * *(const T*)(vbytes + e1.off);
        s2 += e2.val * *(const T*)(vbytes + e2.off);
        s3 += e3.val * *(const T*)(vbytes + e3.off);
      }
      for (; u < KL; ++u) {
        const RecEntry<T> e0 = ep[u * stride];
        s0 += e0.val * *(const T*)(vbytes + e0.off);
      }
      const T sacc = group_sum_g<G>((s0 + s1) + (s2 + s3));
      if (act && c == 0) row[r] = v[by * n + r] - sacc;
    });
    __syncthreads();
    p1.stop(9);
    PhaseClock p2(trace);
    // phase 2: v_row = inv(D) t.  Lane c of row r takes the 16-byte chunks
    // c, c+G, ... of the row's stored column range (one vector load of the
    // inverse and one broadcast load of t per V columns); the trip count is
    // the warp's maximum, out-of-range chunks are skipped by a predicate
    for_rows_g<G>(n, [&](int r, bool act, int c) {
      constexpr int V = 16 / (int)sizeof(T);
      using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
      const int rr = act ? r : 0;
      const int j0 = UPPER ? rr - rr % V : 0;
      const int nch = UPPER ? (n - j0 + V - 1) / V : rr / V + 1;
      constexpr int RW = 32 / G;  // rows per warp
      const int rw = r & ~(RW - 1);
      const int rl = rw + RW - 1 < n ? rw + RW - 1 : n - 1;
      const int nch_w = UPPER ? (n - (rw - rw % V) + V - 1) / V : rl / V + 1;
      const Vec* ip = (const Vec*)(inv + 16 * RecLayout<T>::rec_inv_row(rr, n, UPPER));
      const Vec* tp = (const Vec*)(row + j0);
      T s0 = 0, s1 = 0;
      const int steps = (nch_w + G - 1) / G;
      for (int st = 0; st < steps; ++st) {
        const int q = c + st * G;
        const bool ok = act && q < nch;
        const int qq = ok ? q : 0;
        const Vec a = ip[qq], t = tp[qq];
        if (sizeof(T) == 4) {
          const float4& af = reinterpret_cast<const float4&>(a);
          const float4& tf = reinterpret_cast<const float4&>(t);
          const T w = ok ? (T)1 : (T)0;
          s0 += w * (af.x * tf.x + af.y * tf.y);
          s1 += w * (af.z * tf.z + af.w * tf.w);
        } else {
          const double2& ad = reinterpret_cast<const double2&>(a);
          const double2& td = reinterpret_cast<const double2&>(t);
          const T w = ok ? (T)1 : (T)0;
          s0 += w * (ad.x * td.x);
          s1 += w * (ad.y * td.y);
        }
      }
      const T sacc = group_sum_g<G>(s0 + s1);
      if (act && c == 0) v[by * n + r] = sacc;
    });
    __syncthreads();
    p2.stop(10);
    if (threadIdx.x == 0 && k + pp.nstage < n) {
      fence_proxy_async();
      pipe_issue(pp, R, k + pp.nstage, s);
    }
  }
  return true;
}

// Warp-level asynchronous copies (cp.async, 16 bytes per lane per instruction)
// with group accounting: used to stage Gauss--Seidel coefficient rows.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// One forward lexicographic Gauss--Seidel sweep on a 9-point operator, run by
// warp 0 (the caller synchronises the CTA afterwards).  The coefficient row of
// grid row by+D is copied into a 4-slot staging area while row by is solved.
// Grid row by: every lane forms t_r = b_r - (E, S-row, N-row couplings) x
// for its E consecutive unknowns; the in-row recurrence
// x_r = alpha_r x_{r-1} + t_r / a_C,r (alpha = -a_W/a_C) is an affine map per
// unknown, composed by a warp-wide scan.
template <typename T, int EMAX>
__device__ void gs_rows_warp(int n, const RecSet& R, char* stage, const T* b, T* x,
                             unsigned long long* trace) {
  constexpr int D = 3;            // rows in flight ahead of the one being solved
  constexpr int E = EMAX;         // unknowns per lane (the host packs rows for this width)
  const int lane = threadIdx.x & 31;
  const int r0 = lane * E;
  const int chunks = R.bytes / 16;
  auto copy_row = [&](int row) {
    const char* src = R.recs + (size_t)row * R.bytes;
    char* dst = stage + (size_t)(row % (D + 1)) * R.bytes;
    for (int i = lane; i < chunks; i += 32) cp_async16(dst + 16 * i, src + 16 * i);
  };
  for (int k = 0; k < D; ++k) {
    if (k < n) copy_row(k);
    cp_async_commit();
  }
  for (int by = 0; by < n; ++by) {
    if (by + D < n) copy_row(by + D);
    cp_async_commit();
    cp_async_wait<D>();           // the group of row `by` has landed
    __syncwarp();
    PhaseClock pt(trace);
    const T* cf = (const T*)(stage + (size_t)(by % (D + 1)) * R.bytes);
    T beta[EMAX], alpha[EMAX];
    T A = 1, B = 0;
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      beta[e] = 0;
      alpha[e] = 0;
      const int r = r0 + e;
      if (r < n) {
        const int i = by * n + r;
        auto c = [&](int q) { return cf[(q * E + e) * 32 + lane]; };
        // neighbours outside the grid have coefficient 0: clamp their index
        const bool hasE = r + 1 < n, hasW = r > 0, hasS = by > 0, hasN = by + 1 < n;
        const int iE = hasE ? i + 1 : i;
        const int iS = hasS ? i - n : i, iN = hasN ? i + n : i;
        const T xE = x[iE];
        const T xSW = x[hasW ? iS - 1 : iS], xS = x[iS], xSE = x[hasE ? iS + 1 : iS];
        const T xNW = x[hasW ? iN - 1 : iN], xN = x[iN], xNE = x[hasE ? iN + 1 : iN];
        const T cE = hasE ? c(G_E) : (T)0;
        const T cSW = (hasS && hasW) ? c(G_SW) : (T)0, cS = hasS ? c(G_S) : (T)0;
        const T cSE = (hasS && hasE) ? c(G_SE) : (T)0;
        const T cNW = (hasN && hasW) ? c(G_NW) : (T)0, cN = hasN ? c(G_N) : (T)0;
        const T cNE = (hasN && hasE) ? c(G_NE) : (T)0;
        const T t = b[i] - (((cE * xE + cSW * xSW) + (cS * xS + cSE * xSE)) +
                            ((cNW * xNW + cN * xN) + cNE * xNE));
        alpha[e] = c(G_ALPHA);
        beta[e] = c(G_INVC) * t;
        B = alpha[e] * B + beta[e];
        A = alpha[e] * A;
      }
    }
    pt.stop(12);
    PhaseClock ps(trace);
    // inclusive scan of the lanes' affine maps x_out = A x_in + B
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T Ap = __shfl_up_sync(0xffffffffu, A, o);
      const T Bp = __shfl_up_sync(0xffffffffu, B, o);
      if (lane >= o) {
        B = A * Bp + B;
        A = A * Ap;
      }
    }
    T xin = __shfl_up_sync(0xffffffffu, B, 1);
    if (lane == 0) xin = 0;
    __syncwarp();
#pragma unroll
    for (int e = 0; e < EMAX; ++e) {
      const int r = r0 + e;
      if (r < n) {
        xin = alpha[e] * xin + beta[e];
        x[by * n + r] = xin;
      }
    }
    __syncwarp();
    ps.stop(13);
  }
  cp_async_wait<0>();
}

// A Gauss--Seidel sweep staged through the (idle) record ring.
template <typename T>
__device__ bool gs_sweep(int n, const RecSet& R, Pipe& pp, const T* b, T* x, int* status,
                         unsigned long long* trace = nullptr) {
  if (pp.dead) return false;
  if (threadIdx.x < 32) {
    if (n <= 32) gs_rows_warp<T, 1>(n, R, pp.ring, b, x, trace);
    else if (n <= 64) gs_rows_warp<T, 2>(n, R, pp.ring, b, x, trace);
    else gs_rows_warp<T, 4>(n, R, pp.ring, b, x, trace);
  }
  __syncthreads();
  return true;
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
