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

namespace igm {

constexpr int kBlock = 512;       // threads per CTA of the solve kernels
constexpr int kGroup = 4;         // lanes cooperating on one matrix row
constexpr int kMaxH = 8;          // max h-multigrid levels at p = 1

enum WOp : int { W_GS = 0, W_RESTRICT = 1, W_COARSE = 2, W_PROLONG = 3 };

struct HLevelD {
  int n;                       // unknowns per direction (N_k = n*n)
  const double* A64;           // 9-point stencil [N_k][9], (dy+1)*3 + (dx+1)
  const float* A32;
  const double* G64;           // Gauss--Seidel block inverses: n blocks of n(n+1)/2 (lower packed)
  const float* G32;
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
  // ILUT factors in block-row form
  const int *Lptr, *Lcol, *Uptr, *Ucol;
  const double *Lval64, *Uval64, *Linv64, *Uinv64;
  const float *Lval32, *Uval32, *Linv32, *Uinv32;
  // L2 transfers between order p and order 1 (Sec. 4, Eq. (prolongation))
  int N1;
  const int *Pptr, *Pcol, *PTptr, *PTcol;
  const double *Pval64, *PTval64, *MpL64, *M1L64;
  const float *Pval32, *PTval32, *MpL32, *M1L32;
  // h-multigrid at p = 1
  int nh;
  HLevelD h[kMaxH];
  const double* Cinv;          // coarsest operator inverse [Nc][Nc], FP64
  int nops;
  int ops[160];                // W-cycle program: op | (level << 8)
  // options
  int precision;               // 0 FP64, 1 mixed
  int inner, nu1, nu2, max_cycles;
  double tol;
  // arena layout (element offsets in the smoothing precision)
  int o_r, o_d, o_t, o_u, o_row;
  long arena_bytes;
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

// Warp-uniform loop over rows with kGroup lanes per row: every lane of every
// warp runs the same number of passes, so the group shuffles inside f are
// always executed by the full warp.  f(row, active, lane_in_group).
template <typename F>
__device__ __forceinline__ void for_group_rows(int nrows, F&& f) {
  const int gl = threadIdx.x % kGroup;
  const int per = blockDim.x / kGroup;
  for (int r0 = 0; r0 < nrows; r0 += per) {
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

// Stage 1 of the sum factorisation along xi: tm = (I (x) M1) x, tk = (I (x) K1) x.
template <typename T, typename S>
__device__ void sf_stage1(int n, int p, const T* bM, const T* bK, const S* x, const S* x2, T* tm,
                          T* tk) {
  const int W = 2 * p + 1, N = n * n;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int ix = i % n, row0 = i - ix;
    T sm = 0, sk = 0;
    const T* m = bM + (size_t)ix * W;
    const T* k = bK ? bK + (size_t)ix * W : nullptr;
    for (int o = 0; o < W; ++o) {
      const int jx = ix + o - p;
      if (jx < 0 || jx >= n) continue;
      const T xv = src<T>(x, x2, row0 + jx);
      sm += m[o] * xv;
      if (k) sk += k[o] * xv;
    }
    tm[i] = sm;
    if (tk) tk[i] = sk;
  }
}

// y = A x by sum factorisation on the affine map:
//   stage 1 (along xi):  tm = (I (x) bM) x,  tk = (I (x) bK) x
//   stage 2 (along eta): y  = (bA (x) I) tm + (bcM (x) I) tk
// With bM = M1, bK = K1, bA = M1 + c K1, bcM = c M1 this is
// A = M1 (x) M1 + c (K1 (x) M1 + M1 (x) K1); with bK = bcM = nullptr and
// bA = M1 it is the mass matrix.  If b != nullptr, out = b - y and, when red
// != nullptr, the CTA-wide sum of out^2 is returned; else out = y.
template <typename T, typename S, typename B, typename O>
__device__ double apply_A_affine(int n, int p, const T* bM, const T* bK, const T* bA,
                                 const T* bcM, const S* x, const S* x2, const B* b, O* out, T* tm,
                                 T* tk, double* red) {
  const int W = 2 * p + 1, N = n * n;
  sf_stage1<T>(n, p, bM, bK, x, x2, tm, tk);
  __syncthreads();
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int ix = i % n, iy = i / n;
    const T* a = bA + (size_t)iy * W;
    const T* cm = bcM ? bcM + (size_t)iy * W : nullptr;
    T y = 0;
    for (int o = 0; o < W; ++o) {
      const int jy = iy + o - p;
      if (jy < 0 || jy >= n) continue;
      y += a[o] * tm[ix + n * jy];
      if (cm) y += cm[o] * tk[ix + n * jy];
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

// Curved: y = A x from the (2p+1)^2 stencil; same out/b convention.
template <typename T, typename S, typename B, typename O>
__device__ double apply_stencil(int n, int w, const T* sA, const S* x, const S* x2, const B* b,
                                O* out, double* red) {
  const int W = 2 * w + 1, N = n * n;
  double acc = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
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

// v <- L^{-1} v for a unit lower factor in block-row form.  Grid rows are
// processed in order; within a grid row, t = v - (off-block part) is formed
// in parallel, then v_row = inv(L_D) t by a packed dense product.
template <typename T>
__device__ void block_lower_solve(int n, const int* ptr, const int* col, const T* val, const T* inv,
                                  T* v, T* row) {
  const size_t blk = lower_off(n);
  for (int by = 0; by < n; ++by) {
    for_group_rows(n, [&](int r, bool act, int gl) {
      T s = 0;
      if (act) {
        const int i = by * n + r;
        for (int k = ptr[i] + gl; k < ptr[i + 1]; k += kGroup) s += val[k] * v[col[k]];
      }
      s = group_sum(s);
      if (act && gl == 0) row[r] = v[by * n + r] - s;
    });
    __syncthreads();
    const T* D = inv + (size_t)by * blk;
    for_group_rows(n, [&](int r, bool act, int gl) {
      T s = 0;
      if (act) {
        const T* Dr = D + lower_off(r);
        for (int j = gl; j <= r; j += kGroup) s += Dr[j] * row[j];
      }
      s = group_sum(s);
      if (act && gl == 0) v[by * n + r] = s;
    });
    __syncthreads();
  }
}

// v <- U^{-1} v, grid rows in reverse order, packed upper block inverses.
template <typename T>
__device__ void block_upper_solve(int n, const int* ptr, const int* col, const T* val, const T* inv,
                                  T* v, T* row) {
  const size_t blk = upper_off(n, n);
  for (int by = n - 1; by >= 0; --by) {
    for_group_rows(n, [&](int r, bool act, int gl) {
      T s = 0;
      if (act) {
        const int i = by * n + r;
        for (int k = ptr[i] + gl; k < ptr[i + 1]; k += kGroup) s += val[k] * v[col[k]];
      }
      s = group_sum(s);
      if (act && gl == 0) row[r] = v[by * n + r] - s;
    });
    __syncthreads();
    const T* D = inv + (size_t)by * blk;
    for_group_rows(n, [&](int r, bool act, int gl) {
      T s = 0;
      if (act) {
        const T* Dr = D + upper_off(r, n);
        for (int j = r + gl; j < n; j += kGroup) s += Dr[j - r] * row[j];
      }
      s = group_sum(s);
      if (act && gl == 0) v[by * n + r] = s;
    });
    __syncthreads();
  }
}

// One forward lexicographic Gauss--Seidel sweep on a 9-point operator:
// per grid row, t = b - (E, S-row, N-row couplings) x, then x_row = (D+W)^{-1} t.
template <typename T>
__device__ void gs_sweep(int n, const T* A, const T* ginv, const T* b, T* x, T* row) {
  const size_t blk = lower_off(n);
  for (int by = 0; by < n; ++by) {
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int i = by * n + r;
      const T* a = A + (size_t)i * 9;
      T t = b[i];
      if (r + 1 < n) t -= a[5] * x[i + 1];
      if (by > 0) {
        if (r > 0) t -= a[0] * x[i - n - 1];
        t -= a[1] * x[i - n];
        if (r + 1 < n) t -= a[2] * x[i - n + 1];
      }
      if (by + 1 < n) {
        if (r > 0) t -= a[6] * x[i + n - 1];
        t -= a[7] * x[i + n];
        if (r + 1 < n) t -= a[8] * x[i + n + 1];
      }
      row[r] = t;
    }
    __syncthreads();
    const T* D = ginv + (size_t)by * blk;
    for_group_rows(n, [&](int r, bool act, int gl) {
      T s = 0;
      if (act) {
        const T* Dr = D + lower_off(r);
        for (int j = gl; j <= r; j += kGroup) s += Dr[j] * row[j];
      }
      s = group_sum(s);
      if (act && gl == 0) x[by * n + r] = s;
    });
    __syncthreads();
  }
}

// t = b - A x on a 9-point operator.
template <typename T>
__device__ void residual9(int n, const T* A, const T* b, const T* x, T* t) {
  const int N = n * n;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
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
  for (int I = threadIdx.x; I < Nc; I += blockDim.x) {
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
  for (int i = threadIdx.x; i < Nf; i += blockDim.x) {
    const int fx = i % nf, fy = i / nf;
    int cxs[2], cys[2];
    T wxs[2], wys[2];
    int nxs = 0, nys = 0;
    if (fx & 1) { cxs[0] = (fx - 1) / 2; wxs[0] = 1; nxs = 1; }
    else {
      if (fx / 2 - 1 >= 0) { cxs[nxs] = fx / 2 - 1; wxs[nxs++] = 0.5; }
      if (fx / 2 < nc) { cxs[nxs] = fx / 2; wxs[nxs++] = 0.5; }
    }
    if (fy & 1) { cys[0] = (fy - 1) / 2; wys[0] = 1; nys = 1; }
    else {
      if (fy / 2 - 1 >= 0) { cys[nys] = fy / 2 - 1; wys[nys++] = 0.5; }
      if (fy / 2 < nc) { cys[nys] = fy / 2; wys[nys++] = 0.5; }
    }
    T s = 0;
    for (int b = 0; b < nys; ++b)
      for (int a = 0; a < nxs; ++a) s += wxs[a] * wys[b] * xc[cxs[a] + nc * cys[b]];
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
