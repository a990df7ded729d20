// Batched FP32 operator apply on the affine map (a block of right-hand-side
// columns, e.g. time intervals): y_b = (Y2 (x) X1 + Z2 (x) W1) x_b with the
// 1D interior bands of half-width p (Sec. 2: M = M1 (x) M1, K = K1 (x) M1 +
// M1 (x) K1 on the unit square), by sum factorisation:
//   stage 1 (along xi):  tm = x X1^T, tk = x W1^T  (rows of the n x n grid)
//   stage 2 (along eta): y = Y2 tm + Z2 tk          (columns of the grid)
// Each of the four 1D factors is a combination a M1 + b K1 formed on the fly
// from the FP32 bands of M1 and K1.
//
// One persistent CTA per SM, split into two warp groups that form a pipeline
// over the CTA's columns:
//   * stage-1 warps (0-6) stream column k + nb - 1 into a ring of nb shared
//     slots by 4-byte cp.async (rows padded with p zero columns on each side,
//     so the band windows need no bounds tests), then turn column k into
//     (tm, tk) in one of two shared buffers;
//   * stage-2 warps (7-15) turn the other buffer into y and store it; each
//     half-warp takes one group of J grid rows, its 16 lanes 16 consecutive
//     grid columns.
// Both stages run on packed FP32 FMAs (two lanes per instruction): stage 1
// accumulates the (tm, tk) pair of a grid point with the (X1, W1) band pair,
// stage 2 the pair (Y2 tm, Z2 tk) with the (Y2, Z2) band pair.
// The groups hand the two buffers back and forth by named barriers (bar.arrive
// / bar.sync; hardware waits, no polling).  Both groups keep their band rows in
// registers: a stage-1 thread owns J grid columns of every row it visits, a
// stage-2 thread J grid rows of every column it visits.  All strides are
// compile-time (two layouts, for grids up to 68 and 84 lines), so every band
// tap is an immediate address offset.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "device.cuh"
#include "spmm.h"

namespace igm {

namespace {

constexpr int kG1 = 224;               // stage-1 threads (warps 0-6)
constexpr int kG2 = 288;               // stage-2 threads (warps 7-15): 18 half-warps
constexpr int kThreads = kG1 + kG2;
constexpr int kHalves = kG2 / 16;
constexpr int kMaxSlots = 3;
constexpr int kBarCopy = 1;            // stage-1 group: ring slot ready / released
constexpr int kBarFull = 2;            // + buffer index: (tm, tk) written
constexpr int kBarEmpty = 4;           // + buffer index: (tm, tk) consumed

__device__ __forceinline__ void bar_sync(int id, int cnt) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(cnt) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int cnt) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(cnt) : "memory");
}
// 4-byte copy issued only when on != 0 (predicated inside the asm: no branch)
__device__ __forceinline__ void cp_async4_if(uint32_t dst, const float* src, int on) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %2, 0;\n @q cp.async.ca.shared.global [%0], [%1], 4;\n}"
      ::"r"(dst), "l"(src), "r"(on) : "memory");
}
// 4-byte copy, zero-filled when on == 0 (src-size 0: nothing is read)
__device__ __forceinline__ void cp_async4_zfill(uint32_t dst, const float* src, int on) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src),
               "r"(on ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// all but the nb - 2 most recent copy groups have landed
__device__ __forceinline__ void cp_async_wait_ring(int nb) {
  switch (nb) {
    case 8: cp_async_wait<6>(); break;
    case 7: cp_async_wait<5>(); break;
    case 6: cp_async_wait<4>(); break;
    case 5: cp_async_wait<3>(); break;
    case 4: cp_async_wait<2>(); break;
    case 3: cp_async_wait<1>(); break;
    default: cp_async_wait<0>(); break;
  }
}
// sum of W band taps: the first a packed multiply, the rest packed FMAs
template <int W, class F>
__device__ __forceinline__ float2 taps(F&& term) {
  float2 acc = __fmul2_rn(term(0).x_, term(0).y_);
#pragma unroll
  for (int o = 1; o < W; ++o) acc = __ffma2_rn(term(o).x_, term(o).y_, acc);
  return acc;
}
struct Term {
  float2 x_, y_;
};

// Shared-memory layout for band width W and grids with J*G <= NC (G groups of
// J grid lines), all strides compile-time so that every band tap is an
// immediate offset.  (tm, tk) are stored interleaved, element (r, c) as the
// pair at 2 (r NS + c): stage 1 writes its (tm, tk) accumulator pairs as they
// are, stage 2 reads one pair per 64-bit load.
template <int W, int NC>
struct Lay {
  static constexpr int p = (W - 1) / 2;
  static constexpr int J = W <= 9 ? 4 : 2;            // grid columns / rows per thread
  static constexpr int V = (J + W - 1 + J - 1) / J;   // J-vectors in a stage-1 window
  static constexpr int XS = (NC - J + J * V + 3) / 4 * 4;  // padded x row, data at [p, p + n)
  static constexpr int R = NC + W - 1;                // (tm, tk) rows, data at [p, p + n)
  static constexpr int NS = NC;                       // (tm, tk) row stride in pairs
  static constexpr int BUF = 2 * R * NS;              // floats per (tm, tk) buffer
  static_assert(XS % 4 == 0 && NS % 2 == 0, "vector alignment");
};

template <int W, int NC>
__global__ void __launch_bounds__(kThreads, 1)
    k_spmm32(int n, int nrhs, int nb, const float* __restrict__ M1, const float* __restrict__ K1,
             SpmmCoef cf, const float* __restrict__ x, float* __restrict__ y, long ld) {
  using L = Lay<W, NC>;
  constexpr int p = L::p, J = L::J, V = L::V, XS = L::XS, NS = L::NS;
  using VecJ = typename std::conditional<J == 4, float4, float2>::type;
  const int G = (n + J - 1) / J, slot = n * XS;
  extern __shared__ __align__(16) float sm[];
  float* ring = sm;                               // [nb][n][XS]
  float* tb = sm + (size_t)nb * slot;             // [2][R][NS][tm, tk]
  const int total = nb * slot + 2 * L::BUF;
  for (int i = threadIdx.x; i < total; i += kThreads) sm[i] = 0.0f;  // halos stay zero
  __syncthreads();
  const int cnt = nrhs > (int)blockIdx.x ? (nrhs - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  auto column = [&](int k) { return (size_t)blockIdx.x + (size_t)k * gridDim.x; };

  if (threadIdx.x < kG1) {
    // ------------------------------ stage 1 ------------------------------
    const int t = threadIdx.x;
    const int R1 = kG1 / G, g = t % G, r0 = t / G;
    const bool on = r0 < R1;
    float2 ab[J][W];  // (X1, W1) band pairs of grid columns J g + j
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const int ix = J * g + j;
#pragma unroll
      for (int o = 0; o < W; ++o) {
        const float m = ix < n ? M1[ix * W + o] : 0.0f;
        const float kv = ix < n ? K1[ix * W + o] : 0.0f;
        ab[j][o] = make_float2(fmaf(cf.xk, kv, cf.xm * m), fmaf(cf.wk, kv, cf.wm * m));
      }
    }
    // copies: warp w takes grid rows w, w + 7, ...; lane l columns l, l + 32, l + 64
    const int wq = t >> 5, lane = t & 31;
    const int c0 = lane < n, c1 = lane + 32 < n, c2 = lane + 64 < n;
    const uint32_t ring_s = smem_u32(ring) + 4u * (p + lane);
    auto issue = [&](int k, int s) {  // column k of this CTA into ring slot s
      if (k < cnt) {
        const float* src = x + column(k) * ld + lane;
        const uint32_t dst = ring_s + 4u * (uint32_t)(s * slot);
        for (int iy = wq; iy < n; iy += kG1 / 32) {
          const float* sr = src + iy * n;
          const uint32_t dr = dst + 4u * (uint32_t)(iy * XS);
          cp_async4_if(dr, sr, c0);
          cp_async4_if(dr + 128u, sr + 32, c1);
          cp_async4_if(dr + 256u, sr + 64, c2);
        }
      }
      cp_async_commit();  // empty groups keep the group count uniform
    };
    for (int s = 0; s + 1 < nb; ++s) issue(s, s);
    int sk = 0;  // ring slot of column k
    for (int k = 0; k < cnt; ++k) {
      cp_async_wait_ring(nb);
      bar_sync(kBarCopy, kG1);  // column k complete; slot (k - 1) % nb no longer read
      issue(k + nb - 1, sk == 0 ? nb - 1 : sk - 1);
      const float* xk = ring + sk * slot + J * g;
      float* tm = tb + (k & 1) * L::BUF + 2 * (p * NS + J * g);
      if (k >= 2) bar_sync(kBarEmpty + (k & 1), kThreads);
      if (on) {
        for (int iy = r0; iy < n; iy += R1) {
          // x[iy][J g - p + q] sits at ring[iy][J g + q]
          const VecJ* row = (const VecJ*)(xk + iy * XS);
          float v[J * V];
#pragma unroll
          for (int q = 0; q < V; ++q) {
            const VecJ w = row[q];
            v[J * q] = w.x;
            v[J * q + 1] = w.y;
            if constexpr (J == 4) {
              v[J * q + 2] = w.z;
              v[J * q + 3] = w.w;
            }
          }
          float2 acc[J];  // (tm, tk) of grid columns J g + j
#pragma unroll
          for (int j = 0; j < J; ++j)
            acc[j] = taps<W>([&](int o) { return Term{ab[j][o], make_float2(v[j + o], v[j + o])}; });
          // columns J g + j >= n carry zero bands; they land in the row padding
          float4* d = (float4*)(tm + 2 * iy * NS);
#pragma unroll
          for (int j = 0; j < J; j += 2) d[j / 2] = make_float4(acc[j].x, acc[j].y, acc[j + 1].x, acc[j + 1].y);
        }
      }
      bar_arrive(kBarFull + (k & 1), kThreads);
      sk = sk + 1 == nb ? 0 : sk + 1;
    }
    cp_async_wait<0>();
  } else {
    // ------------------------------ stage 2 ------------------------------
    // half-warp h takes row groups h, h + 18, ...; lane c of it columns c, c + 16, ...
    // (16 consecutive pairs: one 128-byte wavefront per half-warp and load)
    const int u = threadIdx.x - kG1;
    const int h = u >> 4, c = u & 15;
    auto coefs = [&](int gy, float2 (&yz)[J][W]) {  // (Y2, Z2) band pairs of rows J gy + j
#pragma unroll
      for (int j = 0; j < J; ++j) {
        const int iy = J * gy + j;
#pragma unroll
        for (int o = 0; o < W; ++o) {
          const float m = iy < n ? M1[iy * W + o] : 0.0f;
          const float kv = iy < n ? K1[iy * W + o] : 0.0f;
          yz[j][o] = make_float2(fmaf(cf.yk, kv, cf.ym * m), fmaf(cf.zk, kv, cf.zm * m));
        }
      }
    };
    auto rows = [&](int gy, const float2 (&yz)[J][W], const float* tm, float* yb) {
      const float2* tg = (const float2*)tm + J * gy * NS;
      float* yg = yb + (size_t)(J * gy) * n;
      const int jn = J * gy < n ? min(J, n - J * gy) : 0;  // valid rows of the group
      for (int ix = c; ix < n; ix += 16) {
        // (tm, tk)[iy - p + o][ix] sits at row iy + o (halo rows)
        float2 w[J + W - 1];
#pragma unroll
        for (int q = 0; q < J + W - 1; ++q) w[q] = tg[q * NS + ix];
        float* yc = yg + ix;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const float2 acc = taps<W>([&](int o) { return Term{yz[j][o], w[j + o]}; });
          if (j < jn) yc[j * n] = acc.x + acc.y;
        }
      }
    };
    float2 yz[J][W];
    const bool one = G <= kHalves;  // one row group per half-warp: bands stay in registers
    if (one) coefs(h, yz);
    for (int k = 0; k < cnt; ++k) {
      bar_sync(kBarFull + (k & 1), kThreads);
      const float* tm = tb + (k & 1) * L::BUF;
      float* yb = y + column(k) * ld;
      if (one) {
        if (h < G) rows(h, yz, tm, yb);
      } else {
        for (int gy = h; gy < G; gy += kHalves) {
          coefs(gy, yz);
          rows(gy, yz, tm, yb);
        }
      }
      if (k + 2 < cnt) bar_arrive(kBarEmpty + (k & 1), kThreads);
    }
  }
}

// ---------------------------------------------------------------------------
// Row-strip form for grids the persistent layouts do not hold (n > 84, e.g.
// h = 1/128): CTA (s, g) takes grid rows [s SR, s SR + SR) of columns g,
// g + gridDim.y, ...  Per column it stages the strip's rows plus p halo rows
// above and below (zero outside the grid, p zero padding columns each side;
// two stages, the next column copied by 4-byte cp.async while the current one
// is contracted).  Thread t owns grid column ix = t (+ blockDim, ...) and walks
// the staged rows q: stage 1 turns row q into the pair (tm, tk) at ix with the
// (X1, W1) band pair of ix in registers; the pairs of the last 2p + 1 rows sit
// in a register window, and once it is full stage 2 forms y of grid row
// r0 + q - 2p with the (Y2, Z2) band pairs of that row (shared-memory
// broadcasts).  Both stages use packed FMAs.  The halo rows' pairs are
// recomputed by the neighbouring strips (a factor (SR + 2p) / SR on stage 1).
// ---------------------------------------------------------------------------
template <int W>
__global__ void __launch_bounds__(512) k_spmm32_strip(int n, int nrhs, int SR,
                                                      const float* __restrict__ M1,
                                                      const float* __restrict__ K1, SpmmCoef cf,
                                                      const float* __restrict__ x,
                                                      float* __restrict__ y, long ld) {
  constexpr int p = (W - 1) / 2;
  extern __shared__ __align__(16) float sm[];
  const int RS = SR + 2 * p, XW = n + 2 * p, STAGE = RS * XW;
  float2* c2 = (float2*)sm;                 // [SR][W]: (Y2, Z2) of grid row r0 + j, tap o
  float* xs = sm + 2 * SR * W;              // [2][RS][XW]: x[r0 - p + q][c - p] at [q][c]
  const int r0 = blockIdx.x * SR;
  const int rows = min(SR, n - r0);
  const int T = blockDim.x;
  for (int i = threadIdx.x; i < SR * W; i += T) {
    const int j = i / W, o = i - j * W, iy = min(r0 + j, n - 1);
    const float m = M1[iy * W + o], k = K1[iy * W + o];
    c2[i] = make_float2(fmaf(cf.yk, k, cf.ym * m), fmaf(cf.zk, k, cf.zm * m));
  }
  const uint32_t xbase = (uint32_t)__cvta_generic_to_shared(xs);
  auto stage = [&](int b, int s) {
    const float* xb = x + (size_t)b * ld;
    const uint32_t base = xbase + 4u * (uint32_t)(s * STAGE);
    for (int i = threadIdx.x; i < STAGE; i += T) {
      const int q = i / XW, c = i - q * XW;
      const int iy = r0 - p + q, ix = c - p;
      const int on = iy >= 0 && iy < n && ix >= 0 && ix < n;
      cp_async4_zfill(base + 4u * (uint32_t)i, on ? xb + (size_t)iy * n + ix : x, on);
    }
  };
  int b = blockIdx.y;
  if (b < nrhs) stage(b, 0);
  cp_async_commit();
  for (int t = 0; b < nrhs; b += gridDim.y, ++t) {
    if (b + (int)gridDim.y < nrhs) stage(b + gridDim.y, (t + 1) & 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float* xq = xs + (t & 1) * STAGE;
    float* yb = y + (size_t)b * ld;
    for (int ix0 = 0; ix0 < n; ix0 += T) {
      const int ix = min(ix0 + (int)threadIdx.x, n - 1);
      const bool mine = ix0 + (int)threadIdx.x < n;
      float2 a1[W];   // (X1, W1) of grid column ix, tap o
#pragma unroll
      for (int o = 0; o < W; ++o) {
        const float m = M1[ix * W + o], k = K1[ix * W + o];
        a1[o] = make_float2(fmaf(cf.xk, k, cf.xm * m), fmaf(cf.wk, k, cf.wm * m));
      }
      float2 win[W];  // (tm, tk) of staged row q at win[q % W]
      for (int q0 = 0; q0 < RS; q0 += W) {
#pragma unroll
        for (int k = 0; k < W; ++k) {
          const int q = q0 + k;
          if (q < RS) {
            const float* xr = xq + q * XW + ix;   // x[.][ix - p + o] at xr[o]
            float2 acc = __fmul2_rn(a1[0], make_float2(xr[0], xr[0]));
#pragma unroll
            for (int o = 1; o < W; ++o) acc = __ffma2_rn(a1[o], make_float2(xr[o], xr[o]), acc);
            win[k] = acc;
            const int j = q - 2 * p;   // output row r0 + j needs staged rows j .. j + 2p
            if (j >= 0 && j < rows) {
              const float2* cj = c2 + j * W;
              float2 s2 = __fmul2_rn(cj[0], win[(k + 1) % W]);
#pragma unroll
              for (int o = 1; o < W; ++o) s2 = __ffma2_rn(cj[o], win[(k + 1 + o) % W], s2);
              if (mine) yb[(size_t)(r0 + j) * n + ix] = s2.x + s2.y;
            }
          }
        }
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

// strip height, threads and shared bytes of the strip form (SR = 0: does not fit):
// the tallest strip (at most 32 rows) in 100 KB, else in all of smem_max.  (Shorter
// strips for more CTAs per SM measured slower: the halo rows' stage-1 work grows.)
int strip_plan(int n, int p, size_t smem_max, size_t* bytes, int* threads) {
  const int W = 2 * p + 1;
  *threads = std::min(512, (n + 31) / 32 * 32);
  for (const size_t budget : {std::min(smem_max, (size_t)100 * 1024), smem_max}) {
    for (int SR = 32; SR >= 1; SR /= 2) {
      const size_t RS = SR + 2 * p, XW = n + 2 * p;
      const size_t b = 4 * (2 * (size_t)SR * W + 2 * RS * XW);
      if (b <= budget) {
        *bytes = b;
        return SR;
      }
    }
  }
  *bytes = 0;
  return 0;
}

template <int W>
cudaError_t launch_strip_w(int n, int nrhs, const float* M1, const float* K1, SpmmCoef cf,
                           const float* x, float* y, long ld, int sms, size_t smem_max,
                           cudaStream_t st) {
  int pl[5];
  spmm32_strip_plan(n, (W - 1) / 2, nrhs, sms, smem_max, pl);
  const int SR = pl[0], threads = pl[1], bytes = pl[2], strips = pl[3], cg = pl[4];
  if (!SR) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_spmm32_strip<W>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_spmm32_strip<W><<<dim3(strips, cg), threads, bytes, st>>>(n, nrhs, SR, M1, K1, cf, x, y, ld);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Curved map (an assembled (2p+1)^2 stencil per grid point, Sec. 2: M and K
// of a B-spline geometry are not Kronecker products).  CTA (tile, g) takes an
// 8 x 32 tile of grid points; each thread owns one point and keeps its
// (2p+1)^2 FP32 coefficients a = cm M + ck K in registers (p <= 5; read from
// global memory per tap above that), loaded once and reused for every column
// the CTA visits.  Columns go four at a time, interleaved in shared memory as
// float4 over the tile plus p halo rows and columns (zero outside the grid),
// so one 128-bit load feeds four FMAs; the next group of four is staged by
// 4-byte cp.async while the current one is contracted (two stages).
// ---------------------------------------------------------------------------
constexpr int kCurvTR = 8, kCurvTC = 32, kCurvThreads = kCurvTR * 32;


// register caps: the coefficients of one point in registers, and 4 / 3 / 2 / 1 CTAs per SM
// for p = 2 / 3 / 4 / 5 (p >= 6 reads coefficients from global memory)
template <int W>
__global__ void __maxnreg__(W <= 5 ? 56 : W <= 7 ? 80 : W <= 9 ? 128 : W <= 11 ? 168 : 64)
    k_spmm32_curved(
    int n, int nrhs, const float* __restrict__ Mq, const float* __restrict__ Kq, float cm,
    float ck, const float* __restrict__ x, float* __restrict__ y, long ld) {
  constexpr int p = (W - 1) / 2, Q = W * W;
  constexpr bool kReg = Q <= 121;
  constexpr int HR = kCurvTR + 2 * p, HC = kCurvTC + 2 * p, STAGE = HR * HC;
  extern __shared__ __align__(16) float4 xs4[];   // [2][HR][HC]: (iy0 - p + r, ix0 - p + c)
  const int tilesx = (n + kCurvTC - 1) / kCurvTC;
  const int ix0 = (blockIdx.x % tilesx) * kCurvTC, iy0 = (blockIdx.x / tilesx) * kCurvTR;
  const int lane = threadIdx.x & 31, wr = threadIdx.x >> 5;
  const int ix = ix0 + lane, iy = iy0 + wr;
  const bool mine = ix < n && iy < n;
  const size_t N = (size_t)n * n;
  const size_t pt = mine ? (size_t)iy * n + ix : 0;
  // coefficient q (entry (q / W, q % W) of the point's stencil) of cm M + ck K
  auto coef = [&](int q) {
    float a = 0.0f;
    if (Mq) a = cm * __ldg(Mq + q * N + pt);
    if (Kq) a = fmaf(ck, __ldg(Kq + q * N + pt), a);
    return a;
  };
  float v[kReg ? Q : 1];
  if constexpr (kReg) {
#pragma unroll
    for (int q = 0; q < Q; ++q) v[q] = coef(q);
  }
  const int ngroups = (nrhs + 3) / 4;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(xs4);
  auto stage = [&](int g, int s) {
    const uint32_t base = sbase + (uint32_t)(s * STAGE) * 16u;
    for (int e = threadIdx.x; e < 4 * STAGE; e += kCurvThreads) {
      const int b = e & 3, pos = e >> 2, r = pos / HC, c = pos - r * HC;
      const int jy = iy0 - p + r, jx = ix0 - p + c, col = 4 * g + b;
      const int on = jy >= 0 && jy < n && jx >= 0 && jx < n && col < nrhs;
      const float* src = on ? x + (size_t)col * ld + (size_t)jy * n + jx : x;
      cp_async4_zfill(base + 4u * (uint32_t)e, src, on);
    }
  };
  int g = blockIdx.y;
  if (g < ngroups) stage(g, 0);
  cp_async_commit();
  for (int t = 0; g < ngroups; g += gridDim.y, ++t) {
    if (g + (int)gridDim.y < ngroups) stage(g + gridDim.y, (t + 1) & 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();
    const float4* xt = xs4 + (t & 1) * STAGE + wr * HC + lane;
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if constexpr (!kReg) {
      // coefficients from global memory: one stencil row at a time
#pragma unroll 1
      for (int dy = 0; dy < W; ++dy) {
#pragma unroll
        for (int dx = 0; dx < W; ++dx) {
          const float a = coef(dy * W + dx);
          const float4 u = xt[dy * HC + dx];
          acc.x = fmaf(a, u.x, acc.x);
          acc.y = fmaf(a, u.y, acc.y);
          acc.z = fmaf(a, u.z, acc.z);
          acc.w = fmaf(a, u.w, acc.w);
        }
      }
    }
#pragma unroll
    for (int dy = 0; dy < W; ++dy) {
#pragma unroll
      for (int dx = 0; dx < W; ++dx) {
        if constexpr (kReg) {
          const float a = v[dy * W + dx];
          const float4 u = xt[dy * HC + dx];
          acc.x = fmaf(a, u.x, acc.x);
          acc.y = fmaf(a, u.y, acc.y);
          acc.z = fmaf(a, u.z, acc.z);
          acc.w = fmaf(a, u.w, acc.w);
        }
      }
    }
    if (mine) {
      const float r[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
      for (int b = 0; b < 4; ++b)
        if (4 * g + b < nrhs) y[(size_t)(4 * g + b) * ld + pt] = r[b];
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

template <int W>
cudaError_t launch_curved_w(int n, int nrhs, const float* Mq, const float* Kq, float cm, float ck,
                            const float* x, float* y, long ld, int sms, cudaStream_t st) {
  constexpr int p = (W - 1) / 2;
  const size_t bytes = 2 * sizeof(float4) * (size_t)(kCurvTR + 2 * p) * (kCurvTC + 2 * p);
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_spmm32_curved<W>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
  }
  int pl[6];
  spmm32_curved_plan(n, p, nrhs, sms, pl);
  const int tiles = pl[4], cg = pl[5];
  k_spmm32_curved<W><<<dim3(tiles, cg), kCurvThreads, bytes, st>>>(n, nrhs, Mq, Kq, cm, ck, x, y,
                                                                   ld);
  return cudaGetLastError();
}

constexpr int kCaps[] = {68, 84};  // J*G limits of the two layouts

template <int W, int NC>
size_t smem_of(int n, int nb) {
  using L = Lay<W, NC>;
  return sizeof(float) * ((size_t)nb * n * L::XS + 2 * (size_t)L::BUF);
}

// layout cap and ring depth for an n x n grid (cap 0: does not fit)
template <int W>
void plan(int n, size_t smem_max, int* cap, int* nb) {
  constexpr int J = W <= 9 ? 4 : 2;
  const int JG = (n + J - 1) / J * J;
  *cap = 0;
  *nb = 0;
  for (int d = kMaxSlots; d >= 2 && !*cap; --d) {
    if (JG <= kCaps[0] && smem_of<W, kCaps[0]>(n, d) <= smem_max) *cap = kCaps[0];
    else if (JG <= kCaps[1] && smem_of<W, kCaps[1]>(n, d) <= smem_max) *cap = kCaps[1];
    if (*cap) *nb = d;
  }
}

template <int W, int NC>
cudaError_t launch_nc(int n, int nrhs, int nb, const float* M1, const float* K1, SpmmCoef cf,
                      const float* x, float* y, long ld, int grid, cudaStream_t st) {
  const size_t smem = smem_of<W, NC>(n, nb);
  cudaError_t e = cudaFuncSetAttribute(k_spmm32<W, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_spmm32<W, NC><<<grid, kThreads, smem, st>>>(n, nrhs, nb, M1, K1, cf, x, y, ld);
  return cudaGetLastError();
}

template <int W>
int slots_w(int n, size_t smem_max) {
  int cap, nb;
  plan<W>(n, smem_max, &cap, &nb);
  return nb;
}

template <int W>
cudaError_t launch_w(int n, int nrhs, const float* M1, const float* K1, SpmmCoef cf,
                     const float* x, float* y, long ld, int grid, size_t smem_max, cudaStream_t st) {
  int cap, nb;
  plan<W>(n, smem_max, &cap, &nb);
  if (cap == kCaps[0]) return launch_nc<W, kCaps[0]>(n, nrhs, nb, M1, K1, cf, x, y, ld, grid, st);
  if (cap == kCaps[1]) return launch_nc<W, kCaps[1]>(n, nrhs, nb, M1, K1, cf, x, y, ld, grid, st);
  return cudaErrorInvalidValue;
}

}  // namespace

template <int W>
void layout_w(int n, size_t smem_max, int* out) {
  int cap, nb;
  plan<W>(n, smem_max, &cap, &nb);
  out[0] = cap;
  out[1] = nb;
  if (cap == kCaps[0] || cap == kCaps[1]) {
    const bool a = cap == kCaps[0];
    out[2] = a ? Lay<W, kCaps[0]>::J : Lay<W, kCaps[1]>::J;
    out[3] = a ? Lay<W, kCaps[0]>::XS : Lay<W, kCaps[1]>::XS;
    out[4] = a ? Lay<W, kCaps[0]>::NS : Lay<W, kCaps[1]>::NS;
    out[5] = a ? Lay<W, kCaps[0]>::R : Lay<W, kCaps[1]>::R;
    out[6] = (int)(a ? smem_of<W, kCaps[0]>(n, nb) : smem_of<W, kCaps[1]>(n, nb));
  } else {
    out[2] = out[3] = out[4] = out[5] = out[6] = 0;
  }
}

int spmm32_layout(int n, int p, size_t smem_max, int* out) {
  switch (p) {
    case 2: layout_w<5>(n, smem_max, out); break;
    case 3: layout_w<7>(n, smem_max, out); break;
    case 4: layout_w<9>(n, smem_max, out); break;
    case 5: layout_w<11>(n, smem_max, out); break;
    case 6: layout_w<13>(n, smem_max, out); break;
    case 7: layout_w<15>(n, smem_max, out); break;
    case 8: layout_w<17>(n, smem_max, out); break;
    default: return 0;
  }
  return out[0] != 0;
}

int spmm32_slots(int n, int p, size_t smem_max) {
  switch (p) {
    case 2: return slots_w<5>(n, smem_max);
    case 3: return slots_w<7>(n, smem_max);
    case 4: return slots_w<9>(n, smem_max);
    case 5: return slots_w<11>(n, smem_max);
    case 6: return slots_w<13>(n, smem_max);
    case 7: return slots_w<15>(n, smem_max);
    case 8: return slots_w<17>(n, smem_max);
    default: return 0;
  }
}

cudaError_t launch_spmm32_strip(int n, int p, int nrhs, const float* M1, const float* K1,
                                SpmmCoef cf, const float* x, float* y, long ld, int sms,
                                size_t smem_max, cudaStream_t st) {
  switch (p) {
    case 2: return launch_strip_w<5>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    case 3: return launch_strip_w<7>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    case 4: return launch_strip_w<9>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    case 5: return launch_strip_w<11>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    case 6: return launch_strip_w<13>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    case 7: return launch_strip_w<15>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    case 8: return launch_strip_w<17>(n, nrhs, M1, K1, cf, x, y, ld, sms, smem_max, st);
    default: return cudaErrorInvalidValue;
  }
}

int spmm32_strip_rows(int n, int p, size_t smem_max) {
  size_t bytes = 0;
  int threads = 0;
  return (p >= 2 && p <= 8 && n >= 1) ? strip_plan(n, p, smem_max, &bytes, &threads) : 0;
}

void spmm32_strip_plan(int n, int p, int nrhs, int sms, size_t smem_max, int* out) {
  size_t bytes = 0;
  int threads = 0;
  const int SR = (p >= 2 && p <= 8 && n >= 1) ? strip_plan(n, p, smem_max, &bytes, &threads) : 0;
  const int strips = SR ? (n + SR - 1) / SR : 0;
  out[0] = SR;
  out[1] = SR ? threads : 0;
  out[2] = (int)bytes;
  out[3] = strips;
  // about four CTAs per SM over the launch
  out[4] = SR ? std::max(1, std::min(nrhs, (4 * sms + strips - 1) / strips)) : 0;
}

void spmm32_curved_plan(int n, int p, int nrhs, int sms, int* out) {
  const int tiles = ((n + kCurvTC - 1) / kCurvTC) * ((n + kCurvTR - 1) / kCurvTR);
  const int ngroups = (nrhs + 3) / 4;
  out[0] = kCurvTR;
  out[1] = kCurvTC;
  out[2] = kCurvTR + 2 * p;
  out[3] = kCurvTC + 2 * p;
  out[4] = tiles;
  // about four CTAs per SM over the launch; each loads its coefficients once
  out[5] = std::max(1, std::min(ngroups, (4 * sms + tiles - 1) / tiles));
}

cudaError_t launch_spmm32_curved(int n, int p, int nrhs, const float* Mq, const float* Kq,
                                 float cm, float ck, const float* x, float* y, long ld, int sms,
                                 cudaStream_t st) {
  if (n < 1 || (long)n * n > ld) return cudaErrorInvalidValue;
  switch (p) {
    case 2: return launch_curved_w<5>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    case 3: return launch_curved_w<7>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    case 4: return launch_curved_w<9>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    case 5: return launch_curved_w<11>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    case 6: return launch_curved_w<13>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    case 7: return launch_curved_w<15>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    case 8: return launch_curved_w<17>(n, nrhs, Mq, Kq, cm, ck, x, y, ld, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_spmm32(int n, int p, int nrhs, const float* M1, const float* K1, SpmmCoef cf,
                          const float* x, float* y, long ld, int grid, size_t smem_max,
                          cudaStream_t st) {
  switch (p) {
    case 2: return launch_w<5>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    case 3: return launch_w<7>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    case 4: return launch_w<9>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    case 5: return launch_w<11>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    case 6: return launch_w<13>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    case 7: return launch_w<15>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    case 8: return launch_w<17>(n, nrhs, M1, K1, cf, x, y, ld, grid, smem_max, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace igm
