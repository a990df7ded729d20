// C ABI of the library (include/igamgrit.h): host orchestration, device
// uploads and the kernels that run the p-multigrid solves (Sec. 4) and the
// MGRIT sweeps (Sec. 3).
#include <cuda_runtime.h>

#include <algorithm>

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "../../include/igamgrit.h"
#include "host_setup.h"
#include "kernels.h"
#include "phic.h"
#include "spmm.h"

using namespace igm;

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
static thread_local std::string g_err;
static std::atomic<long> g_launches{0};

static igm_status fail(igm_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t _e = (call);                                                              \
    if (_e != cudaSuccess)                                                                \
      return fail(_e == cudaErrorMemoryAllocation ? IGM_ERR_OOM : IGM_ERR_CUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(_e));                    \
  } while (0)

extern "C" const char* igm_last_error(void) { return g_err.c_str(); }
extern "C" long igm_kernel_launches(void) { return g_launches.load(); }

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  ~DevBuf() { if (p) cudaFree(p); }
};

struct Uploader {
  std::vector<std::unique_ptr<DevBuf>> bufs;
  cudaError_t err = cudaSuccess;
  template <typename T>
  T* put(const std::vector<T>& v) {
    if (err != cudaSuccess) return nullptr;
    if (v.empty()) return nullptr;
    auto b = std::make_unique<DevBuf>();
    b->bytes = v.size() * sizeof(T);
    err = cudaMalloc(&b->p, b->bytes);
    if (err != cudaSuccess) return nullptr;
    err = cudaMemcpy(b->p, v.data(), b->bytes, cudaMemcpyHostToDevice);
    T* out = (T*)b->p;
    bufs.push_back(std::move(b));
    return out;
  }
  template <typename T>
  float* put32(const std::vector<T>& v) {
    std::vector<float> f(v.begin(), v.end());
    return put(f);
  }
  void* raw(size_t bytes) {
    if (err != cudaSuccess) return nullptr;
    auto b = std::make_unique<DevBuf>();
    b->bytes = bytes;
    err = cudaMalloc(&b->p, bytes);
    if (err != cudaSuccess) return nullptr;
    err = cudaMemset(b->p, 0, bytes);
    void* out = b->p;
    bufs.push_back(std::move(b));
    return out;
  }
};

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct iga_ops {
  Geometry geom;
  Discretisation hi, lo;   // order p and order 1 on the same knots / rule
  Csr P, PT;               // transfer interior x interior and its transpose
  double kappa = 1.0;
  Uploader up;
  // device copies
  double *bM64 = nullptr, *bK64 = nullptr, *sM64 = nullptr, *sK64 = nullptr;
  float *bM32 = nullptr, *bK32 = nullptr;
  float *sMq32 = nullptr, *sKq32 = nullptr;   // curved map: FP32 stencils, [(2p+1)^2][N]
  std::vector<double> qpts, qwdet;
};

struct pmg_handle {
  const iga_ops* ops = nullptr;
  pmg_opts opts;
  double c = 0.0;
  Csr L, U;
  PmgD d;
  Uploader up;
  bool arena_smem = true;
  long arena_bytes = 0;
  long smem_bytes = 0;      // dynamic shared memory per CTA of the solve kernels
  char* garena = nullptr;   // global arena for grid_capacity CTAs when not in shared memory
  int grid_capacity = 0;
};

static Csr transpose(const Csr& A) {
  Csr T;
  T.rows = A.cols;
  T.cols = A.rows;
  T.ptr.assign(T.rows + 1, 0);
  for (int c : A.col) T.ptr[c + 1]++;
  for (int i = 0; i < T.rows; ++i) T.ptr[i + 1] += T.ptr[i];
  T.col.resize(A.col.size());
  T.val.resize(A.val.size());
  std::vector<int> pos(T.ptr.begin(), T.ptr.end() - 1);
  for (int i = 0; i < A.rows; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int c = A.col[k];
      T.col[pos[c]] = i;
      T.val[pos[c]] = A.val[k];
      pos[c]++;
    }
  return T;
}

static int dev_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v;
}

// ---------------------------------------------------------------------------
// iga_assemble and friends
// ---------------------------------------------------------------------------
extern "C" igm_status iga_basis_eval(int p, int nel, int nx, const double* x, int* span,
                                     double* N, double* dN) {
  if (p < 1 || p > 8 || nel < 1 || nx < 0 || (nx > 0 && (!x || !span || !N)))
    return fail(IGM_ERR_ARG, "iga_basis_eval: p in [1, 8], nel >= 1, non-null x, span, N");
  for (int i = 0; i < nx; ++i)
    if (!(x[i] >= 0.0 && x[i] <= 1.0)) return fail(IGM_ERR_ARG, "iga_basis_eval: x outside [0, 1]");
  const std::vector<double> t = open_uniform_knots(p, nel);
  for (int i = 0; i < nx; ++i) {
    span[i] = find_span(t, p, x[i]);
    basis_on_span(t, p, span[i], x[i], N + (size_t)i * (p + 1),
                  dN ? dN + (size_t)i * (p + 1) : nullptr);
  }
  return IGM_OK;
}

// The map of an iga_desc: the unit square, or the B-spline map with open
// uniform knots.  Returns "" or an error text.
static std::string make_geometry(const iga_desc* desc, Geometry& g) {
  if (desc->geom == 0) {
    g.affine = true;
    return "";
  }
  if (desc->geom != 1) return "geom must be 0 or 1";
  g.affine = false;
  for (int d = 0; d < 2; ++d) {
    g.deg[d] = desc->gdeg[d];
    g.nctrl[d] = desc->gn[d];
    if (g.deg[d] < 1 || g.nctrl[d] <= g.deg[d]) return "invalid geometry net";
    g.knots[d] = open_uniform_knots(g.deg[d], g.nctrl[d] - g.deg[d]);
  }
  if (!desc->gctrl) return "geometry control net missing";
  g.ctrl.assign(desc->gctrl, desc->gctrl + 2 * g.nctrl[0] * g.nctrl[1]);
  return "";
}

extern "C" igm_status iga_assemble_host(const iga_desc* desc, int which, int* n, double* out) {
  if (!desc) return fail(IGM_ERR_ARG, "null argument");
  if (desc->p < 1 || desc->p > 8) return fail(IGM_ERR_ARG, "p must be in [1, 8]");
  if (desc->nel < 2 || desc->nel > 1024) return fail(IGM_ERR_ARG, "nel must be in [2, 1024]");
  if (which < 0 || which > 2) return fail(IGM_ERR_ARG, "which must be 0 (M), 1 (K) or 2 (lumped)");
  Geometry g;
  const std::string ge = make_geometry(desc, g);
  if (!ge.empty()) return fail(IGM_ERR_ARG, ge);
  Discretisation d;
  const int nq = desc->nquad > 0 ? desc->nquad : desc->p + 1;
  const std::string e = assemble(g, desc->p, desc->nel, nq, d);
  if (!e.empty()) return fail(IGM_ERR_ARG, e);
  if (n) *n = d.n;
  if (out) {
    const std::vector<double>& v = which == 0 ? d.M.val : (which == 1 ? d.K.val : d.lumped);
    std::memcpy(out, v.data(), v.size() * sizeof(double));
  }
  return IGM_OK;
}

extern "C" igm_status iga_transfer_host(const iga_desc* desc, int* nnz, int* ptr, int* col,
                                        double* val) {
  if (!desc) return fail(IGM_ERR_ARG, "null argument");
  if (desc->p < 2 || desc->p > 8) return fail(IGM_ERR_ARG, "p must be in [2, 8]");
  if (desc->nel < 2 || desc->nel > 1024) return fail(IGM_ERR_ARG, "nel must be in [2, 1024]");
  Geometry g;
  const std::string ge = make_geometry(desc, g);
  if (!ge.empty()) return fail(IGM_ERR_ARG, ge);
  Discretisation hi, lo;
  const int nq = desc->nquad > 0 ? desc->nquad : desc->p + 1;
  std::string e = assemble(g, desc->p, desc->nel, nq, hi);
  if (e.empty()) e = assemble(g, 1, desc->nel, nq, lo);
  if (!e.empty()) return fail(IGM_ERR_ARG, e);
  const Csr P = transfer(g, hi, lo);
  if (nnz) *nnz = P.nnz();
  if (ptr) std::memcpy(ptr, P.ptr.data(), P.ptr.size() * sizeof(int));
  if (col) std::memcpy(col, P.col.data(), P.col.size() * sizeof(int));
  if (val) std::memcpy(val, P.val.data(), P.val.size() * sizeof(double));
  return IGM_OK;
}

// The p = 1 operator M_1 + c K_1 and its Galerkin h-hierarchy (Sec. 4, Fig. 5):
// coarsen while the element count is even and above coarsest_nel, at most kMaxH levels.
static std::vector<Stencil> hmg_hierarchy(const Discretisation& lo, double c, int coarsest_nel) {
  std::vector<Stencil> H;
  Stencil A1 = lo.M;
  for (size_t i = 0; i < A1.val.size(); ++i) A1.val[i] = lo.M.val[i] + c * lo.K.val[i];
  H.push_back(A1);
  int nel_k = lo.nel;
  while (nel_k > coarsest_nel && nel_k % 2 == 0 && (int)H.size() < kMaxH) {
    H.push_back(galerkin_coarse(H.back()));
    nel_k /= 2;
  }
  return H;
}

extern "C" igm_status pmg_hmg_host(const iga_desc* desc, double kappa_dt, int coarsest_nel,
                                   int level, int* nlevels, int* n, double* out) {
  if (!desc) return fail(IGM_ERR_ARG, "null argument");
  if (desc->nel < 2 || desc->nel > 1024) return fail(IGM_ERR_ARG, "nel must be in [2, 1024]");
  if (coarsest_nel < 2 || level < 0) return fail(IGM_ERR_ARG, "coarsest_nel >= 2, level >= 0");
  Geometry g;
  const std::string ge = make_geometry(desc, g);
  if (!ge.empty()) return fail(IGM_ERR_ARG, ge);
  Discretisation lo;
  const int nq = desc->nquad > 0 ? desc->nquad : desc->p + 1;
  const std::string e = assemble(g, 1, desc->nel, nq, lo);
  if (!e.empty()) return fail(IGM_ERR_ARG, e);
  const std::vector<Stencil> H = hmg_hierarchy(lo, kappa_dt, coarsest_nel);
  if (nlevels) *nlevels = (int)H.size();
  if (level >= (int)H.size()) return fail(IGM_ERR_ARG, "level beyond the coarsest h-level");
  if (n) *n = H[level].n;
  if (out) std::memcpy(out, H[level].val.data(), H[level].val.size() * sizeof(double));
  return IGM_OK;
}

extern "C" igm_status iga_assemble(const iga_desc* desc, iga_ops** out) {
  if (!desc || !out) return fail(IGM_ERR_ARG, "null argument");
  if (desc->p < 2 || desc->p > 8) return fail(IGM_ERR_ARG, "p must be in [2, 8]");
  if (desc->nel < 4 || desc->nel > 1024) return fail(IGM_ERR_ARG, "nel must be in [4, 1024]");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
    return fail(IGM_ERR_CUDA, "no CUDA device");
  auto ops = std::make_unique<iga_ops>();
  ops->kappa = desc->kappa;
  Geometry& g = ops->geom;
  const std::string ge = make_geometry(desc, g);
  if (!ge.empty()) return fail(IGM_ERR_ARG, ge);
  const int nq = desc->nquad > 0 ? desc->nquad : desc->p + 1;
  std::string e = assemble(g, desc->p, desc->nel, nq, ops->hi);
  if (!e.empty()) return fail(IGM_ERR_ARG, e);
  e = assemble(g, 1, desc->nel, nq, ops->lo);
  if (!e.empty()) return fail(IGM_ERR_ARG, e);
  ops->P = transfer(g, ops->hi, ops->lo);
  ops->PT = transpose(ops->P);
  quadrature_points(g, ops->hi, ops->qpts, ops->qwdet);
  Uploader& up = ops->up;
  if (g.affine) {
    ops->bM64 = up.put(ops->hi.M1);
    ops->bK64 = up.put(ops->hi.K1);
    ops->bM32 = up.put32(ops->hi.M1);
    ops->bK32 = up.put32(ops->hi.K1);
  }
  ops->sM64 = up.put(ops->hi.M.val);
  ops->sK64 = up.put(ops->hi.K.val);
  if (!g.affine) {
    // the batched FP32 apply reads coefficient q of all points contiguously
    const int N = ops->hi.N, Q = ops->hi.M.width() * ops->hi.M.width();
    std::vector<float> tm((size_t)Q * N), tk((size_t)Q * N);
    for (int i = 0; i < N; ++i)
      for (int q = 0; q < Q; ++q) {
        tm[(size_t)q * N + i] = (float)ops->hi.M.val[(size_t)i * Q + q];
        tk[(size_t)q * N + i] = (float)ops->hi.K.val[(size_t)i * Q + q];
      }
    ops->sMq32 = up.put(tm);
    ops->sKq32 = up.put(tk);
  }
  if (up.err != cudaSuccess) return fail(IGM_ERR_CUDA, cudaGetErrorString(up.err));
  *out = ops.release();
  return IGM_OK;
}

extern "C" void iga_destroy(iga_ops* ops) { delete ops; }

extern "C" igm_status iga_sizes(const iga_ops* ops, int* n, int* N, int* nqp) {
  if (!ops) return fail(IGM_ERR_ARG, "null handle");
  if (n) *n = ops->hi.n;
  if (N) *N = ops->hi.N;
  if (nqp) *nqp = (int)ops->qwdet.size();
  return IGM_OK;
}

extern "C" igm_status iga_quadrature_points(const iga_ops* ops, double* pts) {
  if (!ops || !pts) return fail(IGM_ERR_ARG, "null argument");
  std::memcpy(pts, ops->qpts.data(), ops->qpts.size() * sizeof(double));
  return IGM_OK;
}

extern "C" igm_status iga_load_vector(const iga_ops* ops, const double* fq, double* out,
                                      igm_stream s) {
  if (!ops || !fq || !out) return fail(IGM_ERR_ARG, "null argument");
  std::vector<double> b;
  load_vector(ops->geom, ops->hi, fq, b);
  CU(cudaMemcpyAsync(out, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice,
                     (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  return IGM_OK;
}

// Banded Cholesky solve of the interior mass matrix (host, FP64).
static std::string mass_solve(const Discretisation& d, std::vector<double>& x) {
  const int N = d.N, n = d.n, p = d.p;
  const int bw = p * n + p;  // half bandwidth in the natural ordering
  std::vector<double> B((size_t)N * (bw + 1), 0.0);  // B[i][k] = A(i, i-k)
  Csr A = d.M.to_csr(false);
  for (int i = 0; i < N; ++i)
    for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) {
      int j = A.col[k];
      if (j <= i) B[(size_t)i * (bw + 1) + (i - j)] = A.val[k];
    }
  for (int i = 0; i < N; ++i) {
    for (int k = std::min(i, bw); k >= 1; --k) {
      int j = i - k;
      double s = B[(size_t)i * (bw + 1) + k];
      for (int l = k + 1; l <= std::min(i, bw); ++l) {
        int m = i - l;          // column index
        int kj = j - m;         // offset in row j
        if (kj > bw || kj < 0) continue;
        s -= B[(size_t)i * (bw + 1) + l] * B[(size_t)j * (bw + 1) + kj];
      }
      B[(size_t)i * (bw + 1) + k] = s / B[(size_t)j * (bw + 1)];
    }
    double s = B[(size_t)i * (bw + 1)];
    for (int l = 1; l <= std::min(i, bw); ++l) s -= B[(size_t)i * (bw + 1) + l] * B[(size_t)i * (bw + 1) + l];
    if (s <= 0.0) return "mass matrix not positive definite";
    B[(size_t)i * (bw + 1)] = std::sqrt(s);
  }
  for (int i = 0; i < N; ++i) {
    double s = x[i];
    for (int l = 1; l <= std::min(i, bw); ++l) s -= B[(size_t)i * (bw + 1) + l] * x[i - l];
    x[i] = s / B[(size_t)i * (bw + 1)];
  }
  for (int i = N - 1; i >= 0; --i) {
    double s = x[i];
    for (int l = 1; l <= std::min(N - 1 - i, bw); ++l) s -= B[(size_t)(i + l) * (bw + 1) + l] * x[i + l];
    x[i] = s / B[(size_t)i * (bw + 1)];
  }
  return "";
}

extern "C" igm_status iga_project(const iga_ops* ops, const double* fq, double* out, igm_stream s) {
  if (!ops || !fq || !out) return fail(IGM_ERR_ARG, "null argument");
  std::vector<double> b;
  load_vector(ops->geom, ops->hi, fq, b);
  std::string e = mass_solve(ops->hi, b);
  if (!e.empty()) return fail(IGM_ERR_NUMERIC, e);
  CU(cudaMemcpyAsync(out, b.data(), b.size() * sizeof(double), cudaMemcpyHostToDevice,
                     (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  return IGM_OK;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
namespace igm {
cudaError_t launch_pmg_solve(int prec, const PmgD& P, int grid, long smem, cudaStream_t st,
                             const double* b, double* x, long ld, int ncycles, int* cycles_out,
                             int* status, char* garena) {
  return prec ? launch_pmg_solve_f32(P, grid, smem, st, b, x, ld, ncycles, cycles_out, status, garena)
              : launch_pmg_solve_f64(P, grid, smem, st, b, x, ld, ncycles, cycles_out, status, garena);
}
cudaError_t launch_ilut_apply(int prec, const PmgD& P, int grid, long smem, cudaStream_t st,
                              const double* r, double* z, long ld, char* garena, int* status) {
  return prec ? launch_ilut_apply_f32(P, grid, smem, st, r, z, ld, garena, status)
              : launch_ilut_apply_f64(P, grid, smem, st, r, z, ld, garena, status);
}
cudaError_t launch_mgrit_sweep(int prec, const SweepArgs& a, int grid, long smem, cudaStream_t st) {
  return prec ? launch_mgrit_sweep_f32(a, grid, smem, st) : launch_mgrit_sweep_f64(a, grid, smem, st);
}
cudaError_t launch_mgrit_level(int prec, const SweepArgs& a, int grid, long smem, cudaStream_t st) {
  return prec ? launch_mgrit_level_f32(a, grid, smem, st) : launch_mgrit_level_f64(a, grid, smem, st);
}
cudaError_t launch_mgrit_batch(int prec, const BatchMember* mem, BatchState* st, int nmem,
                               unsigned long long* ctl, int grid, long smem, cudaStream_t s) {
  return prec ? launch_mgrit_batch_f32(mem, st, nmem, ctl, grid, smem, s)
              : launch_mgrit_batch_f64(mem, st, nmem, ctl, grid, smem, s);
}
int mgrit_sweep_max_resident(int prec, long smem) {
  return prec ? mgrit_sweep_max_resident_f32(smem) : mgrit_sweep_max_resident_f64(smem);
}
cudaError_t set_solver_smem(long bytes) {
  cudaError_t e = set_smem_f32(bytes);
  return e == cudaSuccess ? set_smem_f64(bytes) : e;
}
}  // namespace igm

// ---------------------------------------------------------------------------
// pmg_setup
// ---------------------------------------------------------------------------
extern "C" void pmg_default_opts(pmg_opts* o) {
  if (!o) return;
  o->nu1 = 1;
  o->nu2 = 1;
  o->ilut_droptol = 1e-12;
  o->ilut_fill = 1.0;
  o->hmg_coarsest_nel = 8;
  o->precision = 1;
  o->inner_cycles = 1;
  o->tol = 1e-10;
  o->max_cycles = 50;
  o->trace = 0;
  o->solver = 0;
  o->autotune = 0;
  o->layout = 0;
  o->hmg_fp64 = 0;
}

static void gen_wcycle(int k, int last, std::vector<int>& ops) {
  if (k == last) {
    ops.push_back(W_COARSE | (k << 8));
    return;
  }
  ops.push_back(W_GS | (k << 8));
  ops.push_back(W_RESTRICT | (k << 8));
  gen_wcycle(k + 1, last, ops);
  // the second visit of an exact coarsest solve reproduces the first: skip it
  if (k + 1 != last) gen_wcycle(k + 1, last, ops);
  ops.push_back(W_PROLONG | (k << 8));
  ops.push_back(W_GS | (k << 8));
}

static int align4(int x) { return (x + 3) & ~3; }

// Pack the block-row records of one triangular factor for the wavefront
// sweep (layout: RecLayout in device.cuh).  Record k covers grid row k (lower) or
// n-1-k (upper); every record is padded to the same size (a multiple of 128
// bytes) so that record k starts at k * rec_bytes.
template <typename T>
static std::string pack_records(const BlockTri& B, bool upper, int team, std::vector<char>& out,
                                int& rec_bytes) {
  const int n = B.n;
  const int N = n * n;
  const size_t blk = (size_t)n * (n + 1) / 2;
  std::vector<std::vector<char>> recs;
  int max_bytes = 0;
  for (int k = 0; k < n; ++k) {
    const int by = upper ? n - 1 - k : k;
    const int nb = upper ? by + 1 : by - 1;  // grid row one step back in the sweep
    const int* rp = &B.off.ptr[(size_t)by * n];
    int KF = 0, KN = 0;
    for (int r = 0; r < n; ++r) {
      int f = 0, m = 0;
      for (int e = rp[r]; e < rp[r + 1]; ++e) {
        const int col = B.off.col[e];
        if (col < 0 || col >= N) return "factor column out of range";
        const int g = col / n;
        if (upper ? g <= by : g >= by) return "factor entry not behind its grid row in the sweep";
        (g == nb ? m : f) += 1;
      }
      KF = std::max(KF, f);
      KN = std::max(KN, m);
    }
    const RecLayout<T> lay(n, KF, KN, upper, team);
    if (lay.o_inv % 16 || lay.o_desc % 16) return "factor record parts not 16-byte aligned";
    std::vector<char> rec(lay.bytes, 0);
    int* hdr = (int*)rec.data();
    hdr[0] = KF; hdr[1] = KN; hdr[2] = by; hdr[3] = 0;
    T* fv = (T*)(rec.data() + lay.o_fv);
    uint16_t* fi = (uint16_t*)(rec.data() + lay.o_fi);
    T* nv = (T*)(rec.data() + lay.o_nv);
    uint16_t* ni = (uint16_t*)(rec.data() + lay.o_ni);
    for (int r = 0; r < n; ++r) {
      int f = 0, m = 0;
      for (int e = rp[r]; e < rp[r + 1]; ++e) {
        const int col = B.off.col[e];
        if (col > 0xffff) return "factor column beyond 16-bit indices";
        const size_t pos = (size_t)((col / n == nb) ? m++ : f++) * n + r;
        (col / n == nb ? nv : fv)[pos] = (T)B.off.val[e];
        (col / n == nb ? ni : fi)[pos] = (uint16_t)col;
      }
    }
    // dense inverse in 16-byte chunks (zero outside the triangle): the flat
    // row-major chunk list, then stored lane-step-major with descriptors
    constexpr int V = 16 / (int)sizeof(T);
    const double* src = &B.inv[(size_t)by * blk];
    const int total = RecLayout<T>::rec_inv_row(n, n, upper);
    const int S = RecLayout<T>::wave_steps(n, upper, team);
    std::vector<T> flat((size_t)total * V, (T)0);
    std::vector<int> crow(total), cq(total);
    for (int r = 0; r < n; ++r) {
      const int c0 = RecLayout<T>::rec_inv_row(r, n, upper);
      const int c1 = RecLayout<T>::rec_inv_row(r + 1, n, upper);
      const int j0 = upper ? r - r % V : 0;
      for (int c = c0; c < c1; ++c) {
        crow[c] = r;
        cq[c] = c - c0;
        for (int u = 0; u < V; ++u) {
          const int j = j0 + (c - c0) * V + u;
          double vv = 0.0;
          if (!upper && j <= r) vv = src[(size_t)r * (r + 1) / 2 + j];
          if (upper && j >= r && j < n) vv = src[(size_t)r * n - (size_t)r * (r - 1) / 2 + (j - r)];
          flat[(size_t)c * V + u] = (T)vv;
        }
      }
    }
    T* inv = (T*)(rec.data() + lay.o_inv);
    int* desc = (int*)(rec.data() + lay.o_desc);
    for (int l = 0; l < team; ++l)
      for (int st = 0; st < S; ++st) {
        const int c = l * S + st;
        if (c >= total) continue;
        const int r = crow[c];
        const int tq = (upper ? r / V : 0) + cq[c];
        const int end = std::min((l + 1) * S, total);
        const bool flush = c + 1 == end || c + 1 == RecLayout<T>::rec_inv_row(r + 1, n, upper);
        if (tq > 0xff || r + l > 0x3ff) return "diagonal block too large for the sweep schedule";
        const size_t pos = (size_t)st * team + l;
        std::copy(&flat[(size_t)c * V], &flat[(size_t)c * V] + V, inv + pos * V);
        desc[pos] = tq | ((r + l) << 8) | (flush ? (int)0x80000000u : 0);
      }
    max_bytes = std::max(max_bytes, lay.bytes);
    recs.push_back(std::move(rec));
  }
  rec_bytes = (max_bytes + 127) & ~127;
  out.assign((size_t)rec_bytes * n, 0);
  for (int k = 0; k < n; ++k) std::copy(recs[k].begin(), recs[k].end(), out.begin() + (size_t)k * rec_bytes);
  return "";
}

// 1D transfer factor between the interior order-p functions (rows) and the
// interior order-1 functions (columns) on the same knots with the same rule,
// stored as bands of width w with per-row starts (Sec. 4, Eq. (PM) on the
// affine map: P = P1 (x) P1).  Returns false if a row does not fit the band.
static bool transfer_bands(const Discretisation& hi, const Discretisation& lo, int w,
                           std::vector<int>& js, std::vector<double>& band,
                           std::vector<int>& is, std::vector<double>& tband) {
  const int n = hi.n, n1 = lo.n, p = hi.p, nq = hi.nq;
  std::vector<double> P1((size_t)n * n1, 0.0), gx, gw;
  gauss_legendre(nq, gx, gw);
  std::vector<double> Nh(p + 1), Nl(2);
  for (int e = 0; e < hi.nel; ++e) {
    const double x0 = hi.knots[e + p], x1 = hi.knots[e + p + 1];
    for (int a = 0; a < nq; ++a) {
      const double x = 0.5 * (x1 - x0) * gx[a] + 0.5 * (x0 + x1);
      const double wq = 0.5 * (x1 - x0) * gw[a];
      basis_on_span(hi.knots, p, e + p, x, Nh.data(), nullptr);
      basis_on_span(lo.knots, 1, e + 1, x, Nl.data(), nullptr);
      for (int la = 0; la <= p; ++la)
        for (int lb = 0; lb <= 1; ++lb) {
          const int i = e + la - 1, j = e + lb - 1;
          if (i < 0 || j < 0 || i >= n || j >= n1) continue;
          P1[(size_t)i * n1 + j] += wq * Nh[la] * Nl[lb];
        }
    }
  }
  if (n1 < w || n < w) return false;
  auto fill = [&](int rows, int cols, bool trans, std::vector<int>& st, std::vector<double>& bd) {
    st.assign(rows, 0);
    bd.assign((size_t)rows * w, 0.0);
    for (int r = 0; r < rows; ++r) {
      int lo_c = -1, hi_c = -1;
      for (int c2 = 0; c2 < cols; ++c2) {
        const double v = trans ? P1[(size_t)c2 * n1 + r] : P1[(size_t)r * n1 + c2];
        if (v != 0.0) { if (lo_c < 0) lo_c = c2; hi_c = c2; }
      }
      if (lo_c < 0) lo_c = hi_c = 0;
      if (hi_c - lo_c + 1 > w) return false;
      const int s0 = std::min(lo_c, cols - w);
      st[r] = s0;
      for (int k = 0; k < w; ++k) {
        const int c2 = s0 + k;
        bd[(size_t)r * w + k] = trans ? P1[(size_t)c2 * n1 + r] : P1[(size_t)r * n1 + c2];
      }
    }
    return true;
  };
  return fill(n, n1, false, js, band) && fill(n1, n, true, is, tband);
}

// Set-up of one p-multigrid hierarchy for A = M + kappa_dt K; expl_dt != 0
// also uploads R = M - expl_dt K, the explicit part of a theta-scheme step
// (Sec. 2, Eq. (los)), for the step right-hand side.
static igm_status pmg_setup_ex(const iga_ops* ops, double kappa_dt, double expl_dt,
                               const pmg_opts* opts, pmg_handle** out);

extern "C" igm_status pmg_setup(const iga_ops* ops, double kappa_dt, const pmg_opts* opts,
                                pmg_handle** out) {
  return pmg_setup_ex(ops, kappa_dt, 0.0, opts, out);
}

static igm_status pmg_setup_ex(const iga_ops* ops, double kappa_dt, double expl_dt,
                               const pmg_opts* opts, pmg_handle** out) {
  if (!ops || !out) return fail(IGM_ERR_ARG, "null argument");
  auto h = std::make_unique<pmg_handle>();
  h->ops = ops;
  if (opts) h->opts = *opts; else pmg_default_opts(&h->opts);
  const pmg_opts& o = h->opts;
  if (o.nu1 < 0 || o.nu2 < 0 || o.nu1 + o.nu2 < 1) return fail(IGM_ERR_ARG, "need nu1 + nu2 >= 1");
  if (o.precision != 0 && o.precision != 1) return fail(IGM_ERR_ARG, "precision must be 0 or 1");
  if (o.inner_cycles < 1) return fail(IGM_ERR_ARG, "inner_cycles must be >= 1");
  if (o.max_cycles < 1) return fail(IGM_ERR_ARG, "max_cycles must be >= 1");
  if (!(o.tol >= 0.0)) return fail(IGM_ERR_ARG, "tol must be >= 0");
  if (o.solver != 0 && o.solver != 1) return fail(IGM_ERR_ARG, "solver must be 0 or 1");
  if (o.layout < 0 || o.layout > 6) return fail(IGM_ERR_ARG, "layout must be in [0, 6]");
  if (o.hmg_fp64 != 0 && o.hmg_fp64 != 1) return fail(IGM_ERR_ARG, "hmg_fp64 must be 0 or 1");
  if (o.solver == 1) h->opts.precision = 0;  // CG runs in FP64
  h->c = kappa_dt;
  const Discretisation& hi = ops->hi;
  const Discretisation& lo = ops->lo;
  const int n = hi.n, N = hi.N, p = hi.p, W = 2 * p + 1;
  if (lo.n > 128) return fail(IGM_ERR_ARG, "nel > 129 is not supported by the p=1 sweeps");
  // A = M + c K (Sec. 4: the backward-Euler step matrix)
  Stencil A = hi.M;
  for (size_t i = 0; i < A.val.size(); ++i) A.val[i] = hi.M.val[i] + kappa_dt * hi.K.val[i];
  Csr Acsr = A.to_csr(true);
  std::string e = ilut(Acsr, o.ilut_droptol, o.ilut_fill, h->L, h->U);
  if (!e.empty()) return fail(IGM_ERR_NUMERIC, e);
  BlockTri BL, BU;
  e = block_lower(h->L, n, BL);
  if (e.empty()) e = block_upper(h->U, n, BU);
  if (!e.empty()) return fail(IGM_ERR_NUMERIC, e);
  // p = 1 operator and its h-hierarchy (Sec. 4, Fig. 5)
  std::vector<Stencil> H = hmg_hierarchy(lo, kappa_dt, o.hmg_coarsest_nel);
  std::vector<double> Cinv;
  e = spd_inverse(H.back(), Cinv);
  if (!e.empty()) return fail(IGM_ERR_NUMERIC, e);

  PmgD& d = h->d;
  std::memset(&d, 0, sizeof(d));
  Uploader& up = h->up;
  d.p = p; d.n = n; d.N = N; d.w = p; d.affine = ops->geom.affine ? 1 : 0;
  d.c = kappa_dt;
  if (d.affine) {
    std::vector<double> bA((size_t)n * W), bcM((size_t)n * W);
    for (size_t i = 0; i < bA.size(); ++i) {
      bA[i] = hi.M1[i] + kappa_dt * hi.K1[i];
      bcM[i] = kappa_dt * hi.M1[i];
    }
    d.bM64 = ops->bM64; d.bK64 = ops->bK64; d.bM32 = ops->bM32; d.bK32 = ops->bK32;
    d.bA64 = up.put(bA); d.bcM64 = up.put(bcM);
    d.bA32 = up.put32(bA); d.bcM32 = up.put32(bcM);
  }
  d.sA64 = up.put(A.val);
  d.sA32 = up.put32(A.val);
  d.sM64 = ops->sM64;
  d.solver = o.solver;
  if (o.solver == 1) {
    const int S = (2 * p + 1) * (2 * p + 1);
    std::vector<double> dinv(N);
    for (int i = 0; i < N; ++i) {
      const double a = A.val[(size_t)i * S + S / 2];
      if (!(a > 0.0)) return fail(IGM_ERR_NUMERIC, "non-positive diagonal for CG");
      dinv[i] = 1.0 / a;
    }
    d.dinv64 = up.put(dinv);
  }
  d.expl = expl_dt;
  if (expl_dt != 0.0) {
    Stencil R = hi.M;
    for (size_t i = 0; i < R.val.size(); ++i) R.val[i] = hi.M.val[i] - expl_dt * hi.K.val[i];
    d.sR64 = up.put(R.val);
    if (d.affine) {
      std::vector<double> bR((size_t)n * W), bcR((size_t)n * W);
      for (size_t i = 0; i < bR.size(); ++i) {
        bR[i] = hi.M1[i] - expl_dt * hi.K1[i];
        bcR[i] = -expl_dt * hi.M1[i];
      }
      d.bR64 = up.put(bR);
      d.bcR64 = up.put(bcR);
    }
  }
  // ILUT records in the smoothing precision, packed for the sweep teams
  // (uploaded once the shared-memory layout is chosen below)
  if (n > 256) return fail(IGM_ERR_ARG, "grid rows longer than 256 unknowns are not supported");
  struct Packed {
    std::vector<char> L, U;
    int maxL = 0, maxU = 0;
  };
  auto pack = [&](int team, Packed& pk) {
    std::string err = o.precision == 0 ? pack_records<double>(BL, false, team, pk.L, pk.maxL)
                                       : pack_records<float>(BL, false, team, pk.L, pk.maxL);
    if (err.empty())
      err = o.precision == 0 ? pack_records<double>(BU, true, team, pk.U, pk.maxU)
                             : pack_records<float>(BU, true, team, pk.U, pk.maxU);
    return err;
  };
  Packed pk128;
  e = pack(kSweepTeam, pk128);
  if (!e.empty()) return fail(IGM_ERR_ARG, e);
  // transfers: CSR always (curved), tensor-product bands on the affine map
  d.N1 = lo.N;
  d.n1 = lo.n;
  d.Pptr = up.put(ops->P.ptr); d.Pcol = up.put(ops->P.col);
  d.Pval64 = up.put(ops->P.val); d.Pval32 = up.put32(ops->P.val);
  d.PTptr = up.put(ops->PT.ptr); d.PTcol = up.put(ops->PT.col);
  d.PTval64 = up.put(ops->PT.val); d.PTval32 = up.put32(ops->PT.val);
  d.MpL64 = up.put(hi.lumped); d.MpL32 = up.put32(hi.lumped);
  d.M1L64 = up.put(lo.lumped); d.M1L32 = up.put32(lo.lumped);
  d.wP = p + 2;
  if (d.affine) {
    std::vector<int> js, is;
    std::vector<double> pb, ptb;
    if (transfer_bands(hi, lo, d.wP, js, pb, is, ptb)) {
      d.tp = 1;
      d.Pjs = up.put(js); d.PTis = up.put(is);
      d.Pb64 = up.put(pb); d.PTb64 = up.put(ptb);
      d.Pb32 = up.put32(pb); d.PTb32 = up.put32(ptb);
    }
  }
  // h-levels: 9-point stencils and Gauss--Seidel row records (lane-interleaved)
  d.nh = (int)H.size();
  for (int k = 0; k < d.nh; ++k) {
    const int nk = H[k].n;
    const int E = nk <= 32 ? 1 : (nk <= 64 ? 2 : (nk <= 128 ? 4 : 8));  // lanes' width in gs_sweep
    const bool g64 = o.precision == 0 || o.hmg_fp64;   // GS coefficients in FP64
    const int es_g = g64 ? 8 : 4;
    const int rec_bytes = G_NCOEF * E * 32 * es_g;  // multiple of 128
    std::vector<char> recs((size_t)rec_bytes * nk, 0);
    for (int by = 0; by < nk; ++by) {
      char* rec = recs.data() + (size_t)by * rec_bytes;
      for (int r = 0; r < nk; ++r) {
        const double* a = &H[k].val[(size_t)(by * nk + r) * 9];
        if (a[4] == 0.0) return fail(IGM_ERR_NUMERIC, "zero diagonal at p = 1");
        double g[G_NCOEF];
        g[G_SW] = a[0]; g[G_S] = a[1]; g[G_SE] = a[2]; g[G_E] = a[5];
        g[G_NW] = a[6]; g[G_N] = a[7]; g[G_NE] = a[8];
        g[G_ALPHA] = r > 0 ? -a[3] / a[4] : 0.0;
        g[G_INVC] = 1.0 / a[4];
        const int lane = r / E, e = r % E;
        for (int q = 0; q < G_NCOEF; ++q) {
          const size_t idx = (size_t)(q * E + e) * 32 + lane;
          if (g64) ((double*)rec)[idx] = g[q];
          else ((float*)rec)[idx] = (float)g[q];
        }
      }
    }
    d.h[k].n = nk;
    d.h[k].A64 = up.put(H[k].val);
    d.h[k].A32 = up.put32(H[k].val);
    d.h[k].G.recs = up.put(recs);
    d.h[k].G.bytes = rec_bytes;
  }
  d.Cinv = up.put(Cinv);
  std::vector<int> wops;
  gen_wcycle(0, d.nh - 1, wops);
  if ((int)wops.size() > (int)(sizeof(d.ops) / sizeof(int)))
    return fail(IGM_ERR_ARG, "h-multigrid hierarchy too deep for the W-cycle program");
  d.nops = (int)wops.size();
  for (int i = 0; i < d.nops; ++i) d.ops[i] = wops[i];
  if (o.trace) d.trace = (unsigned long long*)up.raw(sizeof(unsigned long long) * IGM_PH_COUNT);
  d.precision = o.precision;
  d.inner = o.inner_cycles;
  d.nu1 = o.nu1;
  d.nu2 = o.nu2;
  d.max_cycles = o.max_cycles;
  d.tol = o.tol;
  // arena layout, in elements of the smoothing precision:
  // [r][d] (mixed only) [t] [U: FP32/64 SpMM temporaries | h-level vectors + transfer temp]
  // The mixed form's FP64 residual temporaries (2N doubles) alias d, t and U.
  const int es = o.precision == 0 ? 8 : 4;
  int off = 0;
  if (o.precision == 1) {
    d.o_r = off; off = align4(off + N);
    d.o_d = off; off = align4(off + N);
  }
  d.o_t = off; off = align4(off + N);
  d.o_u = off;
  int hsum = 0;
  for (int k = 0; k < d.nh; ++k) {
    d.h[k].ox = d.o_u + hsum; hsum = align4(hsum + H[k].n * H[k].n);
    d.h[k].ob = d.o_u + hsum; hsum = align4(hsum + H[k].n * H[k].n);
    d.h[k].ot = d.o_u + hsum; hsum = align4(hsum + H[k].n * H[k].n);
  }
  d.o_tr = d.o_u + hsum;
  int coarse_part = hsum + align4(n * lo.n);
  d.hmg64 = (o.precision == 1 && o.hmg_fp64) ? 1 : 0;
  if (d.hmg64) {
    // the h-level vectors in doubles (offsets in doubles from the arena's
    // start; o_u is a multiple of 4 floats), then the FP32 transfer
    // temporary and the order-1 vector between transfers and W-cycle
    int hd = 0;
    for (int k = 0; k < d.nh; ++k) {
      const int nk2 = H[k].n * H[k].n;
      d.h[k].ox = d.o_u / 2 + hd; hd = align4(hd + nk2);
      d.h[k].ob = d.o_u / 2 + hd; hd = align4(hd + nk2);
      d.h[k].ot = d.o_u / 2 + hd; hd = align4(hd + nk2);
    }
    d.o_tr = d.o_u + 2 * hd;
    d.o_c1 = d.o_tr + align4(n * lo.n);
    coarse_part = 2 * hd + align4(n * lo.n) + align4(lo.N);
  }
  off += std::max(std::max(align4(2 * N) + align4(N), coarse_part),
                  o.solver == 1 ? 4 * align4(N) : 0);  // CG: p, q and two operator temporaries
  h->arena_bytes = (long)off * es;
  d.arena_bytes = h->arena_bytes;
  if (up.err != cudaSuccess) return fail(IGM_ERR_CUDA, cudaGetErrorString(up.err));
  // shared memory: record ring (as many stages as fit, 4 at most; one sweep
  // team per stage) + mbarriers + the sweep teams' scratch, then the arena if
  // it fits, else a staged copy of the swept vector if that fits
  const long optin = dev_smem_optin() - 1024;
  const long bars = 8 * (kMaxStage + kRowBars);
  const long vst = ((long)N * es + 15) & ~15L;
  // preference (measured on the unit square, nel = 64, p = 2..5): the arena
  // in shared memory with at least 3 stages, else with 2; else the most
  // stages with a staged copy of the swept vector; else the arena in shared
  // memory with one stage; else the most stages with everything in global
  // memory.  Returns the byte offset of the arena (0: nothing fits).
  auto place = [&](int slot, int team, int only) -> long {
    const long sweep = ((long)wave_scratch_bytes(n, es, team) + 15) & ~15L;
    d.arena_smem = 0;
    d.nstage = 0;
    d.o_vstage = -1;
    d.sweep_team = team;
    for (int pass = 0; pass < 5; ++pass) {
      // only = 0: arena in shared memory; 1: staged vector; 2: all global
      if (only == 0 && pass != 0 && pass != 1 && pass != 3) continue;
      if (only == 1 && pass != 2) continue;
      if (only == 2 && pass != 4) continue;
      for (int st = kMaxStage; st >= 1; --st) {
        const long base = (long)st * slot + bars + sweep;
        const bool arena = base + h->arena_bytes <= optin;
        if (pass == 0 && st >= 3 && arena) d.arena_smem = 1;
        else if (pass == 1 && st == 2 && arena) d.arena_smem = 1;
        else if (pass == 2 && base + vst <= optin) d.o_vstage = (int)base;
        else if (pass == 3 && arena) d.arena_smem = 1;
        else if (pass == 4 && base <= optin) {}
        else continue;
        d.nstage = st;
        d.slot_bytes = slot;
        d.o_sweep = (int)((long)st * slot + bars);
        return base + (d.o_vstage >= 0 ? vst : 0);
      }
    }
    return 0;
  };
  auto slot_of = [&](const Packed& pk) { return (std::max(pk.maxL, pk.maxU) + 127) & ~127; };
  // kernel attributes once per process (handles may be set up from several threads)
  static std::once_flag attr_once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(attr_once, [&] { attr_err = set_solver_smem(optin); });
  if (attr_err != cudaSuccess) return fail(IGM_ERR_CUDA, cudaGetErrorString(attr_err));
  long arena_off = place(slot_of(pk128), kSweepTeam, -1);
  if (!arena_off) return fail(IGM_ERR_ARG, "a factor record does not fit in shared memory");
  Packed pk256;
  const Packed* chosen = &pk128;
  if (o.layout > 0) {
    // a forced layout: team of 128 (1..3) or 256 (4..6) threads, placement
    // 0 arena in shared memory, 1 staged vector, 2 all global
    const int team = o.layout <= 3 ? 128 : 256, only = (o.layout - 1) % 3;
    if (team == 256) {
      e = pack(256, pk256);
      if (!e.empty()) return fail(IGM_ERR_ARG, e);
      chosen = &pk256;
    }
    arena_off = place(slot_of(*chosen), team, only);
    if (!arena_off)
      return fail(IGM_ERR_ARG, "layout " + std::to_string(o.layout) +
                                   " does not fit in shared memory for this problem");
  } else if (o.autotune) {
    // time every distinct candidate layout on a probe solve (3 cycles, one
    // right-hand side) and keep the fastest
    e = pack(256, pk256);
    if (!e.empty()) return fail(IGM_ERR_ARG, e);
    std::vector<double> hb(N);
    std::mt19937_64 rng(12345);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (auto& v : hb) v = nd(rng);
    double *db = nullptr, *dx = nullptr;
    int *dst = nullptr, *dcy = nullptr;
    char* garena = nullptr;
    CU(cudaMalloc(&db, sizeof(double) * N));
    CU(cudaMalloc(&dx, sizeof(double) * N));
    CU(cudaMalloc(&dst, sizeof(int)));
    CU(cudaMalloc(&dcy, sizeof(int)));
    CU(cudaMalloc(&garena, h->arena_bytes));
    CU(cudaMemcpy(db, hb.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 0.0f;
    int best_team = kSweepTeam, best_only = -1;
    for (int team : {128, 256})
      for (int only : {0, 1, 2}) {
        const Packed& pk = team == 128 ? pk128 : pk256;
        const long off = place(slot_of(pk), team, only);
        if (!off) continue;
        char *rl = nullptr, *ru = nullptr;
        CU(cudaMalloc(&rl, pk.L.size()));
        CU(cudaMalloc(&ru, pk.U.size()));
        CU(cudaMemcpy(rl, pk.L.data(), pk.L.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(ru, pk.U.data(), pk.U.size(), cudaMemcpyHostToDevice));
        PmgD t = d;
        t.Lrec.recs = rl; t.Lrec.bytes = pk.maxL;
        t.Urec.recs = ru; t.Urec.bytes = pk.maxU;
        t.ring_bytes = off;
        const long smem = off + (t.arena_smem ? h->arena_bytes : 0);
        float ms = 0.0f;
        for (int rep = 0; rep < 2; ++rep) {
          CU(cudaMemset(dx, 0, sizeof(double) * N));
          CU(cudaMemset(dst, 0, sizeof(int)));
          CU(cudaEventRecord(e0, 0));
          CU(launch_pmg_solve(t.precision, t, 1, smem, 0, db, dx, N, 3, dcy, dst, garena));
          CU(cudaEventRecord(e1, 0));
          CU(cudaEventSynchronize(e1));
          CU(cudaEventElapsedTime(&ms, e0, e1));
        }
        int hst = 0;
        CU(cudaMemcpy(&hst, dst, sizeof(int), cudaMemcpyDeviceToHost));
        cudaFree(rl);
        cudaFree(ru);
        if (hst != ST_OK) continue;
        if (best_only < 0 || ms < best) {
          best = ms;
          best_team = team;
          best_only = only;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(db); cudaFree(dx); cudaFree(dst); cudaFree(dcy); cudaFree(garena);
    if (best_only >= 0) {
      chosen = best_team == 128 ? &pk128 : &pk256;
      arena_off = place(slot_of(*chosen), best_team, best_only);
    } else {
      arena_off = place(slot_of(pk128), kSweepTeam, -1);
    }
  }
  d.Lrec.recs = up.put(chosen->L); d.Lrec.bytes = chosen->maxL;
  d.Urec.recs = up.put(chosen->U); d.Urec.bytes = chosen->maxU;
  if (up.err != cudaSuccess) return fail(IGM_ERR_CUDA, cudaGetErrorString(up.err));
  d.ring_bytes = arena_off;
  h->arena_smem = d.arena_smem != 0;
  h->smem_bytes = d.ring_bytes + (d.arena_smem ? h->arena_bytes : 0);
  *out = h.release();
  return IGM_OK;
}

extern "C" igm_status pmg_layout(const pmg_handle* h, int* out) {
  if (!h || !out) return fail(IGM_ERR_ARG, "null argument");
  out[0] = h->d.sweep_team;
  out[1] = h->d.nstage;
  out[2] = h->d.arena_smem;
  out[3] = h->d.o_vstage >= 0 ? 1 : 0;
  return IGM_OK;
}

extern "C" void pmg_destroy(pmg_handle* h) {
  if (!h) return;
  if (h->garena) cudaFree(h->garena);
  delete h;
}

static igm_status ensure_arena(pmg_handle* h, int grid) {
  if (h->arena_smem) return IGM_OK;
  if (h->grid_capacity >= grid) return IGM_OK;
  if (h->garena) cudaFree(h->garena);
  h->garena = nullptr;
  h->grid_capacity = 0;
  CU(cudaMalloc(&h->garena, (size_t)h->arena_bytes * grid));
  h->grid_capacity = grid;
  return IGM_OK;
}

static long smem_of(const pmg_handle* h) { return h->smem_bytes; }

extern "C" igm_status pmg_vcycle(pmg_handle* h, int nrhs, const double* b, double* x, long ld,
                                 int ncycles, int* cycles_out, igm_stream s) {
  if (!h || !b || !x) return fail(IGM_ERR_ARG, "null argument");
  if (nrhs < 0 || ncycles < 0 || ld < h->d.N) return fail(IGM_ERR_ARG, "bad nrhs/ld/ncycles");
  if (nrhs == 0) return IGM_OK;
  cudaStream_t st = (cudaStream_t)s;
  igm_status rs = ensure_arena(h, nrhs);
  if (rs != IGM_OK) return rs;
  int* dcyc = nullptr;
  int* dstat = nullptr;
  CU(cudaMallocAsync(&dcyc, sizeof(int) * (nrhs + 1), st));
  dstat = dcyc + nrhs;
  CU(cudaMemsetAsync(dcyc, 0, sizeof(int) * (nrhs + 1), st));
  CU(launch_pmg_solve(h->d.precision, h->d, nrhs, smem_of(h), st, b, x, ld, ncycles, dcyc, dstat,
                      h->garena));
  g_launches++;
  std::vector<int> hc(nrhs + 1);
  CU(cudaMemcpyAsync(hc.data(), dcyc, sizeof(int) * (nrhs + 1), cudaMemcpyDeviceToHost, st));
  CU(cudaFreeAsync(dcyc, st));
  CU(cudaStreamSynchronize(st));
  if (cycles_out) std::memcpy(cycles_out, hc.data(), sizeof(int) * nrhs);
  if (hc[nrhs] == ST_NUMERIC) return fail(IGM_ERR_NUMERIC, "NaN in a spatial residual");
  if (hc[nrhs] == ST_TIMEOUT) return fail(IGM_ERR_TIMEOUT, "a bounded device wait gave up");
  if (hc[nrhs] == ST_NOT_CONVERGED) return fail(IGM_ERR_NOT_CONVERGED, "spatial solve hit max_cycles");
  return IGM_OK;
}

// ---------------------------------------------------------------------------
// pmg_vcycle_static: the same solve with no allocation at all.  Its scratch
// (status word, per-column cycle counts and, when the working vectors do not
// fit in shared memory, the per-CTA arenas) lives in this file-scope device
// array.  Host code must not use the array's name as a device address: the
// address of the current device's copy comes from cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB on every device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch on the current device.  Looked up on
// every call (cudaGetSymbolAddress does not allocate and is cheap), so the
// address stays valid across a cudaDeviceReset or a new primary context.
static igm_status static_scratch(void** out) {
  void* p = nullptr;
  CU(cudaGetSymbolAddress(&p, g_static_scratch));
  *out = p;
  return IGM_OK;
}

extern "C" igm_status pmg_vcycle_static(pmg_handle* h, int nrhs, const double* b, double* x,
                                        long ld, int ncycles, int* cycles_out, igm_stream s) {
  if (!h || !b || !x) return fail(IGM_ERR_ARG, "null argument");
  if (nrhs < 0 || ncycles < 0 || ld < h->d.N) return fail(IGM_ERR_ARG, "bad nrhs/ld/ncycles");
  if (nrhs == 0) return IGM_OK;
  // layout: [status: 256 B][cycle counts: nrhs ints, 256-aligned][arenas]
  const size_t o_cyc = 256;
  const size_t o_arena = o_cyc + (((size_t)nrhs * sizeof(int) + 255) & ~(size_t)255);
  const size_t arena_total = h->arena_smem ? 0 : (size_t)h->arena_bytes * nrhs;
  const size_t need = o_arena + arena_total;
  if (need > kStaticScratchBytes)
    return fail(IGM_ERR_ARG, "pmg_vcycle_static: " + std::to_string(nrhs) + " columns need " +
                                 std::to_string(need) + " bytes of scratch; the static buffer holds " +
                                 std::to_string(kStaticScratchBytes));
  void* base = nullptr;
  igm_status rs = static_scratch(&base);
  if (rs != IGM_OK) return rs;
  char* scratch = (char*)base;
  int* dstat = (int*)scratch;
  int* dcyc = (int*)(scratch + o_cyc);
  char* garena = h->arena_smem ? nullptr : scratch + o_arena;
  cudaStream_t st = (cudaStream_t)s;
  // the buffer keeps the previous call's contents: clear what must start at zero
  CU(cudaMemsetAsync(scratch, 0, o_arena, st));
  CU(launch_pmg_solve(h->d.precision, h->d, nrhs, smem_of(h), st, b, x, ld, ncycles, dcyc, dstat,
                      garena));
  g_launches++;
  int hstat = 0;
  if (cycles_out)
    CU(cudaMemcpyAsync(cycles_out, dcyc, sizeof(int) * nrhs, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(&hstat, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  if (hstat == ST_NUMERIC) return fail(IGM_ERR_NUMERIC, "NaN in a spatial residual");
  if (hstat == ST_TIMEOUT) return fail(IGM_ERR_TIMEOUT, "a bounded device wait gave up");
  if (hstat == ST_NOT_CONVERGED) return fail(IGM_ERR_NOT_CONVERGED, "spatial solve hit max_cycles");
  return IGM_OK;
}

extern "C" igm_status pmg_ilut_apply(pmg_handle* h, int nrhs, const double* r, double* z, long ld,
                                     igm_stream s) {
  if (!h || !r || !z) return fail(IGM_ERR_ARG, "null argument");
  if (nrhs < 0 || ld < h->d.N) return fail(IGM_ERR_ARG, "bad nrhs/ld");
  if (nrhs == 0) return IGM_OK;
  igm_status rs = ensure_arena(h, nrhs);
  if (rs != IGM_OK) return rs;
  CU(launch_ilut_apply(h->d.precision, h->d, nrhs, smem_of(h), (cudaStream_t)s, r, z, ld,
                       h->garena, nullptr));
  g_launches++;
  return IGM_OK;
}

extern "C" igm_status igm_wait_selftest(long spins, igm_stream s) {
  if (spins < 1) return fail(IGM_ERR_ARG, "spins must be >= 1");
  int* dstat = nullptr;
  cudaStream_t st = (cudaStream_t)s;
  CU(cudaMallocAsync(&dstat, sizeof(int), st));
  CU(cudaMemsetAsync(dstat, 0, sizeof(int), st));
  CU(launch_wait_selftest(spins, dstat, st));
  g_launches++;
  int h = 0;
  CU(cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaFreeAsync(dstat, st));
  CU(cudaStreamSynchronize(st));
  if (h == ST_TIMEOUT) return fail(IGM_ERR_TIMEOUT, "bounded mbarrier wait gave up as intended");
  return IGM_OK;
}

extern "C" igm_status igm_grid_barrier_selftest(int nctas, long long wait_cycles, int hold,
                                                igm_stream s) {
  if (nctas < 1 || nctas > 1024 || wait_cycles < 1)
    return fail(IGM_ERR_ARG, "nctas must be in [1, 1024] and wait_cycles >= 1");
  cudaStream_t st = (cudaStream_t)s;
  int* dstat = nullptr;
  CU(cudaMallocAsync(&dstat, 4 * sizeof(unsigned) + sizeof(int), st));
  unsigned* gbar = (unsigned*)(dstat + 1);
  CU(cudaMemsetAsync(dstat, 0, 4 * sizeof(unsigned) + sizeof(int), st));
  CU(launch_barrier_selftest(nctas, wait_cycles, hold ? 1 : 0, gbar, dstat, st));
  g_launches++;
  int h = 0;
  CU(cudaMemcpyAsync(&h, dstat, sizeof(int), cudaMemcpyDeviceToHost, st));
  CU(cudaFreeAsync(dstat, st));
  CU(cudaStreamSynchronize(st));
  if (h == ST_TIMEOUT) return fail(IGM_ERR_TIMEOUT, "bounded grid barrier wait gave up as intended");
  return IGM_OK;
}

extern "C" igm_status pmg_trace(pmg_handle* h, long long* out, int reset) {
  if (!h || !out) return fail(IGM_ERR_ARG, "null argument");
  if (!h->d.trace) return fail(IGM_ERR_ARG, "handle was set up without trace");
  CU(cudaDeviceSynchronize());
  CU(cudaMemcpy(out, h->d.trace, sizeof(long long) * IGM_PH_COUNT, cudaMemcpyDeviceToHost));
  if (reset) CU(cudaMemset(h->d.trace, 0, sizeof(long long) * IGM_PH_COUNT));
  return IGM_OK;
}

extern "C" igm_status pmg_ilut_factors(const pmg_handle* h, int* nnz_l, int* nnz_u, int* l_ptr,
                                       int* l_col, double* l_val, int* u_ptr, int* u_col,
                                       double* u_val) {
  if (!h) return fail(IGM_ERR_ARG, "null handle");
  if (nnz_l) *nnz_l = h->L.nnz();
  if (nnz_u) *nnz_u = h->U.nnz();
  if (l_ptr) std::memcpy(l_ptr, h->L.ptr.data(), h->L.ptr.size() * sizeof(int));
  if (l_col) std::memcpy(l_col, h->L.col.data(), h->L.col.size() * sizeof(int));
  if (l_val) std::memcpy(l_val, h->L.val.data(), h->L.val.size() * sizeof(double));
  if (u_ptr) std::memcpy(u_ptr, h->U.ptr.data(), h->U.ptr.size() * sizeof(int));
  if (u_col) std::memcpy(u_col, h->U.col.data(), h->U.col.size() * sizeof(int));
  if (u_val) std::memcpy(u_val, h->U.val.data(), h->U.val.size() * sizeof(double));
  return IGM_OK;
}

extern "C" igm_status pmg_ilut_host(int n, const int* ptr, const int* col, const double* val,
                                    double droptol, double fill, int* nnz_l, int* nnz_u,
                                    int* l_ptr, int* l_col, double* l_val, int* u_ptr, int* u_col,
                                    double* u_val) {
  if (n < 1 || !ptr || !col || !val || !(droptol >= 0.0) || !(fill > 0.0))
    return fail(IGM_ERR_ARG, "pmg_ilut_host: n >= 1, non-null CSR arrays, droptol >= 0, fill > 0");
  if (ptr[0] != 0) return fail(IGM_ERR_ARG, "pmg_ilut_host: ptr[0] must be 0");
  for (int i = 0; i < n; ++i)
    if (ptr[i + 1] < ptr[i]) return fail(IGM_ERR_ARG, "pmg_ilut_host: ptr must not decrease");
  for (int k = 0; k < ptr[n]; ++k)
    if (col[k] < 0 || col[k] >= n) return fail(IGM_ERR_ARG, "pmg_ilut_host: column out of range");
  Csr A, L, U;
  A.rows = A.cols = n;
  A.ptr.assign(ptr, ptr + n + 1);
  A.col.assign(col, col + ptr[n]);
  A.val.assign(val, val + ptr[n]);
  const std::string e = ilut(A, droptol, fill, L, U);
  if (!e.empty()) return fail(IGM_ERR_NUMERIC, e);
  if (nnz_l) *nnz_l = L.nnz();
  if (nnz_u) *nnz_u = U.nnz();
  if (l_ptr) std::memcpy(l_ptr, L.ptr.data(), L.ptr.size() * sizeof(int));
  if (l_col) std::memcpy(l_col, L.col.data(), L.col.size() * sizeof(int));
  if (l_val) std::memcpy(l_val, L.val.data(), L.val.size() * sizeof(double));
  if (u_ptr) std::memcpy(u_ptr, U.ptr.data(), U.ptr.size() * sizeof(int));
  if (u_col) std::memcpy(u_col, U.col.data(), U.col.size() * sizeof(int));
  if (u_val) std::memcpy(u_val, U.val.data(), U.val.size() * sizeof(double));
  return IGM_OK;
}

extern "C" igm_status pmg_block_tri_host(int n, int upper, const int* ptr, const int* col,
                                         const double* val, int* nnz_off, int* off_ptr,
                                         int* off_col, double* off_val, double* inv) {
  if (n < 1 || n > 4096 || !ptr || !col || !val)
    return fail(IGM_ERR_ARG, "pmg_block_tri_host: n in [1, 4096], non-null CSR arrays");
  const int N = n * n;
  if (ptr[0] != 0) return fail(IGM_ERR_ARG, "pmg_block_tri_host: ptr[0] must be 0");
  for (int i = 0; i < N; ++i)
    if (ptr[i + 1] < ptr[i]) return fail(IGM_ERR_ARG, "pmg_block_tri_host: ptr must not decrease");
  for (int k = 0; k < ptr[N]; ++k) {
    const int i = (int)(std::upper_bound(ptr, ptr + N + 1, k) - ptr) - 1;
    if (col[k] < 0 || col[k] >= N || (upper ? col[k] < i : col[k] >= i))
      return fail(IGM_ERR_ARG, "pmg_block_tri_host: entry outside the factor's triangle");
  }
  Csr F;
  F.rows = F.cols = N;
  F.ptr.assign(ptr, ptr + N + 1);
  F.col.assign(col, col + ptr[N]);
  F.val.assign(val, val + ptr[N]);
  BlockTri B;
  const std::string e = upper ? block_upper(F, n, B) : block_lower(F, n, B);
  if (!e.empty()) return fail(IGM_ERR_NUMERIC, e);
  if (nnz_off) *nnz_off = B.off.nnz();
  if (off_ptr) std::memcpy(off_ptr, B.off.ptr.data(), B.off.ptr.size() * sizeof(int));
  if (off_col) std::memcpy(off_col, B.off.col.data(), B.off.col.size() * sizeof(int));
  if (off_val) std::memcpy(off_val, B.off.val.data(), B.off.val.size() * sizeof(double));
  if (inv) std::memcpy(inv, B.inv.data(), B.inv.size() * sizeof(double));
  return IGM_OK;
}

extern "C" igm_status iga_apply(const iga_ops* ops, int which, int nrhs, const double* x, double* y,
                                long ld, igm_stream s) {
  if (!ops || !x || !y) return fail(IGM_ERR_ARG, "null argument");
  if ((which != 0 && which != 1) || nrhs < 0 || ld < ops->hi.N)
    return fail(IGM_ERR_ARG, "bad which/nrhs/ld");
  if (nrhs == 0) return IGM_OK;
  PmgD d;
  std::memset(&d, 0, sizeof(d));
  d.p = ops->hi.p; d.n = ops->hi.n; d.N = ops->hi.N; d.w = d.p;
  d.affine = ops->geom.affine ? 1 : 0;
  d.bM64 = ops->bM64; d.bK64 = ops->bK64;
  d.sM64 = ops->sM64; d.sA64 = ops->sK64;
  cudaStream_t st = (cudaStream_t)s;
  double* scratch = nullptr;
  CU(cudaMallocAsync(&scratch, sizeof(double) * 2 * (size_t)d.N * nrhs, st));
  CU(launch_apply_op(d, which, nrhs, x, y, ld, scratch, st));
  g_launches++;
  CU(cudaFreeAsync(scratch, st));
  return IGM_OK;
}

extern "C" igm_status iga_apply_f32_layout(int n, int p, long smem_max, int* out) {
  if (!out || n < 1 || p < 2 || p > 8 || smem_max <= 0)
    return fail(IGM_ERR_ARG, "iga_apply_f32_layout: n >= 1, p in [2, 8], smem_max > 0, out");
  spmm32_layout(n, p, (size_t)smem_max, out);
  return IGM_OK;
}

extern "C" igm_status iga_apply_f32_plan(int form, int n, int p, int nrhs, int sms, long smem_max,
                                         int* out) {
  if (!out || (form != 1 && form != 2) || n < 1 || p < 2 || p > 8 || nrhs < 0 || sms < 1 ||
      smem_max <= 0)
    return fail(IGM_ERR_ARG,
                "iga_apply_f32_plan: form 1 or 2, n >= 1, p in [2, 8], nrhs >= 0, sms >= 1, smem_max > 0, out");
  if (form == 1) spmm32_strip_plan(n, p, nrhs, sms, (size_t)smem_max, out);
  else spmm32_curved_plan(n, p, nrhs, sms, out);
  return IGM_OK;
}

extern "C" igm_status iga_apply_f32(iga_ops* ops, int which, double c, int nrhs, const float* x,
                                    float* y, long ld, igm_stream s) {
  if (!ops || (nrhs > 0 && (!x || !y))) return fail(IGM_ERR_ARG, "null argument");
  if (which < 0 || which > 2 || nrhs < 0 || ld < ops->hi.N) return fail(IGM_ERR_ARG, "bad which/nrhs/ld");
  if (nrhs == 0) return IGM_OK;
  const int n = ops->hi.n, p = ops->hi.p;
  cudaStream_t st = (cudaStream_t)s;
  int sms = 0, dev = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (!ops->geom.affine) {
    // curved map: the assembled stencils, y = (cm M + ck K) x
    const float cm = which == 1 ? 0.0f : 1.0f, ck = which == 0 ? 0.0f : which == 1 ? 1.0f : (float)c;
    CU(launch_spmm32_curved(n, p, nrhs, which == 1 ? nullptr : ops->sMq32,
                            which == 0 ? nullptr : ops->sKq32, cm, ck, x, y, ld, sms, st));
    g_launches++;
    return IGM_OK;
  }
  // y = (Y2 (x) X1 + Z2 (x) W1) x with each factor a M1 + b K1:
  //   M = M1 (x) M1;  K = K1 (x) M1 + M1 (x) K1;  M + c K = (M1 + c K1) (x) M1 + c M1 (x) K1
  const float cf32 = (float)c;
  SpmmCoef cf{1, 0, 0, 0, 1, 0, 0, 0};
  if (which == 1) cf = SpmmCoef{1, 0, 0, 1, 0, 1, 1, 0};
  if (which == 2) cf = SpmmCoef{1, 0, 0, 1, 1, cf32, cf32, 0};
  const size_t smem_max = (size_t)dev_smem_optin();
  if (spmm32_slots(n, p, smem_max) < 2) {
    // grids beyond the persistent layouts: the row-strip form
    if (spmm32_strip_rows(n, p, smem_max) < 1) return fail(IGM_ERR_ARG, "grid too large for iga_apply_f32");
    CU(launch_spmm32_strip(n, p, nrhs, ops->bM32, ops->bK32, cf, x, y, ld, sms, smem_max, st));
    g_launches++;
    return IGM_OK;
  }
  const int grid = std::min(nrhs, sms);
  CU(launch_spmm32(n, p, nrhs, ops->bM32, ops->bK32, cf, x, y, ld, grid, smem_max, st));
  g_launches++;
  return IGM_OK;
}

// ---------------------------------------------------------------------------
// MGRIT (Sec. 3)
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// learned coarse propagator
// ---------------------------------------------------------------------------
struct phic_handle {
  PhicNet net;
  PhicWork work;
  PhicTrain train;
  Uploader up;        // weights
  Uploader upw;       // inference work (regrown on demand)
  Uploader upt;       // training state (per phic_train / phic_grad call)
  Uploader uptw;      // training activations (per phic_train / phic_grad call)
};

// Activations for nb images (keep: also the pre-activations, for training).
static igm_status phic_work(phic_handle* h, Uploader& up, PhicWork& w, int nb, bool keep = false) {
  if (w.cap >= nb && (!keep || w.z[0])) return IGM_OK;
  const size_t N = (size_t)h->net.n * h->net.n, C = h->net.C;
  up = Uploader();
  w = PhicWork();
  w.x0 = (__nv_bfloat16*)up.raw(2 * N * nb);
  for (int l = 0; l < 3; ++l) {
    w.h[l] = (__nv_bfloat16*)up.raw(2 * N * C * nb);
    if (keep) w.z[l] = (__nv_bfloat16*)up.raw(2 * N * C * nb);
  }
  w.z4 = (float*)up.raw(4 * N * nb);
  w.s = (double*)up.raw(8 * (size_t)nb);
  if (up.err != cudaSuccess) return fail(IGM_ERR_OOM, cudaGetErrorString(up.err));
  w.cap = nb;
  return IGM_OK;
}

extern "C" igm_status phic_create(int n, int channels, unsigned long long seed, phic_handle** out) {
  if (!out || n < 1 || n > 1024 || (channels != 16 && channels != 32))
    return fail(IGM_ERR_ARG, "phic_create: need n in [1, 1024] and channels 16 or 32");
  auto h = std::make_unique<phic_handle>();
  PhicNet& net = h->net;
  const int C = channels;
  net.n = n;
  net.C = C;
  net.o[0] = 0;
  net.o[1] = C * 9;
  net.o[2] = net.o[1] + C * C * 9;
  net.o[3] = net.o[2] + C * C * 9;
  net.count = net.o[3] + C * 9;
  // initial weights: K1 normal with standard deviation 1/3, K2 and K3 with
  // 1/(3 sqrt C), K4 = 0 (the network starts as the identity)
  std::vector<float> w(net.count, 0.0f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<double> nd(0.0, 1.0);
  for (int i = 0; i < net.o[1]; ++i) w[i] = (float)(nd(rng) / 3.0);
  for (int i = net.o[1]; i < net.o[3]; ++i) w[i] = (float)(nd(rng) / (3.0 * std::sqrt((double)C)));
  net.wall = h->up.put(w);
  net.wf = (__nv_bfloat16*)h->up.raw(2 * (size_t)2 * C * 9 * C);
  net.wb = (__nv_bfloat16*)h->up.raw(2 * (size_t)2 * C * 9 * C);
  net.w1 = (float*)h->up.raw(4 * (size_t)C * 9);
  net.w4 = (float*)h->up.raw(4 * (size_t)C * 9);
  if (h->up.err != cudaSuccess) return fail(IGM_ERR_OOM, cudaGetErrorString(h->up.err));
  CU(phic_refresh(net, 0));
  CU(cudaStreamSynchronize(0));
  *out = h.release();
  return IGM_OK;
}

extern "C" void phic_destroy(phic_handle* h) { delete h; }

extern "C" igm_status phic_set_weights(phic_handle* h, const float* w) {
  if (!h || !w) return fail(IGM_ERR_ARG, "null argument");
  CU(cudaMemcpy(h->net.wall, w, sizeof(float) * h->net.count, cudaMemcpyHostToDevice));
  CU(phic_refresh(h->net, 0));
  CU(cudaStreamSynchronize(0));
  return IGM_OK;
}

extern "C" igm_status phic_get_weights(const phic_handle* h, float* w, int* count) {
  if (!h || !count) return fail(IGM_ERR_ARG, "null argument");
  *count = h->net.count;
  if (w) CU(cudaMemcpy(w, h->net.wall, sizeof(float) * h->net.count, cudaMemcpyDeviceToHost));
  return IGM_OK;
}

extern "C" igm_status phic_apply(phic_handle* h, int nb, const double* u, long ldu, double* out,
                                 long ldo, igm_stream s) {
  if (!h || (nb > 0 && (!u || !out))) return fail(IGM_ERR_ARG, "null argument");
  const long N = (long)h->net.n * h->net.n;
  if (nb < 0 || ldu < N || ldo < N) return fail(IGM_ERR_ARG, "bad nb or leading dimension");
  if (nb == 0) return IGM_OK;
  igm_status r = phic_work(h, h->upw, h->work, nb);
  if (r != IGM_OK) return r;
  CU(phic_forward(h->net, nb, u, ldu, nullptr, 0, nullptr, 0, out, ldo, h->work, (cudaStream_t)s));
  return IGM_OK;
}

// Training state for npairs pairs and minibatches of `batch`, the pairs
// normalised on the device; idx (DEVICE, [nidx]) receives nothing yet.
static igm_status phic_train_state(phic_handle* h, int npairs, const double* U0, const double* U1,
                                   long ld, int batch, int nloss, int nidx, int** idx,
                                   cudaStream_t st) {
  const long N = (long)h->net.n * h->net.n;
  const size_t C = h->net.C, cnt = h->net.count;
  PhicTrain& t = h->train;
  Uploader& up = h->upt;
  up = Uploader();
  t = PhicTrain();
  t.np = npairs;
  t.X = (float*)up.raw(4 * (size_t)N * npairs);
  t.Y = (float*)up.raw(4 * (size_t)N * npairs);
  t.xf = (float*)up.raw(4 * (size_t)N * batch);
  t.y = (float*)up.raw(4 * (size_t)N * batch);
  t.gy = (float*)up.raw(4 * (size_t)N * batch);
  t.gx = (float*)up.raw(4 * (size_t)N * batch);
  for (int l = 0; l < 3; ++l) t.gz[l] = (__nv_bfloat16*)up.raw(2 * (size_t)N * C * batch);
  t.part = (float*)up.raw(4 * cnt * batch);
  t.gw = (float*)up.raw(4 * cnt);
  t.m = (float*)up.raw(4 * cnt);
  t.v = (float*)up.raw(4 * cnt);
  t.loss = (float*)up.raw(4 * (size_t)std::max(1, nloss));
  *idx = (int*)up.raw(4 * (size_t)std::max(1, nidx));
  if (up.err != cudaSuccess) return fail(IGM_ERR_OOM, cudaGetErrorString(up.err));
  igm_status r = phic_work(h, h->uptw, t.work, batch, true);
  if (r != IGM_OK) return r;
  CU(cudaMemsetAsync(t.loss, 0, 4 * (size_t)std::max(1, nloss), st));
  CU(phic_prepare_pairs(h->net.n, npairs, U0, U1, ld, t.X, t.Y, st));
  return IGM_OK;
}

extern "C" igm_status phic_train(phic_handle* h, int npairs, const double* U0, const double* U1,
                                 long ld, int steps, int batch, double lr, unsigned long long seed,
                                 double* loss, igm_stream s) {
  if (!h || !U0 || !U1) return fail(IGM_ERR_ARG, "null argument");
  const long N = (long)h->net.n * h->net.n;
  if (npairs < 1 || steps < 0 || batch < 1 || ld < N || !(lr > 0.0))
    return fail(IGM_ERR_ARG, "phic_train: need npairs, batch >= 1, steps >= 0, ld >= n*n, lr > 0");
  cudaStream_t st = (cudaStream_t)s;
  int* idx = nullptr;
  igm_status r = phic_train_state(h, npairs, U0, U1, ld, batch, steps, std::max(1, steps) * batch,
                                  &idx, st);
  if (r != IGM_OK) return r;
  PhicTrain& t = h->train;
  CU(cudaMemsetAsync(t.m, 0, 4 * (size_t)h->net.count, st));
  CU(cudaMemsetAsync(t.v, 0, 4 * (size_t)h->net.count, st));
  std::vector<int> hidx((size_t)std::max(1, steps) * batch);
  std::mt19937_64 rng(seed);
  std::uniform_int_distribution<int> ud(0, npairs - 1);
  for (auto& k : hidx) k = ud(rng);
  CU(cudaMemcpyAsync(idx, hidx.data(), sizeof(int) * hidx.size(), cudaMemcpyHostToDevice, st));
  for (int k = 0; k < steps; ++k) {
    CU(phic_backprop(h->net, t, batch, idx + (size_t)k * batch, t.loss + k, false, st));
    CU(phic_adam(h->net, t, k, (float)lr, st));
  }
  if (loss && steps > 0) {
    std::vector<float> hl(steps);
    CU(cudaMemcpyAsync(hl.data(), t.loss, sizeof(float) * steps, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    for (int k = 0; k < steps; ++k) loss[k] = hl[k];
  }
  CU(cudaStreamSynchronize(st));
  return IGM_OK;
}

extern "C" igm_status phic_grad(phic_handle* h, int nb, const double* U0, const double* U1,
                                long ld, double* loss, float* gw, float* gx, igm_stream s) {
  if (!h || !U0 || !U1 || !loss || !gw) return fail(IGM_ERR_ARG, "null argument");
  const long N = (long)h->net.n * h->net.n;
  if (nb < 1 || ld < N) return fail(IGM_ERR_ARG, "phic_grad: need nb >= 1 and ld >= n*n");
  cudaStream_t st = (cudaStream_t)s;
  int* idx = nullptr;
  igm_status r = phic_train_state(h, nb, U0, U1, ld, nb, 1, nb, &idx, st);
  if (r != IGM_OK) return r;
  PhicTrain& t = h->train;
  std::vector<int> hidx(nb);
  for (int k = 0; k < nb; ++k) hidx[k] = k;
  CU(cudaMemcpyAsync(idx, hidx.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st));
  CU(phic_backprop(h->net, t, nb, idx, t.loss, gx != nullptr, st));
  float hl = 0.0f;
  CU(cudaMemcpyAsync(&hl, t.loss, sizeof(float), cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(gw, t.gw, sizeof(float) * h->net.count, cudaMemcpyDeviceToHost, st));
  if (gx) CU(cudaMemcpyAsync(gx, t.gx, sizeof(float) * (size_t)N * nb, cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  *loss = hl;
  return IGM_OK;
}

extern "C" void mgrit_default_opts(mgrit_opts* o) {
  if (!o) return;
  o->T = 1.0;
  o->Nt = 256;
  o->m = 4;
  o->max_levels = 30;
  o->min_coarse = 4;
  o->relax = 1;
  o->tol = 1e-10;
  o->max_iter = 100;
  pmg_default_opts(&o->pmg);
  o->initial_guess = 0;
  o->graphs = 1;
  o->profile = 0;
  o->theta = 1.0;
  o->cycle = 0;
  o->priority = 0;
  o->coarse_cycles = 0;
  o->fused = 1;
}

struct Level {
  int Nl = 0;
  double dt = 0.0;
  pmg_handle* h = nullptr;
  double* W = nullptr;
  double* g = nullptr;
};

struct ProfRec {
  int level, grid, mode;
  cudaEvent_t e0, e1;
};

struct mgrit_handle {
  const iga_ops* ops = nullptr;
  mgrit_opts o;
  std::vector<Level> L;
  std::vector<pmg_handle*> owned;
  Uploader up;
  int max_grid = 1;
  std::vector<int> max_resident;            // per level: CTAs of a cooperative sweep launch
  unsigned* gbar = nullptr;                 // grid barrier of the fused level visits
  double* scratch = nullptr;
  double* norms = nullptr;
  unsigned long long* counters = nullptr;   // [0] solves, [1] cycles
  int* status = nullptr;
  double* dfcoef = nullptr;
  double* hnorms = nullptr;                 // pinned host copy of the norms
  double setup_seconds = 0.0;
  // graphs of one iteration: A = fine relaxation + residual + norm copy,
  // B = coarse levels + corrections; captured for one (U, fhat) pair
  cudaGraphExec_t gA = nullptr, gB = nullptr;
  long gA_launches = 0, gB_launches = 0;    // kernels in each graph
  const double* g_U = nullptr;
  const double* g_fhat = nullptr;
  // the run executes on this stream (graph capture is not allowed on the
  // legacy default stream), ordered after and before the caller's stream
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // per-launch profile of the last run
  std::vector<ProfRec> prof;
  std::vector<unsigned long long> prof_cyc;  // counter snapshots after each launch
  unsigned long long* dlog = nullptr;
  int dlog_cap = 0;
  // learned coarse propagator (two levels, FAS) and its scratch
  phic_handle* phic = nullptr;
  double phic_switch = 0.5;
  double *fas_tau = nullptr, *fas_v = nullptr;
  double* fas_backup = nullptr;             // the iterate before a learned coarse correction
  cudaGraphExec_t gL = nullptr;             // the FAS coarse level, captured per (U, fhat)
  // state of the run in progress (mgrit_run, mgrit_run_batched)
  struct Run {
    double* U = nullptr;
    const double* fhat = nullptr;
    cudaStream_t user = nullptr;
    bool profile = false, graphs = false, done = false;
    int it = 0;
    std::vector<double> hist;
    long launches0 = 0;
    std::chrono::steady_clock::time_point t0;
    igm_status status = IGM_OK;
    bool fallback = false;          // the learned propagator was replaced by backward Euler
    bool learned_prev = false;      // the last correction used the learned propagator
    cudaEvent_t evA = nullptr;      // completion of the fine-level part of an iteration
  } run;
  ~mgrit_handle() {
    if (run.evA) cudaEventDestroy(run.evA);
    if (gL) cudaGraphExecDestroy(gL);
    if (gA) cudaGraphExecDestroy(gA);
    if (gB) cudaGraphExecDestroy(gB);
    for (auto& r : prof) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
    for (auto* h : owned) pmg_destroy(h);
    if (hnorms) cudaFreeHost(hnorms);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (own) cudaStreamDestroy(own);
  }
};

// CTAs of the F-relaxation sweeps on a level of Nl steps: one per interval,
// plus one for a partial last interval
static int f_grid(int Nl, int m) { return Nl / m + (Nl % m != 0); }

extern "C" igm_status mgrit_create(const iga_ops* ops, const mgrit_opts* opts, mgrit_handle** out) {
  if (!ops || !opts || !out) return fail(IGM_ERR_ARG, "null argument");
  const mgrit_opts& o = *opts;
  if (o.Nt < 1 || o.m < 2 || !(o.T > 0.0) || o.max_iter < 0 || o.max_levels < 1 ||
      o.max_iter > 255)
    return fail(IGM_ERR_ARG, "bad MGRIT options (Nt >= 1, m >= 2, T > 0, 0 <= max_iter <= 255)");
  if (o.relax != 0 && o.relax != 1) return fail(IGM_ERR_ARG, "relax must be 0 or 1");
  if (!(o.theta >= 0.0 && o.theta <= 1.0)) return fail(IGM_ERR_ARG, "theta must be in [0, 1]");
  if (o.cycle < 0 || o.cycle > 2) return fail(IGM_ERR_ARG, "cycle must be 0 (V), 1 (F) or 2 (W)");
  if (o.coarse_cycles < 0) return fail(IGM_ERR_ARG, "coarse_cycles must be >= 0");
  if (o.fused != 0 && o.fused != 1) return fail(IGM_ERR_ARG, "fused must be 0 or 1");
  auto t0 = std::chrono::steady_clock::now();
  auto mg = std::make_unique<mgrit_handle>();
  mg->ops = ops;
  mg->o = o;
  const int N = ops->hi.N;
  std::vector<Level>& L = mg->L;
  Level l0;
  l0.Nl = o.Nt;
  l0.dt = o.T / o.Nt;
  L.push_back(l0);
  // coarsen to floor(N_l / m) C-points; a remainder leaves a partial last
  // interval of F-points on level l
  while ((int)L.size() < o.max_levels && L.back().Nl > o.min_coarse && L.back().Nl / o.m >= 1) {
    Level nx;
    nx.Nl = L.back().Nl / o.m;
    nx.dt = L.back().dt * o.m;
    L.push_back(nx);
  }
  const int nlev = (int)L.size();
  Uploader& up = mg->up;
  for (int l = 0; l < nlev; ++l) {
    pmg_handle* h = nullptr;
    igm_status r = pmg_setup_ex(ops, o.theta * ops->kappa * L[l].dt,
                                (1.0 - o.theta) * ops->kappa * L[l].dt, &o.pmg, &h);
    if (r != IGM_OK) return r;
    mg->owned.push_back(h);
    L[l].h = h;
    if (l > 0) {
      L[l].W = (double*)up.raw(sizeof(double) * (size_t)(L[l].Nl + 1) * N);
      L[l].g = (double*)up.raw(sizeof(double) * (size_t)(L[l].Nl + 1) * N);
    }
  }
  for (int l = 0; l < nlev; ++l) mg->max_grid = std::max(mg->max_grid, f_grid(L[l].Nl, o.m));
  mg->scratch = (double*)up.raw(sizeof(double) * 2 * (size_t)N * mg->max_grid);
  mg->norms = (double*)up.raw(sizeof(double) * (size_t)mg->max_grid);
  mg->counters = (unsigned long long*)up.raw(sizeof(unsigned long long) * 2);
  mg->status = (int*)up.raw(sizeof(int));
  mg->gbar = (unsigned*)up.raw(sizeof(unsigned) * 4);
  mg->dfcoef = (double*)up.raw(sizeof(double) * (size_t)(o.Nt + 1));
  if (up.err != cudaSuccess) return fail(IGM_ERR_OOM, cudaGetErrorString(up.err));
  CU(cudaMallocHost(&mg->hnorms, sizeof(double) * mg->max_grid));
  {
    int least = 0, greatest = 0;  // greatest priority = numerically lowest
    CU(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    const int prio = std::max(greatest, least - std::max(0, o.priority));
    CU(cudaStreamCreateWithPriority(&mg->own, cudaStreamNonBlocking, prio));
  }
  CU(cudaEventCreateWithFlags(&mg->ev_in, cudaEventDisableTiming));
  CU(cudaEventCreateWithFlags(&mg->ev_out, cudaEventDisableTiming));
  for (int l = 0; l < nlev; ++l) {
    igm_status r = ensure_arena(L[l].h, mg->max_grid);
    if (r != IGM_OK) return r;
    mg->max_resident.push_back(
        o.fused ? mgrit_sweep_max_resident(L[l].h->d.precision, smem_of(L[l].h)) : 0);
  }
  mg->setup_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  *out = mg.release();
  return IGM_OK;
}

extern "C" void mgrit_destroy(mgrit_handle* mg) { delete mg; }

extern "C" igm_status mgrit_set_coarse_propagator(mgrit_handle* mg, phic_handle* h,
                                                  double switch_ratio) {
  if (!mg) return fail(IGM_ERR_ARG, "null argument");
  if (mg->gL) cudaGraphExecDestroy(mg->gL);
  mg->gL = nullptr;
  if (!h) {
    mg->phic = nullptr;
    return IGM_OK;
  }
  if ((int)mg->L.size() != 2)
    return fail(IGM_ERR_ARG, "the learned coarse propagator needs two time levels (max_levels = 2)");
  if (h->net.n != mg->ops->hi.n) return fail(IGM_ERR_ARG, "propagator grid does not match the problem");
  if (!(switch_ratio > 0.0)) return fail(IGM_ERR_ARG, "switch_ratio must be > 0");
  const int N = mg->ops->hi.N, Nc = mg->L[1].Nl;
  if (!mg->fas_tau) {
    mg->fas_tau = (double*)mg->up.raw(sizeof(double) * (size_t)(Nc + 1) * N);
    mg->fas_v = (double*)mg->up.raw(sizeof(double) * (size_t)(Nc + 1) * N);
    mg->fas_backup = (double*)mg->up.raw(sizeof(double) * (size_t)(mg->o.Nt + 1) * N);
    if (mg->up.err != cudaSuccess) return fail(IGM_ERR_OOM, cudaGetErrorString(mg->up.err));
  }
  igm_status r = phic_work(h, h->upw, h->work, Nc);
  if (r != IGM_OK) return r;
  mg->phic = h;
  mg->phic_switch = switch_ratio;
  return IGM_OK;
}

// Launch one sweep kernel on level l: one mode, or (nmodes > 1) the modes of
// a level visit in one cooperative launch with grid barriers between them.
static igm_status sweep(mgrit_handle* mg, int l, int mode, int grid, double* nrm, double* U,
                        const double* fhat, cudaStream_t st, bool profile,
                        const int* modes = nullptr, int nmodes = 0) {
  const int nlev = (int)mg->L.size();
  std::vector<Level>& L = mg->L;
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.P = L[l].h->d;
  a.mode = mode;
  a.m = mg->o.m;
  a.Nl = L[l].Nl;
  a.nint = L[l].Nl / mg->o.m;
  a.W = l == 0 ? U : L[l].W;
  a.g = l > 0 ? L[l].g : nullptr;
  if (l + 1 < nlev) {
    a.Wc = L[l + 1].W;
    a.gc = L[l + 1].g;
    a.gnext = L[l + 1].g;
  }
  a.norms = nrm;
  a.fhat = (l == 0) ? fhat : nullptr;
  a.fcoef = mg->dfcoef;
  a.dt0 = L[0].dt;
  a.theta = mg->o.theta;
  a.scratch = mg->scratch;
  a.garena = L[l].h->garena;
  a.ncycles = l > 0 ? mg->o.coarse_cycles : 0;
  a.counters = mg->counters;
  a.status = mg->status;
  a.nmodes = nmodes > 1 ? nmodes : 0;
  for (int q = 0; q < nmodes && q < 3; ++q) a.modes[q] = modes[q];
  a.gbar = mg->gbar;
  a.bar_cycles = kWaitCycles;
  ProfRec rec{l, grid, a.nmodes ? (int)MODE_FUSED : mode, nullptr, nullptr};
  if (a.nmodes) CU(cudaMemsetAsync(mg->gbar, 0, sizeof(unsigned) * 4, st));
  if (profile) {
    CU(cudaEventCreate(&rec.e0));
    CU(cudaEventCreate(&rec.e1));
    CU(cudaEventRecord(rec.e0, st));
  }
  if (a.nmodes)
    CU(launch_mgrit_level(a.P.precision, a, grid, smem_of(L[l].h), st));
  else
    CU(launch_mgrit_sweep(a.P.precision, a, grid, smem_of(L[l].h), st));
  g_launches++;
  if (profile) {
    CU(cudaEventRecord(rec.e1, st));
    const int k = (int)mg->prof.size();
    if (k < mg->dlog_cap)
      CU(cudaMemcpyAsync(mg->dlog + 2 * k, mg->counters, 2 * sizeof(unsigned long long),
                         cudaMemcpyDeviceToDevice, st));
    mg->prof.push_back(rec);
  }
  return IGM_OK;
}

#define SWEEP(l, mode, grid, nrm)                                                \
  do {                                                                           \
    igm_status _r = sweep(mg, l, mode, grid, nrm, U, fhat, st, profile);         \
    if (_r != IGM_OK) return _r;                                                 \
  } while (0)
#define SWEEP_FUSED(l, modes, nmodes, grid, nrm)                                 \
  do {                                                                           \
    igm_status _r = sweep(mg, l, 0, grid, nrm, U, fhat, st, profile, modes, nmodes); \
    if (_r != IGM_OK) return _r;                                                 \
  } while (0)

// Whether the relaxation phases of a visit of level l run as one cooperative
// launch: requested, and all the level's CTAs can be resident at once.
static bool fused_level(const mgrit_handle* mg, int l) {
  return mg->o.fused && mg->o.relax == 1 &&
         f_grid(mg->L[l].Nl, mg->o.m) <= mg->max_resident[l];
}

// Part A of an iteration: fine-level relaxation (Sec. 3, FCF or F) and the
// C-point residual, injected into g^(1); copies the per-interval norms.
static igm_status part_A(mgrit_handle* mg, bool first, double* U, const double* fhat,
                         cudaStream_t st, bool profile) {
  const int nint0 = mg->L[0].Nl / mg->o.m, nf0 = f_grid(mg->L[0].Nl, mg->o.m);
  if (mg->o.relax == 1 && fused_level(mg, 0)) {
    // one launch: (F,) C, F + residual with grid barriers between them
    static const int fcf[3] = {MODE_F, MODE_C, MODE_FR};
    SWEEP_FUSED(0, first ? fcf : fcf + 1, first ? 3 : 2, nf0, mg->norms);
  } else if (mg->o.relax == 1) {
    // the leading F-relaxation is skipped after the first iteration: the
    // interpolation has just made the F-points Phi-consistent
    if (first) SWEEP(0, MODE_F, nf0, nullptr);
    SWEEP(0, MODE_C, nint0, nullptr);
    SWEEP(0, MODE_FR, nf0, mg->norms);
  } else if (first) {
    SWEEP(0, MODE_FR, nf0, mg->norms);
  } else {
    SWEEP(0, MODE_R, nint0, mg->norms);
  }
  CU(cudaMemcpyAsync(mg->hnorms, mg->norms, sizeof(double) * nint0, cudaMemcpyDeviceToHost, st));
  return IGM_OK;
}

// One visit of coarse level l >= 1 with a cycle of the given kind (Sec. 3
// algorithm box; Sec. 5 names V-, F-cycles): relaxation and residual into
// g^(l+1), then the visits of level l+1 (V: one V; F: an F then a V; W: two
// W, the second from the first's result; a repeated visit of the exact
// coarsest level is skipped), then the correction with F-relaxation.
static igm_status visit(mgrit_handle* mg, int l, int kind, double* U, const double* fhat,
                        cudaStream_t st, bool profile) {
  const int nlev = (int)mg->L.size(), N = mg->ops->hi.N;
  std::vector<Level>& L = mg->L;
  if (l == nlev - 1) {
    SWEEP(l, MODE_SEQ, 1, nullptr);
    return IGM_OK;
  }
  const int ni = L[l].Nl / mg->o.m, nf = f_grid(L[l].Nl, mg->o.m);
  if (fused_level(mg, l)) {
    static const int fcf[3] = {MODE_F, MODE_C, MODE_FR};
    SWEEP_FUSED(l, fcf, 3, nf, nullptr);
  } else {
    if (mg->o.relax == 1) {
      SWEEP(l, MODE_F, nf, nullptr);
      SWEEP(l, MODE_C, ni, nullptr);
    }
    SWEEP(l, MODE_FR, nf, nullptr);
  }
  CU(cudaMemsetAsync(L[l + 1].W, 0, sizeof(double) * (size_t)(L[l + 1].Nl + 1) * N, st));
  const int sub[3][2] = {{0, -1}, {1, 0}, {2, 2}};
  for (int v = 0; v < 2; ++v) {
    const int k = sub[kind][v];
    if (k < 0 || (v == 1 && l + 1 == nlev - 1)) break;
    igm_status r = visit(mg, l + 1, k, U, fhat, st, profile);
    if (r != IGM_OK) return r;
  }
  SWEEP(l, MODE_CF, nf, nullptr);
  return IGM_OK;
}

// Part B: the coarse levels and the correction with F-relaxation (ideal
// interpolation) of the fine level.
static igm_status part_B(mgrit_handle* mg, double* U, const double* fhat, cudaStream_t st,
                         bool profile) {
  const int N = mg->ops->hi.N;
  std::vector<Level>& L = mg->L;
  CU(cudaMemsetAsync(L[1].W, 0, sizeof(double) * (size_t)(L[1].Nl + 1) * N, st));
  const int kind = mg->o.cycle;
  const int nlev = (int)L.size();
  for (int v = 0; v < 2; ++v) {
    const int k = v == 0 ? kind : (kind == 1 ? 0 : (kind == 2 ? 2 : -1));
    if (k < 0 || (v == 1 && nlev == 2)) break;
    igm_status r = visit(mg, 1, k, U, fhat, st, profile);
    if (r != IGM_OK) return r;
  }
  SWEEP(0, MODE_CF, f_grid(L[0].Nl, mg->o.m), nullptr);
  return IGM_OK;
}

static igm_status capture(mgrit_handle* mg, bool partA, double* U, const double* fhat,
                          cudaStream_t st, cudaGraphExec_t* out) {
  CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const long before = g_launches.load();
  igm_status r = partA ? part_A(mg, false, U, fhat, st, false) : part_B(mg, U, fhat, st, false);
  // the captured kernels launch when the graph does
  const long nk = g_launches.load() - before;
  g_launches -= nk;
  (partA ? mg->gA_launches : mg->gB_launches) = nk;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (r != IGM_OK) { if (g) cudaGraphDestroy(g); return r; }
  if (e != cudaSuccess) return fail(IGM_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(IGM_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  return IGM_OK;
}

// The coarse level of two-level MGRIT with the learned propagator (FAS):
// tau_j = u_{jm} - Phi_c(u_{(j-1)m}) + r_j, v_j = Phi_c(v_{j-1}) + tau_j from
// v_0 = u_0, then the C-point correction u_{jm} <- v_j with F-relaxation.
static igm_status part_learned(mgrit_handle* mg, double* U, const double* fhat, cudaStream_t st) {
  const bool profile = false;
  const int m = mg->o.m, Nc = mg->L[1].Nl, N = mg->ops->hi.N;
  CU(cudaMemcpyAsync(mg->fas_backup, U, sizeof(double) * (size_t)(mg->o.Nt + 1) * N,
                     cudaMemcpyDeviceToDevice, st));
  CU(phic_fas_coarse(mg->phic->net, Nc, m, U, mg->L[1].g, mg->fas_tau, mg->fas_v, mg->L[1].W,
                     mg->phic->work, st));
  SWEEP(0, MODE_CF, f_grid(mg->L[0].Nl, m), nullptr);
  return IGM_OK;
}

// Launch the fine-level part of iteration it (relaxation, residual, norms to
// the host) and record run.evA after it.
static igm_status launch_A(mgrit_handle* mg) {
  auto& R = mg->run;
  cudaStream_t st = mg->own;
  double* U = R.U;
  const double* fhat = R.fhat;
  const bool profile = R.profile;
  if (R.graphs && R.it > 0) {
    if (!mg->gA) {
      igm_status r = capture(mg, true, U, fhat, st, &mg->gA);
      if (r != IGM_OK) return r;
    }
    CU(cudaGraphLaunch(mg->gA, st));
    g_launches += mg->gA_launches;
  } else {
    igm_status r = part_A(mg, R.it == 0, U, fhat, st, profile);
    if (r != IGM_OK) return r;
  }
  CU(cudaEventRecord(R.evA, st));
  return IGM_OK;
}

// Start a run: ordering after the caller's stream, the source factors, the
// initial guess, and the first fine-level part (or the whole sequential
// solve for a single time level).
static igm_status run_begin(mgrit_handle* mg, const double* u0, const double* fhat,
                            const double* fcoef, double* U, cudaStream_t user) {
  if (!mg || !u0 || !U) return fail(IGM_ERR_ARG, "null argument");
  const mgrit_opts& o = mg->o;
  auto& R = mg->run;
  cudaStream_t st = mg->own;
  if (!R.evA) CU(cudaEventCreateWithFlags(&R.evA, cudaEventDisableTiming));
  CU(cudaEventRecord(mg->ev_in, user));
  CU(cudaStreamWaitEvent(st, mg->ev_in, 0));
  const int N = mg->ops->hi.N;
  const int nlev = (int)mg->L.size();
  if (fhat && !fcoef) return fail(IGM_ERR_ARG, "fhat given without fcoef");
  if (!fcoef) fhat = nullptr;
  R.U = U;
  R.fhat = fhat;
  R.user = user;
  R.profile = o.profile != 0;
  R.graphs = o.graphs != 0 && !R.profile && nlev > 1;
  R.done = false;
  R.it = 0;
  R.hist.clear();
  R.status = IGM_OK;
  R.fallback = false;
  R.learned_prev = false;
  R.launches0 = g_launches.load();
  if (fhat)
    CU(cudaMemcpyAsync(mg->dfcoef, fcoef, sizeof(double) * (o.Nt + 1), cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(mg->counters, 0, 2 * sizeof(unsigned long long), st));
  CU(cudaMemsetAsync(mg->status, 0, sizeof(int), st));
  for (auto& r : mg->prof) { cudaEventDestroy(r.e0); cudaEventDestroy(r.e1); }
  mg->prof.clear();
  if (R.profile && !mg->dlog) {
    mg->dlog_cap = 4096;
    mg->dlog = (unsigned long long*)mg->up.raw(sizeof(unsigned long long) * 2 * mg->dlog_cap);
    if (mg->up.err != cudaSuccess) return fail(IGM_ERR_OOM, cudaGetErrorString(mg->up.err));
  }
  if (R.graphs && (mg->g_U != U || mg->g_fhat != fhat)) {
    if (mg->gA) cudaGraphExecDestroy(mg->gA);
    if (mg->gB) cudaGraphExecDestroy(mg->gB);
    if (mg->gL) cudaGraphExecDestroy(mg->gL);
    mg->gA = mg->gB = mg->gL = nullptr;
  }
  // initial guess: U[0] = u0, U[n>=1] = 0 unless the caller's U is to be kept
  CU(cudaMemcpyAsync(U, u0, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  if (!o.initial_guess) CU(cudaMemsetAsync(U + N, 0, sizeof(double) * (size_t)o.Nt * N, st));
  R.t0 = std::chrono::steady_clock::now();
  if (nlev == 1) {
    const bool profile = R.profile;
    SWEEP(0, MODE_SEQ, 1, nullptr);
    R.done = true;
    return IGM_OK;
  }
  return launch_A(mg);
}

// After the fine-level part of an iteration has completed (run.evA): the
// stopping test on the C-point residual norms, then either the end of the
// run or the coarse levels, the correction and the next fine-level part.
static igm_status run_advance(mgrit_handle* mg) {
  const mgrit_opts& o = mg->o;
  auto& R = mg->run;
  cudaStream_t st = mg->own;
  double* U = R.U;
  const double* fhat = R.fhat;
  const bool profile = R.profile;
  const int nlev = (int)mg->L.size();
  const int nint0 = mg->L[0].Nl / o.m;
  double rr = 0.0;
  for (int j = 0; j < nint0; ++j) rr += mg->hnorms[j];
  const double rho = std::sqrt(rr);
  // a learned coarse correction that made the residual non-finite or did not
  // contract enough is undone: the iterate before it is restored, relaxed
  // again, and the run continues with the backward-Euler coarse level
  if (R.learned_prev && !(rho <= mg->phic_switch * R.hist.back())) {
    R.learned_prev = false;
    R.fallback = true;
    const int N = mg->ops->hi.N;
    CU(cudaMemcpyAsync(U, mg->fas_backup, sizeof(double) * (size_t)(o.Nt + 1) * N,
                       cudaMemcpyDeviceToDevice, st));
    return launch_A(mg);
  }
  R.hist.push_back(rho);
  if (!(rho == rho)) return fail(IGM_ERR_NUMERIC, "NaN in the MGRIT residual");
  if (rho == 0.0 || rho <= o.tol * R.hist[0] || R.it >= o.max_iter) {
    R.done = true;
    if (R.graphs) {
      mg->g_U = U;
      mg->g_fhat = fhat;
    }
    return IGM_OK;
  }
  R.learned_prev = false;
  if (mg->phic && !R.fallback) {
    R.learned_prev = true;
    const int Nc = mg->L[1].Nl;
    if (R.graphs) {
      if (!mg->gL) {
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        igm_status r = part_learned(mg, U, fhat, st);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(st, &g);
        if (r != IGM_OK) { if (g) cudaGraphDestroy(g); return r; }
        if (e != cudaSuccess) return fail(IGM_ERR_CUDA, cudaGetErrorString(e));
        e = cudaGraphInstantiate(&mg->gL, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(IGM_ERR_CUDA, cudaGetErrorString(e));
      }
      CU(cudaGraphLaunch(mg->gL, st));
    } else {
      igm_status r = part_learned(mg, U, fhat, st);
      if (r != IGM_OK) return r;
    }
    g_launches += 5 * (Nc + 1) + 2 + 1;
  } else if (R.graphs) {
    if (!mg->gB) {
      igm_status r = capture(mg, false, U, fhat, st, &mg->gB);
      if (r != IGM_OK) return r;
    }
    CU(cudaGraphLaunch(mg->gB, st));
    g_launches += mg->gB_launches;
  } else {
    igm_status r = part_B(mg, U, fhat, st, profile);
    if (r != IGM_OK) return r;
  }
  ++R.it;
  return launch_A(mg);
}

// End of a run: order the caller's stream after it, collect the counters and
// fill stats; the status reflects spatial-solve failures and convergence.
static igm_status run_finish(mgrit_handle* mg, mgrit_stats* stats) {
  const mgrit_opts& o = mg->o;
  auto& R = mg->run;
  cudaStream_t st = mg->own;
  const int nlev = (int)mg->L.size();
  CU(cudaEventRecord(mg->ev_out, st));
  CU(cudaStreamWaitEvent(R.user, mg->ev_out, 0));
  CU(cudaStreamSynchronize(st));
  auto t1 = std::chrono::steady_clock::now();
  unsigned long long hc[2] = {0, 0};
  int hstat = 0;
  CU(cudaMemcpy(hc, mg->counters, sizeof(hc), cudaMemcpyDeviceToHost));
  CU(cudaMemcpy(&hstat, mg->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (R.profile) {
    const int k = std::min((int)mg->prof.size(), mg->dlog_cap);
    mg->prof_cyc.assign(2 * (size_t)k, 0);
    if (k) CU(cudaMemcpy(mg->prof_cyc.data(), mg->dlog, sizeof(unsigned long long) * 2 * k,
                         cudaMemcpyDeviceToHost));
  }
  const auto& hist = R.hist;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->iters = R.it;
    stats->levels = nlev;
    for (size_t k = 0; k < hist.size() && k < 256; ++k) stats->res_hist[k] = hist[k];
    stats->solves = (long)hc[0];
    stats->vcycles = (long)hc[1];
    stats->vcyc_mean = hc[0] ? (double)hc[1] / (double)hc[0] : 0.0;
    stats->seconds = std::chrono::duration<double>(t1 - R.t0).count();
    stats->setup_seconds = mg->setup_seconds;
    stats->launches = g_launches.load() - R.launches0;
    stats->coarse_fallback = R.fallback ? 1 : 0;
  }
  if (hstat == ST_NUMERIC) return fail(IGM_ERR_NUMERIC, "NaN in a spatial residual");
  if (hstat == ST_TIMEOUT) return fail(IGM_ERR_TIMEOUT, "a bounded device wait gave up");
  if (hstat == ST_NOT_CONVERGED) return fail(IGM_ERR_NOT_CONVERGED, "a spatial solve hit max_cycles");
  if (nlev > 1 && !hist.empty() && !(hist.back() <= o.tol * hist[0]) && hist.back() != 0.0)
    return fail(IGM_ERR_NOT_CONVERGED, "MGRIT hit max_iter");
  return IGM_OK;
}

extern "C" igm_status mgrit_run(mgrit_handle* mg, const double* u0, const double* fhat,
                                const double* fcoef, double* U, mgrit_stats* stats, igm_stream s) {
  igm_status r = run_begin(mg, u0, fhat, fcoef, U, (cudaStream_t)s);
  while (r == IGM_OK && !mg->run.done) {
    CU(cudaEventSynchronize(mg->run.evA));
    r = run_advance(mg);
  }
  if (r != IGM_OK) {
    cudaStreamSynchronize(mg->own);
    return r;
  }
  return run_finish(mg, stats);
}

extern "C" igm_status mgrit_run_batched(int nprob, mgrit_handle* const* mgs,
                                        const double* const* u0, const double* const* fhat,
                                        const double* const* fcoef, double* const* U,
                                        mgrit_stats* stats, float* latency_ms, igm_stream s) {
  if (nprob < 0 || (nprob > 0 && (!mgs || !u0 || !U))) return fail(IGM_ERR_ARG, "null argument");
  if (nprob == 0) return IGM_OK;
  for (int i = 0; i < nprob; ++i)
    for (int k = 0; k < i; ++k)
      if (mgs[i] == mgs[k]) return fail(IGM_ERR_ARG, "a handle appears twice in the batch");
  cudaStream_t user = (cudaStream_t)s;
  cudaEvent_t start = nullptr;
  std::vector<cudaEvent_t> ends(nprob, nullptr);
  CU(cudaEventCreate(&start));
  for (auto& e : ends) CU(cudaEventCreate(&e));
  CU(cudaEventRecord(start, user));
  std::vector<igm_status> st(nprob, IGM_OK);
  std::vector<char> active(nprob, 1);
  int left = nprob;
  for (int i = 0; i < nprob; ++i) {
    st[i] = run_begin(mgs[i], u0[i], fhat ? fhat[i] : nullptr, fcoef ? fcoef[i] : nullptr, U[i],
                      user);
    if (st[i] != IGM_OK || mgs[i]->run.done) {
      if (st[i] == IGM_OK) CU(cudaEventRecord(ends[i], mgs[i]->own));
      active[i] = 0;
      --left;
    }
  }
  // host scheduler: advance whichever problem's fine-level part has finished
  while (left > 0) {
    bool progressed = false;
    for (int i = 0; i < nprob; ++i) {
      if (!active[i]) continue;
      const cudaError_t q = cudaEventQuery(mgs[i]->run.evA);
      if (q == cudaErrorNotReady) continue;
      if (q != cudaSuccess) {
        st[i] = fail(IGM_ERR_CUDA, cudaGetErrorString(q));
      } else {
        st[i] = run_advance(mgs[i]);
        if (st[i] == IGM_OK && mgs[i]->run.done) CU(cudaEventRecord(ends[i], mgs[i]->own));
      }
      progressed = true;
      if (st[i] != IGM_OK || mgs[i]->run.done) {
        active[i] = 0;
        --left;
      }
    }
    if (!progressed) std::this_thread::yield();
  }
  igm_status first = IGM_OK;
  for (int i = 0; i < nprob; ++i) {
    if (st[i] == IGM_OK) st[i] = run_finish(mgs[i], stats ? &stats[i] : nullptr);
    else cudaStreamSynchronize(mgs[i]->own);
    if (latency_ms) {
      float ms = -1.0f;
      if (st[i] == IGM_OK || st[i] == IGM_ERR_NOT_CONVERGED) cudaEventElapsedTime(&ms, start, ends[i]);
      latency_ms[i] = ms;
    }
    if (first == IGM_OK && st[i] != IGM_OK) first = st[i];
  }
  cudaEventDestroy(start);
  for (auto& e : ends) cudaEventDestroy(e);
  return first;
}

// ---------------------------------------------------------------------------
// Device-scheduled batch (one persistent launch): each member's run as a
// program of phases, the same launches part_A / part_B / visit issue.
// ---------------------------------------------------------------------------
static void prog_partA(const mgrit_handle* mg, bool first, std::vector<BatchPhase>& v) {
  const int m = mg->o.m, nint0 = mg->L[0].Nl / m, nf0 = f_grid(mg->L[0].Nl, m);
  if (mg->o.relax == 1) {
    if (first) v.push_back({0, MODE_F, nf0, BOP_SWEEP});
    v.push_back({0, MODE_C, nint0, BOP_SWEEP});
    v.push_back({0, MODE_FR, nf0, BOP_SWEEP});
  } else {
    v.push_back(first ? BatchPhase{0, MODE_FR, nf0, BOP_SWEEP} : BatchPhase{0, MODE_R, nint0, BOP_SWEEP});
  }
  v.push_back({0, 0, 1, BOP_TEST});
}

static void prog_zero(const mgrit_handle* mg, int l, std::vector<BatchPhase>& v) {
  v.push_back({l, 0, std::min(64, mg->L[l].Nl + 1), BOP_ZERO});
}

static void prog_visit(const mgrit_handle* mg, int l, int kind, std::vector<BatchPhase>& v) {
  const int nlev = (int)mg->L.size(), m = mg->o.m;
  if (l == nlev - 1) {
    v.push_back({l, MODE_SEQ, 1, BOP_SWEEP});
    return;
  }
  const int ni = mg->L[l].Nl / m, nf = f_grid(mg->L[l].Nl, m);
  if (mg->o.relax == 1) {
    v.push_back({l, MODE_F, nf, BOP_SWEEP});
    v.push_back({l, MODE_C, ni, BOP_SWEEP});
  }
  v.push_back({l, MODE_FR, nf, BOP_SWEEP});
  prog_zero(mg, l + 1, v);
  const int sub[3][2] = {{0, -1}, {1, 0}, {2, 2}};
  for (int q = 0; q < 2; ++q) {
    const int k = sub[kind][q];
    if (k < 0 || (q == 1 && l + 1 == nlev - 1)) break;
    prog_visit(mg, l + 1, k, v);
  }
  v.push_back({l, MODE_CF, nf, BOP_SWEEP});
}

static void prog_partB(const mgrit_handle* mg, std::vector<BatchPhase>& v) {
  const int nlev = (int)mg->L.size(), kind = mg->o.cycle;
  prog_zero(mg, 1, v);
  for (int q = 0; q < 2; ++q) {
    const int k = q == 0 ? kind : (kind == 1 ? 0 : (kind == 2 ? 2 : -1));
    if (k < 0 || (q == 1 && nlev == 2)) break;
    prog_visit(mg, 1, k, v);
  }
  v.push_back({0, MODE_CF, f_grid(mg->L[0].Nl, mg->o.m), BOP_SWEEP});
}

// The arguments of level l's sweeps (the mode is given per phase).
static SweepArgs level_args(mgrit_handle* mg, int l, double* U, const double* fhat) {
  const int nlev = (int)mg->L.size();
  std::vector<Level>& L = mg->L;
  SweepArgs a;
  std::memset(&a, 0, sizeof(a));
  a.P = L[l].h->d;
  a.m = mg->o.m;
  a.Nl = L[l].Nl;
  a.nint = L[l].Nl / mg->o.m;
  a.W = l == 0 ? U : L[l].W;
  a.g = l > 0 ? L[l].g : nullptr;
  if (l + 1 < nlev) {
    a.Wc = L[l + 1].W;
    a.gc = L[l + 1].g;
    a.gnext = L[l + 1].g;
  }
  a.norms = l == 0 ? mg->norms : nullptr;
  a.fhat = l == 0 ? fhat : nullptr;
  a.fcoef = mg->dfcoef;
  a.dt0 = L[0].dt;
  a.theta = mg->o.theta;
  a.scratch = mg->scratch;
  a.garena = L[l].h->garena;
  a.ncycles = l > 0 ? mg->o.coarse_cycles : 0;
  a.counters = mg->counters;
  a.status = mg->status;
  return a;
}

extern "C" igm_status mgrit_run_batched_device(int nprob, mgrit_handle* const* mgs,
                                               const double* const* u0, const double* const* fhat,
                                               const double* const* fcoef, double* const* U,
                                               mgrit_stats* stats, float* latency_ms,
                                               igm_stream s) {
  if (nprob < 0 || (nprob > 0 && (!mgs || !u0 || !U))) return fail(IGM_ERR_ARG, "null argument");
  if (nprob == 0) return IGM_OK;
  for (int i = 0; i < nprob; ++i) {
    if (!mgs[i] || !u0[i] || !U[i]) return fail(IGM_ERR_ARG, "null member");
    for (int k = 0; k < i; ++k)
      if (mgs[i] == mgs[k]) return fail(IGM_ERR_ARG, "a handle appears twice in the batch");
    if (mgs[i]->phic) return fail(IGM_ERR_ARG, "the device-scheduled batch has no learned coarse propagator");
    if (mgs[i]->L[0].h->d.precision != mgs[0]->L[0].h->d.precision)
      return fail(IGM_ERR_ARG, "all members of a device-scheduled batch need the same precision");
  }
  const int prec = mgs[0]->L[0].h->d.precision;
  cudaStream_t st = (cudaStream_t)s;
  auto t0 = std::chrono::steady_clock::now();
  // every member's run starts as mgrit_run does: initial guess, source factors, counters
  std::vector<BatchMember> hm(nprob);
  std::vector<std::vector<SweepArgs>> args(nprob);
  std::vector<std::vector<BatchPhase>> progs(nprob);
  long smem = 0;
  size_t nargs = 0, nph = 0;
  for (int i = 0; i < nprob; ++i) {
    mgrit_handle* mg = mgs[i];
    const mgrit_opts& o = mg->o;
    const int N = mg->ops->hi.N, nlev = (int)mg->L.size();
    const double* fh = fhat ? fhat[i] : nullptr;
    const double* fc = fcoef ? fcoef[i] : nullptr;
    if (fh && !fc) return fail(IGM_ERR_ARG, "fhat given without fcoef");
    if (!fc) fh = nullptr;
    if (fh) CU(cudaMemcpyAsync(mg->dfcoef, fc, sizeof(double) * (o.Nt + 1), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(mg->counters, 0, 2 * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(mg->status, 0, sizeof(int), st));
    CU(cudaMemcpyAsync(U[i], u0[i], sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    if (!o.initial_guess) CU(cudaMemsetAsync(U[i] + N, 0, sizeof(double) * (size_t)o.Nt * N, st));
    for (int l = 0; l < nlev; ++l) {
      args[i].push_back(level_args(mg, l, U[i], fh));
      smem = std::max(smem, smem_of(mg->L[l].h));
    }
    std::vector<BatchPhase>& v = progs[i];
    int nA0 = 0, nB = 0, nA = 0;
    if (nlev == 1) {
      v.push_back({0, MODE_SEQ, 1, BOP_SWEEP});
      v.push_back({0, 0, 1, BOP_TEST});
      nA0 = 2;
    } else {
      prog_partA(mg, true, v);
      nA0 = (int)v.size();
      prog_partB(mg, v);
      nB = (int)v.size() - nA0;
      prog_partA(mg, false, v);
      nA = (int)v.size() - nA0 - nB;
    }
    hm[i].nA0 = nA0;
    hm[i].nB = nB;
    hm[i].nA = nA;
    hm[i].nint0 = nlev == 1 ? 0 : mg->L[0].Nl / o.m;
    hm[i].norms = mg->norms;
    hm[i].tol = o.tol;
    hm[i].max_iter = o.max_iter;
    nargs += args[i].size();
    nph += v.size();
  }
  // one upload: [members][states][level arguments][programs][control]
  const size_t o_st = ((sizeof(BatchMember) * nprob + 255) / 256) * 256;
  const size_t o_args = o_st + ((sizeof(BatchState) * nprob + 255) / 256) * 256;
  const size_t o_prog = o_args + ((sizeof(SweepArgs) * nargs + 255) / 256) * 256;
  const size_t o_ctl = o_prog + ((sizeof(BatchPhase) * nph + 255) / 256) * 256;
  const size_t total = o_ctl + 256;
  char* dbuf = nullptr;
  CU(cudaMallocAsync((void**)&dbuf, total, st));
  std::vector<char> hbuf(total, 0);
  {
    SweepArgs* da = (SweepArgs*)(dbuf + o_args);
    BatchPhase* dp = (BatchPhase*)(dbuf + o_prog);
    size_t ka = 0, kp = 0;
    for (int i = 0; i < nprob; ++i) {
      hm[i].lv = da + ka;
      hm[i].prog = dp + kp;
      std::memcpy(hbuf.data() + o_args + sizeof(SweepArgs) * ka, args[i].data(),
                  sizeof(SweepArgs) * args[i].size());
      std::memcpy(hbuf.data() + o_prog + sizeof(BatchPhase) * kp, progs[i].data(),
                  sizeof(BatchPhase) * progs[i].size());
      ka += args[i].size();
      kp += progs[i].size();
    }
    std::memcpy(hbuf.data(), hm.data(), sizeof(BatchMember) * nprob);
  }
  CU(cudaMemcpyAsync(dbuf, hbuf.data(), total, cudaMemcpyHostToDevice, st));
  // one persistent CTA per SM (a CTA of the solver holds a whole SM's registers)
  int dev = 0, sms = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = std::max(1, sms);
  BatchState* dst = (BatchState*)(dbuf + o_st);
  unsigned long long* ctl = (unsigned long long*)(dbuf + o_ctl);
  CU(launch_mgrit_batch(prec, (const BatchMember*)dbuf, dst, nprob, ctl, grid, smem, st));
  g_launches++;
  std::vector<BatchState> hs(nprob);
  unsigned long long hctl[3] = {0, 0, 0};
  CU(cudaMemcpyAsync(hs.data(), dst, sizeof(BatchState) * nprob, cudaMemcpyDeviceToHost, st));
  CU(cudaMemcpyAsync(hctl, ctl, sizeof(hctl), cudaMemcpyDeviceToHost, st));
  CU(cudaFreeAsync(dbuf, st));
  CU(cudaStreamSynchronize(st));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  igm_status first = IGM_OK;
  for (int i = 0; i < nprob; ++i) {
    mgrit_handle* mg = mgs[i];
    const int nlev = (int)mg->L.size();
    unsigned long long hc[2] = {0, 0};
    int hstat = 0;
    CU(cudaMemcpy(hc, mg->counters, sizeof(hc), cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(&hstat, mg->status, sizeof(int), cudaMemcpyDeviceToHost));
    const BatchState& S = hs[i];
    const int nh = std::min(S.nhist, kBatchHist);
    if (stats) {
      mgrit_stats& t = stats[i];
      std::memset(&t, 0, sizeof(t));
      t.iters = S.it;
      t.levels = nlev;
      if (nlev > 1)
        for (int k = 0; k < nh && k < 256; ++k) t.res_hist[k] = S.hist[k];
      t.solves = (long)hc[0];
      t.vcycles = (long)hc[1];
      t.vcyc_mean = hc[0] ? (double)hc[1] / (double)hc[0] : 0.0;
      t.seconds = secs;
      t.setup_seconds = mg->setup_seconds;
      t.launches = 1;
    }
    if (latency_ms) latency_ms[i] = S.finished ? (float)((double)(S.t_end - hctl[2]) * 1e-6) : -1.0f;
    igm_status r = IGM_OK;
    if (!S.finished || hctl[1]) r = fail(IGM_ERR_TIMEOUT, "the batch scheduler gave up waiting for work");
    else if (hstat == ST_NUMERIC || (nh > 0 && !(S.hist[nh - 1] == S.hist[nh - 1])))
      r = fail(IGM_ERR_NUMERIC, "NaN in a residual");
    else if (hstat == ST_TIMEOUT) r = fail(IGM_ERR_TIMEOUT, "a bounded device wait gave up");
    else if (hstat == ST_NOT_CONVERGED) r = fail(IGM_ERR_NOT_CONVERGED, "a spatial solve hit max_cycles");
    else if (nlev > 1 && nh > 0 && !(S.hist[nh - 1] <= mg->o.tol * S.hist[0]) && S.hist[nh - 1] != 0.0)
      r = fail(IGM_ERR_NOT_CONVERGED, "MGRIT hit max_iter");
    if (first == IGM_OK && r != IGM_OK) first = r;
  }
  return first;
}

extern "C" igm_status mgrit_profile(const mgrit_handle* mg, int cap, int* count, int* level,
                                    int* grid, int* mode, float* ms, long* cycles) {
  if (!mg || !count) return fail(IGM_ERR_ARG, "null argument");
  const int k = std::min(cap, (int)std::min(mg->prof.size(), (size_t)mg->dlog_cap));
  for (int i = 0; i < k; ++i) {
    const ProfRec& r = mg->prof[i];
    if (level) level[i] = r.level;
    if (grid) grid[i] = r.grid;
    if (mode) mode[i] = r.mode;
    if (ms) {
      float t = 0.f;
      CU(cudaEventElapsedTime(&t, r.e0, r.e1));
      ms[i] = t;
    }
    if (cycles) {
      const unsigned long long prev = i ? mg->prof_cyc[2 * (i - 1) + 1] : 0ull;
      cycles[i] = (long)(mg->prof_cyc[2 * i + 1] - prev);
    }
  }
  *count = k;
  return IGM_OK;
}

extern "C" igm_status mgrit_solve(const iga_ops* ops, const mgrit_opts* opts, const double* u0,
                                  const double* fhat, const double* fcoef, double* U,
                                  mgrit_stats* stats, igm_stream s) {
  mgrit_handle* mg = nullptr;
  igm_status r = mgrit_create(ops, opts, &mg);
  if (r != IGM_OK) return r;
  r = mgrit_run(mg, u0, fhat, fcoef, U, stats, s);
  mgrit_destroy(mg);
  return r;
}
