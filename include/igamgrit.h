/*
 * igamgrit.h -- C ABI of the GB300 (sm_103a) solver for the IgA-discretised
 * heat equation with MGRIT in time and p-multigrid in space
 * (Tielen, Moeller, Vuik, arXiv 2107.05337).
 *
 * Problem (Sec. 2, Eq. (heat)): d_t u - kappa Laplace(u) = f on
 * Omega = F((0,1)^2), u = 0 on the boundary, u(.,0) = u0.  B-splines of order
 * p on a uniform open knot vector with nel elements per direction (Sec. 2);
 * the theta-scheme of Sec. 2, Eq. (los), backward Euler (theta = 1) by default:
 *     (M + theta kappa dt K) u^{k+1} = (M - (1-theta) kappa dt K) u^k + dt f.
 * Each such spatial solve is done by the p-multigrid cycle of Sec. 4 (ILUT
 * smoother, L2-projection transfers to p = 1, one h-multigrid W-cycle with
 * Gauss--Seidel at p = 1, direct coarsest solve).  The time stepping is
 * solved parallel-in-time by MGRIT (Sec. 3: FCF relaxation, injection, ideal
 * interpolation, V-cycle over rediscretised levels dt_l = m^l dt).
 *
 * Conventions shared by every entry point:
 *  - Unknowns: the (Dirichlet-eliminated) interior coefficients, n = nel+p-2
 *    per direction, N = n*n, numbered i = ix + n*iy (xi fastest).
 *  - Vectors passed as pointers are DEVICE memory owned by the caller unless
 *    the argument says "host".  Handles are owned by the library and freed by
 *    the matching *_destroy call.
 *  - Every call returns an igm_status and never throws; on failure the
 *    thread-local message igm_last_error() says why.  Work is enqueued on the
 *    CUDA stream passed in (0 = legacy default stream); calls that need a
 *    device result on the host (mgrit_solve, cycles_out) synchronise it.
 *  - There is no CPU fallback: without a usable sm_103a device every call
 *    that touches the GPU returns IGM_ERR_CUDA.
 */
#ifndef IGAMGRIT_H
#define IGAMGRIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IGM_OK = 0,
  IGM_ERR_ARG = -1,           /* invalid argument or unsupported size */
  IGM_ERR_CUDA = -2,          /* CUDA runtime error (message has the CUDA text) */
  IGM_ERR_OOM = -3,           /* device or host allocation failed */
  IGM_ERR_NOT_CONVERGED = -4, /* a spatial solve or MGRIT hit its cycle limit */
  IGM_ERR_TIMEOUT = -5,       /* a bounded device wait gave up */
  IGM_ERR_NUMERIC = -6        /* zero pivot in ILUT, NaN/Inf in a residual */
} igm_status;

typedef void* igm_stream; /* a cudaStream_t */

/* ---------------------------------------------------------------------------
 * Discretisation (Sec. 2).
 * ------------------------------------------------------------------------ */
typedef struct {
  int p;          /* B-spline order (Sec. 2, Cox--de Boor): 2..8 for iga_assemble,
                     1..8 for the host-side calls */
  int nel;        /* elements per direction (uniform open knot vector, span 1/nel) */
  int nquad;      /* Gauss points per direction per element; 0 -> p+1 */
  int geom;       /* 0: unit square (affine, F = identity);
                     1: B-spline geometry map given by gdeg, gn, gctrl */
  int gdeg[2];    /* geometry degrees (xi, eta) when geom == 1 */
  int gn[2];      /* control points per direction when geom == 1 */
  const double* gctrl; /* HOST, [gn[1]][gn[0]][2], xi fastest; uniform open knots */
  double kappa;   /* diffusion coefficient (Sec. 2, Eq. (heat)) */
} iga_desc;

typedef struct iga_ops iga_ops;

/* Assemble M, K (Sec. 2), the order-1 matrices on the same knots, the
 * transfer matrix P_1^p and the row-sum lumped masses (Sec. 4, Eq. (PM)) on
 * the host with Gauss quadrature, and upload them.  *out receives a handle.
 * Errors: IGM_ERR_ARG for p outside [2, 8], nel outside [4, 1024] or an
 * invalid geometry control net (the map is assumed regular: the quadrature
 * uses |det J|); IGM_ERR_CUDA without a device; IGM_ERR_OOM when the upload
 * fails. */
igm_status iga_assemble(const iga_desc* desc, iga_ops** out);
void iga_destroy(iga_ops* ops);

/* Sizes: n per direction, N = n*n unknowns, number of quadrature points of
 * the whole mesh (nel^2 * nquad^2) used by the two calls below. */
igm_status iga_sizes(const iga_ops* ops, int* n, int* N, int* nquad_points);

/* HOST [nqp][4] array of (xi, eta, x, y) at every quadrature point, in the
 * order the two calls below expect their function values. */
igm_status iga_quadrature_points(const iga_ops* ops, double* pts);

/* b_i = int_Omega f Phi_i (interior i) from HOST values fq[nqp] of f at the
 * quadrature points; writes DEVICE out[N]. */
igm_status iga_load_vector(const iga_ops* ops, const double* fq, double* out, igm_stream s);

/* The univariate B-spline basis of order p on the open uniform knot vector of
 * nel elements on [0, 1] (Sec. 2: the Cox--de Boor recursion, knots repeated
 * p+1 times at the ends), evaluated on the HOST; needs no device.  For each of
 * the nx HOST points x[i] in [0, 1]: span[i] = the index s of the knot span
 * holding x[i] (knots[s] <= x[i] < knots[s+1]; the last non-empty span at
 * x = 1), so that the nonzero functions are s-p .. s; N[i*(p+1) + k] and
 * dN[i*(p+1) + k] = the value and first derivative of function s-p+k (HOST
 * outputs [nx][p+1]; dN may be NULL).  The same code serves the assembly of
 * iga_assemble.  IGM_ERR_ARG for p outside [1, 8], nel < 1, a null array or a
 * point outside [0, 1]. */
igm_status iga_basis_eval(int p, int nel, int nx, const double* x, int* span, double* N,
                          double* dN);

/* The matrices iga_assemble builds (Sec. 2: M_ij = int phi_i phi_j, K_ij =
 * int grad phi_i . grad phi_j over the mapped domain, Gauss quadrature), on
 * the HOST; needs no device.  which = 0: M, 1: K, as stencils of the interior
 * unknowns (i = ix + n*iy): out[i*(2p+1)^2 + (dy+p)*(2p+1) + (dx+p)] = the
 * entry coupling i to (ix+dx) + n*(iy+dy), 0 where that point lies outside
 * the grid (HOST out [n*n*(2p+1)^2]); which = 2: the lumped masses (full-basis
 * row sums of M on the interior rows, HOST out [n*n]).  *n = interior
 * unknowns per direction; out may be NULL to query n.  The descriptor is
 * iga_assemble's, with p in [1, 8] and nel in [2, 1024]; IGM_ERR_ARG for
 * invalid input. */
igm_status iga_assemble_host(const iga_desc* desc, int which, int* n, double* out);

/* The transfer matrix of the p-multigrid (Sec. 4, Eq. (PM): P_ij = int phi_i
 * psi_j, phi of order p, psi of order 1 on the same knot spans and quadrature),
 * interior x interior, as iga_assemble builds it, on the HOST; needs no
 * device.  CSR over the N = n^2 order-p rows (ptr [N+1], col, val: columns are
 * the interior order-1 unknowns); call once with NULL arrays for *nnz, then
 * with arrays of that size.  The descriptor is iga_assemble's (p in [2, 8], nel in
 * [2, 1024]);
 * IGM_ERR_ARG for invalid input. */
igm_status iga_transfer_host(const iga_desc* desc, int* nnz, int* ptr, int* col, double* val);

/* Consistent L2 projection onto the spline space (Sec. 3: g^0 is u^0
 * projected onto V_{h,p}): solves M u = b(fq); writes DEVICE out[N]. */
igm_status iga_project(const iga_ops* ops, const double* fq, double* out, igm_stream s);

/* y = M x, y = K x (FP64) on a block of nrhs DEVICE columns with leading
 * dimension ld (column j at x + j*ld).  which: 0 = M, 1 = K. */
igm_status iga_apply(const iga_ops* ops, int which, int nrhs, const double* x, double* y,
                     long ld, igm_stream s);

/* Batched FP32 apply: y_b = M x_b (which = 0), K x_b (1) or (M + c K) x_b
 * (2) for b < nrhs, x, y DEVICE [nrhs][ld] FP32, ld >= N, any alignment, x
 * and y not overlapping; c is rounded to FP32.  The operator of Eq. (los)
 * applied to a block of right-hand sides such as the time points of an
 * interval.
 * Affine map (the unit square): sum factorisation (Sec. 2: M = M1 (x) M1,
 * K = K1 (x) M1 + M1 (x) K1) in shared memory: one persistent CTA per SM
 * pipelines its columns (one warp group streams a column in and contracts
 * along xi while the other contracts the previous column along eta).  Grids
 * the persistent layouts do not hold (n > 84; iga_apply_f32_layout reports
 * the plan) are applied by a row-strip form instead: each CTA stages a strip
 * of grid rows with p halo rows above and below for a group of columns (the
 * h = 1/128 grids); IGM_ERR_ARG when not even one grid row fits in shared
 * memory.
 * Curved map (a B-spline geometry, Sec. 2: M and K assembled): the
 * (2p+1)^2-point stencils of every grid point, held in FP32 on the device
 * since iga_assemble, coefficients of cm M + ck K formed once per CTA and
 * applied to four columns at a time. */
igm_status iga_apply_f32(iga_ops* ops, int which, double c, int nrhs, const float* x, float* y,
                         long ld, igm_stream s);

/* The shared-memory plan iga_apply_f32 uses for an n x n grid at order p on a
 * device with smem_max bytes of opt-in shared memory per block (HOST out[7]):
 * the grid-line cap of the chosen layout (68 or 84; 0 when the grid does not
 * fit and iga_apply_f32 refuses it), the copy-ring depth, grid lines per
 * thread, the padded row stride of the staged columns, the row stride and row
 * count of the (tm, tk) buffers, and the dynamic shared bytes per CTA.  Host
 * only (needs no device).  IGM_ERR_ARG for p outside [2, 8] or n < 1. */
igm_status iga_apply_f32_layout(int n, int p, long smem_max, int* out);

/* The launch plan of iga_apply_f32's other two forms for an n x n grid at
 * order p, nrhs columns, a device with sms SMs and smem_max bytes of opt-in
 * shared memory per block (HOST out; needs no device).  form 1, the row-strip
 * form (out[5]): rows per strip (0 when not even one row fits), threads per
 * CTA, dynamic shared bytes, strips (grid x), column groups (grid y).  form 2,
 * the curved form (out[6]): tile rows and columns, staged rows and columns
 * (the tile plus p halo lines on each side; two stages of float4 of them in
 * shared memory), tiles (grid x), column groups (grid y).  IGM_ERR_ARG for
 * invalid input. */
igm_status iga_apply_f32_plan(int form, int n, int p, int nrhs, int sms, long smem_max, int* out);

/* ---------------------------------------------------------------------------
 * p-multigrid (Sec. 4) for A = M + c K, c = kappa*dt.
 * ------------------------------------------------------------------------ */
typedef struct {
  int nu1, nu2;           /* pre/post ILUT smoothing steps (Sec. 4, steps 1 and 5) */
  double ilut_droptol;    /* ILUT drop tolerance relative to ||a_i||_2 (default 1e-12) */
  double ilut_fill;       /* ILUT fill factor: keep ceil(fill*nnz) per row part (default 1) */
  int hmg_coarsest_nel;   /* h-multigrid coarsening stops at this element count (default 8) */
  int precision;          /* 0: FP64 throughout; 1: FP32 smoothing, SpMM, transfers and
                             Gauss--Seidel, FP64 outer residual b - A x with iterative
                             refinement and FP64 coarsest p=1 direct solve */
  int inner_cycles;       /* precision 1: FP32 V-cycles per FP64 refinement step (default 1) */
  double tol;             /* spatial stop: ||b - A x||_2 <= tol ||b||_2 (default 1e-10) */
  int max_cycles;         /* cycle limit of one spatial solve (default 50) */
  int trace;              /* 1: accumulate SM clock cycles per solver phase (pmg_trace) */
  int solver;             /* 0: p-multigrid cycles (default); 1: conjugate gradients with a
                             diagonal preconditioner (the comparison solver of Sec. 5), always
                             in FP64 (precision is set to 0), one "cycle" = one CG iteration,
                             max_cycles = the iteration limit */
  int autotune;           /* 0: the fixed layout policy (default); 1: time the candidate layouts
                             of the ILUT sweeps (sweep team of 128 or 256 threads; arena in shared
                             memory, swept vector staged in shared memory, or everything in global
                             memory) on a probe solve at setup and keep the fastest */
  int layout;             /* 0: the fixed policy or autotune (default); 1..6 force one layout
                             of the ILUT sweeps (for tests and measurements): sweep teams of
                             128 (1..3) or 256 (4..6) threads, with the working vectors in
                             shared memory (1, 4), the swept vector staged in shared memory and
                             the working vectors in global memory (2, 5), or everything in
                             global memory (3, 6); pmg_setup returns IGM_ERR_ARG when the
                             forced layout does not fit in shared memory */
  int hmg_fp64;           /* precision 1 only: 0 (default) the p = 1 W-cycle (Gauss--Seidel,
                             residuals, bilinear transfers) in FP32 like the rest of the cycle,
                             with the coarsest direct solve in FP64; 1 the whole W-cycle in
                             FP64 (the order-p <-> order-1 transfers stay FP32) */
} pmg_opts;

typedef struct pmg_handle pmg_handle;

/* Fill *o with the defaults listed above. */
void pmg_default_opts(pmg_opts* o);

/* Build the p-multigrid hierarchy for A = M + kappa_dt K: ILUT factors in
 * natural order with their block-row (grid-row) form and dense
 * diagonal-block inverses, the p=1 operator and its Galerkin h-hierarchy
 * (9-point stencils), and the coarsest dense inverse.  Host setup plus one
 * upload.  Errors: IGM_ERR_ARG for invalid options or a mesh the p = 1
 * sweeps do not support (nel > 129), IGM_ERR_NUMERIC on a zero ILUT pivot or
 * a coarsest operator that is not positive definite, IGM_ERR_OOM/CUDA when
 * the upload fails. */
igm_status pmg_setup(const iga_ops* ops, double kappa_dt, const pmg_opts* opts, pmg_handle** out);
void pmg_destroy(pmg_handle* h);

/* Spatial solves on nrhs independent right-hand sides b (DEVICE, column j at
 * b + j*ld), updating the initial guesses x in place.  ncycles > 0: exactly
 * that many cycles (p-multigrid V-cycles in the FP64 form; FP64 refinement
 * steps of inner_cycles FP32 V-cycles in the mixed form); ncycles == 0: cycle
 * until the stop test holds or max_cycles.  cycles_out: HOST [nrhs] or NULL.
 * Synchronises the stream (the cycle counts and the status word are read
 * back).  Returns IGM_ERR_NOT_CONVERGED if some column hit max_cycles,
 * IGM_ERR_NUMERIC on a NaN residual, IGM_ERR_TIMEOUT if a bounded device wait
 * gave up (the solve was abandoned part way and x is incomplete). */
igm_status pmg_vcycle(pmg_handle* h, int nrhs, const double* b, double* x, long ld, int ncycles,
                      int* cycles_out, igm_stream s);

/* pmg_vcycle for callers that cannot allocate device memory.  This entry point
 * has no counterpart in the paper; it exists for users of the library whose
 * device memory is committed elsewhere (a host application that reserves
 * the GPU's memory up front for its own pool, or a real-time loop in which an
 * allocation would synchronise the device and break its timing): it calls no
 * cudaMalloc, cudaFree or other allocating routine.  Same arguments, results
 * and statuses as pmg_vcycle; the handle must already be set up (pmg_setup
 * allocates).  Its scratch (status word, per-column cycle counts, and the
 * per-column working vectors when they do not fit in shared memory) lives in
 * one static 16 MiB device buffer that every device which loads the library
 * holds until the process exits.  Calls needing more than 16 MiB of scratch
 * return IGM_ERR_ARG with the required size in igm_last_error().  The first
 * call looks up the buffer's device address on the current device (which
 * allocates nothing).  Like pmg_vcycle it synchronises the stream before it
 * returns, to read the status word back.  All calls share the buffer, which
 * keeps the last call's contents (the call clears what must start at zero):
 * calls that overlap on the GPU (other streams, other host threads) race. */
igm_status pmg_vcycle_static(pmg_handle* h, int nrhs, const double* b, double* x, long ld,
                             int ncycles, int* cycles_out, igm_stream s);

/* Block-row triangular sweeps with the ILUT factors (diagnostics and tests):
 * z = (L U)^{-1} r on nrhs DEVICE columns, in the handle's precision. */
igm_status pmg_ilut_apply(pmg_handle* h, int nrhs, const double* r, double* z, long ld,
                          igm_stream s);

/* Solver phases timed when opts.trace = 1 (SM clock cycles of CTA thread 0,
 * summed over all CTAs and calls since setup or the last reset). */
typedef enum {
  IGM_PH_RESIDUAL64 = 0,  /* FP64 residual b - A x and its norm */
  IGM_PH_RESIDUAL = 1,    /* residuals in the smoothing precision */
  IGM_PH_ILUT = 2,        /* ILUT sweeps L then U (Sec. 4, smoother) */
  IGM_PH_RESTRICT = 3,    /* restriction p -> 1 (Sec. 4, step 2) */
  IGM_PH_WCYCLE = 4,      /* h-multigrid W-cycle at p = 1 (Sec. 4, step 3) */
  IGM_PH_PROLONG = 5,     /* prolongation 1 -> p (Sec. 4, step 4) */
  IGM_PH_RHS = 6,         /* MGRIT step right-hand side M u + dt f */
  IGM_PH_GS = 7,          /* Gauss--Seidel sweeps inside the W-cycle */
  IGM_PH_ILUT_WAIT = 8,   /* ILUT, first sweep team: waits for its records and for the
                             preceding grid rows */
  IGM_PH_ILUT_OFF = 9,    /* ILUT, first sweep team: off-block couplings of its grid rows */
  IGM_PH_ILUT_DIAG = 10,  /* ILUT, first sweep team: diagonal-block products and row
                             completion */
  IGM_PH_GS_WAIT = 11,    /* Gauss--Seidel, warp 0: waits for the preceding grid row */
  IGM_PH_GS_ROW = 12,     /* Gauss--Seidel: couplings to later unknowns (all threads) */
  IGM_PH_GS_SCAN = 13,    /* Gauss--Seidel, warp 0: couplings to the preceding row, in-row
                             recurrence (warp scan) and stores */
  IGM_PH_COUNT = 14
} igm_phase;

/* The layout of the ILUT sweeps chosen at setup (HOST out[4]): threads per
 * sweep team, record ring slots, 1 if the working vectors are in shared
 * memory, 1 if the swept vector is staged in shared memory. */
igm_status pmg_layout(const pmg_handle* h, int* out);

/* Copy the accumulated phase clocks (HOST out[IGM_PH_COUNT]); reset = 1
 * zeroes them afterwards.  The handle must have been set up with trace = 1. */
igm_status pmg_trace(pmg_handle* h, long long* out, int reset);

/* Host copies of the ILUT factors in CSR (L strictly lower, U upper with the
 * diagonal), for pattern comparisons.  Pass NULL arrays to query sizes
 * (*nnz_l, *nnz_u).  Values are FP64. */
igm_status pmg_ilut_factors(const pmg_handle* h, int* nnz_l, int* nnz_u, int* l_ptr, int* l_col,
                            double* l_val, int* u_ptr, int* u_col, double* u_val);

/* The ILUT factorisation of pmg_setup (Sec. 4's smoother; dual threshold in
 * natural order, the drop tolerance relative to each row's 2-norm, at most
 * ceil(fill * nnz) entries per strictly-lower and strictly-upper row part),
 * applied to a caller's HOST CSR matrix of n rows (ptr[n+1], col, val; any
 * column order within a row).  Outputs as pmg_ilut_factors: L strictly lower,
 * U upper with the diagonal; call once with NULL arrays for *nnz_l, *nnz_u,
 * then with arrays of those sizes (l_ptr, u_ptr [n+1]).  Needs no device.
 * IGM_ERR_ARG for malformed CSR or parameters, IGM_ERR_NUMERIC for a zero pivot. */
igm_status pmg_ilut_host(int n, const int* ptr, const int* col, const double* val, double droptol,
                         double fill, int* nnz_l, int* nnz_u, int* l_ptr, int* l_col,
                         double* l_val, int* u_ptr, int* u_col, double* u_val);

/* The order-1 operator M_1 + kappa_dt K_1 of the p-multigrid's coarse
 * correction and its h-multigrid hierarchy as pmg_setup builds it (Sec. 4,
 * Fig. 5: bilinear prolongation, Galerkin coarse operators P^T A P, coarsening
 * while the element count is even and above coarsest_nel), on the HOST; needs
 * no device.  Level 0 is the operator on the descriptor's mesh.  *nlevels =
 * the number of h-levels; *n = interior nodes per direction of the level;
 * out (HOST [n*n*9], may be NULL) = its 9-point stencil, out[i*9 + (dy+1)*3 +
 * (dx+1)] coupling node i = ix + n*iy to (ix+dx) + n*(iy+dy), 0 outside the
 * grid.  The descriptor is iga_assemble's (its p only sets the quadrature
 * rule, p+1 points, unless nquad > 0).  IGM_ERR_ARG for invalid input or a
 * level beyond the coarsest. */
igm_status pmg_hmg_host(const iga_desc* desc, double kappa_dt, int coarsest_nel, int level,
                        int* nlevels, int* n, double* out);

/* The block-row form in which the ILUT sweeps consume a factor (Sec. 4's
 * smoother: L y = r and U z = y, solved one grid row at a time), on the HOST;
 * needs no device.  Input: an ILUT factor of an n x n grid of unknowns (N =
 * n^2, i = ix + n*iy) as HOST CSR (ptr[N+1], col, val): upper = 0: L strictly
 * lower (unit diagonal implied), upper = 1: U upper with the diagonal.
 * Outputs: the entries coupling to other grid rows as CSR (call once with
 * NULL arrays for *nnz_off, then with off_ptr [N+1] and arrays of that size),
 * and inv (HOST [n * n(n+1)/2], may be NULL) = the inverse of each grid row's
 * diagonal block, packed per block iy: for L, row r holds columns 0..r at
 * r(r+1)/2 + j; for U, row r holds columns r..n-1 at r*n - r(r-1)/2 + (j-r).
 * IGM_ERR_ARG for malformed input or an entry outside the triangle,
 * IGM_ERR_NUMERIC for a zero diagonal of U. */
igm_status pmg_block_tri_host(int n, int upper, const int* ptr, const int* col, const double* val,
                              int* nnz_off, int* off_ptr, int* off_col, double* off_val,
                              double* inv);

/* ---------------------------------------------------------------------------
 * MGRIT (Sec. 3).
 * ------------------------------------------------------------------------ */
typedef struct {
  double T;        /* final time */
  int Nt;          /* fine time steps */
  int m;           /* coarsening factor (Sec. 3: dt_C = m dt_F) */
  int max_levels;  /* time levels including the fine one (2 = two-level) */
  int min_coarse;  /* stop coarsening once a level has <= min_coarse steps; a level of N_l
                      steps coarsens to floor(N_l/m) (needs N_l >= m); when m does not divide
                      N_l its last N_l mod m points are F-points of a partial interval */
  int relax;       /* 0: F-relaxation, 1: FCF-relaxation (Sec. 3) */
  double tol;      /* stop when rho_k <= tol * rho_0 (C-point residual 2-norm) */
  int max_iter;    /* iteration limit */
  pmg_opts pmg;    /* spatial solver options used on every level */
  int initial_guess; /* 0: u_n = 0 for n >= 1; 1: start from the U passed in (a warm
                        restart from an earlier run's iterate; the stopping test is relative
                        to this run's first residual, so a restart aiming at the original
                        target passes tol scaled by the earlier run's residual reduction) */
  int graphs;      /* 1: replay each iteration's launches as CUDA graphs (default 1) */
  int profile;     /* 1: record CUDA events around every sweep launch (mgrit_profile) */
  double theta;    /* theta-scheme of Sec. 2, Eq. (los): 1 backward Euler (default),
                      0.5 Crank-Nicolson, 0 forward Euler; in [0, 1] */
  int cycle;       /* MGRIT hierarchy (Sec. 5): 0 V-cycle (default), 1 F-cycle, 2 W-cycle */
  int priority;    /* scheduling priority of the handle's work against other work on the
                      GPU: 0 normal (default), k > 0 k levels more urgent (clamped to the
                      device's range of stream priorities) */
  int coarse_cycles; /* spatial solves on the coarse time levels: 0 = to pmg.tol like the
                        fine level (default); k > 0 = exactly k p-multigrid cycles (an
                        inexact coarse propagator; the fine level, and with it the
                        converged answer, is unchanged) */
  int fused;       /* 1 (default): with FCF relaxation, the relaxation phases of one visit
                      of a level (F, C, F + C-point residual) run as one cooperative launch
                      of one CTA per interval with a bounded grid-wide barrier between the
                      phases, when all the level's CTAs can be resident at once (else, and
                      with 0, one launch per phase); results are identical either way */
} mgrit_opts;

typedef struct {
  int iters;             /* MGRIT iterations (coarse corrections) done */
  int levels;            /* time levels used */
  double res_hist[256];  /* rho_k, k = 0..iters (fine-level C-point residual norms) */
  double vcyc_mean;      /* mean cycles per spatial solve */
  long solves;           /* spatial solves done (all levels, all columns) */
  long vcycles;          /* cycles done (all solves) */
  double seconds;        /* wall time of the iteration loop (setup excluded) */
  double setup_seconds;  /* p-multigrid setup of all levels */
  long launches;         /* kernel launches of the run */
  int coarse_fallback;   /* 1 if a learned coarse propagator was replaced by backward Euler */
} mgrit_stats;

typedef struct mgrit_handle mgrit_handle;

void mgrit_default_opts(mgrit_opts* o);

/* Set up MGRIT (Sec. 3) for the time grid in opts: the level hierarchy
 * dt_l = m^l dt, one p-multigrid hierarchy per level (rediscretised operator
 * M + theta kappa dt_l K; the step's right-hand side uses
 * M - (1 - theta) kappa dt_l K), and the device work buffers.  Host setup plus uploads;
 * no solve.  The handle keeps a pointer to ops, which must outlive it. */
igm_status mgrit_create(const iga_ops* ops, const mgrit_opts* opts, mgrit_handle** out);
void mgrit_destroy(mgrit_handle* mg);

/* Solve the space-time system of Sec. 3 by MGRIT with the handle's options.
 * u0: DEVICE [N] initial coefficients (g^0); fhat: DEVICE [N] load vector of
 * the spatial source profile or NULL; fcoef: HOST [Nt+1] time factors c(t_n)
 * of a separable source f(x,t) = c(t) fhat(x) or NULL; U: DEVICE [Nt+1][N],
 * caller-owned, receives all time levels (U[0] = u0).  Reads one FP64 vector
 * of C-point residual norms back per iteration for the stopping test.
 * Returns IGM_ERR_NOT_CONVERGED when max_iter is reached first (or a spatial
 * solve hit its cycle limit), IGM_ERR_NUMERIC on a NaN residual,
 * IGM_ERR_TIMEOUT if a bounded device wait gave up (U is then incomplete). */
igm_status mgrit_run(mgrit_handle* mg, const double* u0, const double* fhat, const double* fcoef,
                     double* U, mgrit_stats* stats, igm_stream s);

/* Run nprob independent MGRIT solves (each as mgrit_run on its own handle,
 * with its own problem size, order, time grid and kappa) concurrently: every
 * handle works on its own internal stream, replaying its iteration graphs,
 * and one host thread advances whichever problem's fine-level relaxation has
 * finished (the stopping test of Sec. 3 needs one norm read-back per
 * iteration).  Arrays of length nprob: mgs (distinct handles), u0, U (DEVICE
 * pointers as in mgrit_run), fhat and fcoef (either array pointer may be NULL
 * for no sources; entries as in mgrit_run), stats (HOST, may be NULL),
 * latency_ms (HOST, may be NULL): per problem the time from the start of the
 * batch on stream s to the end of that problem's solve, measured with CUDA
 * events (-1 for a problem that failed).  All problems run to the end;
 * returns the first non-OK status in problem order.  There is no counterpart
 * in the paper: it schedules several of the paper's solves on one GPU. */
igm_status mgrit_run_batched(int nprob, mgrit_handle* const* mgs, const double* const* u0,
                             const double* const* fhat, const double* const* fcoef,
                             double* const* U, mgrit_stats* stats, float* latency_ms,
                             igm_stream s);

/* The same batch as mgrit_run_batched in ONE persistent kernel launch, with
 * no host scheduler: each member's run is a program of phases (the sweeps of
 * Sec. 3's relaxation, residual, coarse visits and correction, and the
 * stopping test after every fine-level residual), and one CTA per SM
 * repeatedly claims a task (one interval of the current phase of a member;
 * members are scanned in array order, so put the short ones first for
 * shortest-job-first service); the CTA that completes a phase's last task
 * moves that member on, and the stopping test runs on the device from the
 * device-side residual norms.  No task waits for another; an idle CTA gives
 * up (IGM_ERR_TIMEOUT) after about a second in which no task completed.
 * Results are bit-identical to mgrit_run of each member.  All members must
 * use the same precision and no learned coarse propagator.  latency_ms: per
 * member, the time from the launch's start to the end of its run (device
 * clock).  stats[i].launches = 1 (the batch's single launch).  There is no
 * counterpart in the paper. */
igm_status mgrit_run_batched_device(int nprob, mgrit_handle* const* mgs, const double* const* u0,
                                    const double* const* fhat, const double* const* fcoef,
                                    double* const* U, mgrit_stats* stats, float* latency_ms,
                                    igm_stream s);

/* ---------------------------------------------------------------------------
 * Learned coarse propagator Phi_c (no counterpart in the paper, whose coarse
 * levels rediscretise the time step, Sec. 3).  A convolutional network on the
 * n x n grid of interior coefficients (zero padding: the homogeneous
 * Dirichlet condition), BF16 weights and activations with FP32 accumulation
 * (the C -> C layers, their input gradients and weight gradients on the
 * tensor cores):
 *   x = u / s, s = max |u|;  h1 = g(K1 * x), h2 = g(K2 * h1), h3 = g(K3 * h2),
 *   Phi_c(u) = u + s * K4 * h3,  g(z) = z (1 + erf(z / sqrt 2)) / 2 (GELU),
 * K1: 1 -> C, K2, K3: C -> C, K4: C -> 1 channels, 3 x 3 kernels, no biases.
 * Weights (FP32 master copy) in one array [K1 (C,1,3,3) | K2 (C,C,3,3) |
 * K3 (C,C,3,3) | K4 (1,C,3,3)] of count = 9 (2C + 2C^2) floats, the last two
 * indices the kernel row (eta) and column (xi).
 * ------------------------------------------------------------------------ */
typedef struct phic_handle phic_handle;

/* n = interior coefficients per direction, channels C = 32 (16 for small
 * tests); K1, K2, K3 random (seeded), K4 = 0 (the network starts as the
 * identity). */
igm_status phic_create(int n, int channels, unsigned long long seed, phic_handle** out);
void phic_destroy(phic_handle* h);
/* HOST w[count]; phic_get_weights also returns count (w may be NULL). */
igm_status phic_set_weights(phic_handle* h, const float* w);
igm_status phic_get_weights(const phic_handle* h, float* w, int* count);
/* out_b = Phi_c(u_b) for nb DEVICE vectors of n*n FP64 values (row strides ldu, ldo). */
igm_status phic_apply(phic_handle* h, int nb, const double* u, long ldu, double* out, long ldo,
                      igm_stream s);
/* Train on npairs DEVICE pairs (U0 row b -> U1 row b, stride ld, FP64): each
 * pair is normalised by max |U0_b|; mean squared error of Phi_c(U0_b)/s -
 * U1_b/s over minibatches of `batch` pairs drawn uniformly (seeded), `steps`
 * Adam steps (beta 0.9, 0.999, eps 1e-8) with learning rate lr.  loss: HOST
 * [steps] per-step minibatch losses, or NULL.  Synchronises the stream. */
igm_status phic_train(phic_handle* h, int npairs, const double* U0, const double* U1, long ld,
                      int steps, int batch, double lr, unsigned long long seed, double* loss,
                      igm_stream s);
/* The loss of phic_train on the nb pairs (U0 row b -> U1 row b, DEVICE, stride
 * ld, normalised by max |U0_b|) as one minibatch, and its gradient by back
 * propagation with the current weights: HOST *loss, gw[count] (the weight
 * gradient, master layout), gx[nb][n*n] (the gradient with respect to the
 * normalised inputs U0_b / s_b; may be NULL).  No weight update.
 * Synchronises the stream. */
igm_status phic_grad(phic_handle* h, int nb, const double* U0, const double* U1, long ld,
                     double* loss, float* gw, float* gx, igm_stream s);
/* Use h (NULL: backward Euler again) as the coarse propagator of a two-level
 * MGRIT handle (max_levels = 2), with the FAS coarse equation
 * tau_j = u_{jm} - Phi_c(u_{(j-1)m}) + r_j, v_j = Phi_c(v_{j-1}) + tau_j.  The
 * fine propagator is unchanged, so the converged answer is sequential
 * stepping.  When the residual after a learned correction is not finite or
 * its contraction rho_k / rho_{k-1} exceeds switch_ratio (0.5 recommended),
 * that correction is undone (the iterate before it is restored and relaxed
 * again) and the run continues with the backward-Euler coarse level
 * (mgrit_stats.coarse_fallback = 1).  The handle h must outlive the MGRIT
 * handle's use of it. */
igm_status mgrit_set_coarse_propagator(mgrit_handle* mg, phic_handle* h, double switch_ratio);

/* One-shot convenience: mgrit_create + mgrit_run + mgrit_destroy. */
igm_status mgrit_solve(const iga_ops* ops, const mgrit_opts* opts, const double* u0,
                       const double* fhat, const double* fcoef, double* U, mgrit_stats* stats,
                       igm_stream s);

/* Per-launch record of the last mgrit_run with opts.profile = 1:
 * HOST arrays of capacity cap: level, grid (CTAs), mode, duration in ms and
 * spatial cycles done by the launch.  Returns the number of launches recorded
 * in *count (at most cap). */
igm_status mgrit_profile(const mgrit_handle* mg, int cap, int* count, int* level, int* grid,
                         int* mode, float* ms, long* cycles);

/* Failure-detection self-test: launches one kernel whose bounded mbarrier
 * wait (the same wait the solver uses for its streamed factor records) has
 * nothing to wait for; after `spins` polls the kernel records the timeout and
 * returns, and the call returns IGM_ERR_TIMEOUT with the device still usable.
 * Returns IGM_OK only if the wait completed, which would be a fault. */
igm_status igm_wait_selftest(long spins, igm_stream s);

/* Failure-detection self-test of the grid-wide barrier that separates the
 * phases of a fused level visit (mgrit_opts.fused): nctas CTAs in one
 * cooperative launch pass two barriers.  hold = 0: returns IGM_OK.  hold = 1:
 * CTA 0 does not arrive at the first barrier, so every CTA's bounded wait runs
 * out after wait_cycles SM clocks; the kernel records the timeout and returns,
 * and the call returns IGM_ERR_TIMEOUT with the device still usable.
 * IGM_ERR_ARG for nctas outside [1, 1024] or wait_cycles < 1. */
igm_status igm_grid_barrier_selftest(int nctas, long long wait_cycles, int hold, igm_stream s);

/* Thread-local text of the last error (empty string if none). */
const char* igm_last_error(void);

/* Number of device kernel launches issued by this library since load
 * (all entry points, all threads). */
long igm_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* IGAMGRIT_H */
