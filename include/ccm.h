/*
 * ccm.h -- C ABI of the GB300 fourth-order cut-cell elliptic solver.
 *
 * Problem (Sec. 1, eq. ccEllipticEq; Sec. 3.3 boundary operators):
 *     a u_x1x1 + b u_x1x2 + c u_x2x2 = f   in Omega,   b^2 - 4ac < 0,
 *     u = g (Dirichlet)  or  n . grad u = g (Neumann, n the outward unit normal)  on dOmega,
 * discretised on the Cartesian cells of the box R = [x0, x0 + nx h] x [y0, y0 + ny h] by the
 * paper's fourth-order finite-volume cut-cell method (Sec. 3): cell averages of u and f,
 * boundary-piece averages of g, L u + N g = f (eq. PoissonLinearDiscretization), solved by a
 * geometric multigrid on the level hierarchy of Sec. 4.
 *
 * Conventions shared by every entry point:
 *   - Cell (i, j) is (x0 + i h, x0 + (i+1) h) x (y0 + j h, y0 + (j+1) h); cell arrays are
 *     row-major [ny][nx] (i fastest), one FP64 value per Cartesian cell.  Empty cells and cells
 *     merged into a neighbour by Alg. 1 are ignored on input and written as 0 on output; a
 *     merged cell's value lives at its survivor (see ccm_cell_map).
 *   - Boundary data: one FP64 value per boundary segment, in the order of
 *     ccm_boundary_segments.  A segment is the whole boundary piece S_i of one (survivor)
 *     cell, box-wall edges included when the box is part of dOmega.
 *   - Array arguments of ccm_apply / ccm_apply_T / ccm_solve / ccm_solve_T and the level
 *     entry points are DEVICE pointers on the current device unless a parameter says
 *     "host".  The caller owns every buffer it passes; the handle owns its level arrays and
 *     work space.  A handle is used from one stream at a time.
 *   - stream is a cudaStream_t (0 = legacy default stream); calls are asynchronous on it
 *     unless documented otherwise.
 *   - Return value: 0 on success, a negative CCM_E* code otherwise (ccm_strerror names it).
 *     Invalid arguments are rejected before any work is queued.
 */
#ifndef CCM_H
#define CCM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* curve kinds: parameters p[] (t in [0, 2 pi), counter-clockwise)
 *   CCM_CIRCLE  p = (cx, cy, r)              gamma = c + r (cos t, sin t)
 *   CCM_ELLIPSE p = (cx, cy, a, b, phi)      gamma = c + Rot(phi) (a cos t, b sin t)
 *   CCM_STAR    p = (cx, cy, r0, amp, k)     gamma = c + (r0 + amp cos k t)(cos t, sin t)
 *   CCM_POLYGON pts = (x0, y0, ..., x_{n-1}, y_{n-1}), npts = n >= 3 vertices in
 *               counter-clockwise order, no self-intersection; edge k is traversed at
 *               constant speed for t in [2 pi k / n, 2 pi (k + 1) / n), so corners are kinks
 *               of gamma and every integral along a piece is split there
 *   CCM_SPLINE  pts, npts as for CCM_POLYGON: the periodic cubic spline through the points
 *               (each coordinate), knots at the cumulative chord lengths scaled to [0, 2 pi)
 *               (boundaries of the Yin sets Y_c, Sec. 2); integrals are split at the knots */
enum { CCM_CIRCLE = 1, CCM_ELLIPSE = 2, CCM_STAR = 3, CCM_POLYGON = 4, CCM_SPLINE = 5 };
/* boundary conditions (Sec. 3.3): NONE only for box_bc (the box is not part of dOmega);
 * ROBIN (curves only) is gamma1 u + gamma2 du/dn = g with the curve's robin[] = (gamma1,
 * gamma2), n the unit normal pointing out of Omega */
enum { CCM_NONE = 0, CCM_DIRICHLET = 1, CCM_NEUMANN = 2, CCM_ROBIN = 3 };
/* arithmetic of the multigrid cycle */
enum { CCM_FP64 = 0, CCM_MIXED = 1 };

enum {
  CCM_OK = 0,
  CCM_EINVAL = -1,     /* null pointer, b^2-4ac >= 0, h <= 0, bad sizes, nx/ny not divisible */
  CCM_EGEOM = -2,      /* curve leaves the box, mixed BC types (or Robin coefficients) in one
                          cell, isolated pieces */
  CCM_EPLG = -3,       /* no poised stencil within the search radius */
  CCM_ESINGULAR = -4,  /* zero pivot in a block or bottom factorisation */
  CCM_ENOCONV = -5,    /* max_iter reached; u holds the last iterate */
  CCM_ETIMEOUT = -6,   /* a bounded device wait ran out */
  CCM_ECUDA = -7,      /* a CUDA runtime call failed */
  CCM_ENOMEM = -8,     /* device or host allocation failed */
  CCM_ENOTFINITE = -9, /* a residual norm became NaN or Inf */
  CCM_ETOOLARGE = -10  /* the grid does not fit the fixed scratch of ccm_apply_noalloc */
};

typedef struct {
  int kind;        /* CCM_CIRCLE | CCM_ELLIPSE | CCM_STAR */
  double p[8];     /* parameters, see above */
  int orient;      /* +1: Omega lies inside the curve; -1: the curve bounds a hole */
  int bc;          /* CCM_DIRICHLET | CCM_NEUMANN | CCM_ROBIN */
  double robin[2]; /* CCM_ROBIN: (gamma1, gamma2), finite, not both zero; ignored otherwise */
  int npts;        /* CCM_POLYGON, CCM_SPLINE: point count; ignored otherwise */
  const double* pts; /* CCM_POLYGON, CCM_SPLINE: host array of 2 npts coordinates (copied) */
} ccm_curve;

typedef struct {
  double a, b, c;          /* constant coefficients, b^2 - 4ac < 0 */
  double x0, y0, h;        /* box origin and cell size */
  int nx, ny;              /* cells per side */
  int box_bc;              /* CCM_DIRICHLET | CCM_NEUMANN | CCM_NONE */
  int ncurves;
  const ccm_curve* curves; /* host array of ncurves curves (copied by ccm_setup) */
} ccm_problem;

typedef struct {
  double omega;      /* weight of the Jacobi smoother SMO-1 (Sec. 4.1) */
  int nu1, nu2;      /* pre- and post-smoothing sweeps (Alg. 2) */
  double theta;      /* merging threshold of Alg. 1 */
  int coarsest;      /* the hierarchy stops at the first level with <= coarsest cells per side */
  int precision;     /* CCM_FP64 | CCM_MIXED (FP32 cycles inside FP64 refinement) */
  double rtol;       /* stop when ||r - L u||_inf <= rtol ||r||_inf, r = f - N g */
  int max_iter;      /* outer iterations (V-cycles) */
  int ras_passes;    /* passes of the overlapping block solve used for SMO-2 */
  int ras_block;     /* core size of an SMO-2 block (unknowns) */
  int ras_overlap;   /* overlap of an SMO-2 block on each side (unknowns) */
  int nthreads;      /* host threads for ccm_setup (0 = all cores) */
  int ras_exact;     /* levels with at most this many irregular cells use one exact block */
  int inner_cycles;  /* CCM_MIXED: FP32 V-cycles per FP64 residual evaluation */
  int smoother;      /* 0: SMO-1 then SMO-2 from the new regular values (Sec. 4.1, two launches);
                        1: block-Jacobi form, both from the old iterate (one launch per sweep) */
  int coarse_n;      /* levels with at most coarse_n cells a side run their part of every V-cycle
                        as one launch of one thread-block cluster (16 or 8 CTAs of 1024
                        threads, cluster barriers between the phases of Alg. 2); smoother 1
                        with ras_passes <= 1 only; 0: never */
  int batch;         /* CCM_MIXED: right-hand sides ccm_solve advances together (1 - 4096).
                        The handle's FP32 work arrays and its level-0 FP64 iterate and
                        right-hand side hold `batch` copies, and every kernel launch of an
                        outer iteration covers all of them (the right-hand side is the
                        grid's y index).  Needs the persistent kernels on every level of
                        64^2 cells or more, the block-Jacobi smoother and coarse_n 0; else
                        the handle runs one right-hand side at a time (ccm_info.batch). */
  int cycle;         /* CCM_MIXED: 0, every inner cycle of an outer iteration is a V-cycle
                        (Alg. 2); 1, the first one is an FMG cycle (Sec. 4, the FMG figure:
                        the residual restricted to the bottom level, then one V-cycle per
                        level from the prolonged coarse solution) and the others V-cycles. */
  int setup_device;  /* ccm_setup: 1, the weighted least-squares fits of every candidate PLG
                        stencil (Sec. 3.3) and the condition numbers of the chosen ones run on
                        the GPU (one warp per stencil), the candidates being enumerated on host
                        threads; 0, everything on host threads.  Same stencils either way,
                        coefficients equal to rounding. */
  int krylov;        /* CCM_MIXED: 0, the correction of an outer iteration is the inner cycles'
                        result e = M r (plain iterative refinement); m in 1 - 8, it is the
                        GMRES(m) solution of L e = r with M as right preconditioner (m
                        applications of M, FP32 basis, FP64 dot products, all on the device),
                        for problems where the cycle alone converges slowly or not at all.
                        One right-hand side at a time (ccm_info.batch = 1). */
} ccm_params;

typedef struct {
  int nx, ny, levels;
  int64_t n_cells;      /* non-empty (survivor) cells on the finest level */
  int64_t n_regular;    /* regular cells (finest level) */
  int64_t n_irregular;  /* irregular cells (finest level) */
  int64_t n_segments;   /* boundary segments (finest level) */
  int64_t device_bytes; /* device memory held by the handle */
  double setup_ms;      /* host + upload time of ccm_setup */
  double plg_cond_max;  /* largest 2-norm condition number of a chosen FV sample matrix */
  int batch;            /* right-hand sides ccm_solve advances together (1 unless params.batch > 1
                           and the conditions stated there hold) */
  /* wall time of the phases of ccm_setup (ms), the columns of the paper's setup tables:
   * cut cells, moments and merging of every level (Sec. 3.1, Alg. 1); PLG stencils and
   * weighted fits (Sec. 3.3); the boundary order of Alg. 3 with the SMO-2 block inverses and
   * the packing; the coarsest level's dense inverse; the upload and device configuration */
  double setup_geometry_ms, setup_fits_ms, setup_blocks_ms, setup_bottom_ms, setup_upload_ms;
} ccm_info;

typedef struct {
  int iterations;           /* outer iterations (V-cycles) performed */
  double rel_residual;      /* ||r - L u||_inf / ||r||_inf at exit (FP64) */
  double history[64];       /* relative residual after each iteration (first 64) */
} ccm_stats;

typedef struct ccm_handle ccm_handle;
typedef struct ccm_group ccm_group;

/* Fill p with the defaults: omega 0.7, nu1 = nu2 = 3, theta 0.3, coarsest 16, CCM_MIXED,
 * rtol 1e-10, max_iter 100, ras_passes 1, ras_block 64, ras_overlap 24, nthreads 0,
 * ras_exact 0, inner_cycles 3, smoother 1, coarse_n 0, batch 1, cycle 0, setup_device 1, krylov 0. */
int ccm_default_params(ccm_params* p);

/* Host setup (Sec. 3.1 - 3.4, Sec. 4): cut cells and moments (Green's formula, Sec. 2.4),
 * Alg. 1 merging, regular/irregular classification, PLG stencils and weighted min-norm
 * fits (eq. derivedCoefAgain) on every level h 2^m, the boundary ordering of Alg. 3, and the
 * upload of the packed level arrays to the current device.  params may be NULL (defaults).
 * Blocking; *out receives a new handle, release it with ccm_free.  Errors: CCM_EINVAL,
 * CCM_EGEOM, CCM_EPLG, CCM_ESINGULAR, CCM_ENOMEM, CCM_ECUDA. */
int ccm_setup(const ccm_problem* prob, const ccm_params* params, ccm_handle** out);

/* Sizes and statistics of a handle (host struct). */
int ccm_query(const ccm_handle* h, ccm_info* info);

/* Host arrays describing the finest level:
 *   status[ny*nx]: 0 empty (or merged away), 1 pure, 2 cut / merged survivor;
 *   owner[ny*nx]: linear index of the cell that holds this cell's unknown (-1 if empty);
 *   regular[ny*nx]: 1 for regular cells (eq. stdLap stencil), 0 otherwise;
 *   vol[ny*nx]: volume of the (merged) cut cell in units of h^2.
 * Any pointer may be NULL.  Blocking. */
int ccm_cell_map(const ccm_handle* h, int8_t* status, int32_t* owner, int8_t* regular, double* vol);

/* Boundary segments of the finest level in ĝ order (host arrays of n_segments, any may be
 * NULL): cell = linear index of the owning cell, bc = CCM_DIRICHLET | CCM_NEUMANN | CCM_ROBIN,
 * length = arc length of the piece (physical units).  Blocking. */
int ccm_boundary_segments(const ccm_handle* h, int32_t* cell, int32_t* bc, double* length);

/* Boundary operator of every finest-level segment in the general form gamma1 u + gamma2 du/dn
 * (Sec. 3.3): gamma[2 s] = gamma1, gamma[2 s + 1] = gamma2 of segment s (host array of
 * 2 n_segments): (1, 0) for Dirichlet, (0, 1) for Neumann, the curve's robin[] for Robin.
 * The boundary datum g of a segment is the average of that operator applied to u.  Blocking. */
int ccm_boundary_robin(const ccm_handle* h, double* gamma);

/* Fitted rows of level `level` of the handle (host arrays, any may be NULL; call with NULL
 * arrays to read *n_rows first): cell[n] the row's cell, cols[n][15] its stencil cells
 * (linear indices of that level's grid), beta[n][15] the coefficients and nb[n] the boundary
 * coefficient in physical units, seg[n] the boundary segment or -1.  The same layout as
 * ccm_host_rows, so that a handle's setup can be compared with the host-only one. */
int ccm_level_rows(const ccm_handle* h, int level, int64_t* n_rows, int32_t* cell, int32_t* cols, double* beta,
                   double* nb, int32_t* seg);

/* Quadrature rules that reproduce the averages the discretisation expects (Sec. 3.2,
 * eq. iteratedIntegral): for every non-pure non-empty cell, nodes and weights whose weighted
 * sum over f is the integral of f over the (merged) cut cell; for every boundary segment,
 * nodes, arc-length weights and outward unit normals along its pieces.  Pure cells are plain
 * squares (ccm_cell_averages applies a tensor Gauss rule to them).  Call with NULL arrays to get the counts
 * in *n_cell_nodes / *n_bdry_nodes, then again with host arrays of those sizes:
 *   cell_of[n]: linear cell index, cxy[2n]: (x, y), cw[n]: weight (area units);
 *   seg_of[m]: segment index, bxy[2m]: (x, y), bw[m]: weight (length), bn[2m]: normal. */
int ccm_quadrature(const ccm_handle* h, int64_t* n_cell_nodes, int64_t* n_bdry_nodes,
                   int32_t* cell_of, double* cxy, double* cw,
                   int32_t* seg_of, double* bxy, double* bw, double* bn);

/* Input averages the discretisation expects (Sec. 3.2, eq. iteratedIntegral), with the
 * caller's functions evaluated at the library's nodes.  The library calls f (or g) with host
 * arrays of n node coordinates, possibly several times, and the function fills out[0, n):
 *   ccm_field_fn: out = f(x, y);
 *   ccm_grad_fn:  u, ux, uy = u(x, y) and its gradient.
 * ccm_cell_averages: out[ny][nx] (host) = the average of f over every non-empty (survivor)
 *   cell: the 5 x 5 tensor Gauss rule on pure cells, the cut-cell rule of ccm_quadrature on
 *   cut and merged cells; 0 on the other cells.
 * ccm_boundary_averages: out[n_segments] (host) = the average over every boundary segment of
 *   its operator gamma1 u + gamma2 du/dn (ccm_boundary_robin; n the outward unit normal), by
 *   the rule of ccm_quadrature along the segment's pieces.
 * Blocking, host only.  Errors: CCM_EINVAL (NULL arguments). */
typedef void (*ccm_field_fn)(void* ctx, int64_t n, const double* x, const double* y, double* out);
typedef void (*ccm_grad_fn)(void* ctx, int64_t n, const double* x, const double* y, double* u, double* ux,
                            double* uy);
int ccm_cell_averages(const ccm_handle* h, ccm_field_fn f, void* ctx, double* out);
int ccm_boundary_averages(const ccm_handle* h, ccm_grad_fn g, void* ctx, double* out);

/* out = L u + N g (eq. PoissonLinearDiscretization) on the finest level, physical units.
 * u, out: device [nrhs][ny][nx] FP64; g: device [nrhs][n_segments] FP64 (may be NULL: g = 0).
 * Runs in FP64 (regular stencil, Sec. 3.2; fitted irregular rows, eq. goalOfApproximation). */
int ccm_apply(ccm_handle* h, const double* u, const double* g, double* out, int nrhs, void* stream);

/* Allocation-free operator application.  Same result as ccm_apply with nrhs = 1
 * (out = L u + N g on the finest level, physical units; u, out: device [ny][nx] FP64, g:
 * device [n_segments] FP64 or NULL).  It is for callers that must not allocate device memory
 * at call time: a host framework whose caching allocator owns all device memory (a second
 * allocator beside it fragments the device and can fail where the framework would not), or a
 * latency-bound loop that cannot afford cudaMalloc / cudaFree, which may synchronise the
 * device.  The handle is set up beforehand, and its device must be the current device
 * (CCM_EINVAL otherwise, before any work is queued).  Unlike ccm_apply, this call does not use
 * the handle's work arrays.  It uses a fixed file-scope device array (the library keeps
 * CCM_NOALLOC_SCRATCH_BYTES = 16 MiB on every device that loads it, until the process exits).
 * That array holds two padded FP64 grids of at most CCM_NOALLOC_MAX_PADDED cells each, where
 * the padded size is ((nx + 4) rounded up to a multiple of 32) * (ny + 4); larger grids are
 * rejected with CCM_ETOOLARGE before any work is queued.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.  The first call on a device looks up the array's device address
 * (once per device), so make that first call before any stream capture.  Every call shares
 * the array, so calls that overlap on the GPU (other streams, other handles) race; the call
 * clears the part of the array it uses before filling it.  The paper has no counterpart of
 * this entry point: it exists for the memory model of its callers. */
#define CCM_NOALLOC_MAX_PADDED (1L << 20)
#define CCM_NOALLOC_SCRATCH_BYTES (2L * CCM_NOALLOC_MAX_PADDED * 8L)
int ccm_apply_noalloc(const ccm_handle* h, const double* u, const double* g, double* out, void* stream);

/* Transposed operator: out_u = L^T v, out_g = N^T v (either may be NULL).  v, out_u:
 * device [nrhs][ny][nx]; out_g: device [nrhs][n_segments]; FP64.  Uses the point-symmetric
 * regular stencil on regular rows and a precomputed transposed CSR of the fitted rows. */
int ccm_apply_T(ccm_handle* h, const double* v, double* out_u, double* out_g, int nrhs, void* stream);

/* Solve L u = f - N g (eq. PoissonResidualForm) by V-cycles (Alg. 2) to rtol.  One outer
 * iteration (CCM_FP64: one FP64 V-cycle; CCM_MIXED: inner_cycles FP32 V-cycles on the FP32
 * image of the FP64 residual, then u += e in FP64) runs as one CUDA graph, captured on the
 * first call; the FP64 residual norm is read back after every outer iteration.
 * f: device [nrhs][ny][nx] cell averages; g: device [nrhs][n_segments] (NULL: g = 0);
 * u: device [nrhs][ny][nx], in: initial guess, out: solution.  CCM_MIXED handles with
 * ccm_info.batch > 1 advance up to that many right-hand sides per graph replay, until the
 * worst of them meets rtol (the others iterate on).  stats (host, nullable) receives the
 * outer iteration count of the last group and, per iteration, the largest relative residual
 * of its right-hand sides.
 * Synchronises the stream once per outer iteration (the convergence test).  The first call
 * captures the graphs, so make it outside any caller's stream capture.
 * Errors: CCM_ENOCONV (u holds the last iterate), CCM_ENOTFINITE, CCM_ECUDA. */
int ccm_solve(ccm_handle* h, const double* f, const double* g, double* u, int nrhs,
              void* stream, ccm_stats* stats);

/* ccm_solve with HOST arrays: f [nrhs][ny][nx], g [nrhs][n_segments] (may be NULL) and u
 * [nrhs][ny][nx] (in: initial guess, out: solution) in host memory, same layouts.  Pinned host
 * memory (cudaHostAlloc, cudaHostRegister, a pinned torch tensor) is read and written by the
 * packing kernels directly over the host link, with no staging copy: only the non-empty
 * cells of f and u are read and only the non-empty cells of u are written (the cells outside
 * the domain hold no unknown and keep the values the caller's u had there; ccm_solve sets
 * them to 0).  Pageable memory is accessed the
 * same way where the device reads pageable memory coherently (Grace systems), else through
 * device staging buffers and copies.  Device pointers are accepted too.  Returns after u
 * is complete on the host (the stream is synchronised).  Errors as ccm_solve, plus
 * CCM_ENOMEM for a staging buffer. */
int ccm_solve_host(ccm_handle* h, const double* f, const double* g, double* u, int nrhs,
                   void* stream, ccm_stats* stats);

/* Many problems, one graph launch.  A group holds `count` set-up handles (distinct; each
 * its own geometry, grid size, coefficients and precision) and one CUDA graph in which the
 * outer iterations of all of them run: a device-side loop that, per pass, runs the outer
 * iteration of every member whose relative residual is still above its rtol (and below
 * its max_iter), each member's work on its own branch of the graph, then a one-thread-block
 * kernel that reads the members' FP64 residual norms and retires the converged ones.  The
 * arithmetic of a member is that of ccm_solve with one right-hand side; only the
 * convergence test moves from the host to the device.
 * ccm_group_create captures every member's iteration (it synchronises `stream` and uses
 * each member's private capture stream; call it outside any stream capture, after
 * ccm_set_cycle_params).  members[] is copied; the handles must outlive the group, and no
 * other call may use them while a group solve is in flight.  Errors: CCM_EINVAL (NULL, a
 * handle given twice), CCM_ENOMEM, CCM_ECUDA (the runtime rejected the graph).
 * ccm_group_solve: f[k], u[k] device [ny_k][nx_k] and g[k] device [n_segments_k] (g or
 * g[k] may be NULL: zero boundary data) of member k, the same layouts as ccm_solve; u[k] is
 * the initial guess on entry, the solution on return.  stats (host, nullable) is an array
 * of count entries.  Launches the right-hand side set-up of every member, then the graph,
 * then synchronises the stream once.  Returns the first member's error in member order
 * (CCM_ENOCONV, CCM_ENOTFINITE, CCM_ETIMEOUT) or CCM_ECUDA; stats tell which member.
 * ccm_group_query: members, and 1 when the members' kernels keep their programmatic
 * (overlapped-launch) edges inside the graph, 0 when they were captured without them. */
int ccm_group_create(ccm_handle* const* members, int count, void* stream, ccm_group** out);
int ccm_group_solve(ccm_group* g, const double* const* f, const double* const* gb, double* const* u,
                    void* stream, ccm_stats* stats);
int ccm_group_query(const ccm_group* g, int* members, int* programmatic);
void ccm_group_free(ccm_group* g);

/* Adjoint solve L^T lambda = rhs (transpose of eq. PoissonResidualForm) by the same V-cycle on
 * the hierarchy of the transposed operators (L^(m))^T: cells whose column of L is the plain
 * point-symmetric stencil keep it, every other cell gets an explicit transposed row, with its
 * own boundary order, SMO-2 blocks and bottom inverse.  The first call builds that hierarchy
 * on the host and uploads it (blocking, allocates); later calls reuse it.  lambda in: initial
 * guess, out: solution; rhs, lambda: device [nrhs][ny][nx].  Gradients of a loss J(u(f, g)):
 * dJ/df = lambda, dJ/dg = -N^T lambda (ccm_apply_T of lambda). */
int ccm_solve_T(ccm_handle* h, const double* rhs, double* lambda, int nrhs, void* stream,
                ccm_stats* stats);

/* ---- level components of the V-cycle (one call = one step of the path, for testing and
 *      composition).  Level arrays use the user layout of that level: [ny_m][nx_m] FP64
 *      device arrays with nx_m = nx >> m, values in physical units of level m. */

/* out = L^(m) u on level m (no boundary term). */
int ccm_level_apply(ccm_handle* h, int level, const double* u, double* out, void* stream);
/* One smoother step on level m (Sec. 4.1): SMO-1 (weighted Jacobi on the regular cells)
 * then SMO-2 (block update of the irregular cells) for L^(m) u = r; u is updated in place.
 * precision CCM_FP64 or CCM_MIXED (FP32 arithmetic, FP64 in and out). */
int ccm_level_smooth(ccm_handle* h, int level, double* u, const double* r, int precision, void* stream);
/* Coarse residual (Alg. 2): rc = Restrict(r - L^(m) u) on level m + 1. */
int ccm_level_restrict(ccm_handle* h, int level, const double* u, const double* r, double* rc, void* stream);
/* Prolongation (Alg. 2): u += Prolong(uc), uc on level m + 1. */
int ccm_level_prolong(ccm_handle* h, int level, const double* uc, double* u, void* stream);
/* The first post-smoothing sweep of Alg. 2 with the prolongation fused, as the V-cycle runs
 * it: one smoother step on level m (as ccm_level_smooth) from the iterate u + Prolong(uc),
 * the parent's value added on the regular cells (Sec. 4.1); u (level m) is updated in place,
 * uc is level m + 1's iterate, r level m's right-hand side, all in the user layout of their
 * level.  precision as ccm_level_smooth.  Where level m's tiles are staged by TMA this is one
 * launch (the persistent sweep reads u + Prolong(uc) on the fly), else a prolongation and a
 * sweep.  Errors: CCM_EINVAL (level out of range or the coarsest, a NULL array), CCM_ECUDA. */
int ccm_level_prolong_smooth(ccm_handle* h, int level, double* u, const double* uc, const double* r, int precision,
                             void* stream);
/* Bottom solve on the coarsest level M: u = (L^(M))^-1 r. */
int ccm_bottom_solve(ccm_handle* h, const double* r, double* u, void* stream);
/* One V-cycle (Alg. 2) on level 0 for L u = r (physical units, FP64 in and out). */
int ccm_vcycle(ccm_handle* h, double* u, const double* r, int precision, void* stream);

/* Change the cycle parameters of a set-up handle (and of its transposed hierarchy, if built)
 * without repeating the host setup: omega (0, 1.5], nu1, nu2 (0 - 16, nu1 + nu2 >= 1),
 * inner_cycles (1 - 16), cycle (0 V, 1 FMG first).  Synchronises the device and drops the
 * captured iteration graphs (the next solve recaptures them).  Used by the autotuner.  The
 * paper fixes omega = 0.5, nu1 = nu2 = 3 (Sec. 5); these are free parameters of Alg. 2.
 * Errors: CCM_EINVAL, CCM_ECUDA. */
int ccm_set_cycle_params(ccm_handle* h, double omega, int nu1, int nu2, int inner_cycles, int cycle);

/* Rebuild the SMO-2 blocks of a set-up handle (and of its transposed hierarchy, if built):
 * on every level with fitted rows, cores of `block` consecutive rows of the boundary order
 * (Alg. 3) widened by `overlap` rows on each side, with the widened blocks' L22 inverses
 * (Sec. 4.1, eq. updateByBlock, solved by overlapping dense blocks).  block 8 - 128, overlap
 * 0 - 64; levels set up with one exact block (ras_exact) keep it.  The host recomputes the
 * inverses and uploads them, no other setup is repeated.  Blocking; drops the captured
 * iteration graphs.  Used by the autotuner.  Errors: CCM_EINVAL, CCM_ESINGULAR, CCM_ENOMEM,
 * CCM_ECUDA. */
int ccm_set_smo2_blocks(ccm_handle* h, int block, int overlap);

/* Launch shape of the persistent kernels (testing and tuning; not part of the method).  The
 * smoothing sweep of a level with TMA-staged tiles is one launch whose work items are the
 * level's SMO-2 blocks and its 64 x 32 tiles with a regular cell (Sec. 4.1), and the residual
 * + restriction is one launch over the fine tiles that restriction visits (Alg. 2).  Each CTA
 * takes items c, c + G, c + 2 G, ... through a two-stage copy ring, G = the CTAs given to one
 * right-hand side: min(items, resident CTAs of the GPU / nrhs, launch cap).
 * ccm_set_launch_cap: at most max_ctas CTAs per right-hand side in both kernels on every
 *   level (0: no cap, the default), so that small grids also run every CTA through many ring
 *   items.  Results do not depend on it.  Synchronises the device and drops the captured
 *   iteration graphs.  Errors: CCM_EINVAL, CCM_ECUDA.
 * ccm_level_launch: the shape of level `level`'s sweep and restriction launches for
 *   precision CCM_FP64 or CCM_MIXED when nrhs right-hand sides run together (1 for
 *   ccm_level_smooth, ccm_level_restrict, ccm_vcycle and single solves).  Counts are 0 where
 *   the level does not use that persistent kernel (small levels, the bottom level, the
 *   sequential smoother).  Host-only, no device work.  Errors: CCM_EINVAL. */
typedef struct {
  int sweep_items;     /* work items of one sweep launch (SMO-2 blocks + tiles) */
  int sweep_blocks;    /* of which SMO-2 block items */
  int sweep_ctas;      /* CTAs per right-hand side */
  int restrict_items;  /* tiles of one residual + restriction launch */
  int restrict_ctas;   /* CTAs per right-hand side */
  int64_t block_inv_entries;  /* entries of the SMO-2 block inverse rows one sweep reads */
} ccm_launch_info;
int ccm_set_launch_cap(ccm_handle* h, int max_ctas);
int ccm_level_launch(const ccm_handle* h, int level, int precision, int nrhs, ccm_launch_info* out);

/* One FMG cycle (Sec. 4, the FMG figure) for L u = r on the finest level, from the zero guess:
 * r restricted level by level to the bottom level and solved there, then one V-cycle (Alg. 2)
 * per finer level whose initial guess is the prolonged coarse solution.  r: device [ny][nx]
 * (unscaled), u: device [ny][nx], output only.  precision CCM_FP64 or CCM_MIXED (FP32 cycle).
 * Errors: CCM_EINVAL, CCM_ECUDA. */
int ccm_fmg(ccm_handle* h, double* u, const double* r, int precision, void* stream);

/* Self-test of the failure path of the bounded device waits: one CTA waits, with the wait
 * helper every TMA-staged kernel uses, on an mbarrier phase that nothing completes.  The wait
 * runs out after about 4 ms of SM clock, sets the handle's device error word, and the kernel
 * returns, so the context stays usable.  Returns CCM_ETIMEOUT (the expected outcome; the error
 * word is cleared again), CCM_OK if the wait did not run out, or CCM_ECUDA.  Blocking. */
int ccm_wait_selftest(ccm_handle* h, void* stream);

/* ---- accounting and profiling (not part of the method).
 * ccm_launch_count: kernels launched by this library in this process so far (all handles).
 * ccm_profile: record CUDA events on the handle's stream around every launch of one class:
 *   CCM_PROF_RESID_FP64  level-0 FP64 residual of the regular cells (outer iteration),
 *   CCM_PROF_SMO1_FP32   level-0 smoothing sweep in FP32 (SMO-1 with the SMO-2 blocks of the
 *                        block-Jacobi smoother), except the first post-smoothing sweep;
 *                        CCM_PROF_SMO1_FP64 the same in FP64,
 *   CCM_PROF_VCYCLE      one whole V-cycle,
 *   CCM_PROF_SMO2_FP32   level-0 SMO-2 block step in FP32,
 *   CCM_PROF_PROLONG_SMO1_FP32  level-0 first post-smoothing sweep with the prolongation fused,
 *   CCM_PROF_RESTRICT_FP32      level-0 residual + restriction in FP32;
 * 0 switches profiling off.
 * ccm_profile_read: total device time (ms) and launch count recorded since the last read;
 * waits for the recorded events. */
enum { CCM_PROF_OFF = 0, CCM_PROF_RESID_FP64 = 1, CCM_PROF_SMO1_FP32 = 2, CCM_PROF_SMO1_FP64 = 3,
       CCM_PROF_VCYCLE = 4, CCM_PROF_SMO2_FP32 = 5, CCM_PROF_PROLONG_SMO1_FP32 = 6, CCM_PROF_RESTRICT_FP32 = 7 };
int64_t ccm_launch_count(void);
int ccm_profile(ccm_handle* h, int kernel_class);
int ccm_profile_read(ccm_handle* h, double* ms, int64_t* launches);

/* ---- host-only view of the setup (no device memory is touched; usable without a GPU).
 * ccm_host_build runs the same host setup as ccm_setup and keeps the result on the host so
 * its discrete choices can be inspected and checked. */
typedef struct ccm_host_setup ccm_host_setup;
int ccm_host_build(const ccm_problem* prob, const ccm_params* params, ccm_host_setup** out);
/* sizes of level m: cells per side, fitted rows, boundary segments */
int ccm_host_level_sizes(const ccm_host_setup* s, int level, int* nx, int* ny, int64_t* n_irregular,
                         int64_t* n_segments);
/* fitted rows of level m (host arrays): cell[n2] linear index; cols[n2*15] linear indices
 * (row-major, cell first); beta[n2*15] and nb[n2] in physical units (L = h^-2 * scaled);
 * seg[n2] boundary segment or -1.  Any pointer may be NULL. */
int ccm_host_rows(const ccm_host_setup* s, int level, int32_t* cell, int32_t* cols, double* beta, double* nb,
                  int32_t* seg);
/* cell map of level m (see ccm_cell_map) and per-cell moments mom[ny*nx*15] in the cell frame
 * (units of h, graded monomial order (0,0),(1,0),(0,1),(2,0),...); any pointer may be NULL. */
int ccm_host_cell_map(const ccm_host_setup* s, int level, int8_t* status, int32_t* owner, int8_t* regular,
                      double* vol, double* mom);
void ccm_host_free(ccm_host_setup* s);

void ccm_free(ccm_handle* h);
const char* ccm_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* CCM_H */
