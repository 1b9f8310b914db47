/*
 * topo.h -- C-ABI of the GB300 SIMP hot-path library (libtopo.so).
 *
 * The calls follow the problem statement of arXiv 2012.08208 (Section 4: the
 * program main(nelx, nely[, nelz], volfrac, penal, rmin); Section 5: 3D,
 * other supports, several load cases, passive elements) on structured grids of
 * unit Q4 (2D, plane stress) / H8 (3D) elements.
 *
 * Conventions shared by every call
 *   - Numbering: node (i,j[,k]) = i + (nelx+1)*(j + (nely+1)*k); element
 *     (i,j[,k]) = i + nelx*(j + nely*k); DOF = dim*node + component.
 *   - Host arrays are borrowed for the duration of the call only.  Where a call
 *     takes `on_device`, a nonzero value means the pointer is device memory of
 *     the problem's device (e.g. a PyTorch tensor on the problem's stream);
 *     zero means host memory.
 *   - Ownership: the library allocates and owns every device buffer of a
 *     problem; tp_destroy_problem frees them.
 *   - Errors: every call returns a tp_status; no exception crosses the ABI.
 *     After an error the handle stays valid and tp_last_error() describes it.
 *     Calls on one handle are not thread-safe.  All work is enqueued on the
 *     stream given at creation; calls that return scalars synchronise it.
 *   - Order: create, set_fixed, set_loads, [set_passive], set_density, then per
 *     SIMP iteration solve, sensitivities, filter, oc_update (or tp_simp_step).
 *     A call whose inputs are not ready returns TP_ERR_STATE.
 */
#ifndef TOPO_H
#define TOPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TP_OK = 0,
  TP_ERR_ARG = 1,            /* invalid argument (size, range, NaN, null pointer) */
  TP_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  TP_ERR_OOM = 3,            /* device allocation failed */
  TP_ERR_NOT_CONVERGED = 4,  /* solve hit max_it before the tolerance */
  TP_ERR_BREAKDOWN = 5,      /* CG breakdown (p^T K p <= 0 or not finite) */
  TP_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired */
  TP_ERR_STATE = 7           /* call out of order (inputs not set) */
} tp_status;

/* Problem parameters (Section 4: nelx, nely, volfrac, penal, rmin; Section 5.1
 * adds nelz).  E0/Emin/nu: modified-SIMP moduli and Poisson ratio;
 * move/dmin: OC move limit and lower density bound (Eq. "update");
 * n_cases: number of load cases (Section 5.3), 1..8. */
typedef struct tp_params {
  int dim;      /* 2 (Q4, plane stress) or 3 (H8) */
  int nelx, nely, nelz;  /* elements per axis; nelz ignored in 2D */
  double E0, Emin, nu, penal, volfrac, rmin, move, dmin;
  int n_cases;
} tp_params;

enum { TP_PREC_F64 = 0, TP_PREC_MIXED = 1, TP_PREC_DW = 2 };
enum { TP_WARM_ZERO = 0, TP_WARM_PREVIOUS = 1, TP_WARM_USER = 2 };
/* Preconditioner of tp_solve.  TP_PRECOND_JACOBI: the persistent Jacobi-PCG
 * described above.  TP_PRECOND_MG: CG preconditioned by one geometric
 * multigrid V-cycle in FP32 per iteration (nested structured grids coarsened
 * 2:1 while the element counts are even, then by their smallest common odd
 * factor, down to the first grid of at most 4096 DOFs; Galerkin coarse
 * operators; degree-2 Chebyshev smoothing on the l1-Jacobi scaling; a dense
 * FP32 inverse of the coarsest operator formed on the device at every rebuild,
 * TP_ERR_BREAKDOWN if it meets a non-positive pivot), in
 * segments that solve for an FP32 correction and restart from the FP64 true
 * residual (FP64 vectors and operator after a segment that gains less than
 * 100x).  The iterations run as replays of a CUDA graph.
 * TP_PRECOND_MG_FUSED: the same method with each FP32 segment in one
 * persistent cooperative kernel.  Both need element counts that reach such a
 * coarsest grid (else TP_ERR_ARG); `precision` = TP_PREC_F64 starts with FP64
 * segments; `update_drop` is ignored. */
enum { TP_PRECOND_JACOBI = 0, TP_PRECOND_MG = 1, TP_PRECOND_MG_FUSED = 2 };
enum { TP_FILTER_SENSITIVITY = 0, TP_FILTER_DENSITY = 1, TP_FILTER_HELMHOLTZ = 2 };
/* Quantities for tp_get / tp_set (all FP64):
 *   TP_RHO   design densities rho[n_el]
 *   TP_U     displacements u[n_cases][n_dof] (the solution, or the warm start)
 *   TP_DC    raw sensitivities dc[n_el] (after tp_sensitivities)
 *   TP_DCF   filtered sensitivities dc~[n_el] (after tp_filter)
 *   TP_CE    element energies sum_k u_e^T K0 u_e [n_el] (after tp_sensitivities)
 *   TP_RHO_PHYS  physical densities used for stiffness [n_el] (rho, or rho~ in
 *                the density and Helmholtz filter modes) */
enum { TP_RHO = 0, TP_U = 1, TP_DC = 2, TP_DCF = 3, TP_CE = 4, TP_RHO_PHYS = 5 };

/* Solver options.  tol: target TRUE relative residual ||f - K u||_2 / ||f||_2
 * per case, checked in FP64 at exit.  max_it: maximum CG iterations.
 * precision TP_PREC_F64: all vectors and the operator in FP64.
 * precision TP_PREC_MIXED: operator and CG vectors in FP32, dot products in FP64,
 * and the solution accumulated in FP64 with reliable updates: whenever the FP32
 * recurrence residual has dropped by `update_drop` (e.g. 1e-2) since the last
 * update, the FP64 true residual f - K u replaces it.  warm_start: TP_WARM_*.
 * TP_WARM_USER uses the displacement set by tp_set(TP_U, ...) or by the learned
 * warm start (tp_warm_start_nn, topo_nn.h); if its true relative residual
 * exceeds warm_max_rel in any case, the solve falls back to u = 0 and reports
 * warm_fallback. */
typedef struct tp_solve_opts {
  double tol;
  int max_it;
  int precision;
  int warm_start;
  double update_drop;
  double warm_max_rel;  /* TP_WARM_USER: largest accepted starting true relative
                           residual (0 means 1, i.e. no worse than u = 0) */
  int precond;          /* TP_PRECOND_JACOBI (default), TP_PRECOND_MG or TP_PRECOND_MG_FUSED */
} tp_solve_opts;

typedef struct tp_solve_info {
  int iters;            /* CG iterations (shared by all cases) */
  int updates;          /* FP64 true-residual evaluations */
  int converged;        /* 1 if every case met tol */
  int status;           /* tp_status of the solve */
  double rel_res[8];    /* final true relative residual per case */
  double ms;            /* device time of the solve */
  double rel_res_init[8];  /* true relative residual of the starting guess per case */
  int warm_fallback;    /* 1 if a TP_WARM_USER start was dropped for u = 0 */
} tp_solve_info;

typedef struct tp_step_info {
  tp_solve_info solve;
  double compliance;    /* sum_k f_k^T u_k */
  double lambda;        /* OC multiplier */
  double volume;        /* sum rho_new */
  double change;        /* max |rho_new - rho| */
  int oc_passes;        /* passes over the elements in the OC multiplier search */
  int oc_root;          /* how lambda was fixed: 1 closed form on a bracket with no
                           clamp change, 2 exact piecewise root, 0 bisection midpoint */
} tp_step_info;

typedef struct tp_problem tp_problem;

/* Create a problem on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Validates sizes and ranges:
 * dim in {2,3}, element counts >= 1, 0 < volfrac <= 1, rmin > 0, penal >= 1,
 * 0 <= nu < 0.5, 0 < Emin < E0, 0 < dmin < 1, move > 0, 1 <= n_cases <= 8. */
tp_status tp_create_problem(const tp_params* params, void* cuda_stream, tp_problem** out);
void tp_destroy_problem(tp_problem* p);
const char* tp_last_error(const tp_problem* p);

/* Dirichlet DOFs (Section 4.2; DirichletBC): fixed[n_dof] (host), nonzero = u = 0.
 * Rejected if no DOF is fixed (K would be singular). */
tp_status tp_set_fixed(tp_problem* p, const uint8_t* fixed);
/* Nodal loads f[n_cases][n_dof] (host, FP64; Section 4.2 loads, Section 5.3 load
 * cases).  Loads on fixed DOFs are ignored.  Rejects NaN/Inf and an all-zero case. */
tp_status tp_set_loads(tp_problem* p, const double* f);
/* Passive elements passive[n_el] (host; Section 5.4): 1 = void, held at dmin. */
tp_status tp_set_passive(tp_problem* p, const int8_t* passive);
/* Design densities rho[n_el] (FP64, host or device).  Must lie in (0, 1]. */
tp_status tp_set_density(tp_problem* p, const double* rho, int on_device);

/* Solve K(rho) u_k = f_k for every case (replaces the sparse LU of Section 4.3)
 * by preconditioned CG: opts->precond selects the persistent Jacobi-PCG launch
 * or the multigrid-PCG (TP_PRECOND_*).  Fills `info` (may be NULL).  Returns TP_ERR_NOT_CONVERGED / TP_ERR_BREAKDOWN / TP_ERR_TIMEOUT when the
 * solve did not reach opts->tol (the solution is still stored). */
tp_status tp_solve(tp_problem* p, const tp_solve_opts* opts, tp_solve_info* info);

/* Compliance c = sum_k f_k^T u_k and sensitivities
 * dc_e = -p rho_e^(p-1) (E0 - Emin) sum_k u_e^T K0 u_e (Section 3.2 sensitivity,
 * Section 4.4, Section 5.3).  `compliance` (host, may be NULL) receives c. */
tp_status tp_sensitivities(tp_problem* p, double* compliance);

/* Mesh-independency filter (Section 3.2.2, Eq. "filter", "filter_cond"; Eq.
 * "filter_mat"): W_ab = max(0, rmin - |x_a - x_b|) over element midpoints, rows
 * truncated at the mesh boundary.
 * mode TP_FILTER_SENSITIVITY (the paper's): dc~_a = sum_b W_ab rho_b dc_b /
 *   (rho_a sum_b W_ab).
 * mode TP_FILTER_DENSITY: the stiffness uses the filtered densities
 *   rho~ = W rho / rowsum (tp_set_filter_mode); dc then holds d c / d rho~
 *   and this call applies the chain rule dc~ = W^T (dc / rowsum).  The OC
 *   update keeps its volume constraint on rho.
 * mode TP_FILTER_HELMHOLTZ: the PDE filter of the paper's parallel runs
 *   (Section "Parallel implementation of topology optimization", after Lazarov
 *   and Sigmund): rho~ = H rho with H = T^T (R^2 K_F + M_F)^-1 T, K_F and M_F
 *   the bilinear / trilinear Laplacian stiffness and mass with natural
 *   (Neumann) boundaries, T the element-to-node integral of the shape
 *   functions, R = rmin / (2 sqrt 3).  H is symmetric, so dc~ = H dc.  Each
 *   application solves the nodal system by FP64 iterative refinement around
 *   FP32 Jacobi-PCG solves until the FP64 true relative residual is at most
 *   1e-14 (TP_ERR_NOT_CONVERGED otherwise) and synchronises.
 * `mode` must equal the problem's filter mode (else TP_ERR_STATE). */
tp_status tp_filter(tp_problem* p, int mode);
/* Filter mode of the problem (default TP_FILTER_SENSITIVITY); also the mode
 * tp_simp_step uses.  TP_FILTER_DENSITY and TP_FILTER_HELMHOLTZ make tp_solve /
 * tp_sensitivities use the filtered densities rho~ (TP_RHO_PHYS). */
tp_status tp_set_filter_mode(tp_problem* p, int mode);

/* OC update with bisection on lambda (Section 3.2, Eq. "update", Section 3.2.1):
 * rho_new = max(dmin, max(rho - m, min(1, min(rho + m, rho sqrt(-dc~ / lambda))))),
 * lambda such that sum rho_new = volfrac * n_el (passive held at dmin), bracket
 * [0, 1e9] widened x10 as needed, stopped at width <= 1e-10 (l1 + l2).  Replaces
 * rho by rho_new.  Outputs (host, each may be NULL): lambda, volume, change. */
tp_status tp_oc_update(tp_problem* p, double* lambda, double* volume, double* change);

/* One SIMP iteration: solve, sensitivities, sensitivity filter, OC update. */
tp_status tp_simp_step(tp_problem* p, const tp_solve_opts* opts, tp_step_info* info);

/* Copy a quantity out (TP_RHO, TP_U, TP_DC, TP_DCF, TP_CE, TP_RHO_PHYS) to `dst`. */
tp_status tp_get(tp_problem* p, int what, void* dst, int on_device);
/* Set a quantity: TP_U (warm start for TP_WARM_USER / TP_WARM_PREVIOUS),
 * TP_DC (raw sensitivities, e.g. to filter given values), TP_DCF (filtered
 * sensitivities, e.g. to run the OC update on given values). */
tp_status tp_set(tp_problem* p, int what, const void* src, int on_device);

/* Apply the boundary-conditioned operator: y = K(rho) u on free DOFs with the
 * fixed entries of u read as 0, and y_i = u_i on fixed DOFs.  precision
 * TP_PREC_F64: u, y are double[n_dof]; TP_PREC_MIXED: float[n_dof] (FP32 operator);
 * TP_PREC_DW: double[n_dof], the operator in double-word FP32 arithmetic
 * (about 48 significant bits; the form of the multigrid solver's true
 * residual at tolerances >= 1e-8 in 3D).
 * `ncopies` > 1 applies it to that many consecutive vectors (stride n_dof). */
tp_status tp_matvec(tp_problem* p, const void* u, void* y, int precision, int ncopies,
                    int on_device);

/* Launch accounting: number of kernels this library enqueued since creation. */
long long tp_launch_count(const tp_problem* p);

/* ---------------------------------------------------------------------------
 * Batches of independent 2D problems (one persistent launch for all solves).
 *
 * A batch holds n independent 2D Q4 problems (one load case each, same nu),
 * each with its own grid, volfrac, rmin, penal, move and dmin (Section 4
 * problem statement per instance).  tp_batch_step performs one SIMP iteration
 * of every instance:
 *   - one persistent cooperative CG launch solves all instances (FP32
 *     operator and vectors, FP64 reductions and true-residual updates inside
 *     the launch, previous displacement as warm start);
 *   - then sensitivities, the sensitivity filter and the per-instance OC
 *     bisection follow, all as batched kernels.
 * The step's kernels are captured once in a CUDA graph and replayed while the
 * options stay the same.  Densities start at each instance's volfrac.
 * Instances are independent: none of these calls exchanges data between them.
 * Errors as for single problems; tp_batch_last_error describes the last one. */
typedef struct tp_batch tp_batch;
typedef struct tp_batch_info {
  int max_iters;        /* CG iterations of the slowest instance */
  int updates;          /* FP64 true-residual evaluations (max over instances) */
  int converged;        /* 1 if every instance met tol */
  int graph;            /* 1 if the step ran as a replayed CUDA graph */
  int tile_rows;        /* node rows per tile (tiles are 32 nodes wide) */
  int ctas;             /* CTAs of the persistent launch */
  double max_rel_res;   /* largest final true relative residual */
  double ms;            /* device time of the step */
} tp_batch_info;

/* params[n]: dim 2, n_cases 1, equal nu.  Allocates all device state. */
tp_status tp_batch_create(int n, const tp_params* params, void* cuda_stream, tp_batch** out);
void tp_batch_destroy(tp_batch* b);
const char* tp_batch_last_error(const tp_batch* b);
/* Instance i: fixed[2 * nodes_i], loads f[2 * nodes_i] (host, ABI DOF layout),
 * densities rho[n_el_i] (host, in (0, 1]). */
tp_status tp_batch_set_fixed(tp_batch* b, int i, const uint8_t* fixed);
tp_status tp_batch_set_loads(tp_batch* b, int i, const double* f);
tp_status tp_batch_set_density(tp_batch* b, int i, const double* rho);
/* Tile shape of the CG launch: tile_rows in {4, 8, 16}, ctas_per_sm in 1..8. */
tp_status tp_batch_set_tiles(tp_batch* b, int tile_rows, int ctas_per_sm);
/* Autotuner: times a short CG for every tile_rows x ctas_per_sm in
 * {4, 8, 16} x {1, 2, 4} and keeps the fastest.  The choice is cached in the JSON
 * file `cache_path` (may be NULL) under a key naming the size class (instance
 * count, total nodes to 2 significant digits, SM count); a cached key skips the
 * sweep.  Outputs (may be NULL): the chosen shape. */
tp_status tp_batch_autotune(tp_batch* b, const char* cache_path, int* tile_rows, int* ctas_per_sm);
/* One SIMP iteration of every instance.  opts->precision must be
 * TP_PREC_MIXED; warm_start is always the previous displacement.  compliance
 * (host, n doubles, may be NULL) receives each instance's c = f^T u. */
tp_status tp_batch_step(tp_batch* b, const tp_solve_opts* opts, tp_batch_info* info, double* compliance);
/* Copy TP_RHO, TP_DC, TP_DCF (n_el_i) or TP_U (2 * nodes_i) of instance i to host
 * `dst` (may be NULL); scalars (host, 6 doubles, may be NULL) receives compliance,
 * lambda, volume, change, CG iterations and final true relative residual. */
tp_status tp_batch_get(tp_batch* b, int i, int what, double* dst, double* scalars);
long long tp_batch_launch_count(const tp_batch* b);

/* Allocation-free OC update.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they update the
 * design -- e.g. a host framework whose allocator already holds the device
 * memory budget, a plugin host that forbids device allocations after start-up,
 * or a tight loop that must not pay for cudaMalloc/cudaFree and the device-wide
 * synchronisation cudaFree can imply.  It computes exactly what tp_oc_update
 * computes (same kernel, same readings), without a problem handle and without
 * allocating anything: its scratch (about 8.3 MB) is one static device array
 * that each GPU loading this library keeps until the process exits.
 *
 * Arguments: rho[n_el], dcf[n_el] (filtered sensitivities) and rho_new[n_el]
 * are device pointers on the current device; passive[n_el] (device, 1 = void) may
 * be NULL; rho_new must not alias rho or dcf.  volfrac, move, dmin as in
 * tp_params.  cuda_stream: the stream to run on (NULL = legacy default stream).
 * lambda, volume, change (host, each may be NULL) receive the multiplier, the new
 * volume and max |rho_new - rho|.  The call synchronises the stream before it
 * returns.
 * Limits and errors: 1 <= n_el <= TP_NOALLOC_MAX_ELEMENTS, else TP_ERR_ARG (the
 * scratch holds one double per element); bad ranges or NULL arrays give
 * TP_ERR_ARG; CUDA failures TP_ERR_CUDA.
 * Sharing: every call uses the same scratch array, which keeps the last call's
 * contents (the call clears what must start at zero).  Calls whose work overlaps
 * on the GPU -- e.g. from two threads or on two streams at once -- race and give
 * undefined results; serialise them.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before any
 * stream capture. */
#define TP_NOALLOC_MAX_ELEMENTS 1048576LL
tp_status tp_oc_update_noalloc(const double* rho, const double* dcf, const int8_t* passive, long long n_el,
                               double volfrac, double move, double dmin, double* rho_new, void* cuda_stream,
                               double* lambda, double* volume, double* change);

/* Dense SPD inverse in FP32: the coarsest-level solve of the multigrid
 * preconditioner (TP_PRECOND_MG), exposed on its own.  Not in the paper, which
 * factorises K directly; a multigrid coarsest grid small enough for a dense
 * inverse is this library's choice.
 * Method: a blocked symmetric sweep (Gauss-Jordan elimination without
 * pivoting, 64-row pivot blocks, the upper triangle only; Beaton-Goodnight
 * sweep operator in block form), every rank-64 update on the device in FP32.
 * Arguments: a[n * n] (host, row-major; the upper triangle j >= i is read, the
 * matrix is taken as symmetric) and ainv[n * n] (host, receives the full
 * inverse); 1 <= n <= TP_SPD_INVERSE_MAX_N.  cuda_stream: the stream to run on
 * (NULL = legacy default stream).  The call allocates n * n + 192 n + 8192
 * floats of device memory for its duration and synchronises before it returns.
 * Errors: TP_ERR_ARG for NULL arrays or n out of range; TP_ERR_BREAKDOWN when a
 * pivot is not positive and finite (the matrix is not positive definite, or
 * not in FP32; ainv then holds no inverse); TP_ERR_OOM, TP_ERR_CUDA. */
#define TP_SPD_INVERSE_MAX_N 16384
tp_status tp_spd_inverse_f32(const float* a, float* ainv, int n, void* cuda_stream);

/* The paper's own elements (Section 4 "Discretization the problem", Section 5
 * "Working with 3D problems"): the boundary-conditioned operator
 * y = K(rho) u for vector P1 on the structured grid of unit squares cut into 2
 * triangles each, or unit cubes cut into the 6 Kuhn tetrahedra, one density
 * per cell, sigma = 2 mu eps + lambda tr(eps) I (Section 4.3) scaled by
 * Emin + rho^penal (1 - Emin).  FP64.
 * Cells: square / cube e = i + nelx (j + nely k) holds cells 2 e, 2 e + 1 (2D)
 * or 6 e .. 6 e + 5 (3D).  diagonal (2D): 0 cuts along (i, j)-(i+1, j+1) into
 * (v00, v10, v11), (v00, v11, v01); 1 along (i+1, j)-(i, j+1) into
 * (v00, v10, v01), (v10, v11, v01); 2 alternates by row (even rows 0, odd
 * rows 1).  3D (diagonal 0): cell 6 e + t is the Kuhn tetrahedron of the
 * t-th axis ordering in lexicographic order (012, 021, 102, 120, 201, 210):
 * the path from the cube's lowest corner stepping along those axes.
 * Arguments (device pointers on the current device): rho[n_cells];
 * fixed[n_dof] (1 = Dirichlet DOF); u, y [ncases][n_dof] with DOF = dim *
 * node + component, nodes x fastest.  y = u on fixed rows; u is read as 0 on
 * fixed DOFs elsewhere.  nelz = 0 in 2D.  The call synchronises the stream.
 * The cell matrices travel with each launch (kernel parameters), so calls on
 * different streams or threads may overlap.  Errors: TP_ERR_ARG for sizes, dim, diagonal, material
 * (mu > 0, lambda + 2 mu / dim > 0), Emin outside [0, 1), penal outside
 * [1, 10], ncases outside 1..8 or NULL pointers; TP_ERR_CUDA. */
tp_status tp_p1_matvec(int dim, int nelx, int nely, int nelz, int diagonal, double lam, double mu, double Emin,
                       double penal, const double* rho, const uint8_t* fixed, const double* u, double* y,
                       int ncases, void* cuda_stream);

/* Host-side cell shapes of tp_p1_matvec (no device work): for each shape t
 * (4 in 2D: types 0, 1 = the cells of a "right" cut square, 2, 3 = of a
 * "left" cut square; 6 in 3D: the Kuhn tetrahedra in the order of
 * tp_p1_matvec), K[t][nd][nd] (nd = dim (dim + 1), unit modulus, DOF order
 * vertex-major then component) and offsets[t][dim + 1][dim] (vertex offsets
 * within the unit square / cube).  K holds 4 * 36 (2D) or 6 * 144 (3D)
 * doubles, offsets 4 * 3 * 2 or 6 * 4 * 3 ints.  TP_ERR_ARG for a bad
 * dimension, material or NULL pointer. */
tp_status tp_p1_shape_matrices(int dim, double lam, double mu, double* K, int* offsets);

/* Host-side filter stencil for the P1 cells (no device work): the paper's
 * weights W = max(0, rmin - distance) between cell midpoints (centroids),
 * for a centre cell of each type (the types of tp_p1_shape_matrices; in 2D
 * the types a diagonal pattern does not use get no entries).  An entry is
 * the neighbour cell local index l of the square / cube displaced by
 * (dx, dy, dz) from the centre's; in 2D the neighbour's cut follows from its
 * row.  Outputs (host): count[ntypes] entries per type, entries[n][4] =
 * (dx, dy, dz, l) grouped by type, weights[n]; n_entries = n.  cap is the
 * capacity of entries / weights.  Rows are not truncated at the domain
 * boundary: a caller skips neighbours outside the grid.  TP_ERR_ARG for a bad
 * dim, diagonal, rmin (0 < rmin <= 16), NULL pointers or too small a cap. */
tp_status tp_p1_filter_stencil(int dim, int diagonal, double rmin, int cap, int* count, int* entries,
                               double* weights, int* n_entries);

/* ---------------------------------------------------------------------------
 * The SIMP loop on the paper's own elements (Section 4 "Discretization the
 * problem": triangles, P1 displacements, one density per cell; Section 5
 * "Working with 3D problems": tetrahedra; the material and form of the
 * Section 4.3 listing).  The grid and cells are those of tp_p1_matvec: unit
 * squares cut into 2 triangles (diagonal 0 "right", 1 "left", 2 alternating
 * by row) or unit cubes cut into the 6 Kuhn tetrahedra (diagonal 0); cell
 * index = 2 e + l (2D) or 6 e + l (3D) for square / cube e.  Stiffness
 * sigma = 2 mu eps + lambda tr(eps) I scaled by Emin + rho^penal (1 - Emin).
 * Calls, conventions and errors as for the Q4 / H8 problem (tp_status,
 * borrowed pointers, tp_p1_last_error, calls on one handle not thread-safe):
 *   tp_p1_solve          K(rho) u_k = f_k by Jacobi-preconditioned CG in FP64
 *                        (opts->precision TP_PREC_F64, opts->precond
 *                        TP_PRECOND_JACOBI, else TP_ERR_ARG), all cases
 *                        together, until the TRUE relative residual
 *                        ||f - K u|| / ||f|| <= opts->tol (recomputed
 *                        whenever the recurrence meets it);
 *                        warm_start TP_WARM_ZERO, TP_WARM_PREVIOUS or
 *                        TP_WARM_USER (the TP_U set by tp_p1_set)
 *   tp_p1_sensitivities  c = sum_k f_k^T u_k, ce_e = sum_k u_e^T K_e u_e (unit
 *                        modulus), dc_e = -penal rho_e^(penal-1) (1 - Emin) ce_e
 *                        (Section 3.2, Section 4.4; the cell energy is a
 *                        uniform multiple of the paper's DG0 projection)
 *   tp_p1_filter         dc~_a = sum_b W_ab rho_b dc_b / (rho_a sum_b W_ab),
 *                        W_ab = max(0, rmin - |m_a - m_b|) between cell
 *                        centroids, rows truncated at the grid boundary
 *                        (Eq. "filter", "filter_mat")
 *   tp_p1_oc_update      the OC update of tp_oc_update on the cells
 *                        (Eq. "update"; passive cells held at dmin)
 *   tp_p1_simp_step      solve, sensitivities, filter, OC update
 *   tp_p1_apply          y = K(rho) u (boundary-conditioned as in tp_matvec)
 *                        for all cases: u, y [n_cases][n_dof]; with
 *                        on_device = 1 the call only enqueues the kernel
 * tp_p1_set_fixed: fixed[n_dof] (host, nonzero = u = 0; at least one).
 * tp_p1_set_loads: f[n_cases][n_dof] (host, finite; loads on fixed DOFs do not
 * enter the solve).  tp_p1_set_passive: passive[n_cells] (host, 1 = void).
 * tp_p1_set_density: rho[n_cells] in (0, 1].  tp_p1_get: TP_RHO (= TP_RHO_PHYS),
 * TP_U, TP_DC, TP_DCF, TP_CE.  tp_p1_set: TP_U, TP_DC, TP_DCF.
 * Parameters: dim 2 or 3; nelx, nely >= 1, nelz >= 1 in 3D and 0 in 2D;
 * mu > 0, lambda + 2 mu / dim > 0; 0 < Emin < 1; 1 <= penal <= 10;
 * 0 < volfrac <= 1; 0 < rmin <= 4; move > 0; 0 < dmin < 1; 1..8 cases. */
typedef struct tp_p1_params {
  int dim, nelx, nely, nelz;
  int diagonal;
  double lam, mu, Emin, penal, volfrac, rmin, move, dmin;
  int n_cases;
} tp_p1_params;
typedef struct tp_p1_problem tp_p1_problem;
tp_status tp_p1_create(const tp_p1_params* params, void* cuda_stream, tp_p1_problem** out);
void tp_p1_destroy(tp_p1_problem* p);
const char* tp_p1_last_error(const tp_p1_problem* p);
long long tp_p1_launch_count(const tp_p1_problem* p);
tp_status tp_p1_set_fixed(tp_p1_problem* p, const uint8_t* fixed);
tp_status tp_p1_set_loads(tp_p1_problem* p, const double* f);
tp_status tp_p1_set_passive(tp_p1_problem* p, const int8_t* passive);
tp_status tp_p1_set_density(tp_p1_problem* p, const double* rho, int on_device);
tp_status tp_p1_solve(tp_p1_problem* p, const tp_solve_opts* opts, tp_solve_info* info);
tp_status tp_p1_sensitivities(tp_p1_problem* p, double* compliance);
tp_status tp_p1_filter(tp_p1_problem* p);
tp_status tp_p1_oc_update(tp_p1_problem* p, double* lambda, double* volume, double* change);
tp_status tp_p1_simp_step(tp_p1_problem* p, const tp_solve_opts* opts, tp_step_info* info);
tp_status tp_p1_apply(tp_p1_problem* p, const double* u, double* y, int on_device);
tp_status tp_p1_get(tp_p1_problem* p, int what, void* dst, int on_device);
tp_status tp_p1_set(tp_p1_problem* p, int what, const void* src, int on_device);

/* Phase tracing of the persistent CG (not in the paper; a profiling aid).
 * When enabled, CTA 0 of every CG launch records %globaltimer (ns) at eight
 * points of each iteration into a ring of 32 iterations: 0 start, 1 operator
 * done, 2 CTA partial written, 3 first grid barrier passed, 4 scalars of the
 * first phase published, 5 vector update done, 6 second grid barrier passed,
 * 7 totals of the second phase read.  tp_get_trace copies the ring (32 x 8
 * int64, row = iteration mod 32) to `out` (host).  Tracing adds one store per
 * point and stays off by default. */
tp_status tp_set_trace(tp_problem* p, int enable);
tp_status tp_get_trace(tp_problem* p, long long* out);

/* Wait limit of the grid barriers (not in the paper; a test aid for the
 * failure path).  Every grid-wide wait of the persistent Jacobi-PCG and of the
 * OC kernel gives up after `cycles` SM clock cycles (0 restores the default,
 * about 1 s at 2 GHz), records TP_ERR_TIMEOUT and returns, so the context and
 * the handle stay usable.  A tiny value (e.g. 1) makes the next solve return
 * TP_ERR_TIMEOUT.  Synchronises the problem's stream.  TP_ERR_ARG outside
 * [0, 4e9]. */
tp_status tp_set_wait_budget(tp_problem* p, long long cycles);

/* Launch timing of the multigrid solver (profiling aid).  When enabled, the
 * dominant kernel of each multigrid solve is bracketed by CUDA event pairs on
 * the problem's stream: with TP_PRECOND_MG every finest-level sweep launch
 * (mg_sweep_kernel; event nodes in the replayed graph), with
 * TP_PRECOND_MG_FUSED every persistent segment launch.  tp_get_profile writes
 * out[4] (host): the number of timed launches, their total device time in ms,
 * their total algorithmic bytes (a sweep: the finest moduli and l1 scale, per
 * case u and b read and y written; a segment: one V-cycle plus, per CG
 * iteration, a V-cycle, the operator phase and the vector update, each value
 * read or written once per phase and operator data once per sweep) and the
 * number of multigrid levels.  Enabling resets the totals. */
tp_status tp_set_profile(tp_problem* p, int enable);
tp_status tp_get_profile(tp_problem* p, double* out);

#ifdef __cplusplus
}
#endif
#endif /* TOPO_H */
