/*
 * libpair: GB300 (sm_103a) pAIR inside S_N source iteration for upwind-DG
 * transport.  Method: Hanophy, Southworth, Li, Morel, Manteuffel, "Parallel
 * approximate ideal restriction multigrid for solving the S_N transport
 * equations" (arXiv 1910.11463).
 *
 * Conventions (every entry point):
 *  - Array arguments are caller-owned DEVICE pointers (CUDA global memory,
 *    contiguous) unless a comment says "host".  The library never frees them.
 *  - Hierarchies (pair_hier) are library-owned and released by air_free().
 *  - Work is ordered on the caller's stream ('stream' is a cudaStream_t; 0 is
 *    the legacy default stream).  Calls that return host-visible results
 *    (sizes, convergence info) synchronise that stream before returning.
 *  - Every call returns a pair_status; no C++ exception crosses this boundary.
 *    On error the outputs are unspecified and pair_last_error() returns a
 *    message (per calling thread).
 *  - Indices are 0-based int32; CSR column indices must be sorted ascending
 *    within each row.  Floating point data is IEEE binary64 unless stated.
 *  - A handle must not be used from two streams at the same time.
 *  - Device memory the library allocates comes from its own stream-ordered memory
 *    pool on each device; memory a call frees stays in that pool for later calls
 *    (the pool keeps its peak size until the process exits).
 */
#ifndef PAIR_H
#define PAIR_H

#include <stdint.h>

#if defined(__GNUC__)
#define PAIR_API __attribute__((visibility("default")))
#else
#define PAIR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PAIR_OK = 0,
    PAIR_ERR_ARG = -1,            /* invalid argument (null pointer, size, parameter range) */
    PAIR_ERR_OOM = -2,            /* device allocation failed, or the memory budget
                                   * holds less than one direction's hierarchy */
    PAIR_ERR_SINGULAR = -3,       /* singular element block or sweep cycle block (zero pivot) */
    PAIR_ERR_NOT_CONVERGED = -4,  /* iteration limit reached before the tolerance */
                                  /* -5 and -7 are not used: coarsening that stalls
                                   * (n_c = 0 or n_c >= 0.9 n) ends the hierarchy
                                   * there, which is not an error, and no kernel of
                                   * this library waits on the device */
    PAIR_ERR_NAN = -6,            /* NaN/Inf found in an input or a residual */
    PAIR_ERR_CUDA = -8,           /* a CUDA runtime call failed */
    PAIR_ERR_UNSUPPORTED = -9,    /* size outside what this build handles (message says which) */
    PAIR_ERR_DEVICE = -10,        /* a kernel reported an internal bound violation */
    PAIR_ERR_COMM = -11           /* the scalar-flux reduction function reported an error */
} pair_status;

typedef struct pair_hier_s *pair_hier;

/* AIR parameters (Sec. 1.2 AIR, Sec. 4 parameter choices, Eq. soc).
 *  distance      1 or 2: neighbourhood of the lAIR local solves (Sec. 1.2, Sec. 4.1.1)
 *  theta         strength threshold for the CF splitting (paper: 0.25, Sec. 4)
 *  eps_R         strength threshold for the R sparsity pattern (Eq. soc; paper 0.01)
 *  phi_R         filter applied to R after it is built (Sec. 4.1.2; 0 = off)
 *  phi_A         filter applied to every coarse operator, diagonal kept (0 = off)
 *  max_levels    level cap (including the finest)
 *  max_coarse    a level with at most this many rows is the coarsest
 *  coarse_sweeps pointwise Jacobi sweeps from zero on the coarsest level (one CTA
 *                per matrix in shared memory while a matrix's coarsest level fits
 *                40 KB; larger coarsest levels sweep grid-wide, one launch per sweep)
 *  seed          PMIS key hash seed
 *  precision     0: hierarchy values and V-cycle in FP64;
 *                1: FP32 hierarchy and V-cycle under FP64 iterative refinement
 *                   (FP64 outer residual and iterate);
 *                2: as 1, but on the structured hex block form the outer residual
 *                   is computed in double-float arithmetic (pairs of floats with
 *                   exact two-sum / two-product, ~2^-44 relative) on the FP32 pipe,
 *                   and the iterate is held as a float pair during each solve
 *                   (other meshes and generic matrices: as 1)
 *  f_sweeps      F-point Jacobi sweeps of the post-relaxation before its C-point
 *                sweep (1: F-C, 2: F-F-C)
 *  nair          0: R from lAIR local solves; 1: nAIR of degree 1 (Sec. 1.2, the
 *                Neumann-expansion variant; Sec. 4.1.2 runs it with phi_R = 0.1):
 *                Z_i = -A_CF^s[i,:] (I + N) D_FF^{-1}, N = I - D_FF^{-1} A_FF^s, where
 *                ^s keeps the eps_R-strong entries (and the diagonal), on the
 *                distance-2 pattern; `distance` is then not used */
typedef struct {
    int distance;
    double theta, eps_R, phi_R, phi_A;
    int max_levels, max_coarse, coarse_sweeps;
    uint64_t seed;
    int precision;
    int f_sweeps;
    int nair;
} air_params;

/* Fills the defaults: distance 1, theta 0.25, eps_R 0.01, phi_R 0, phi_A 0,
 * max_levels 25, max_coarse 100, coarse_sweeps 20, seed 3, precision 1,
 * f_sweeps 2, nair 0. */
PAIR_API void air_params_default(air_params *p);

/* A square CSR matrix in device memory. */
typedef struct {
    int n;              /* rows = columns */
    int nnz;            /* rowptr[n] */
    const int *rowptr;  /* n + 1 */
    const int *col;     /* nnz, ascending within a row */
    const double *val;  /* nnz */
} pair_csr;

/* Per-level sizes of one matrix of a (possibly batched) hierarchy. */
typedef struct {
    int n;          /* rows of this level */
    int nnz;        /* stored entries of A_l */
    int nc;         /* coarse points (0 on the coarsest level) */
    int nnz_R;      /* stored entries of Z (R = [Z, I] has nnz_R + nc) */
    int coarsest;   /* 1 on the last level of this matrix */
    int pmis_rounds;
    int n_singular; /* lAIR local systems found singular (their R row is injection) */
} pair_level_info;

typedef struct {
    int iters;          /* V-cycles (refinement steps) taken by the slowest matrix */
    double rel_resid;   /* max over matrices of ||b - A x|| / ||b|| at exit (FP64) */
    double rho;         /* mean convergence factor (||r_k||/||r_0||)^(1/k) over matrices */
} air_solve_info;

/*
 * air_setup: AIR hierarchies for 'count' independent square matrices A[0..count-1]
 * (Sec. 1.2; Sec. 4.1.1 Eq. soc; Sec. 4.1.2), built together: every level of
 * all matrices is processed by one launch per setup step.
 * Steps per level: strength (|a_ij| >= theta max_{k!=i}|a_ik|), PMIS CF
 * splitting with key (lambda_i, hash(seed, level, i), i), one-point
 * interpolation to the strongest C neighbour, lAIR restriction R = [Z, I]
 * from FP64 LU solves on distance-1/2 strong F neighbourhoods (pattern from
 * eps_R), optional phi_R filter, Galerkin A_c = R A P, optional phi_A filter.
 * All setup arithmetic is FP64 in the order documented with the kernels: the
 * compiler contracts nothing (no implicit fused multiply-add), and the LU
 * updates, the Neumann series and the Galerkin sums use an explicit fma()
 * exactly where that order writes one, so results are reproducible bit for bit.
 *   A      host array of 'count' descriptors of device CSR matrices (copied)
 *   out    receives the new handle
 * Errors: PAIR_ERR_ARG (count < 1, null pointers, n < 1, distance not 1/2),
 * PAIR_ERR_UNSUPPORTED (an lAIR pattern larger than the local-solve limit).
 */
PAIR_API pair_status air_setup(const pair_csr *A, int count, const air_params *prm, void *stream, pair_hier *out);

/* One V-cycle on every matrix of the batch (Sec. 1.2): x <- x + V(b - A x).
 * No pre-relaxation; restrict the residual with R, recurse with zero initial
 * guess, prolong with P (one-point), post-relax with f_sweeps F-Jacobi sweeps
 * then one C-Jacobi sweep (omega = 1); coarsest level: coarse_sweeps Jacobi
 * sweeps.  The level-0
 * residual is FP64; the cycle runs in the hierarchy's precision.
 *   b, x   concatenation of the right-hand sides / iterates of all matrices
 *          (length = sum of n), x updated in place. */
PAIR_API pair_status air_vcycle(pair_hier h, const double *b, double *x, void *stream);

/* Repeats air_vcycle until ||b - A x||_2 <= tol ||b||_2 for every matrix (FP64
 * residual) or maxit cycles (Sec. 2.1 solve loop).  Matrices that converge
 * stop being updated.  'info' (host, may be NULL) receives the totals.
 * Returns PAIR_ERR_NOT_CONVERGED if a matrix misses the tolerance. */
PAIR_API pair_status air_solve(pair_hier h, const double *b, double *x, double tol, int maxit, void *stream,
                      air_solve_info *info);

/* Number of matrices in the batch and levels of matrix 'mat' (host out). */
PAIR_API pair_status air_hier_nlevels(pair_hier h, int mat, int *nlevels);
PAIR_API pair_status air_level_info(pair_hier h, int mat, int level, pair_level_info *out);

/* Copies level 'level' of matrix 'mat' to HOST arrays (any may be NULL), with
 * indices local to that matrix: A_l (rowptr n+1, col nnz, val nnz), the CF
 * splitting cf (n bytes: 1 C, 0 F; undefined on the coarsest level), pmap (n:
 * coarse column of P for each row or -1), cpts (nc: fine index of each coarse
 * point) and Z (zrowptr nc+1, zcol nnz_R fine indices, zval nnz_R). */
PAIR_API pair_status air_level_export(pair_hier h, int mat, int level, int *rowptr, int *col, double *val,
                             signed char *cf, int *pmap, int *cpts, int *zrowptr, int *zcol, double *zval);

PAIR_API void air_free(pair_hier h);

/* ---------------------------------------------------------------------------
 * Upwind DG transport (Eq. weak_form_transport) on two mesh kinds:
 *  PAIR_MESH_HEX: the unit cube split into n^3 hexahedra, Q1 elements, element
 *    e = ix + n (iy + n iz), DOF 8 e + a, local node a = ax + 2 ay + 4 az;
 *  PAIR_MESH_TET: tetrahedra, P1 elements, DOF 4 t + a, local node a = vertex
 *    tets[4t + a]; face f of a tet is the triangle without its vertex f.
 * Vacuum boundaries unless g_inflow != 0.
 * ------------------------------------------------------------------------- */
#define PAIR_MESH_HEX 0
#define PAIR_MESH_TET 1
typedef struct {
    int kind;              /* PAIR_MESH_HEX or PAIR_MESH_TET */
    int n;                 /* hex: elements per axis */
    int ntet;              /* tet: number of tetrahedra */
    const double *verts;   /* tet: device, vertex coordinates, 3 per vertex */
    const int *tets;       /* tet: device, 4 vertex ids per tetrahedron */
    const int *nbr;        /* tet: device, 4 per tetrahedron: the tet across face f, -1 on the boundary */
} pair_mesh;

typedef struct {
    int M;                  /* directions */
    const double *omega;    /* HOST, M x 3 direction cosines */
    const double *w;        /* HOST, M weights (sum 4 pi for a full set) */
} pair_quad;

/* Stored entries of the block-scaled operator A = D^{-1} L of direction
 * 'omega' (host, 3 doubles): 8 per row for the identity diagonal plus 4 per
 * inflow face with an upwind neighbour (Sec. 1.3). */
PAIR_API pair_status dg_hex_nnz(const pair_mesh *mesh, const double *omega, int *nnz);

/* Assembles A = D^{-1} L for one direction (Eq. weak_form_transport, block
 * scaling of Sec. 1.3) into caller-allocated device CSR arrays (rowptr N+1,
 * col/val dg_hex_nnz entries).  Diagonal block = identity (stored as its
 * diagonal); off-diagonal face blocks D_K^{-1} L_KK' (8 x 4).  FP64, element
 * blocks factored by LU with partial pivoting; no compiler contraction, with an
 * explicit fma() in each LU update and substitution step.
 *   sigma_t  device, n^3 values.
 * PAIR_ERR_SINGULAR: an element block with a zero pivot. */
PAIR_API pair_status dg_assemble_hex(const pair_mesh *mesh, const double *omega, const double *sigma_t,
                            int *rowptr, int *col, double *val, void *stream);

/* Tetrahedral counterpart of dg_assemble_hex (P1, block size 4, coupling
 * blocks 4 x 3).  The row pointer (N + 1 = 4 ntet + 1 entries) is always
 * written and *nnz receives the entry count; col and val (capacity entries)
 * are written only when non-NULL and capacity >= *nnz, so a first call with
 * col = val = NULL sizes the arrays.  Tetrahedra are tested for zero volume
 * (PAIR_ERR_SINGULAR). */
PAIR_API pair_status dg_assemble_tet(const pair_mesh *mesh, const double *omega, const double *sigma_t, int *rowptr,
                                     int *col, double *val, int capacity, int *nnz, void *stream);

/* Scalar-flux reduction for angular decomposition (Sec. 5, parallel in angle: each
 * process holds the whole mesh and a subset of the directions, and the scalar
 * flux is summed over the processes once per source iteration).  si_solve, given
 * a quadrature subset, calls it once per SI iteration with v = a device array of
 * n = N + 1 doubles: the partial flux sum_{m in subset} w_m psi_m (N values), then
 * this process's status (0, or 1 if one of its direction solves missed inner_tol).
 * The function must replace all n values by their sums over the processes (for
 * example an all-reduce) with the work complete on the device when it returns,
 * and return 0; any other return ends si_solve with PAIR_ERR_COMM.  Every process
 * then holds the same flux and takes the same stopping decision; a summed status
 * above 0 ends every process's si_solve with PAIR_ERR_NOT_CONVERGED.  Each process
 * passes the same mesh, cross sections and initial phi.  The function runs on the
 * thread that called si_solve, between kernels of the library's private stream. */
typedef int (*pair_reduce_fn)(double *v, long long n, void *ctx);

/* Source-iteration controls. */
typedef struct {
    double tol;          /* stop when ||phi^{n+1} - phi^n|| <= tol ||phi^{n+1}|| (2-norm) */
    int max_iters;       /* SI iterations (1 = exactly one iteration) */
    double inner_tol;    /* per-direction solve: ||b - A psi|| <= inner_tol ||b|| */
    int inner_maxit;     /* V-cycles per direction solve */
    int batch;           /* directions per batch (0: all that fit the memory budget) */
    double mem_budget_gb;/* device memory for hierarchies (0: 60% of free memory) */
    double g_inflow;     /* isotropic inflow angular flux on the inflow boundary (0: vacuum) */
    int use_graphs;      /* capture the V-cycle of a batch in a CUDA graph */
    int fixed_iters;     /* 1: run exactly max_iters SI iterations (stop early only at tol)
                          * and return PAIR_OK with the last change in info; 0: missing
                          * tol after max_iters > 1 iterations is PAIR_ERR_NOT_CONVERGED */
    int solver;          /* 0: AIR per direction (the method); 1: exact GPU sweep of the
                          * block-scaled system (Sec. 1.1, the comparison of Sec. 6):
                          * upwind wavefronts on hexahedral meshes, a level schedule
                          * with cyclic components solved as dense blocks on
                          * tetrahedral meshes (see pair_sweep); air is then not used */
    int inner_cycles;    /* 0: every direction solved to inner_tol from psi = 0 (the
                          * method); l > 0: exactly l V-cycles from psi = 0, a fixed
                          * approximate inverse, so SI converges to the modified problem
                          * it defines (Sec. 3, inexact solves; inner_tol is not used) */
    const double *q_ang; /* NULL, or device array M*N (direction-major) of nodal values of
                          * an angular source density added to each direction's source
                          * (sigma_s phi + q) / (4 pi), e.g. the manufactured-solution
                          * source of the Appendix; caller-owned */
    pair_reduce_fn phi_reduce; /* NULL, or the scalar-flux reduction of a direction subset
                          * (Sec. 5, parallel in angle), see pair_reduce_fn */
    void *reduce_ctx;    /* passed to phi_reduce unchanged */
    int concurrent;      /* direction groups solved at the same time (si_solve and
                          * si_adjoint), each batch on its own stream from its own host
                          * thread, when every hierarchy is resident (0: min(M, 3); 1:
                          * one batch after another).  The
                          * directions are split into at least this many batches; each
                          * group sums its batches' w_m psi_m and phi^{n+1} adds the
                          * group sums in group order, so the flux is deterministic for
                          * a given value (and differs between values only by rounding).
                          * The exact sweep (solver 1) always runs one batch at a time. */
    int timing;          /* k >= 1: CUDA events around the level-0 kernels and each
                          * coarse level's sweeps in the V-cycles of SI iterations k, 2k,
                          * ... (counting from 1; the per-kernel times and traffic of
                          * si_info, summed over those cycles), the concurrent groups
                          * then running one after another so that no other group's
                          * kernels fall between a kernel's events; 0: none.  An event
                          * between two kernels of a captured cycle ends their
                          * programmatic overlap, so timed cycles replay graphs of their
                          * own and run slower (~10% on the 32^3 S4 batch); the other
                          * iterations replay graphs without events. */
} si_params;

PAIR_API void si_params_default(si_params *p);   /* 1e-8, 500, 1e-8, 100, 0, 0, 0, 1, 0, 0, 0, NULL, NULL, NULL, 0, 0 */

typedef struct {
    int si_iters;
    double si_change;        /* last ||phi^{n+1}-phi^n|| / ||phi^{n+1}|| */
    int vcycles;             /* total V-cycles (refinement steps) over all solves */
    double max_inner_resid;  /* max final relative FP64 residual over direction solves */
    int batches;             /* direction batches per SI iteration */
    int rebuilt;             /* 1 if hierarchies were rebuilt every SI iteration */
    double t_setup_ms;       /* assembly + AIR setup time (host clock around each batch's
                              * setup; with concurrent groups the longest batch's) */
    double t_solve_ms;       /* RHS build + solves + scalar-flux sums (device events; with
                              * concurrent groups the wall time less the setup) */
    int levels_max;          /* deepest hierarchy */
    double op_complexity;    /* sum_l nnz(A_l) / nnz(A_0), mean over directions */
    /* device-event timings of the level-0 kernels and their algorithmic traffic
     * (bytes the method must move: operator entries, vectors read and written),
     * summed over batches; with concurrent groups a kernel's events also span the
     * other groups' kernels that ran beside it */
    double t_res0_ms;        /* FP64 residual r = b - A psi, all launches */
    int n_res0;
    double gb_res0;          /* algorithmic GB over those launches */
    double t_relax0_ms;      /* level-0 F- and C-Jacobi passes, all launches */
    int n_relax0;
    double gb_relax0;
    double t_setup_phase_ms[4]; /* strength+PMIS, P+lAIR, Galerkin RAP, other setup (with
                                 * concurrent groups: those of the longest batch setup) */
    double t_relaxc_ms;      /* F- and C-Jacobi passes on levels >= 1 (SELL copies) and
                              * the grid-wide coarsest sweeps of levels >= 1, all cycles */
    int n_relaxc;            /* cycles measured */
    double gb_relaxc;        /* algorithmic GB of those passes */
    double t_res32_ms;       /* FP32 inner residuals r - A d of the refinement steps */
    int n_res32;
    double gb_res32;
    int outer_residuals;     /* outer (FP64-accurate) residuals that read the operator, over all
                              * direction solves (the first one of a solve from psi = 0 is b) */
    double t_relaxc_level_ms[8]; /* t_relaxc_ms by level: entry k is level k + 1 (the last
                                  * entry also holds deeper levels) */
    int timed_iters;         /* SI iterations whose cycles the kernel timings cover
                              * (si_params.timing) */
    double t_xfer_ms;        /* grid transfers: every level's restriction (R_l applied to
                              * b_l) and one-point prolongation, all cycles */
    int n_xfer;              /* cycles measured */
    double gb_xfer;          /* algorithmic GB of those transfers */
} si_info;

/* Source iteration (Eq. sn_transport with Eq. angular_quad): each iteration
 * solves every direction m with AIR, A_m psi_m = D_m^{-1} M (sigma_s phi^n + q)/(4 pi),
 * from psi = 0 to inner_tol, then phi^{n+1} = sum_m w_m psi_m (FP64, fixed m
 * order).
 *   sigma_t, sigma_s, q   per-element values (n^3 or ntet)
 *   phi      N DOFs (8 n^3 or 4 ntet): in = initial guess, out = result
 *   psi      N*M (direction-major) or NULL
 * These arrays (and sp->q_ang) may be device memory or HOST memory (pinned,
 * registered or pageable), each on its own: a host array is copied to a device
 * buffer on 'stream' before the solve and phi / psi are copied back after it (so
 * a host phi or psi is complete when si_solve returns); pinned host memory makes
 * the copies asynchronous DMA.
 *   air      AIR parameters (precision selects FP64 or FP32-refined)
 *   info     host, may be NULL.
 * Errors: PAIR_ERR_NAN if sigma_t, sigma_s, q, the initial phi or q_ang holds a
 * NaN or Inf (checked before any other work), or a residual or the scalar flux
 * turns non-finite; PAIR_ERR_SINGULAR for a zero-volume tetrahedron or a
 * singular element block (checked right after assembly, before the setup);
 * PAIR_ERR_OOM when sp->mem_budget_gb (or, at 0, the free device memory) is below
 * the estimated footprint of one direction; PAIR_ERR_NOT_CONVERGED as described
 * for fixed_iters.  After any error the library holds no state of the call, and
 * later calls work normally. */
PAIR_API pair_status si_solve(const pair_mesh *mesh, const pair_quad *quad, const double *sigma_t, const double *sigma_s,
                     const double *q, const air_params *air, const si_params *sp, double *phi, double *psi,
                     void *stream, si_info *info);

/* Adjoint source iteration and cross-section gradients of J = g^T phi, the
 * discrete adjoint of si_solve's fixed point (the paper has no adjoint; the
 * forward equations are Eq. sn_transport and Eq. angular_quad):
 *   A_m^T y_m = phis,  phis <- g + sigma_s (sum_m w_m W_m^T y_m) / (4 pi),
 *   W_m = D_m^{-1} M (so W_m^T y_m = M D_m^{-T} y_m, M symmetric);
 *   dJ/dsigma_t,K = -sum_m w_m y_{m,K}^T W_{m,K} psi_{m,K}
 *   dJ/dsigma_s,K =  sum_m w_m y_{m,K}^T W_{m,K} phi_K / (4 pi)
 *   dJ/dq_K       =  sum_m w_m y_{m,K}^T W_{m,K} 1 / (4 pi)
 * Each A_m^T gets its own AIR hierarchy (all directions batched); with
 * sp->solver = 1 each A_m^T y_m = phis is instead solved exactly by the GPU
 * sweep (the level schedule of pair_sweep on the transposed operator).
 *   psi            device N*M, the converged forward angular fluxes (si_solve's psi)
 *   g              device N, dJ/dphi (e.g. detector weights)
 *   dJ_dsigma_t, dJ_dsigma_s, dJ_dq   device per-element outputs (n^3 or ntet)
 *   phi_adjoint    device N output (adjoint scalar flux) or NULL
 * Every direction's hierarchy must fit the memory budget (PAIR_ERR_OOM otherwise).
 * Hexahedral (8 DOFs per element) and tetrahedral (4 DOFs per element) meshes. */
PAIR_API pair_status si_adjoint(const pair_mesh *mesh, const pair_quad *quad, const double *sigma_t,
                                const double *sigma_s, const double *q, const double *psi, const double *g,
                                const air_params *air, const si_params *sp, double *dJ_dsigma_t,
                                double *dJ_dsigma_s, double *dJ_dq, double *phi_adjoint, void *stream,
                                si_info *info);

/* Transpose of a device CSR matrix into caller-allocated device arrays
 * (trowptr n+1, tcol and tval nnz), columns ascending in every row. */
PAIR_API pair_status pair_csr_transpose(const pair_csr *A, int *trowptr, int *tcol, double *tval, void *stream);

/* Exact solve A x = b of one block-scaled upwind operator by a level-scheduled
 * GPU sweep (Sec. 1.1, the transport sweep that pAIR replaces; Sec. 6).  A is
 * the operator of one direction after block-inverse scaling (Sec. 1.3), as
 * dg_assemble_* returns it: rows in element blocks of nb = 4 (P1 tetrahedra)
 * or 8 (Q1 hexahedra) DOFs, each diagonal block the identity.  Elements are
 * grouped by upwind level (level = 1 + the largest level upwind) and each
 * level is one launch: x_K = b_K - sum A_KK' x_K' over the rows' entries
 * outside the element, in stored order, multiply and subtract unfused.  A
 * cycle of the element graph (possible on tetrahedra) is a strongly connected
 * component solved as one dense block by LU with partial pivoting; a component
 * may have at most 32 unknowns (8 tetrahedra), and an element may reference at
 * most as many elements as it has faces.
 *   A          device CSR (n = nb * elements rows, global column indices)
 *   b, x       device, n doubles each (x is written, b is read)
 *   n_cycles   host, may be NULL: number of cyclic components solved
 *   n_levels   host, may be NULL: number of levels of the schedule
 * The schedule is built, used once and released (device memory at most
 * 50 bytes per element while it runs); the call synchronises the stream.
 * PAIR_ERR_ARG: nb not 4 or 8, n not a multiple of nb or a column out of
 * range; PAIR_ERR_UNSUPPORTED: a larger cycle or more references than faces;
 * PAIR_ERR_SINGULAR: a singular cyclic component. */
PAIR_API pair_status pair_sweep(const pair_csr *A, int nb, const double *b, double *x, void *stream, int *n_cycles,
                                int *n_levels);

PAIR_API const char *pair_last_error(void);

/* ---------------------------------------------------------------------------
 * Allocation-free residual.  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need a
 * residual, for example code running inside a memory arena or pool that
 * forbids cudaMalloc/cudaFree (an allocation there would synchronise the
 * device or bypass the arena's accounting), or an application that has
 * already reserved all device memory for its own buffers.
 *
 * r = b - A x and rnorm[0] = ||r||_2 (FP64, deterministic), for one CSR
 * matrix.  All arrays are caller-owned device memory: A's arrays, b, x, r (n
 * doubles each) and rnorm (one double).  The call allocates nothing: its only
 * scratch, one partial sum per 256 rows, lives in a static device array of
 * PAIR_NOALLOC_MAX_ROWS / 256 doubles (512 KiB) that every GPU which loads the
 * library holds until the process exits.  Matrices with more than
 * PAIR_NOALLOC_MAX_ROWS rows are rejected with PAIR_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address; make that
 * first call before any stream capture.  The address is kept with the id of
 * the CUDA context it was found in, so after a device reset the next call
 * looks it up again (make that call before any capture as well).  All calls share the one array, so
 * calls whose work overlaps on the GPU (different streams, no ordering) race
 * and must not be issued; each call writes every scratch entry it reads, so
 * nothing needs clearing between calls.  Ordered on 'stream'.
 * ------------------------------------------------------------------------- */
#define PAIR_NOALLOC_MAX_ROWS (1 << 24)
PAIR_API pair_status pair_residual_norm_noalloc(const pair_csr *A, const double *b, const double *x, double *r,
                                                double *rnorm, void *stream);

/* Library kernels launched so far by this process (graph replays count each
 * captured kernel once per replay).  Instrumentation for benchmarks; not
 * thread-safe with concurrent library calls. */
PAIR_API long long pair_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* PAIR_H */
