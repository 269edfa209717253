/*
 * gamblet.h - C ABI of the GB300 gamblet multiresolution solver.
 *
 * Problem (Sec. 5.1, discrete system (eqhuiuhiuhuiu)): given the fine
 * stiffness matrix A = A^(q) of -div(a grad u) = g (symmetric positive
 * definite, CSR) and a nested dyadic measurement hierarchy, compute the
 * gamblet transform (Sec. 4, Algorithms 1 and 2 of Sec. 5) and the solution
 * u of A u = g as the sum of its level components (Theorem thmgugyug2).
 *
 * Hierarchy (Sec. 4.1, Definition defindextree / Construction defmulires,
 * H = 1/2): every fine unknown i carries a level-q lattice cell
 * (x_i, y_i), 0 <= x_i, y_i < 2^q, all distinct.  The level-k subdomain of i
 * is the cell (x_i >> (q-k), y_i >> (q-k)); I^(k) is the set of non-empty
 * level-k cells, pi^(k-1,k) aggregates children into parents
 * (Eq. eq:eigdeiud3dd).  Each level-(k-1) cell has m <= 4 children.  The
 * detail basis W^(k) is Construction const2 (Sec. 4.6: normalised rows of
 * U^(m), Lemma const0; children ordered row-major by (y & 1, x & 1)).
 *
 * Pointers: every array argument may be host memory (pageable or pinned) or
 * device memory of the current CUDA device; the library tells them apart with
 * cudaPointerGetAttributes and copies as needed.  The caller owns all input
 * and output buffers; the handle owns every device buffer of the hierarchy.
 *
 * Errors: every function returns a gamblet_status.  No call aborts or
 * throws; gamblet_last_error() returns a thread-local message describing the
 * last failure.  A handle whose call failed with GAMBLET_ERR_CUDA should be
 * destroyed.
 *
 * Streams: work is issued on opts.stream (a cudaStream_t, 0 = legacy
 * default stream).  gamblet_setup and gamblet_solve return after their
 * results are complete (they synchronise that stream once at the end).
 */
#ifndef GAMBLET_H
#define GAMBLET_H

#include <stdint.h>

#if defined(__GNUC__)
#define GAMBLET_API __attribute__((visibility("default")))
#else
#define GAMBLET_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GAMBLET_OK = 0,
  GAMBLET_ERR_INVALID_ARG = 1,     /* bad size, pointer, layout or option   */
  GAMBLET_ERR_NOT_SPD = 2,         /* non-positive pivot in a Cholesky      */
  GAMBLET_ERR_NOT_CONVERGED = 3,   /* iteration cap hit; result still written */
  GAMBLET_ERR_CUDA = 4,            /* CUDA runtime error                    */
  GAMBLET_ERR_OUT_OF_MEMORY = 5,   /* device allocation failed              */
  GAMBLET_ERR_UNSUPPORTED = 6      /* valid input outside this build's limits */
} gamblet_status;

/* Square sparse matrix in CSR form with 0-based int32 indices. */
typedef struct {
  int32_t n;               /* rows = columns                                */
  int64_t nnz;             /* number of stored entries                      */
  const int32_t* rowptr;   /* n + 1 offsets                                 */
  const int32_t* colind;   /* nnz column indices                            */
  const double* val;       /* nnz values                                    */
} gamblet_csr;

typedef enum {
  GAMBLET_FP64 = 0,   /* every stage in float64                              */
  GAMBLET_MIXED = 1   /* patch factorisations, Galerkin products and level
                         matrix-vector products in float32 with float32
                         accumulation; dots, residuals, the coarsest solve and
                         the outer refinement in float64                     */
} gamblet_precision;

typedef struct {
  /* Localization radius rho (Sec. 4.10 / Definition defb), in level-(k-1)
   * cells.  rho <= 0 selects the exact, non-localized transform of
   * Algorithm 1 (dense levels; small problems only).                        */
  double rho;
  /* Neighbourhood rule for i^rho: 0 = Euclidean distance between closed
   * squares <= rho (the paper's rule), 1 = Chebyshev box max(|dx|,|dy|)<=rho. */
  int32_t nbr_rule;
  int32_t precision;        /* gamblet_precision                           */
  double level_tol;         /* relative residual target of each level CG   */
  int32_t level_max_iter;   /* iteration cap of each level CG              */
  double refine_tol;        /* outer float64 relative residual target      */
  int32_t refine_max_iter;  /* cap on outer flexible-CG iterations; 0 = the
                               one-pass transform of Algorithm 2 only      */
  /* Patch systems of Definition defb: > 0 = block-Jacobi preconditioned CG
   * to this relative residual (Sec. 5.4 / Thm tmdiscreteaccuracy allow
   * inexact patch solves); 0 = default (1e-3 mixed, 1e-12 float64);
   * < 0 = dense Cholesky (exact to rounding).  An inexact patch solve only
   * changes R (any full-rank R keeps R A R^T SPD), so the mixed default
   * trades a slightly weaker preconditioner for fewer patch iterations;
   * the outer float64 iteration restores the accuracy.                    */
  double patch_tol;
  int32_t use_graph;        /* capture repeated launch sequences in CUDA graphs */
  int32_t profile;          /* 1: time every kernel phase with CUDA events on
                               the library's stream (gamblet_kernel_stats)  */
  int32_t autotune;         /* 1: pick launch shapes (patch solver and its
                               lanes per neighbour parent, Galerkin kernel,
                               lanes and threads per CTA, level-CG SpMV
                               tile) by timing candidates on a sample of
                               each large level, once per geometry and
                               precision in a process; 0: fixed rules      */
  int32_t galerkin_variant; /* -1: automatic; 0..8: use that Galerkin
                               kernel on every level (3, 4, 5: the tile
                               kernel with 8, 4, 16 lanes per output;
                               6, 7, 8: the tile kernel with 4, 8, 16
                               lanes per horizontal pair of outputs;
                               see gamblet_launch_shapes)                  */
  int32_t patch_gather;     /* -1: automatic; 0, 1, 2: use the SIMT patch
                               CG with that block gather on every level;
                               3, 4: the tensor-core patch solves
                               (tcgen05, float16 block-Jacobi-scaled patch
                               matrices, float32 accumulation) with windows
                               of 1 x 1 or 2 x 2 coarse cells per CTA on
                               every level - mixed path only, UNSUPPORTED
                               otherwise.  Automatic considers the
                               tensor-core solves on the mixed path when
                               patch_tol >= 4.8e-4 (their float16 rounding
                               of the scaled matrix is 2^-11 relative)     */
  void* stream;             /* cudaStream_t                                */
} gamblet_opts;

typedef struct {
  int32_t status;           /* gamblet_status of the call                   */
  int32_t q;                /* number of levels                             */
  int32_t outer_iters;      /* outer float64 iterations performed           */
  int32_t level_iters[32];  /* level CG iterations summed over the call, [k] */
  double rel_residual;      /* |g - A u|_2 / |g|_2 in float64 at exit       */
  double setup_ms;          /* device time of the last gamblet_setup        */
  double solve_ms;          /* device time of this call                     */
  int32_t patch_iters_max;  /* largest patch CG iteration count in setup (0 = Cholesky) */
  double patch_iters_mean;  /* mean patch CG iterations per patch in setup  */
} gamblet_info;

typedef struct gamblet_ctx* gamblet_handle;

/* Fill *opts with defaults: rho = 3, Euclidean rule, FP64, level_tol 1e-8,
 * level_max_iter 1000, refine_tol 1e-13, refine_max_iter 50, graphs on,
 * profiling off, autotuning on (no forced kernel variants), default
 * stream. */
GAMBLET_API void gamblet_default_opts(gamblet_opts* opts);

/*
 * Fine-to-coarse setup (Algorithm 1 lines 7-15 for rho <= 0, Algorithm 2
 * lines 7-15 with Definition defb otherwise), with psi^(q) = phi (the
 * initialisation described after Algorithm 1 in Sec. 5.2: A^(q) = A).
 *   A      fine stiffness, symmetric positive definite; A->n = number of
 *          fine unknowns (>= 1).  Entries may couple only cells within the
 *          same or adjacent level-(q-1) cells' stencil reach (any sparse
 *          pattern; the stored pattern must be symmetric).
 *   q      number of levels, 2 <= q <= 15.
 *   cells  n x 2 int32, row-major: cells[2 i] = x_i, cells[2 i + 1] = y_i.
 *   opts   options (NULL = defaults).
 *   out    receives the handle.
 * Returns INVALID_ARG for malformed input (duplicate or out-of-range cells,
 * bad CSR), NOT_SPD if a factorisation meets a non-positive pivot,
 * UNSUPPORTED if a patch exceeds the on-chip capacity of this build.
 */
GAMBLET_API gamblet_status gamblet_setup(const gamblet_csr* A, int32_t q, const int32_t* cells,
                             const gamblet_opts* opts, gamblet_handle* out);

/*
 * Setup with the level-q initialisation by the mass matrix (Algorithm 1,
 * lines 1-5; Algorithm 2, lines 2a-5 with Definition deflocinvm): the
 * level-q gamblets psi^(q)_i = sum_j (M^-1,loc)_{j,i} phi_j, where column i
 * of M^-1,loc solves the mass system restricted to the nodes whose cells lie
 * within distance rho_q of node i's cell (same rule as opts->nbr_rule) with
 * right-hand side e_i.  The hierarchy is built on
 * A^(q),loc = (M^-1,loc)^T A M^-1,loc (symmetrised), with g^(q) = g (the
 * nodal values of the right-hand side, Algorithm 1 line 4).  gamblet_solve
 * on the handle solves A^(q),loc U = g and returns the nodal coefficients
 * u = M^-1,loc U (with an unbounded rho_q: the solution of A u = M g).
 *   A, M    fine stiffness and mass matrices (same size, symmetric positive
 *           definite; cell offsets between coupled unknowns at most 5).
 *   rho_q   patch radius of M^-1,loc in level-q cell units (> 0).
 *   Other arguments as for gamblet_setup.  gamblet_grad is not available on
 *   the handle (UNSUPPORTED).  info->setup_ms includes the initialisation.
 */
GAMBLET_API gamblet_status gamblet_setup_mass(const gamblet_csr* A, const gamblet_csr* M,
                                              int32_t q, const int32_t* cells, double rho_q,
                                              const gamblet_opts* opts, gamblet_handle* out);

/*
 * Setup of nprob independent problems (each its own fine stiffness,
 * lattice and coefficient field, Sec. 5 per problem) as ONE hierarchy, so
 * that every level's patch solves, Galerkin products and level CGs of all
 * problems run in one launch per level.  The problems are placed, largest
 * first, in disjoint aligned subtrees of one 2^Q x 2^Q lattice (Q the
 * smallest with 4^Q >= sum_p 4^q[p]); the combined fine operator is block
 * diagonal.  On the levels where a problem still spans several cells, its
 * gamblets, R rows and level operators equal those of its own hierarchy
 * (patches that reach into a neighbouring subtree see zero coupling there);
 * above its own level 1 the measurement cells hold several problems, which
 * is again a nested hierarchy of the combined operator (Sec. 4.1), so the
 * solve is exact for every problem.
 *   nprob    number of problems (>= 1).
 *   A, q     arrays of nprob: fine stiffness and level count (1..15) of
 *            each problem, as for gamblet_setup (host or device arrays).
 *   cells    array of nprob pointers: n_p x 2 int32 cells of problem p in
 *            its own 2^q[p] lattice.
 *   opts     options (NULL = defaults); rho must be > 0.
 *   out      receives the handle; gamblet_solve on it takes g and u of
 *            sum_p n_p entries, problem after problem.
 *   offsets  NULL or host array of nprob + 1: problem p owns entries
 *            [offsets[p], offsets[p + 1]) of those vectors.
 * info->setup_ms includes packing the problems.  Returns INVALID_ARG for
 * malformed input (a column index or cell outside its problem), UNSUPPORTED
 * when the packed lattice would exceed 2^15 cells per side or the combined
 * CSR int32 indexing.
 */
GAMBLET_API gamblet_status gamblet_setup_batched(int32_t nprob, const gamblet_csr* A,
                                                 const int32_t* q, const int32_t* const* cells,
                                                 const gamblet_opts* opts, gamblet_handle* out,
                                                 int32_t* offsets);

/*
 * Solve A u = g (Eqs. eqyguugy6t, eqsdjoejddi1, eqsdjoejddi2, Theorem
 * thddwedmgugyug): restrict g through the levels, solve the independent
 * level systems B^(k) w^(k) = W^(k) g^(k) by CG and A^(1) U^(1) = g^(1)
 * directly, prolongate and sum.  With refine_max_iter > 0 this gamblet
 * operator preconditions a float64 flexible CG on A^(q) (Sec. 5.4: use as a
 * preconditioner) until |g - A u| <= refine_tol |g|.
 *   g           n float64 right-hand side.
 *   u           n float64 output.
 *   components  NULL, or q x n float64 output: row 0 = u^(1), row k-1 =
 *               u^(k) - u^(k-1) in fine coordinates (one-pass transform of
 *               g; their sum is the one-pass solution).
 *   info        NULL or receives iteration counts and residuals.
 * Returns NOT_CONVERGED (u still written) if a cap was hit.
 */
GAMBLET_API gamblet_status gamblet_solve(gamblet_handle h, const double* g, double* u,
                             double* components, gamblet_info* info);

/*
 * Several right-hand sides with one hierarchy (Sec. 5.4, subsequent
 * solves).  Right-hand sides go through the gamblet operator in groups of
 * up to four: the restriction, the level CG, the prolongation and the
 * float64 outer product read each matrix (Rhat, the level blocks, RT,
 * Ahat^(q)) once for the whole group (a sparse matrix times a block of
 * vectors); each right-hand side keeps its own outer flexible CG and stops
 * when it reaches refine_tol.
 *   nrhs  number of right-hand sides (>= 1).
 *   G     nrhs x n float64, row-major: right-hand side r at G + r * n.
 *   U     nrhs x n float64 output, same layout.
 *   info  NULL or receives the largest outer iteration count and the
 *         worst final relative residual.
 * Returns NOT_CONVERGED (U still written) if a right-hand side hit the cap.
 * Localized transform only.
 */
GAMBLET_API gamblet_status gamblet_solve_many(gamblet_handle h, int32_t nrhs, const double* G,
                                              double* U, gamblet_info* info);

/*
 * Truncated one-pass solve (Sec. 5.4, subsequent solves): u^(k) = u^(1) +
 * sum_{l=2..k} (u^(l) - u^(l-1)), the Galerkin approximation of u in the
 * span of the level-k gamblets psi^(k) (Theorem thddwedmgugyug, Eq.
 * eqhuhiuv), in fine coordinates.  The restriction runs to level 1, the
 * level systems 2..k are solved, and the levels above k only interpolate
 * (v^(l) = R^(l,l-1) v^(l-1)); no outer refinement.  k = q gives the
 * one-pass solution (gamblet_solve with refine_max_iter = 0).
 *   k   1 <= k <= q.   g, u, info as for gamblet_solve.
 */
GAMBLET_API gamblet_status gamblet_solve_truncated(gamblet_handle h, int32_t k, const double* g,
                                                   double* u, gamblet_info* info);

/*
 * Diagnostics: estimates of the extreme eigenvalues of B^(k) = W A^(k) W^T
 * (the level systems whose condition numbers the paper bounds uniformly in
 * k, Theorem thmodhehiudhehd) by the Lanczos process on the stored detail
 * blocks, steps iterations (capped at |J^(k)|) from a fixed pseudo-random
 * start, extremes of the Lanczos matrix by Sturm bisection.  Localized
 * transform only.  cond(B^(k)) ~ lmax / lmin.
 *   construction  2: W of Construction const2 (orthonormal rows, the basis
 *                 the library stores); 1: Construction const1 (row t of a
 *                 parent = child t minus child t + 1), for which
 *                 W1 A W1^T = M B M^T with the per-parent change of basis M
 *                 (Sec. 4.6; the paper compares the two constructions'
 *                 condition numbers).  Anything else: INVALID_ARG.
 */
GAMBLET_API gamblet_status gamblet_level_condition(gamblet_handle h, int32_t k,
                                                   int32_t construction, int32_t steps,
                                                   double* lmin, double* lmax);

/*
 * Compression in the normalised gamblet basis (Sec. 5.1, Example 1: the
 * representation of u in psi^(1)_i / ||psi^(1)_i||_a and chi^(k)_j /
 * ||chi^(k)_j||_a is sparse).  Runs the one-pass transform of g, forms the
 * normalised coefficients c^(1)_i = U_i sqrt(A^(1)_ii) and c^(k)_j =
 * w^(k)_j sqrt(B^(k)_jj), keeps those with |c| >= eps * max |c| and rebuilds
 * u from them (zeroed coefficients dropped from the level recursion).
 *   eps     relative threshold (>= 0; 0 keeps everything: the one-pass u).
 *   u       n float64 output (nodal coefficients after a mass setup).
 *   kept, total  NULL or receive the kept and the total coefficient counts.
 * Localized transform only (UNSUPPORTED for rho <= 0).
 */
GAMBLET_API gamblet_status gamblet_compress(gamblet_handle h, const double* g, double eps,
                                            double* u, int64_t* kept, int64_t* total);

/*
 * Adjoint gradient of J = 1/2 |u - u_obs|^2 with respect to theta_c =
 * log a_c for a cellwise-constant coefficient (the paper has no adjoint; the
 * discrete adjoint of A(theta) u = g):  A lambda = u - u_obs is solved with
 * the same hierarchy as gamblet_solve, then
 *   dJ/dtheta_c = -a_c sum_{p,r} lambda_{cell_nodes[4c+p]} K_ref[4p+r] u_{cell_nodes[4c+r]}
 * over the cell's corners (entries -1 = Dirichlet corner, skipped).
 *   ncell       number of cells.
 *   cell_nodes  ncell x 4 int32 fine unknown of each corner, or -1.
 *   cell_a      ncell float64 coefficient a_c.
 *   K_ref       4 x 4 float64 reference element matrix (row-major).
 *   u, u_obs    n float64: the current solution and the observation.
 *   dJ          ncell float64 output.
 *   J           NULL or receives J.
 */
GAMBLET_API gamblet_status gamblet_grad(gamblet_handle h, int32_t ncell, const int32_t* cell_nodes,
                            const double* cell_a, const double* K_ref, const double* u,
                            const double* u_obs, double* dJ, double* J, gamblet_info* info);

/*
 * Gradient of J = 1/2 |u_loc - u_obs|^2 through the ONE-PASS localized
 * transform: u_loc = G_loc g is the output of Algorithm 2 (lines 15-18: the
 * restriction with the localized R^(k-1,k), the level solves, the
 * prolongation and sum) with the handle's patch and level solves and no
 * outer refinement, and the derivative follows its dependence on the
 * coefficient through the localized setup (lines 7-13: the patch solves of
 * Definition defb, R^(k-1,k) and the Galerkin products).  The paper has no
 * such derivative; this is reverse-mode differentiation of those steps:
 *   dJ/dtheta_c = a_c sum_{p,r} sym(Abar^(q))_{cell_nodes[4c+p], cell_nodes[4c+r]} K_ref[4p+r],
 * theta_c = log a_c, Abar^(q) the adjoint of A^(q) after the reverse pass.
 * It is exact for the map that the handle computes when the patch and level
 * solves are exact; with tolerances it carries their error (tight
 * tolerances, e.g. patch_tol 1e-13 and level_tol 1e-13, give the derivative
 * of Algorithm 2 with exact solves).
 *   ncell, cell_nodes, cell_a, K_ref  as for gamblet_grad.
 *   g, u_obs    n float64: right-hand side and observation.
 *   u           NULL or n float64: receives u_loc.
 *   dJ          ncell float64 output.
 *   dJ_dg       NULL or n float64: receives dJ/dg = G_loc (u_loc - u_obs).
 *   J           NULL or receives J.
 * Host or device buffers.  Needs a localized handle of one problem, set up
 * with gamblet_setup and patch_tol >= 0; anything else returns UNSUPPORTED.
 * The reverse pass runs in the handle's working precision: float64 for
 * precision 0; float32 on the mixed path's float32 hierarchy (J, the misfit
 * and the outputs in float64), which gives the derivative of the float32
 * one-pass map to float32 accuracy (about 1e-4 relative with patch and level
 * tolerances of 1e-6).  NOT_CONVERGED if a level solve hit its cap (all
 * outputs still written).  Device work memory: about
 * e (|S_k| + 4 |S_k + N|) n_(k-1) bytes at the finest level k = q, e the
 * element size (a few hundred MB at 256 x 256 cells, rho = 3, float64),
 * released before return.
 */
GAMBLET_API gamblet_status gamblet_grad_onepass(gamblet_handle h, int32_t ncell,
                                                const int32_t* cell_nodes, const double* cell_a,
                                                const double* K_ref, const double* g,
                                                const double* u_obs, double* u, double* dJ,
                                                double* dJ_dg, double* J, gamblet_info* info);

/*
 * J = 1/2 |u - u_obs|^2, the objective that gamblet_grad also returns, for
 * callers that cannot allocate device memory when they need it: applications
 * whose framework allocator already holds the free device memory (a caching
 * allocator grows to fill the GPU, so a side cudaMalloc can fail), programs
 * under a hard device-memory budget, and loops that evaluate J many times
 * (an optimiser's line search) and cannot accept the device-wide
 * synchronisation of cudaFree.  The paper has no counterpart; this is a
 * service entry point.
 *   n       number of unknowns, 1 <= n <= GAMBLET_NOALLOC_MAX_N; larger n
 *           returns UNSUPPORTED.
 *   u, u_obs  device pointers of the current device, n float64 each; a host
 *           pointer or another GPU's memory returns INVALID_ARG.
 *   J       device pointer (current device) or host pointer to one float64;
 *           with a host pointer the call copies J back and waits for the
 *           stream.
 *   stream  cudaStream_t for the two kernels (0 = legacy default stream).
 * Allocates nothing: the partial sums live in a fixed 8.2 KB device array
 * that every GPU loading the library keeps until exit.  The first call on a
 * device looks up that array's address (cudaGetSymbolAddress) with the
 * device current; make that first call before any stream capture.  Calls
 * share the array, so calls that overlap on the GPU race; each call
 * overwrites every slot it reads, so no clearing is needed between calls.
 */
#define GAMBLET_NOALLOC_MAX_N 2097152
GAMBLET_API gamblet_status gamblet_objective_noalloc(int32_t n, const double* u,
                                                     const double* u_obs, double* J,
                                                     void* stream);

/*
 * Values of the fine operator of Sec. 5.1 (Eq. eqhuiuhiuhuiu) for a
 * coefficient constant on each cell: A = sum_c exp(log_a[c]) K_ref restricted
 * to the cell's interior corners, written into an existing CSR pattern.
 *   n, rowptr, colind, nnz  the pattern (device pointers); every pair of
 *                 interior corners of a cell must be present in it.
 *   ncell, cell_nodes  ncell x 4 int32 fine unknown of each corner, -1 on the
 *                 Dirichlet boundary (device pointer).
 *   log_a         ncell float64 (device pointer).
 *   K_ref         4 x 4 float64 element matrix (host or device).
 *   val           nnz float64 output (device pointer), overwritten.
 *   cell_a        NULL or ncell float64 output (device): exp(log_a).
 * Returns INVALID_ARG if a corner pair is missing from the pattern.
 */
GAMBLET_API gamblet_status gamblet_assemble_cells(int32_t n, const int32_t* rowptr,
                                                  const int32_t* colind, int64_t nnz,
                                                  int32_t ncell, const int32_t* cell_nodes,
                                                  const double* log_a, const double* K_ref,
                                                  double* val, double* cell_a, void* stream);

/* Launch shapes the setup used at level k (2 <= k <= q, localized
 * transform), chosen by the autotuner or by the fixed rules:
 *   shapes[0]  patch-CG threads per neighbour parent (1, 2, 4; 0 = Cholesky or
 *              tensor-core patch solves)
 *   shapes[1]  patch-CG block gather (0 thread per block, 1 half-warp per block,
 *              2 four lanes per block), or 3, 4 for the tensor-core patch
 *              solves with windows of 1 x 1 or 2 x 2 coarse cells
 *   shapes[2]  Galerkin kernel (0 thread per position, 1 warp-cooperative,
 *              2 warp per row, 3, 4, 5 2 x 2 row tiles with 8, 4, 16 lanes
 *              per output target)
 *   shapes[3]  level-CG SpMV threads per parent (1: 16 x 16 tiles, 4: 8 x 8,
 *              16: 4 x 4) */
GAMBLET_API gamblet_status gamblet_launch_shapes(gamblet_handle h, int32_t k, int32_t* shapes);

/* Number of nodes n_k = |I^(k)| and detail rows |J^(k)| at level k. */
GAMBLET_API gamblet_status gamblet_level_size(gamblet_handle h, int32_t k, int32_t* n_k, int32_t* nJ_k);

/*
 * Copy one level operator to caller memory as COO triplets in the oracle's
 * index order (level q: the caller's unknown order; level k < q: cells
 * sorted row-major by (y, x); J^(k): by parent, then t = 1..m-1).
 *   which  0 = A^(k) (n_k x n_k), 1 = R^(k-1,k) (n_{k-1} x n_k, k >= 2),
 *          2 = B^(k) (|J^(k)| x |J^(k)|, k >= 2).
 *   capacity  size of rows/cols/vals; *nnz receives the count.  Call with
 *          capacity 0 to query the count.  Entries that are structurally
 *          present but zero may be included.
 */
GAMBLET_API gamblet_status gamblet_get_operator(gamblet_handle h, int32_t which, int32_t k, int64_t capacity,
                                    int64_t* nnz, int32_t* rows, int32_t* cols, double* vals);

/* Per-kernel statistics accumulated since the handle was created or last
 * reset, when opts.profile = 1: CUDA-event time on the library's stream, the
 * number of launches, and the algorithmic bytes moved and flops performed
 * (counted from the data the operation must read and write once, not from
 * hardware counters).  Writes up to capacity entries; returns the number of
 * entries available (call with capacity 0 to query). */
typedef struct {
  char name[48];
  int64_t launches;
  double ms;
  double bytes;
  double flops;
} gamblet_kernel_stat;
GAMBLET_API int32_t gamblet_kernel_stats(gamblet_handle h, gamblet_kernel_stat* out,
                                         int32_t capacity);
GAMBLET_API void gamblet_reset_kernel_stats(gamblet_handle h);

/*
 * Host-only consistency check of the symbolic plan (needs no GPU): builds the
 * plan of a full 2^q x 2^q square (Q1 block stencil, patches i^rho of
 * Sec. 4.10 with rule nbr_rule) and verifies its tables against their
 * definitions derived independently - the half-plane of every symmetric
 * block stencil (one block per pair of opposite offsets), the patch block
 * lists and per-row adjacency (Definition defb), the tensor-core windows
 * (union of the patches, membership bits, blocks, right-hand-side offsets,
 * output map), the phase-1 lists of the tiled Galerkin product (every
 * contribution Ahat[o][u] Rhat_r(j) with u = r + N_j - O_o at a position the
 * outputs read, exactly once), its phase-2 lists, single and paired (every
 * incidence of an output target c with a window position c + N_j,
 * Eq. eqhuhiuv), and the next level's block stencil and conversion map
 * (every coupling of the coarse cell stencil in exactly one block).
 *   q         2..12; rho in (0, 8]; nbr_rule 0 (Euclidean) or 1 (box).
 *   counts    NULL or 5 int64: levels, phase-1 entries, phase-1 items,
 *             phase-2 incidences, half-plane offsets (summed over levels).
 * Returns INVALID_ARG with the first violated property in gamblet_last_error.
 */
GAMBLET_API gamblet_status gamblet_plan_check(int32_t q, double rho, int32_t nbr_rule,
                                              int64_t* counts);

/* Total CUDA kernel launches issued by this library in this process. */
GAMBLET_API int64_t gamblet_kernel_launches(void);

/* Device bytes held by the handle. */
GAMBLET_API int64_t gamblet_device_bytes(gamblet_handle h);

/* Release every resource of the handle (NULL is ignored). */
GAMBLET_API void gamblet_destroy(gamblet_handle h);

GAMBLET_API const char* gamblet_status_string(int32_t status);
GAMBLET_API const char* gamblet_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GAMBLET_H */
