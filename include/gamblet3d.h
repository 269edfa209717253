/*
 * gamblet3d.h - C ABI of the three-dimensional gamblet solver.
 *
 * The method of Sec. 4 and 5 is stated for a domain of R^d; this is its
 * d = 3 instance: nested dyadic cubes (Construction defmulires with
 * H = 1/2, so a cube has up to eight children), the detail basis W^(k) of
 * Construction const2 (normalised Helmert rows of Lemma const0 on the
 * active children, ordered by the slot (x & 1) + 2 (y & 1) + 4 (z & 1)),
 * the localized patch systems of Definition defb (Algorithm 2 line 11),
 * R^(k-1,k) = pibar + D W (line 12), the Galerkin products
 * A^(k-1) = R A^(k) R^T (line 13) and the solve by restriction, level CG,
 * prolongation and sum (lines 15-18), refined by a float64 flexible CG on
 * the fine operator that uses the gamblet operator as its preconditioner.
 *
 * Every computation runs in float64 on the current CUDA device.  Shared
 * types (gamblet_csr, gamblet_opts, gamblet_info, gamblet_status) and the
 * pointer, error and stream conventions are those of gamblet.h.
 */
#ifndef GAMBLET3D_H
#define GAMBLET3D_H

#include "gamblet.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gamblet3d_ctx* gamblet3d_handle;

/*
 * Fine-to-coarse setup with psi^(q) = phi (A^(q) = A).
 *   A      fine stiffness, symmetric positive definite, A->n >= 1 unknowns.
 *   q      number of levels, 2 <= q <= 8.
 *   cells  n x 3 int32, row-major: the level-q lattice cell (x, y, z) of
 *          each unknown, 0 <= x, y, z < 2^q, all distinct.  The level-k
 *          cell is the coordinates shifted right by q - k bits.
 *   opts   NULL = defaults (gamblet_default_opts).  Honoured fields: rho
 *          (patch radius in level-(k-1) cells; rho <= 0 = unbounded, the
 *          exact transform of Algorithm 1), nbr_rule (0 Euclidean distance
 *          between closed cubes, 1 Chebyshev box), level_tol,
 *          level_max_iter, refine_tol, refine_max_iter, patch_tol (> 0: the
 *          relative residual of the block-Jacobi CG of each patch system;
 *          0: 1e-12), profile (per-kernel device times,
 *          gamblet3d_kernel_stats) and stream.
 *          precision must be GAMBLET_FP64 (MIXED returns UNSUPPORTED).
 *   out    receives the handle.
 * Returns INVALID_ARG for malformed input (a cell outside the lattice or
 * shared by two unknowns, a column index out of range, bad sizes), NOT_SPD
 * if a block-Jacobi factor or the level-1 Cholesky meets a non-positive
 * pivot, UNSUPPORTED when a patch or a Galerkin row exceeds the shared
 * memory of one CTA (patch radius too large for the level sizes), and
 * NOT_CONVERGED when a patch CG hit its iteration cap (the handle is still
 * returned and usable).
 */
GAMBLET_API gamblet_status gamblet3d_setup(const gamblet_csr* A, int32_t q, const int32_t* cells,
                                           const gamblet_opts* opts, gamblet3d_handle* out);

/*
 * Solve A u = g: the one-pass gamblet transform (restriction, the
 * independent level systems B^(k) w^(k) = W^(k) g^(k) by block-Jacobi CG,
 * A^(1) U^(1) = g^(1) by Cholesky, prolongation and sum), refined by a
 * float64 flexible CG on A with that operator as preconditioner until
 * |g - A u| <= refine_tol |g| (refine_max_iter = 0: the one-pass solution).
 *   g, u        n float64 (host or device).
 *   components  NULL or q x n float64: row 0 = u^(1), row k-1 =
 *               u^(k) - u^(k-1) of the one-pass transform of g.
 *   info        NULL or receives iteration counts, residual and times.
 * Returns NOT_CONVERGED (u still written) if a cap was hit.
 */
GAMBLET_API gamblet_status gamblet3d_solve(gamblet3d_handle h, const double* g, double* u,
                                           double* components, gamblet_info* info);

/* Number of nodes n_k = |I^(k)| and detail rows |J^(k)| at level k. */
GAMBLET_API gamblet_status gamblet3d_level_size(gamblet3d_handle h, int32_t k, int32_t* n_k,
                                                int32_t* nJ_k);

/*
 * Copy one level operator to caller memory as COO triplets in the oracle's
 * index order: level q in the caller's unknown order; level k < q by the
 * cells' row-major key (z, y, x) (x fastest); rows of W^(k) by parent, then
 * t = 1..m-1.
 *   which  0 = A^(k) (n_k x n_k), 1 = R^(k-1,k) (n_(k-1) x n_k, k >= 2),
 *          2 = B^(k) (|J^(k)| x |J^(k)|, k >= 2).
 *   capacity  size of rows, cols and vals (host arrays); *nnz receives the
 *          count.  capacity 0 queries the count.  Structurally present zeros
 *          may be included.
 */
GAMBLET_API gamblet_status gamblet3d_get_operator(gamblet3d_handle h, int32_t which, int32_t k,
                                                  int64_t capacity, int64_t* nnz, int32_t* rows,
                                                  int32_t* cols, double* vals);

/* Launch geometry of level k (2 <= k <= q): geom[0] = patch neighbours NB,
 * geom[1] = block offsets |O_k| of A^(k), geom[2] = patch CG iterations
 * (largest), geom[3] = dilated offsets of the Galerkin rows. */
GAMBLET_API gamblet_status gamblet3d_level_geometry(gamblet3d_handle h, int32_t k, int32_t* geom);

/* Per-kernel statistics of the handle's setup and solves when opts.profile
 * = 1 (CUDA-event time on the library's stream, launches, and algorithmic
 * bytes and flops), as for gamblet_kernel_stats; returns the number of
 * entries available (capacity 0 queries it). */
GAMBLET_API int32_t gamblet3d_kernel_stats(gamblet3d_handle h, gamblet_kernel_stat* out,
                                           int32_t capacity);
GAMBLET_API void gamblet3d_reset_kernel_stats(gamblet3d_handle h);

/* Device bytes held by the handle. */
GAMBLET_API int64_t gamblet3d_device_bytes(gamblet3d_handle h);

/* Release every resource of the handle (NULL is ignored). */
GAMBLET_API void gamblet3d_destroy(gamblet3d_handle h);

#ifdef __cplusplus
}
#endif

#endif /* GAMBLET3D_H */
