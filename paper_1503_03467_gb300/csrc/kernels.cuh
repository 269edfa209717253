// kernels.cuh - launch wrappers of the gamblet device kernels.
//
// All launches take the stream explicitly and return immediately; the host
// orchestration in gamblet.cu checks cudaGetLastError after each phase.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

// ---------------------------------------------------------------- hierarchy
// cells (n x 2, device) -> Morton index of every fine unknown; flag[0] = 2
// when a cell lies outside [0, 2^q), flag[1] = largest Morton index.
void launch_cells_to_morton(const int32_t* cells, int n, int q, int32_t* morton_of, int* flag,
                            cudaStream_t s);
// Inverse map (Morton -> unknown or -1) and child masks of the level-q
// parents; flag[0] = 1 when two unknowns share a cell.
void launch_scatter_cells(const int32_t* morton_of, int n, int32_t* unknown_of,
                          uint32_t* pmask_q, int* flag, cudaStream_t s);
// ---------------------------------------------------------------- diagnostics
// y = B^(k) x on the detail slots of transformed level-k vectors (float64).
template <typename T>
void launch_detail_spmv(const T* Bd, const int2* off, int noff, int Lpar, int64_t npar,
                        const double* x, double* y, cudaStream_t s);
// deterministic pseudo-random start vector on the active detail slots
void launch_detail_start(int64_t npar, const uint32_t* pmask, double* v, cudaStream_t s);
// detail vectors from the stored Helmert basis to Construction const1:
// out = M in (transpose 0) or M^T in (1), per parent; W1 A W1^T = M B M^T
void launch_detail_basis(int64_t npar, const uint32_t* pmask, const double* in, double* out,
                         int transpose, cudaStream_t s);
// out = a x + b y + c z (y, z may be NULL)
void launch_lanczos_step(int64_t n, double a, const double* x, const double* y, double b,
                         const double* z, double c, double* out, cudaStream_t s);

// ---------------------------------------------------------------- compression
// max over the level's detail coefficients of |w_j| sqrt(B_jj), as the bit
// pattern of a non-negative double (atomicMax into *cmax).
template <typename T>
void launch_coef_max(const T* w, const T* Bd, int o0, int64_t npar, const uint32_t* pmask,
                     unsigned long long* cmax, cudaStream_t s);
// zero the w_j with |w_j| sqrt(B_jj) < thr; *kept += the others.
template <typename T>
void launch_coef_threshold(T* w, const T* Bd, int o0, int64_t npar, const uint32_t* pmask,
                           double thr, unsigned long long* kept, cudaStream_t s);

// ---------------------------------------------------------------- mass initialisation
// Largest |cell offset| (x, y) between the rows and columns of a fine CSR.
void launch_csr_node_extent(int n, const int32_t* rowptr, const int32_t* colind,
                            const int32_t* morton_of, int* ext, int* bad, cudaStream_t s);
// Fine CSR -> per-node stencil St[i][s] over the (2 rx + 1) x (2 ry + 1)
// cell offsets (row-major in (dy, dx)); St must be zeroed.
void launch_csr_to_stencil(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                           const int32_t* morton_of, int rx, int ry, double* St, cudaStream_t s);
// Minv[i][j]: column i of the localized mass inverse (Definition deflocinvm)
// on the patch nodes c_i + N_j; status receives DEV_NOT_SPD on a
// non-positive pivot.
void launch_mass_patch_inverse(int n, int NB, int jc, const int2* nbr, const double* Mst, int mrx,
                               int mry, const int32_t* morton_of, const int32_t* unknown_of,
                               int L, int64_t ncell, double* Minv, int* status, int num_sms,
                               cudaStream_t s);
size_t mass_patch_smem_bytes(int NB);
// Node-level lists of the product (M^-1,loc)^T A M^-1,loc (as the Galerkin
// lists, with scalar entries): window offsets W and pairs (s, j) with
// W_w + A_s = N_j; output offsets D and pairs (j, w) with W_w = D_d + N_j.
struct MassTripleGeom {
  int NB, nast;
  int nwin;
  const int2* win;
  const int* l1_ptr;
  const int2* l1;
  int nout;
  const int2* out;
  const int* l2_ptr;
  const int2* l2;
};
void launch_mass_triple(int n, MassTripleGeom g, const double* Ast, const double* Minv,
                        const int32_t* morton_of, const int32_t* unknown_of, int L, int64_t ncell,
                        double* out, cudaStream_t s);
void launch_stencil_counts(int n, const int2* off, int noff, const int32_t* morton_of,
                           const int32_t* unknown_of, int L, int64_t ncell, int32_t* count,
                           cudaStream_t s);
void launch_stencil_to_csr(int n, const int2* off, const int* mirror, int noff, const double* X,
                           const int32_t* morton_of, const int32_t* unknown_of, int L,
                           int64_t ncell, const int32_t* rowptr, int32_t* colind, double* val,
                           cudaStream_t s);
// u[j] = (M^-1,loc U)_j.
void launch_mass_apply(int n, int NB, const int2* nbr, const double* Minv, const double* U,
                       const int32_t* morton_of, const int32_t* unknown_of, int L, int64_t ncell,
                       double* u, cudaStream_t s);

// One problem of a batched setup: its unknowns start at row0 and its
// stored entries at nnz0 of the combined CSR; its 2^q lattice is the
// subtree with lower-left cell (x0, y0) of the combined lattice.
struct BatchSeg {
  int64_t row0, nnz0;
  int32_t n, q;
  int32_t x0, y0;
};
// In place on the concatenated arrays: rowptr += nnz0, colind += row0,
// cells += (x0, y0) per problem; flag = 1 for a column index outside its
// problem, 2 for a cell outside its problem's lattice.
void launch_batch_fixup(int nprob, const BatchSeg* seg, int64_t n, int64_t nnz, int32_t* rowptr,
                        int32_t* colind, int32_t* cells, int* flag, cudaStream_t s);
// Child masks of the npar_km1 level-(k-1) parents from the masks of the
// npar_k level-k parents: parent p at level k is active iff pmask_k[p] != 0.
void launch_coarsen_masks(const uint32_t* pmask_k, int64_t npar_k, uint32_t* pmask_km1,
                          int64_t npar_km1, cudaStream_t s);

// ---------------------------------------------------------------- fine operator
// Largest |parent offset| in x and y over the stored entries (atomicMax).
void launch_csr_offset_extent(int n, const int32_t* rowptr, const int32_t* colind,
                              const int32_t* morton_of, int* ext, int* bad_flag,
                              cudaStream_t s);
// Scatter A^(q) into a block stencil (rows/cols in slot space, untransformed).
// Offsets form the box [-rx, rx] x [-ry, ry], index (dy + ry) * (2 rx + 1) + dx + rx.
void launch_csr_to_blocks(int n, const int32_t* rowptr, const int32_t* colind,
                          const double* val, const int32_t* morton_of, int rx, int ry,
                          int64_t npar, double* blk, cudaStream_t s);

// Fine CSR -> node stencil in Morton order, St[s][c] (s over the box
// (2 rx + 1) x (2 ry + 1), row-major in (dy, dx)); St must be zeroed.
void launch_csr_to_mstencil(int n, const int32_t* rowptr, const int32_t* colind,
                            const double* val, const int32_t* morton_of, int rx, int ry,
                            int64_t ncell, double* St, cudaStream_t s);
// yhat = Q (A x): node-stencil SpMV on the untransformed level-q vector x,
// transformed output (one thread per parent).
void launch_stencil_spmv_q(const double* St, const int2* off, int ns, int L, int64_t ncell,
                           int64_t npar, const uint32_t* pmask, const double* x, double* yhat,
                           cudaStream_t s);
// out(o, p) = Q blk(o, p) Q'^T in float32 from an untransformed float64 stencil.
void launch_transform_blocks_f32(const double* blk, float* out, const int2* off, int noff,
                                 int64_t npar, int Lpar, const uint32_t* pmask, cudaStream_t s);

// ---------------------------------------------------------------- transforms
// In place: blk(o, p) <- Q_{mask p} blk(o, p) Q_{mask p+off_o}^T.
void launch_transform_blocks(double* blk, const int2* off, int noff, int64_t npar,
                             int Lpar, const uint32_t* pmask, cudaStream_t s);
// Copy a float64 block stencil to float32.
void launch_convert_f64_f32(const double* in, float* out, int64_t n, cudaStream_t s);
void launch_convert_f32_f64(const float* in, double* out, int64_t n, cudaStream_t s);

// x_hat = Q x (dir = +1) or x = Q^T x_hat (dir = -1) on a level vector whose
// parents have child masks pmask (4 * npar entries).
template <typename T>
void launch_transform_vec(const T* in, T* out, int64_t npar, const uint32_t* pmask, int dir,
                          cudaStream_t s);

// Gather unknown-ordered values to Morton order (inactive cells 0) and back.
void launch_gather_morton(const double* in_unknown, const int32_t* unknown_of, int64_t ncell,
                          double* out_morton, cudaStream_t s);
void launch_scatter_unknown(const double* in_morton, const int32_t* morton_of, int n,
                            double* out_unknown, cudaStream_t s);

// ---------------------------------------------------------------- patches
struct PatchGeom {
  int NB;              // neighbour offsets N_j (level k-1 cell units)
  int jc;              // index of (0, 0) in N
  const int2* nbr;     // N_j
  const int* pair_idx; // NB x NB: index in O_k of N_b - N_a, or -1
  int Lpar;            // side of the level-(k-1) lattice
  int64_t npatch;      // stored level-(k-1) cells (4^(k-1) for a full square)
};
// Localized patch solves of Definition defb for every coarse cell of level
// k-1; writes Rhat rows (SoA [NB * 4][npatch]).  status receives DEV_NOT_SPD
// on a non-positive pivot.
template <typename T>
void launch_patch_solve(const T* Ahat, const uint32_t* pmask_k, PatchGeom g, T* Rhat,
                        int* status, int num_sms, cudaStream_t s);
template <typename T>
size_t patch_smem_bytes(int NB);
// Same rows by block-Jacobi preconditioned CG to relative residual tol
// (at most max_iter iterations), on the patch's nonzero 3x3 blocks;
// iter_stats (device, 3 ints) accumulates the maximum and the sum of
// iterations and the number of patches.
struct PatchPcgGeom {
  int NB, jc;
  const int2* nbr;
  const int* pair_idx;  // NB x NB
  int Lpar;
  int64_t npatch;
  int nhalf;            // block slots in shared memory (stored blocks plus padding)
  const int4* half;     // per slot (ja, jb, o, 0) of a stored block ja >= jb, or ja = -1
  int nadj;             // adjacency entries (2 x stored blocks - NB)
  const int* adj_ptr;   // NB + 1
  const int4* adj;      // (stored block, other neighbour, transposed, 0)
  const int* diag_h;    // NB: stored block of (j, j)
  int spp;              // threads per neighbour parent: 1, 2 or 4
  int64_t i_begin, i_end;  // coarse cells solved: [i_begin, i_end) (all: 0, npatch)
  int gather;           // block gather: 0 thread per block, 1 half-warp per block,
                        // 2 four lanes (one row each) per block
};
template <typename T>
void launch_patch_pcg(const T* Ahat, const uint32_t* pmask_k, PatchPcgGeom g, T* Rhat, double tol,
                      int max_iter, int* iter_stats, int num_sms, cudaStream_t s);
template <typename T>
size_t patch_pcg_smem_bytes(const PatchPcgGeom& g);
// The same patch systems with right-hand sides rhs ([i][NB][4], detail
// slots; the adjoint solves of the reverse pass), solutions written to out
// in Rhat's layout with a zero average slot.
template <typename T>
void launch_patch_pcg_adjoint(const T* Ahat, const uint32_t* pmask_k, PatchPcgGeom g,
                              const T* rhs, T* out, double tol, int max_iter, int* iter_stats,
                              int num_sms, cudaStream_t s);

// Patch CG over a thread-block cluster (patch_cluster.cu) for patches whose
// blocks exceed one CTA's shared memory: CTA c of each cluster of cs keeps
// the block rows jsplit[c] <= j < jsplit[c + 1] (one warp per row, at most
// max_rows rows and max_blocks blocks per CTA); the direction vector and the
// inner products are exchanged through distributed shared memory.  Same
// iteration, stopping rule and iter_stats as launch_patch_pcg.  Returns the
// launch status (the cluster shape is checked by the runtime).
struct PatchClusterGeom {
  PatchPcgGeom pg;
  int cs;           // CTAs per cluster: 2, 4, 8 or 16
  int max_rows;     // rows of the largest range (32 threads each)
  int max_blocks;   // stored blocks of the largest range
  int jsplit[17];   // row ranges of the cs CTAs
};
template <typename T>
cudaError_t launch_patch_pcg_cluster(const T* Ahat, const uint32_t* pmask_k,
                                     const PatchClusterGeom& c, T* Rhat, double tol,
                                     int max_iter, int* iter_stats, cudaStream_t s);
template <typename T>
size_t patch_cluster_smem_bytes(const PatchClusterGeom& c);

// Tensor-core patch solves (patch_mma.cu, float32 path): the patches of the
// G x G coarse cells i = NP w .. NP w + NP - 1 (NP = G^2, Morton order) share
// one CTA, which gathers the block-Jacobi-scaled union matrix B^(k)|_U once
// (float16, tcgen05 kind::f16) and runs their CG solves as one product per
// iteration.  Windows [w_begin, w_end) are solved; status receives
// DEV_NOT_SPD on a non-positive diagonal-block pivot and DEV_TIMEOUT if a
// tensor-core completion wait gives up.  iter_stats as for the patch CG, plus
// [3] += tensor-core products issued (one per window and iteration).
struct PatchMmaGeom {
  int NP, nU, n, Kp, Mt;  // patches per window, union parents, unknowns, padded K, M-tiles
  int npair;              // stored union blocks a > b
  int NB, jc, diag_o, Lpar;
  int64_t npatch, w_begin, w_end;
  const int2* U;          // union offsets relative to the window's first cell
  const int* ubits;       // per union parent: bit c set when it lies in patch c
  const int4* pairs;      // (a, b, o, 0): block of B^(k) between union parents a > b
  const int* rhs_o;       // [c][u]: offset index of cell c seen from parent u, or -1
  const int* outmap;      // [c][j]: union index of cell c + N_j
};
void launch_patch_mma(const float* Ahat, const uint32_t* pmask_k, PatchMmaGeom g, float* Rhat,
                      double tol, int max_iter, int* iter_stats, int* status, int num_sms,
                      cudaStream_t s);
size_t patch_mma_smem_bytes(const PatchMmaGeom& g);

// ---------------------------------------------------------------- Galerkin
struct GalerkinGeom {
  int NB;
  const int2* nbr;       // N_j
  int nwin;              // window positions WIN_w (relative to coarse cell i)
  const int2* win;
  const int* l1_ptr;     // nwin + 1
  const int2* l1_pairs;  // (j, o): N_j - WIN_w = O_o
  int nout;              // output cell offsets S_d
  const int2* out;
  const int* l2_ptr;     // nout + 1
  const int2* l2_pairs;  // (j, w): WIN_w = S_d + N_j
  int Lpar;              // side of the level-(k-1) lattice (= parent lattice of level k)
  int64_t nrow;          // stored level-(k-1) cells (4^(k-1) for a full square)
  int64_t i_begin, i_end;  // rows computed: [i_begin, i_end) (all: 0, nrow)
  int variant;           // 0: thread per window position / output, 1: warp-cooperative,
                         // 2: warp per row, 3, 4, 5: 2 x 2 row tiles with 8, 4 or 16
                         // lanes per output target
  int tile_wmin, tile_W; // tiles: window box [wmin, wmin + W)^2 from the tile origin
  int tile_threads;      // tiles: threads per CTA (256, or 128 for more CTAs per SM)
  const int2* t1;        // (o, j per row packed in bytes, 0xff = none)
  int nt1u;              // window positions read by phase 2 (cid < nt1u)
  int nitems;            // phase-1 work items: (u | cid << 16, t1 begin, t1 end, 0), one
  const int4* t1_items;  // per read position, by decreasing length
  int nt2;
  const int4* t2;        // (c.x, c.y, d0 | d1 << 16, d2 | d3 << 16), d = -1: none
  const int* t2p_ptr;    // nt2 + 1
  const int* t2p;        // per target: (j | cid << 8) with c + N_j = window position cid
  int nt3;               // target pairs (c, c + (1, 0)), variants 6-8:
  const int4* t3;        // two t2-style records per pair (second: d = -1 if alone)
  const int* t3p_ptr;    // nt3 + 1
  const uint32_t* t3p;   // per pair: cid | ja << 16 | jb << 24 (0xff = none)
};
// Shared memory of k_galerkin_tile: four Rhat rows and four window boxes.
size_t galerkin_tile_smem_bytes(const GalerkinGeom& g, size_t elem);
// A'(d, i) = (Rhat Ahat Rhat^T)_{i, i + S_d} for every level-(k-1) cell i.
template <typename T>
void launch_galerkin(const T* Ahat, const T* Rhat, const uint32_t* pmask_k, GalerkinGeom g,
                     T* Aout, cudaStream_t s);
// Level-(k-1) cell stencil (S offsets, [d][i]) -> transformed block stencil
// at level k-1 (offsets O, [o][P][16]) using masks of level k-1 parents.
// map: nO x 16 index into S of 2*Delta + c' - c for (a = c, b = c'), or -1.
template <typename T>
void launch_cells_to_blocks(const T* Acell, int64_t ncell, const int* map, int nO,
                            const int2* Ooff, int Lpar, int64_t npar, const uint32_t* pmask,
                            T* blk, cudaStream_t s);
// A^(1) (4 x 4) from the level-1 cell stencil of the nrow <= 4 existing
// level-1 cells (map[4 i + j] = index in S of cell_j - cell_i, or -1),
// factored in place (lower Cholesky, float64; absent cells get unit rows).
template <typename T>
void launch_level1_factor(const T* Acell, int nrow, const int* map, double* L1, int* status,
                          cudaStream_t s);
// U = A^(1)^-1 g from the factor.
template <typename T>
void launch_level1_solve(const double* L1, const T* g, T* U, cudaStream_t s);

// ---------------------------------------------------------------- solve
// g^(k-1)_i = sum_{j, c} Rhat[j, c, i] ghat^(k)[4 (i + N_j) + c]; if
// pmask_km1 != nullptr the result is also transformed by Q^(k-1) in place.
template <typename T>
void launch_restrict(const T* Rhat, int NB, const int2* nbr, int Lpar, int64_t nrow,
                     const T* ghat_k, T* g_km1, const uint32_t* pmask_km1, cudaStream_t s);
// RT[p][j] = Rhat[p - N_j][j] (interpolation rows regrouped by parent).
template <typename T>
void launch_transpose_rhat(const T* Rhat, int NB, const int2* nbr, int Lpar, int64_t npar, T* RT,
                           cudaStream_t s);
// vhat^(k) = Rhat^T v^(k-1) + [w^(k); 0] from the regrouped rows RT; if
// inverse, v^(k) = Q^T vhat^(k).
template <typename T>
void launch_prolong(const T* RT, int NB, const int2* nbr, int Lpar, int64_t npar,
                    const T* v_km1, const T* w_k, const uint32_t* pmask_k, int inverse,
                    T* out, cudaStream_t s);

// Batched, block-Jacobi preconditioned level CG over several levels at once
// (levelcg.cu).
struct CgLevel {
  const void* Bd;     // detail blocks, SoA [noff][9][npar] (T)
  const void* Bq;     // or NULL: the blocks of the offsets d of the half-plane
                      // H of O_k (d.y > 0, or d.y = 0 and d.x >= 0) as 32-byte
                      // float16 records [nhoff][npar][16] (entries 0..8, the
                      // rest zero), scaled by a power of two; B^(k) is
                      // symmetric, so the block of -d at p is the transpose
                      // of the block of d at p - d
  const float* bq_inv_scale;  // device: the inverse of that scale (with Bq)
  const void* Dinv;   // inverse diagonal detail blocks [9][npar] (T)
  const int2* off;
  int noff;
  const int2* hoff;   // with Bq: the offsets of H
  int nhoff;
  int R;              // largest |offset component| (halo radius)
  int Lpar;
  int64_t npar;
  void* x;            // solution (AoS4, slot 3 unused)
  void* r;
  void* z;
  void* p;
  void* Ap;
  const void* b;      // right-hand side (transformed vector; slots 0..2 used)
  int block_begin;    // first CTA of this level in the vector-kernel grid
  int spmv_begin;     // first CTA of this level in the SpMV grid
  int spp;            // SpMV threads per parent (1: 16 x 16 tiles, 4: 8 x 8, 16: 4 x 4)
  int64_t rstride;    // several right-hand sides: distance between their vectors
};
struct CgScalars {
  double rz, rz_new, rr, rr_new, pAp, rr0, beta;
  int active, iters;
};
size_t cg_spmv_smem_bytes(int max_ts, size_t elem);
// Bq[h][p][0..8] = float16(Ahat[hidx[h]][p] detail block * 2^s), entries
// 9..15 zero, for the nh offsets hidx of the half-plane; 2^s puts the
// largest |entry| of the level's detail blocks, *amax (the bits of the
// largest diagonal entry, from launch_cg_level_setup), in [2^14, 2^15);
// *inv_scale = 2^-s.
void launch_cg_block_records(const float* Ahat, const int* hidx, int nh, int64_t npar,
                             const unsigned* amax, void* Bq, float* inv_scale, cudaStream_t s);
// Side of the square parent tile of one level-CG SpMV CTA (256 threads):
// 16 with one thread per parent, 8 with four, 4 with sixteen (wide stencils:
// more CTAs per level and more lanes splitting the offsets).
__host__ __device__ inline int cg_tile_side(int spp) { return spp >= 16 ? 4 : (spp >= 4 ? 8 : 16); }
template <typename T>
void prepare_cg_spmv(int max_ts);
template <typename T>
void launch_cg_init(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc,
                    cudaStream_t s);
// Activates the levels l < nlev_on whose right-hand side is nonzero.
void launch_cg_start(CgScalars* sc, int nlev, int nlev_on, double tol2, int* any_active,
                     cudaStream_t s);
// Accumulate per-level iteration counts into stats[2..31], a not-converged
// flag into stats[32] and the device-side loop's passes (loop_count, or
// NULL) into stats[33] on the device (nlev <= 30).
void launch_cg_collect(const CgScalars* sc, int nlev, int kmax, double tol2,
                       const int* loop_count, int* stats, cudaStream_t s);
// One CG iteration = launch_cg_spmv (Ap = B p, p.Ap) then launch_cg_rest
// (x, r, z update with r.z and r.r; scalars and convergence; p = z + beta p).
template <typename T>
void launch_cg_spmv(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc, int max_ts,
                    cudaStream_t s);  // total_blocks: SpMV grid size
// Inside a device-side while loop (use_cond = 1) the scalar kernel sets the
// loop condition `cond`: continue while a level iterates and fewer than
// loop_limit passes ran (*loop_count counts them).
template <typename T>
void launch_cg_rest(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc, double tol2,
                    int max_iter, int* any_active, cudaStream_t s,
                    cudaGraphConditionalHandle cond = 0, int use_cond = 0,
                    int* loop_count = nullptr, int loop_limit = 0);
// Coalesced detail-block copy (Bd, or NULL to skip it) and block-Jacobi
// inverses of one level; with amax (one device word, or NULL) also the bits
// of the level's largest active diagonal entry, which bounds every entry of
// the SPD operator.
template <typename T>
void launch_cg_level_setup(const T* Ahat, int noff, int o0, int64_t npar, const uint32_t* pmask,
                           T* Bd, T* Dinv, unsigned* amax, cudaStream_t s);
// Bd[o][3a+b][p] = detail block (a, b) of Ahat[o][p]: the coalesced copy alone.
template <typename T>
void launch_extract_detail(const T* Ahat, int noff, int64_t npar, T* Bd, cudaStream_t s);

// Outer float64 operations on transformed level-q vectors.
// dots[i] += a_i . b_i for up to 3 pairs (nullptr pairs skipped).
void launch_dots(int64_t n, const double* a0, const double* b0, const double* a1,
                 const double* b1, const double* a2, const double* b2, double* dots,
                 cudaStream_t s);
void launch_axpy(int64_t n, const double* alpha_num, const double* alpha_den, double sign,
                 const double* x, double* y, cudaStream_t s);
void launch_xpby(int64_t n, const double* x, const double* beta_num, const double* beta_den,
                 double sign, double* p, cudaStream_t s);
// u += (num / den) p, r -= (num / den) q and *rr += r.r (updated r), one pass.
void launch_update_ur(int64_t n, const double* num, const double* den, const double* p,
                      const double* q, double* u, double* r, double* rr, cudaStream_t s);
// z = (double) zf and *zq += z.q, one pass.
void launch_widen_dot(int64_t n, const float* zf, double* z, const double* q, double* zq,
                      cudaStream_t s);

// Adjoint contraction: dJ_c = -a_c sum_{p,r} lam[n_p] K[p][r] u[n_r].
void launch_adjoint_contract(int ncell, const int32_t* cell_nodes, const double* cell_a,
                             const double* lam, const double* u, double* dJ,
                             cudaStream_t s);
void launch_set_kref(const double* K_ref_host);
// CSR values of sum_c exp(log_a_c) K_ref (val must be zeroed; columns sorted
// within each row); *missing is set if a corner pair is not in the pattern.
void launch_assemble_cells(int n, const int32_t* rowptr, const int32_t* colind, int ncell,
                           const int32_t* cell_nodes, const double* log_a, double* val,
                           double* cell_a, int* missing, cudaStream_t s);

// ---------------------------------------------------------------- dense (exact path)
void launch_dense_from_blocks(const double* blk, const int2* off, int noff, int Lpar,
                              int64_t npar, double* D, cudaStream_t s);
void launch_dense_transform(const double* in, int64_t npar, const uint32_t* pmask, double* out,
                            cudaStream_t s);
// C (m x n) = alpha * op(A) * op(B) + beta * C; op(A) is m x kk, op(B) kk x n.
// Row-major, leading dimensions = column counts of the stored matrices.
void launch_dgemm_t(int m, int n, int kk, double alpha, const double* A, int transA,
                    const double* B, int transB, double beta, double* C, cudaStream_t s);
void launch_dgemm(int m, int n, int kk, double alpha, const double* A, const double* B,
                  int transB, double beta, double* C, cudaStream_t s);
// In-place lower Cholesky of an n x n row-major matrix (single CTA).
void launch_dpotrf(double* A, int n, int* status, cudaStream_t s);
// Solve (L L^T) X = B for nrhs columns of B (n x nrhs row-major), in place.
void launch_dpotrs(const double* L, int n, double* B, int nrhs, cudaStream_t s);
// Gather helpers for the dense path.
void launch_gather_rows_cols(const double* D, int ld, const int32_t* rows, int nr,
                             const int32_t* cols, int nc, double alpha_scale,
                             const double* col_scale, double* out, cudaStream_t s);
void launch_dense_rhat(const double* Y, const int32_t* det, int nJ, const int32_t* par, int nA,
                       const uint32_t* pmask, int64_t npar, double* Rh, cudaStream_t s);
void launch_scatter_det(const double* wc, const int32_t* det, int nJ, double* w, cudaStream_t s);
void launch_gather_det(const double* w, const int32_t* det, int nJ, double* wc, cudaStream_t s);
void launch_level1_factor_dense(const double* A, double* L, int* status, cudaStream_t s);

// ---------------------------------------------------------------- several right-hand sides
// Up to kMaxRhs vectors per pass; each is a separate vector, the one of
// right-hand side r at base + r * stride.  The matrix data (Rhat, RT, the
// level blocks, Ahat^(q)) is read once for all of them.
constexpr int kMaxRhs = 4;
template <typename T>
void launch_restrict_m(const T* Rhat, int NB, const int2* nbr, int Lpar, int64_t nrow,
                       const T* ghat_k, int64_t gstride, T* g_km1, int64_t ostride,
                       const uint32_t* pmask_km1, int nrhs, cudaStream_t s);
template <typename T>
void launch_prolong_m(const T* RT, int NB, const int2* nbr, int Lpar, int64_t npar,
                      const T* v_km1, int64_t vstride, const T* w_k, int64_t wstride,
                      const uint32_t* pmask_k, int inverse, T* out, int64_t ostride, int nrhs,
                      cudaStream_t s);
// The batched level CG over (level, right-hand side): scalars sc[l * nrhs + r],
// vectors of right-hand side r at CgLevel pointer + r * rstride.
template <typename T>
void launch_cgm_init(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc, int nrhs,
                     cudaStream_t s);
void launch_cgm_start(CgScalars* sc, int n, double tol2, int* any_active, cudaStream_t s);
template <typename T>
void launch_cgm_iteration(const CgLevel* lv, int nlev, int spmv_blocks, int total_blocks,
                          CgScalars* sc, int nrhs, int max_ts, double tol2, int max_iter,
                          int* any_active, cudaStream_t s);
size_t cgm_spmv_smem_bytes(int max_ts, size_t elem, int nrhs);

// ---------------------------------------------------------------- one-pass gradient
// Reverse pass through the localized setup and one-pass solve (onepass_grad.cu;
// E = float or double, the working precision of the hierarchy).  Y arrays:
// adjoints of the transformed level operators ([o][P][16]); oidx: box lookup
// (2 obox + 1)^2 of block offsets -> index.
template <typename E>
void launch_rbar_outer(E* Rbar, const int2* nbr, int NB, int L, int64_t nrow, const E* v,
                       const E* gbar, const E* ubar, const E* ghat, cudaStream_t s);
template <typename E>
void launch_ybar_level(E* Y, int noff, const int2* off, int L, int64_t npar, const E* lam,
                       const E* w, cudaStream_t s);
template <typename E>
void launch_abar1(E* A1bar, const E* lam1, const E* U1, cudaStream_t s);
template <typename E>
void launch_xbar_cells(E* X, int nS, const int2* S, int L, int64_t ncell, const E* A1bar,
                       const E* Y, int64_t npar_prev, const int* oidx, int obox,
                       const uint32_t* pmask_prev, cudaStream_t s);
template <typename E>
void launch_window_product(E* T, int nTW, const int* tw_ptr, const int2* tw_pairs, const E* X,
                           const int2* S, const E* Rhat, int NB, int L, int64_t nrow,
                           cudaStream_t s);
template <typename E>
void launch_rbar_galerkin(E* Rbar, const E* T, int nTW, const int* rg, const E* Ahat, int noff,
                          const int2* off, const int2* nbr, int NB, int L, int64_t nrow,
                          cudaStream_t s);
template <typename E>
void launch_ybar_galerkin(E* Y, int noff, const int2* off, const int2* yg, const E* T, int nTW,
                          const E* Rhat, const E* M, const int2* nbr, int NB, int L, int64_t npar,
                          cudaStream_t s);
template <typename E>
void launch_grad_cells(double* out, int ncell, const int32_t* cell_nodes, const double* cell_a,
                       const double* Kref, const int32_t* morton_of, const E* Y, int64_t npar,
                       const int* oidx, int obox, const uint32_t* pmask, cudaStream_t s);

}  // namespace gb
