// d3.cuh - the three-dimensional gamblet path: device helpers and kernel
// launch wrappers (kernels in d3_kernels.cu, orchestration in d3_host.cu).
//
// The method is the same in every dimension (Sec. 4: a domain of R^d with
// nested dyadic subdivisions; Sec. 5.4 states the complexity in d).  In 3-D
// a level-(k-1) cube has up to eight children, so every per-parent object
// of the 2-D path grows from 4 to 8 slots:
//  * A level-k vector is indexed by the Morton code of its lattice cell
//    (x, y, z), 0 <= x, y, z < 2^k: bit b of x, y, z at positions 3b, 3b+1,
//    3b+2.  The children of level-(k-1) cell p are the entries 8p + c with
//    slot c = (x & 1) + 2 (y & 1) + 4 (z & 1), the sibling order of W^(k).
//  * Every level stores its full lattice (8^k cells, 8^(k-1) parents);
//    cells without a fine unknown below them are inactive (zero rows).
//  * Parent p carries an 8-bit mask of its active children.  Its
//    orthonormal 8x8 transform Q_p has rows t = 0..m-2 = the normalised
//    Helmert rows of Lemma const0 (Construction const2) on the active
//    children, zero rows m-1..6, and row 7 = 1/sqrt(m) on the children.
//    x_hat = Q x splits a level vector into W^(k) x (slots 0..6) and
//    sqrt(m) pibar x (slot 7).
//  * A level operator is stored as 8x8 blocks between parent p and parent
//    p + o for the offsets o of a set O_k: Ahat[(o * npar + p) * 64 + 8a + b]
//    = (Q_p A(p, p + o) Q_(p+o)^T)[a][b].  The detail-detail part
//    (a, b <= 6) is B^(k) = W A W^T.
//  * The interpolation of coarse cell i (Alg. 2 line 12) is stored in the
//    same transformed coordinates over its patch parents P_i + N_j:
//    Rhat[(i * NB + j) * 8 + c].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gb {
namespace d3 {

__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
  v &= 0x3ffu;
  v = (v | (v << 16)) & 0x030000ffu;
  v = (v | (v << 8)) & 0x0300f00fu;
  v = (v | (v << 4)) & 0x030c30c3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t v) {
  v &= 0x09249249u;
  v = (v | (v >> 2)) & 0x030c30c3u;
  v = (v | (v >> 4)) & 0x0300f00fu;
  v = (v | (v >> 8)) & 0x030000ffu;
  v = (v | (v >> 16)) & 0x3ffu;
  return v;
}
__host__ __device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}
__host__ __device__ __forceinline__ void demorton3(uint32_t m, int& x, int& y, int& z) {
  x = (int)compact3(m);
  y = (int)compact3(m >> 1);
  z = (int)compact3(m >> 2);
}
// Morton index of cell + (dx, dy, dz) on a side-L lattice, or -1 outside.
__host__ __device__ __forceinline__ int shift3(int x, int y, int z, int dx, int dy, int dz, int L) {
  const int nx = x + dx, ny = y + dy, nz = z + dz;
  if ((unsigned)nx >= (unsigned)L || (unsigned)ny >= (unsigned)L || (unsigned)nz >= (unsigned)L)
    return -1;
  return (int)morton3((uint32_t)nx, (uint32_t)ny, (uint32_t)nz);
}

// Entry (a, c) of Q for child mask m (see the header comment).
__host__ __device__ __forceinline__ double q8(int m, int a, int c) {
  if (!((m >> c) & 1)) return 0.0;
  const int cnt = __popc_portable(m & 255);
  const int j = __popc_portable(m & ((1 << c) - 1));
  if (a == 7) return 1.0 / sqrt((double)cnt);
  if (a >= cnt - 1) return 0.0;
  const double nrm = 1.0 / sqrt((double)((a + 1) * (a + 2)));
  if (j <= a) return nrm;
  if (j == a + 1) return -(double)(a + 1) * nrm;
  return 0.0;
}

// Offsets travel as int4 (x, y, z, 0).  A box lookup maps an offset with
// |components| <= R to its index in a set, or -1: idx[((z + R) S + y + R) S
// + x + R], S = 2R + 1.
struct OffLookup {
  const int* idx;
  int R;
  __device__ __forceinline__ int find(int x, int y, int z) const {
    if (x < -R || x > R || y < -R || y > R || z < -R || z > R) return -1;
    const int S = 2 * R + 1;
    return idx[((z + R) * S + y + R) * S + x + R];
  }
};

// The first failed index guard of the setup kernels since the last call
// (0 = none), cleared on read.
int guard_take();

// ---------------------------------------------------------------- launches
// cells (n x 3) -> Morton code of every unknown; flag[0] = 2 for a cell
// outside [0, 2^q)^3.
void launch_cells_to_morton3(const int32_t* cells, int n, int q, int32_t* morton_of, int* flag,
                             cudaStream_t s);
// unknown_of[morton_of[i]] = i (flag[0] = 1 if two unknowns share a cell) and
// the level-q child masks.
void launch_scatter3(const int32_t* morton_of, int n, int32_t* unknown_of, uint32_t* pmask_q,
                     int* flag, cudaStream_t s);
// Level k-1 masks from level k: child c of P is active iff pmask_k[8P + c] != 0.
void launch_coarsen3(const uint32_t* pmask_k, int64_t npar_km1, uint32_t* pmask_km1,
                     cudaStream_t s);
// Largest |parent offset| per axis over the stored entries (ext[0]);
// flag = 3 for a column index outside [0, n).
void launch_csr_extent3(int n, const int32_t* rowptr, const int32_t* colind,
                        const int32_t* morton_of, int* ext, int* flag, cudaStream_t s);
// Scatter the fine CSR into untransformed blocks (blk must be zeroed).
void launch_csr_to_blocks3(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                           const int32_t* morton_of, OffLookup lk, int q, int64_t npar,
                           double* blk, cudaStream_t s);
// dst(o, p) = Q_p sym(src)(o, p) Q_(p+o)^T, where sym averages each entry
// with its mirror in block (-o, p + o) when symmetrize != 0 (the Galerkin
// product's two evaluations of each pair; mirror[o] = index of -o) and is
// the identity otherwise.  qtab holds the 256 transforms Q (64 doubles per
// mask).  src and dst may alias only when symmetrize == 0.
void launch_transform_blocks3(const double* src, double* dst, const int4* off, const int* mirror,
                              int noff, int64_t npar, int Lpar, const uint32_t* pmask,
                              int symmetrize, const double* qtab, cudaStream_t s);
// Block-Jacobi factors: Dinv[p] = inverse of the active detail block of
// Ahat(0, p) (zero outside), 64 doubles per parent; status = DEV_NOT_SPD on
// a non-positive pivot.
void launch_detail_inverse3(const double* Ahat, int o0, int64_t npar, const uint32_t* pmask,
                            double* Dinv, int* status, cudaStream_t s);

struct Patch3Geom {
  int NB, jc;
  int noff;             // |O_k| (blocks per parent of Ahat)
  const int4* nbr;      // NB neighbour offsets N_j (level k-1 cell units)
  const int* pair_idx;  // NB x NB: index in O_k of N_b - N_a, or -1
  int Lpar;             // side of the level-(k-1) lattice
  int64_t npatch;       // 8^(k-1)
};
// Patch systems of Definition defb by block-Jacobi preconditioned CG, one
// CTA per coarse cell; writes Rhat.  iter_stats[0] = max iterations (atomic),
// [1] = sum, [2] = patches solved.
void launch_patch_cg3(const double* Ahat, const double* Dinv, const uint32_t* pmask_k,
                      Patch3Geom g, double tol, int max_iter, double* Rhat, int* iter_stats,
                      cudaStream_t s);
size_t patch_cg3_smem(int NB);

struct Galerkin3Geom {
  int NB;
  const int4* nbr;
  int Lpar;             // side of the level-(k-1) lattice
  int64_t npatch;       // 8^(k-1) coarse cells
  int nD;               // dilated offsets d (level k-1 cell units)
  const int* l1_ptr;    // nD + 1
  const int2* l1;       // (j, o): N_j + O_o = d
  int nE;               // output offsets e
  const int4* E;
  const int* l2_ptr;    // nE + 1
  const int2* l2;       // (j, d): e + N_j = D_d
  OffLookup out_lk;     // block offsets of level k-1 (level k-2 cell units)
  int noff;             // |O_k|
  int noff_out;         // |O_(k-1)|
  int64_t npar_out;     // 8^(k-2)
};
// A^(k-1) = R A^(k) R^T (Alg. 2 line 13) in node form, scattered into
// untransformed level-(k-1) blocks (out zeroed).
void launch_galerkin3(const double* Ahat, const double* Rhat, const uint32_t* pmask_k,
                      Galerkin3Geom g, double* out, cudaStream_t s);
size_t galerkin3_smem(int NB, int nD);

// x_hat = Q x (dir +1) or x = Q^T x_hat (dir -1) per parent, 8 entries each.
void launch_transform_vec3(const double* in, double* out, int64_t npar, const uint32_t* pmask,
                           int dir, const double* qtab, cudaStream_t s);
// g^(k-1)_i = sum_j Rhat_i[j] . ghat^(k)[P_i + N_j] for the active coarse cells.
void launch_restrict3(const double* Rhat, const double* ghat, const uint32_t* pmask_k,
                      Patch3Geom g, double* gc, cudaStream_t s);
// v^(k) = Q^T (Rhat^T v^(k-1) + [w; 0]) per parent (v_coarse or w may be NULL).
void launch_prolong3(const double* Rhat, const double* v_coarse, const double* w,
                     const uint32_t* pmask_k, Patch3Geom g, const double* qtab, double* v,
                     cudaStream_t s);

// ---------------------------------------------------------------- level CG
struct Lcg3Level {
  const double* A;      // Ahat^(k)
  const double* Dinv;   // block-Jacobi factors
  const int4* off;      // O_k
  int noff;
  int Lpar;
  int64_t npar;
  int64_t v0;           // offset of the level's vectors (8 npar entries)
  int blk0, nblk;       // CTAs of the level in the batched launches
};
struct Lcg3Scalars {
  double rz, bb, alpha, beta;
  int active;  // 1 running, 0 converged (or zero right-hand side), -1 iteration cap hit
  int iters;
  int pad[2];
};
// One block-Jacobi PCG step on all levels with active != 0; partial
// reductions in part (3 doubles per CTA).
void launch_lcg3_start(const Lcg3Level* lv, int nlev, int nblk, const double* b, double* x,
                       double* r, double* z, double* p, double* part, cudaStream_t s);
void launch_lcg3_init_scalars(const Lcg3Level* lv, int nlev, const double* part,
                              Lcg3Scalars* sc, double tol, cudaStream_t s);
void launch_lcg3_spmv(const Lcg3Level* lv, int nlev, int nblk, const Lcg3Scalars* sc,
                      const double* p, double* Ap, double* part, cudaStream_t s);
void launch_lcg3_alpha(const Lcg3Level* lv, int nlev, const double* part, Lcg3Scalars* sc,
                       cudaStream_t s);
void launch_lcg3_update(const Lcg3Level* lv, int nlev, int nblk, const Lcg3Scalars* sc,
                        const double* p, const double* Ap, double* x, double* r, double* z,
                        double* part, cudaStream_t s);
void launch_lcg3_beta(const Lcg3Level* lv, int nlev, const double* part, Lcg3Scalars* sc,
                      double tol, int max_iter, cudaStream_t s);
void launch_lcg3_direction(const Lcg3Level* lv, int nlev, int nblk, const Lcg3Scalars* sc,
                           const double* z, double* p, cudaStream_t s);

// ---------------------------------------------------------------- level 1 and fine level
// Solve Ahat^(1) U_hat = Q g^(1) on the active slots of the single level-0
// parent and return U^(1) = Q^T U_hat (8 entries); status DEV_NOT_SPD.
void launch_coarsest3(const double* A1hat, uint32_t mask, const double* g1, const double* qtab,
                      double* U1, int* status, cudaStream_t s);
// out_m[m] = in[unknown_of[m]] (0 where -1) and back.
void launch_gather3(const double* in, const int32_t* unknown_of, int64_t ncell, double* out,
                    cudaStream_t s);
void launch_scatter_unknown3(const double* in_m, const int32_t* morton_of, int n, double* out,
                             cudaStream_t s);
// y = A x for the fine CSR (eight lanes per row).
void launch_csr_spmv3(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                      const double* x, double* y, cudaStream_t s);
// Deterministic dot products: part[b] = sum over CTA b of x . y (and x . w
// in part[nb + b] when w != NULL); dot_finish sums them into out[0..1].
int dot3_blocks(int64_t n);
void launch_dot3(int64_t n, const double* x, const double* y, const double* w, double* part,
                 cudaStream_t s);
void launch_dot3_finish(const double* part, int nb, int nout, double* out, cudaStream_t s);
// y = a x + b y (elementwise, n entries)
void launch_axpby3(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s);

}  // namespace d3
}  // namespace gb
