// onepass_grad.cu - reverse-mode pass through the localized setup and the
// one-pass solve (Algorithm 2), float64: the gradient of
// J = 1/2 |u_loc - u_obs|^2 with respect to the level operators, level by
// level from the coarsest, ending in dJ/dlog a per fine cell.
//
// Notation (all in the transformed coordinates the forward kernels use):
//  * Rhat[i][j][c]: row i (a level-(k-1) cell) of R^(k-1,k) Q^T on the
//    children c of the neighbour parent p_ij = i + N_j.
//  * Ahat_k[o][P][a][b]: the block of Q A^(k) Q^T coupling parent P and
//    parent P + O_o.
//  * Y_k: the adjoint of Ahat_k in the same layout, accumulated without
//    symmetrisation (only its symmetric part enters: A^(k) is symmetric).
//  * X: the symmetric part of the adjoint of A^(k-1) in plain level-(k-1)
//    coordinates, as a cell stencil X[d][i] = Xbar(i, i + S_d).
//  * T = X Rhat (row i over the window i + TW_w, four children each),
//    stored [w][i][4].
// With those, for k = 2..q (the reverse of Alg. 2 lines 13, 12, 11, 7):
//   Rbar += 2 T Ahat_k (on the pattern of Rhat),  M_i = B_i^-1 Rbar_i (patch
//   solves with the adjoint right-hand side), Y_k += Rhat^T (T - M) on the
//   pattern of Ahat_k; the solve adds the outer products of Alg. 2 lines 15
//   and 17 to Rbar and -lambda w^T to the detail blocks of Y_k.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

// The per-parent transforms of the 16 child masks, Qs[m * 16 + 4 a + c] =
// Q_m[a][c], staged in shared memory by the first 256 threads of a block.
__device__ void stage_q(double* Qs) {
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    Qs[t] = qv<double>(t >> 4, (t >> 2) & 3, t & 3);
  __syncthreads();
}

// Plain entry (i, i') of a level operator whose transformed blocks are Y
// ([o][P][4][4]; P = i >> 2, slot a = i & 3), zero off the block pattern:
// sum_{alpha, beta} Q_P[alpha][a] Y[o][P][alpha][beta] Q_P'[beta][b].
__device__ double plain_entry(const double* __restrict__ Y, int64_t npar,
                              const int* __restrict__ oidx, int obox,
                              const uint32_t* __restrict__ pmask, const double* Qs, int64_t i,
                              int64_t ip) {
  const int64_t P = i >> 2, Pp = ip >> 2;
  const int a = (int)(i & 3), b = (int)(ip & 3);
  int x, y, xp, yp;
  demorton((uint32_t)P, x, y);
  demorton((uint32_t)Pp, xp, yp);
  const int dx = xp - x, dy = yp - y;
  if (dx < -obox || dx > obox || dy < -obox || dy > obox) return 0.0;
  const int o = oidx[(dy + obox) * (2 * obox + 1) + (dx + obox)];
  if (o < 0) return 0.0;
  const double* Qr = Qs + 16 * ((int)pmask[P] & 15);
  const double* Qc = Qs + 16 * ((int)pmask[Pp] & 15);
  const double* B = Y + ((int64_t)o * npar + P) * 16;
  double s = 0.0;
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    const double qa = Qr[4 * al + a];
    if (qa == 0.0) continue;
    double t = 0.0;
#pragma unroll
    for (int be = 0; be < 4; ++be) t += B[4 * al + be] * Qc[4 * be + b];
    s += qa * t;
  }
  return s;
}

// Rbar[i][j][c] = v[i] ubar[4 p + c] + gbar[i] ghat[4 p + c], p = i + N_j
// (the outer products of the prolongation and restriction chains).
__global__ void k_rbar_outer(double* __restrict__ Rbar, const int2* __restrict__ nbr, int NB,
                             int L, int64_t nrow, const double* __restrict__ v,
                             const double* __restrict__ gbar, const double* __restrict__ ubar,
                             const double* __restrict__ ghat) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrow * NB) return;
  const int64_t i = t / NB;
  const int j = (int)(t - i * NB);
  int x, y;
  demorton((uint32_t)i, x, y);
  const int p = shift_cell(x, y, nbr[j].x, nbr[j].y, L, nrow);
  double* out = Rbar + t * 4;
  for (int c = 0; c < 4; ++c)
    out[c] = p < 0 ? 0.0 : v[i] * ubar[4 * (int64_t)p + c] + gbar[i] * ghat[4 * (int64_t)p + c];
}

// Y[o][P][a][b] -= lambda[4 P + a] w[4 P' + b], a, b < 3 (P' = P + O_o):
// the adjoint of B^(k) w^(k) = W g^(k) (Alg. 2 line 8).
__global__ void k_ybar_level(double* __restrict__ Y, int noff, const int2* __restrict__ off,
                             int L, int64_t npar, const double* __restrict__ lam,
                             const double* __restrict__ w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t P = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)P, x, y);
  const int Pp = shift_cell(x, y, off[o].x, off[o].y, L, npar);
  if (Pp < 0) return;
  double* B = Y + t * 16;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) B[4 * a + b] -= lam[4 * P + a] * w[4 * (int64_t)Pp + b];
}

// Abar^(1) = -lambda^(1) U^(1)^T (Alg. 2 line 16), plain 4 x 4.
__global__ void k_abar1(double* __restrict__ A1bar, const double* __restrict__ lam1,
                        const double* __restrict__ U1) {
  const int t = threadIdx.x;
  if (t < 16) A1bar[t] = -lam1[t >> 2] * U1[t & 3];
}

// X[d][i] = sym(Abar^(k-1))(i, i + S_d) in plain level-(k-1) coordinates,
// from the transformed blocks Y of level k-1 (or, for k - 1 = 1, the plain
// 4 x 4 Abar^(1)).
__global__ void k_xbar_cells(double* __restrict__ X, int nS, const int2* __restrict__ S, int L,
                             int64_t ncell, const double* __restrict__ A1bar,
                             const double* __restrict__ Y, int64_t npar_prev,
                             const int* __restrict__ oidx, int obox,
                             const uint32_t* __restrict__ pmask_prev) {
  __shared__ double Qs[256];
  stage_q(Qs);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nS * ncell) return;
  const int d = (int)(t / ncell);
  const int64_t i = t - (int64_t)d * ncell;
  int x, y;
  demorton((uint32_t)i, x, y);
  const int ip = shift_cell(x, y, S[d].x, S[d].y, L, ncell);
  double v = 0.0;
  if (ip >= 0) {
    if (A1bar) {
      v = 0.5 * (A1bar[4 * i + ip] + A1bar[4 * ip + i]);
    } else {
      v = 0.5 * (plain_entry(Y, npar_prev, oidx, obox, pmask_prev, Qs, i, ip) +
                 plain_entry(Y, npar_prev, oidx, obox, pmask_prev, Qs, ip, i));
    }
  }
  X[t] = v;
}

// T[w][i][c] = sum over (d, j) with S_d + N_j = TW_w of X[d][i] Rhat[i + S_d][j][c]
// (window position outermost, so consecutive threads take consecutive rows:
// the X reads and T writes coalesce).
__global__ void k_window_product(double* __restrict__ T, int nTW, const int* __restrict__ tw_ptr,
                                 const int2* __restrict__ tw_pairs, const double* __restrict__ X,
                                 const int2* __restrict__ S, const double* __restrict__ Rhat,
                                 int NB, int L, int64_t nrow) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrow * nTW) return;
  const int w = (int)(t / nrow);
  const int64_t i = t - (int64_t)w * nrow;
  int x, y;
  demorton((uint32_t)i, x, y);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int e = tw_ptr[w]; e < tw_ptr[w + 1]; ++e) {
    const int2 dj = tw_pairs[e];
    const double xv = X[(int64_t)dj.x * nrow + i];
    if (xv == 0.0) continue;
    const int ip = shift_cell(x, y, S[dj.x].x, S[dj.x].y, L, nrow);
    if (ip < 0) continue;
    const double* r = Rhat + ((int64_t)ip * NB + dj.y) * 4;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[c] += xv * r[c];
  }
  double* out = T + t * 4;
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = acc[c];
}

// Rbar[i][j][c] += 2 sum_o sum_c' T[i][N_j - O_o][c'] Ahat[o][p - O_o][c'][c]
// (the adjoint of Alg. 2 line 13 with respect to R, on the pattern of Rhat).
__global__ void k_rbar_galerkin(double* __restrict__ Rbar, const double* __restrict__ T, int nTW,
                                const int* __restrict__ rg, const double* __restrict__ Ahat,
                                int noff, const int2* __restrict__ off,
                                const int2* __restrict__ nbr, int NB, int L, int64_t nrow) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrow * NB) return;
  const int64_t i = t / NB;
  const int j = (int)(t - i * NB);
  int x, y;
  demorton((uint32_t)i, x, y);
  const int p = shift_cell(x, y, nbr[j].x, nbr[j].y, L, nrow);
  if (p < 0) return;
  int px, py;
  demorton((uint32_t)p, px, py);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int o = 0; o < noff; ++o) {
    const int w = rg[j * noff + o];
    if (w < 0) continue;
    const int Pp = shift_cell(px, py, -off[o].x, -off[o].y, L, nrow);
    if (Pp < 0) continue;
    const double* B = Ahat + ((int64_t)o * nrow + Pp) * 16;
    const double* tv = T + ((int64_t)w * nrow + i) * 4;
#pragma unroll
    for (int cp = 0; cp < 4; ++cp)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += tv[cp] * B[4 * cp + c];
  }
  double* out = Rbar + t * 4;
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] += 2.0 * acc[c];
}

// Y[o][P] += sum_j Rhat[i][j]^T (T[i][N_j + O_o] - M[i][j']) with i = P - N_j
// and N_j' = N_j + O_o: the adjoint of Alg. 2 line 13 with respect to A^(k)
// and of the patch solves (line 11) with respect to their matrices and
// right-hand sides, both in transposed form (Y is symmetrised when used).
__global__ void k_ybar_galerkin(double* __restrict__ Y, int noff, const int2* __restrict__ off,
                                const int2* __restrict__ yg, const double* __restrict__ T, int nTW,
                                const double* __restrict__ Rhat, const double* __restrict__ M,
                                const int2* __restrict__ nbr, int NB, int L, int64_t npar) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t P = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)P, x, y);
  if (shift_cell(x, y, off[o].x, off[o].y, L, npar) < 0) return;
  double acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = 0.0;
  for (int j = 0; j < NB; ++j) {
    const int i = shift_cell(x, y, -nbr[j].x, -nbr[j].y, L, npar);
    if (i < 0) continue;
    const int2 wj = yg[o * NB + j];
    const double* r = Rhat + ((int64_t)i * NB + j) * 4;
    double z[4] = {0.0, 0.0, 0.0, 0.0};
    if (wj.x >= 0) {
      const double* tv = T + ((int64_t)wj.x * npar + i) * 4;
#pragma unroll
      for (int c = 0; c < 4; ++c) z[c] = tv[c];
    }
    if (wj.y >= 0) {
      const double* mv = M + ((int64_t)i * NB + wj.y) * 4;
#pragma unroll
      for (int c = 0; c < 4; ++c) z[c] -= mv[c];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[4 * a + b] += r[a] * z[b];
  }
  double* B = Y + t * 16;
#pragma unroll
  for (int e = 0; e < 16; ++e) B[e] += acc[e];
}

// dJ/dlog a_c = a_c sum_{p,r} sym(Abar^(q))(p, r) K_ref[p][r] over the
// interior corners of cell c (A^(q) = sum_c a_c K_c, Sec. 5.1).
__global__ void k_grad_cells(double* __restrict__ out, int ncell,
                             const int32_t* __restrict__ cell_nodes,
                             const double* __restrict__ cell_a, const double* __restrict__ Kref,
                             const int32_t* __restrict__ morton_of, const double* __restrict__ Y,
                             int64_t npar, const int* __restrict__ oidx, int obox,
                             const uint32_t* __restrict__ pmask) {
  __shared__ double Qs[256];
  stage_q(Qs);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  int64_t m[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int u = cell_nodes[4 * c + p];
    m[p] = u >= 0 ? (int64_t)morton_of[u] : -1;
  }
  double s = 0.0;
  for (int p = 0; p < 4; ++p) {
    if (m[p] < 0) continue;
    for (int r = 0; r < 4; ++r) {
      if (m[r] < 0) continue;
      const double xv = 0.5 * (plain_entry(Y, npar, oidx, obox, pmask, Qs, m[p], m[r]) +
                               plain_entry(Y, npar, oidx, obox, pmask, Qs, m[r], m[p]));
      s += xv * Kref[4 * p + r];
    }
  }
  out[c] = cell_a[c] * s;
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

void launch_rbar_outer(double* Rbar, const int2* nbr, int NB, int L, int64_t nrow, const double* v,
                       const double* gbar, const double* ubar, const double* ghat,
                       cudaStream_t s) {
  if (nrow * NB <= 0) return;
  count_launch();
  k_rbar_outer<<<nblk(nrow * NB, 256), 256, 0, s>>>(Rbar, nbr, NB, L, nrow, v, gbar, ubar, ghat);
}
void launch_ybar_level(double* Y, int noff, const int2* off, int L, int64_t npar,
                       const double* lam, const double* w, cudaStream_t s) {
  if ((int64_t)noff * npar <= 0) return;
  count_launch();
  k_ybar_level<<<nblk((int64_t)noff * npar, 256), 256, 0, s>>>(Y, noff, off, L, npar, lam, w);
}
void launch_abar1(double* A1bar, const double* lam1, const double* U1, cudaStream_t s) {
  count_launch();
  k_abar1<<<1, 32, 0, s>>>(A1bar, lam1, U1);
}
void launch_xbar_cells(double* X, int nS, const int2* S, int L, int64_t ncell,
                       const double* A1bar, const double* Y, int64_t npar_prev, const int* oidx,
                       int obox, const uint32_t* pmask_prev, cudaStream_t s) {
  if ((int64_t)nS * ncell <= 0) return;
  count_launch();
  k_xbar_cells<<<nblk((int64_t)nS * ncell, 256), 256, 0, s>>>(X, nS, S, L, ncell, A1bar, Y,
                                                               npar_prev, oidx, obox, pmask_prev);
}
void launch_window_product(double* T, int nTW, const int* tw_ptr, const int2* tw_pairs,
                           const double* X, const int2* S, const double* Rhat, int NB, int L,
                           int64_t nrow, cudaStream_t s) {
  if (nrow * nTW <= 0) return;
  count_launch();
  k_window_product<<<nblk(nrow * nTW, 256), 256, 0, s>>>(T, nTW, tw_ptr, tw_pairs, X, S, Rhat,
                                                          NB, L, nrow);
}
void launch_rbar_galerkin(double* Rbar, const double* T, int nTW, const int* rg,
                          const double* Ahat, int noff, const int2* off, const int2* nbr, int NB,
                          int L, int64_t nrow, cudaStream_t s) {
  if (nrow * NB <= 0) return;
  count_launch();
  k_rbar_galerkin<<<nblk(nrow * NB, 128), 128, 0, s>>>(Rbar, T, nTW, rg, Ahat, noff, off, nbr,
                                                        NB, L, nrow);
}
void launch_ybar_galerkin(double* Y, int noff, const int2* off, const int2* yg, const double* T,
                          int nTW, const double* Rhat, const double* M, const int2* nbr, int NB,
                          int L, int64_t npar, cudaStream_t s) {
  if ((int64_t)noff * npar <= 0) return;
  count_launch();
  k_ybar_galerkin<<<nblk((int64_t)noff * npar, 128), 128, 0, s>>>(Y, noff, off, yg, T, nTW, Rhat,
                                                                   M, nbr, NB, L, npar);
}
void launch_grad_cells(double* out, int ncell, const int32_t* cell_nodes, const double* cell_a,
                       const double* Kref, const int32_t* morton_of, const double* Y,
                       int64_t npar, const int* oidx, int obox, const uint32_t* pmask,
                       cudaStream_t s) {
  if (ncell <= 0) return;
  count_launch();
  k_grad_cells<<<nblk(ncell, 128), 128, 0, s>>>(out, ncell, cell_nodes, cell_a, Kref, morton_of,
                                                 Y, npar, oidx, obox, pmask);
}

}  // namespace gb
