// onepass_grad.cu - reverse-mode pass through the localized setup and the
// one-pass solve (Algorithm 2), in the handle's working precision E (float64,
// or float32 on the mixed path's float32 hierarchy): the gradient of
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
template <typename E>
__device__ void stage_q(E* Qs) {
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    Qs[t] = qv<E>(t >> 4, (t >> 2) & 3, t & 3);
  __syncthreads();
}

// One 4-element entry (16-byte aligned) as vector loads.
__device__ __forceinline__ void ld4v(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void ld4v(const double* p, double* v) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}

// Plain entry (i, i') of a level operator whose transformed blocks are Y
// ([o][P][4][4]; P = i >> 2, slot a = i & 3), zero off the block pattern:
// sum_{alpha, beta} Q_P[alpha][a] Y[o][P][alpha][beta] Q_P'[beta][b].
template <typename E>
__device__ E plain_entry(const E* __restrict__ Y, int64_t npar, const int* __restrict__ oidx,
                         int obox, const uint32_t* __restrict__ pmask, const E* Qs, int64_t i,
                         int64_t ip) {
  const int64_t P = i >> 2, Pp = ip >> 2;
  const int a = (int)(i & 3), b = (int)(ip & 3);
  int x, y, xp, yp;
  demorton((uint32_t)P, x, y);
  demorton((uint32_t)Pp, xp, yp);
  const int dx = xp - x, dy = yp - y;
  if (dx < -obox || dx > obox || dy < -obox || dy > obox) return E(0);
  const int o = oidx[(dy + obox) * (2 * obox + 1) + (dx + obox)];
  if (o < 0) return E(0);
  const E* Qr = Qs + 16 * ((int)pmask[P] & 15);
  const E* Qc = Qs + 16 * ((int)pmask[Pp] & 15);
  const E* B = Y + ((int64_t)o * npar + P) * 16;
  E s = E(0);
#pragma unroll
  for (int al = 0; al < 4; ++al) {
    const E qa = Qr[4 * al + a];
    if (qa == E(0)) continue;
    E t = E(0);
#pragma unroll
    for (int be = 0; be < 4; ++be) t += B[4 * al + be] * Qc[4 * be + b];
    s += qa * t;
  }
  return s;
}

// Rbar[i][j][c] = v[i] ubar[4 p + c] + gbar[i] ghat[4 p + c], p = i + N_j
// (the outer products of the prolongation and restriction chains).
template <typename E>
__global__ void k_rbar_outer(E* __restrict__ Rbar, const int2* __restrict__ nbr, int NB,
                             int L, int64_t nrow, const E* __restrict__ v,
                             const E* __restrict__ gbar, const E* __restrict__ ubar,
                             const E* __restrict__ ghat) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrow * NB) return;
  const int64_t i = t / NB;
  const int j = (int)(t - i * NB);
  int x, y;
  demorton((uint32_t)i, x, y);
  const int p = shift_cell(x, y, nbr[j].x, nbr[j].y, L, nrow);
  E* out = Rbar + t * 4;
  for (int c = 0; c < 4; ++c)
    out[c] = p < 0 ? E(0) : v[i] * ubar[4 * (int64_t)p + c] + gbar[i] * ghat[4 * (int64_t)p + c];
}

// Y[o][P][a][b] -= lambda[4 P + a] w[4 P' + b], a, b < 3 (P' = P + O_o):
// the adjoint of B^(k) w^(k) = W g^(k) (Alg. 2 line 8).
template <typename E>
__global__ void k_ybar_level(E* __restrict__ Y, int noff, const int2* __restrict__ off,
                             int L, int64_t npar, const E* __restrict__ lam,
                             const E* __restrict__ w) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t P = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)P, x, y);
  const int Pp = shift_cell(x, y, off[o].x, off[o].y, L, npar);
  if (Pp < 0) return;
  E* B = Y + t * 16;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) B[4 * a + b] -= lam[4 * P + a] * w[4 * (int64_t)Pp + b];
}

// Abar^(1) = -lambda^(1) U^(1)^T (Alg. 2 line 16), plain 4 x 4.
template <typename E>
__global__ void k_abar1(E* __restrict__ A1bar, const E* __restrict__ lam1,
                        const E* __restrict__ U1) {
  const int t = threadIdx.x;
  if (t < 16) A1bar[t] = -lam1[t >> 2] * U1[t & 3];
}

// X[d][i] = sym(Abar^(k-1))(i, i + S_d) in plain level-(k-1) coordinates,
// from the transformed blocks Y of level k-1 (or, for k - 1 = 1, the plain
// 4 x 4 Abar^(1)).
template <typename E>
__global__ void k_xbar_cells(E* __restrict__ X, int nS, const int2* __restrict__ S, int L,
                             int64_t ncell, const E* __restrict__ A1bar,
                             const E* __restrict__ Y, int64_t npar_prev,
                             const int* __restrict__ oidx, int obox,
                             const uint32_t* __restrict__ pmask_prev) {
  __shared__ E Qs[256];
  stage_q<E>(Qs);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nS * ncell) return;
  const int d = (int)(t / ncell);
  const int64_t i = t - (int64_t)d * ncell;
  int x, y;
  demorton((uint32_t)i, x, y);
  const int ip = shift_cell(x, y, S[d].x, S[d].y, L, ncell);
  E v = E(0);
  if (ip >= 0) {
    if (A1bar) {
      v = E(0.5) * (A1bar[4 * i + ip] + A1bar[4 * ip + i]);
    } else {
      v = E(0.5) * (plain_entry(Y, npar_prev, oidx, obox, pmask_prev, Qs, i, ip) +
                 plain_entry(Y, npar_prev, oidx, obox, pmask_prev, Qs, ip, i));
    }
  }
  X[t] = v;
}

// T[w][i][c] = sum over (d, j) with S_d + N_j = TW_w of X[d][i] Rhat[i + S_d][j][c]
// (window position outermost, so consecutive threads take consecutive rows:
// the X reads and T writes coalesce).
template <typename E>
__global__ void k_window_product(E* __restrict__ T, int nTW, const int* __restrict__ tw_ptr,
                                 const int2* __restrict__ tw_pairs, const E* __restrict__ X,
                                 const int2* __restrict__ S, const E* __restrict__ Rhat,
                                 int NB, int L, int64_t nrow) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrow * nTW) return;
  const int w = (int)(t / nrow);
  const int64_t i = t - (int64_t)w * nrow;
  int x, y;
  demorton((uint32_t)i, x, y);
  E acc[4] = {E(0), E(0), E(0), E(0)};
  // four pairs per step in float32, their loads issued before any is used:
  // the chain pair -> X -> Rhat row is otherwise a dependent latency per
  // pair (in float64 the extra registers cost more occupancy than the
  // overlap gains: one pair per step measured fastest)
  constexpr int U = sizeof(E) == 4 ? 4 : 1;
  const int e1 = tw_ptr[w + 1];
  for (int e = tw_ptr[w]; e < e1; e += U) {
    int2 dj[U];
#pragma unroll
    for (int u = 0; u < U; ++u) dj[u] = e + u < e1 ? tw_pairs[e + u] : make_int2(-1, 0);
    E xv[U];
    int ip[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      xv[u] = E(0);
      ip[u] = -1;
      if (dj[u].x >= 0) {
        xv[u] = X[(int64_t)dj[u].x * nrow + i];
        const int2 sd = S[dj[u].x];
        ip[u] = shift_cell(x, y, sd.x, sd.y, L, nrow);
      }
    }
    E r[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (ip[u] >= 0 && xv[u] != E(0)) {
        ld4v(Rhat + ((int64_t)ip[u] * NB + dj[u].y) * 4, r[u]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) r[u][c] = E(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += xv[u] * r[u][c];
  }
  E* out = T + t * 4;
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] = acc[c];
}

// Rbar[i][j][c] += 2 sum_o sum_c' T[i][N_j - O_o][c'] Ahat[o][p - O_o][c'][c]
// (the adjoint of Alg. 2 line 13 with respect to R, on the pattern of Rhat).
template <typename E>
__global__ void k_rbar_galerkin(E* __restrict__ Rbar, const E* __restrict__ T, int nTW,
                                const int* __restrict__ rg, const E* __restrict__ Ahat,
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
  E acc[4] = {E(0), E(0), E(0), E(0)};
  for (int o = 0; o < noff; ++o) {
    const int w = rg[j * noff + o];
    if (w < 0) continue;
    const int Pp = shift_cell(px, py, -off[o].x, -off[o].y, L, nrow);
    if (Pp < 0) continue;
    const E* B = Ahat + ((int64_t)o * nrow + Pp) * 16;
    E tv[4], b[16];
    ld4v(T + ((int64_t)w * nrow + i) * 4, tv);
#pragma unroll
    for (int cp = 0; cp < 4; ++cp) ld4v(B + 4 * cp, b + 4 * cp);
#pragma unroll
    for (int cp = 0; cp < 4; ++cp)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] += tv[cp] * b[4 * cp + c];
  }
  E* out = Rbar + t * 4;
#pragma unroll
  for (int c = 0; c < 4; ++c) out[c] += 2.0 * acc[c];
}

// Y[o][P] += sum_j Rhat[i][j]^T (T[i][N_j + O_o] - M[i][j']) with i = P - N_j
// and N_j' = N_j + O_o: the adjoint of Alg. 2 line 13 with respect to A^(k)
// and of the patch solves (line 11) with respect to their matrices and
// right-hand sides, both in transposed form (Y is symmetrised when used).
template <typename E>
__global__ void k_ybar_galerkin(E* __restrict__ Y, int noff, const int2* __restrict__ off,
                                const int2* __restrict__ yg, const E* __restrict__ T, int nTW,
                                const E* __restrict__ Rhat, const E* __restrict__ M,
                                const int2* __restrict__ nbr, int NB, int L, int64_t npar) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t P = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)P, x, y);
  if (shift_cell(x, y, off[o].x, off[o].y, L, npar) < 0) return;
  E acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = E(0);
  for (int j = 0; j < NB; ++j) {
    const int i = shift_cell(x, y, -nbr[j].x, -nbr[j].y, L, npar);
    if (i < 0) continue;
    const int2 wj = yg[o * NB + j];
    E r[4], z[4] = {E(0), E(0), E(0), E(0)}, m[4] = {E(0), E(0), E(0), E(0)};
    ld4v(Rhat + ((int64_t)i * NB + j) * 4, r);
    if (wj.x >= 0) ld4v(T + ((int64_t)wj.x * npar + i) * 4, z);
    if (wj.y >= 0) ld4v(M + ((int64_t)i * NB + wj.y) * 4, m);
#pragma unroll
    for (int c = 0; c < 4; ++c) z[c] -= m[c];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[4 * a + b] += r[a] * z[b];
  }
  E* B = Y + t * 16;
#pragma unroll
  for (int e = 0; e < 16; ++e) B[e] += acc[e];
}

// dJ/dlog a_c = a_c sum_{p,r} sym(Abar^(q))(p, r) K_ref[p][r] over the
// interior corners of cell c (A^(q) = sum_c a_c K_c, Sec. 5.1).
template <typename E>
__global__ void k_grad_cells(double* __restrict__ out, int ncell,
                             const int32_t* __restrict__ cell_nodes,
                             const double* __restrict__ cell_a, const double* __restrict__ Kref,
                             const int32_t* __restrict__ morton_of, const E* __restrict__ Y,
                             int64_t npar, const int* __restrict__ oidx, int obox,
                             const uint32_t* __restrict__ pmask) {
  __shared__ E Qs[256];
  stage_q<E>(Qs);
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
      const double xv = 0.5 * ((double)plain_entry(Y, npar, oidx, obox, pmask, Qs, m[p], m[r]) +
                               (double)plain_entry(Y, npar, oidx, obox, pmask, Qs, m[r], m[p]));
      s += xv * Kref[4 * p + r];
    }
  }
  out[c] = cell_a[c] * s;
}

static unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename E>
void launch_rbar_outer(E* Rbar, const int2* nbr, int NB, int L, int64_t nrow, const E* v,
                       const E* gbar, const E* ubar, const E* ghat, cudaStream_t s) {
  if (nrow * NB <= 0) return;
  count_launch();
  k_rbar_outer<E><<<nblk(nrow * NB, 256), 256, 0, s>>>(Rbar, nbr, NB, L, nrow, v, gbar, ubar,
                                                        ghat);
}
template <typename E>
void launch_ybar_level(E* Y, int noff, const int2* off, int L, int64_t npar, const E* lam,
                       const E* w, cudaStream_t s) {
  if ((int64_t)noff * npar <= 0) return;
  count_launch();
  k_ybar_level<E><<<nblk((int64_t)noff * npar, 256), 256, 0, s>>>(Y, noff, off, L, npar, lam, w);
}
template <typename E>
void launch_abar1(E* A1bar, const E* lam1, const E* U1, cudaStream_t s) {
  count_launch();
  k_abar1<E><<<1, 32, 0, s>>>(A1bar, lam1, U1);
}
template <typename E>
void launch_xbar_cells(E* X, int nS, const int2* S, int L, int64_t ncell, const E* A1bar,
                       const E* Y, int64_t npar_prev, const int* oidx, int obox,
                       const uint32_t* pmask_prev, cudaStream_t s) {
  if ((int64_t)nS * ncell <= 0) return;
  count_launch();
  k_xbar_cells<E><<<nblk((int64_t)nS * ncell, 256), 256, 0, s>>>(X, nS, S, L, ncell, A1bar, Y,
                                                                  npar_prev, oidx, obox,
                                                                  pmask_prev);
}
template <typename E>
void launch_window_product(E* T, int nTW, const int* tw_ptr, const int2* tw_pairs, const E* X,
                           const int2* S, const E* Rhat, int NB, int L, int64_t nrow,
                           cudaStream_t s) {
  if (nrow * nTW <= 0) return;
  count_launch();
  k_window_product<E><<<nblk(nrow * nTW, 256), 256, 0, s>>>(T, nTW, tw_ptr, tw_pairs, X, S,
                                                             Rhat, NB, L, nrow);
}
template <typename E>
void launch_rbar_galerkin(E* Rbar, const E* T, int nTW, const int* rg, const E* Ahat, int noff,
                          const int2* off, const int2* nbr, int NB, int L, int64_t nrow,
                          cudaStream_t s) {
  if (nrow * NB <= 0) return;
  count_launch();
  k_rbar_galerkin<E><<<nblk(nrow * NB, 128), 128, 0, s>>>(Rbar, T, nTW, rg, Ahat, noff, off,
                                                           nbr, NB, L, nrow);
}
template <typename E>
void launch_ybar_galerkin(E* Y, int noff, const int2* off, const int2* yg, const E* T, int nTW,
                          const E* Rhat, const E* M, const int2* nbr, int NB, int L, int64_t npar,
                          cudaStream_t s) {
  if ((int64_t)noff * npar <= 0) return;
  count_launch();
  k_ybar_galerkin<E><<<nblk((int64_t)noff * npar, 128), 128, 0, s>>>(Y, noff, off, yg, T, nTW,
                                                                      Rhat, M, nbr, NB, L, npar);
}
template <typename E>
void launch_grad_cells(double* out, int ncell, const int32_t* cell_nodes, const double* cell_a,
                       const double* Kref, const int32_t* morton_of, const E* Y, int64_t npar,
                       const int* oidx, int obox, const uint32_t* pmask, cudaStream_t s) {
  if (ncell <= 0) return;
  count_launch();
  k_grad_cells<E><<<nblk(ncell, 128), 128, 0, s>>>(out, ncell, cell_nodes, cell_a, Kref,
                                                    morton_of, Y, npar, oidx, obox, pmask);
}

#define GB_ONEPASS_INSTANTIATE(E)                                                                \
  template void launch_rbar_outer<E>(E*, const int2*, int, int, int64_t, const E*, const E*,     \
                                     const E*, const E*, cudaStream_t);                          \
  template void launch_ybar_level<E>(E*, int, const int2*, int, int64_t, const E*, const E*,     \
                                     cudaStream_t);                                              \
  template void launch_abar1<E>(E*, const E*, const E*, cudaStream_t);                           \
  template void launch_xbar_cells<E>(E*, int, const int2*, int, int64_t, const E*, const E*,     \
                                     int64_t, const int*, int, const uint32_t*, cudaStream_t);   \
  template void launch_window_product<E>(E*, int, const int*, const int2*, const E*,             \
                                         const int2*, const E*, int, int, int64_t,               \
                                         cudaStream_t);                                          \
  template void launch_rbar_galerkin<E>(E*, const E*, int, const int*, const E*, int,            \
                                        const int2*, const int2*, int, int, int64_t,             \
                                        cudaStream_t);                                           \
  template void launch_ybar_galerkin<E>(E*, int, const int2*, const int2*, const E*, int,        \
                                        const E*, const E*, const int2*, int, int, int64_t,      \
                                        cudaStream_t);                                           \
  template void launch_grad_cells<E>(double*, int, const int32_t*, const double*, const double*, \
                                     const int32_t*, const E*, int64_t, const int*, int,         \
                                     const uint32_t*, cudaStream_t);
GB_ONEPASS_INSTANTIATE(float)
GB_ONEPASS_INSTANTIATE(double)
#undef GB_ONEPASS_INSTANTIATE

}  // namespace gb
