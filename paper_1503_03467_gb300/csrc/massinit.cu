// massinit.cu - level-q initialisation by the mass matrix (Algorithm 1,
// lines 1-5; Algorithm 2, lines 2a-5 with Definition deflocinvm).
//
// The level-q gamblets psi^(q)_i = sum_j (M^-1,loc)_{j,i} phi_j have
// integral delta_ij against phi_j for j in the patch i^{rho_q}: column i of
// M^-1,loc solves the mass system restricted to the patch with right-hand
// side e_i.  The method then runs on A^(q),loc = (M^-1,loc)^T A M^-1,loc and
// the solution's nodal coefficients are u_phi = M^-1,loc U.
//
// Data: nodes are the fine unknowns; their cells give the geometry.  Fine
// operators are held as per-node stencils St[i][s] = X_{i, node(c_i + S_s)}
// over the offsets S of their CSR extent; M^-1,loc as Minv[i][j], the entry
// of patch node c_i + N_j in column i.  All arithmetic is float64.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

// Largest |cell offset| in x and y over the stored entries (atomicMax);
// bad = 1 for a column index out of range or a decreasing rowptr.
__global__ void k_csr_node_extent(int n, const int32_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ colind,
                                  const int32_t* __restrict__ morton_of, int* ext, int* bad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int xi, yi;
  demorton((uint32_t)morton_of[i], xi, yi);
  const int b = rowptr[i], e = rowptr[i + 1];
  if (e < b) {
    atomicExch(bad, 1);
    return;
  }
  int mx = 0, my = 0;
  for (int t = b; t < e; ++t) {
    const int j = colind[t];
    if ((unsigned)j >= (unsigned)n) {
      atomicExch(bad, 1);
      continue;
    }
    int xj, yj;
    demorton((uint32_t)morton_of[j], xj, yj);
    mx = max(mx, abs(xj - xi));
    my = max(my, abs(yj - yi));
  }
  atomicMax(&ext[0], mx);
  atomicMax(&ext[1], my);
}

void launch_csr_node_extent(int n, const int32_t* rowptr, const int32_t* colind,
                            const int32_t* morton_of, int* ext, int* bad, cudaStream_t s) {
  if (n > 0) { count_launch(); k_csr_node_extent<<<(n + 127) / 128, 128, 0, s>>>(n, rowptr, colind, morton_of, ext, bad); }
}

// St[i][s] = X_{i, j} for every stored entry with cell offset c_j - c_i = S_s
// (S: the (2 rx + 1) x (2 ry + 1) box, row-major in (dy, dx)).
__global__ void k_csr_to_stencil(int n, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind,
                                 const double* __restrict__ val,
                                 const int32_t* __restrict__ morton_of, int rx, int ry,
                                 double* St) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int xi, yi;
  demorton((uint32_t)morton_of[i], xi, yi);
  const int ns = (2 * rx + 1) * (2 * ry + 1);
  for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    const int j = colind[t];
    if ((unsigned)j >= (unsigned)n) continue;
    int xj, yj;
    demorton((uint32_t)morton_of[j], xj, yj);
    const int dx = xj - xi, dy = yj - yi;
    if (dx < -rx || dx > rx || dy < -ry || dy > ry) continue;
    St[(int64_t)i * ns + (dy + ry) * (2 * rx + 1) + dx + rx] += val[t];
  }
}

void launch_csr_to_stencil(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                           const int32_t* morton_of, int rx, int ry, double* St, cudaStream_t s) {
  if (n > 0) { count_launch(); k_csr_to_stencil<<<(n + 127) / 128, 128, 0, s>>>(n, rowptr, colind, val, morton_of, rx, ry, St); }
}

// Node of the cell (x + dx, y + dy) of the level-q lattice, or -1.
__device__ __forceinline__ int node_at(int x, int y, int dx, int dy, int L, int64_t ncell,
                                       const int32_t* __restrict__ unknown_of) {
  const int c = shift_cell(x, y, dx, dy, L, ncell);
  return c >= 0 ? unknown_of[c] : -1;
}

// Column i of M^-1,loc: Cholesky of M restricted to the patch nodes
// c_i + N_j (absent nodes get unit rows), then L L^T y = e_{jc}.  One CTA of
// 64 threads per node, the patch matrix in shared memory.
__global__ void __launch_bounds__(64) k_mass_patch_inverse(
    int n, int NB, int jc, const int2* __restrict__ nbr, const double* __restrict__ Mst,
    int mrx, int mry, const int32_t* __restrict__ morton_of,
    const int32_t* __restrict__ unknown_of, int L, int64_t ncell, double* Minv, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* Lm = reinterpret_cast<double*>(smem_raw);  // NB x NB
  double* y = Lm + (size_t)NB * NB;
  int* pnode = reinterpret_cast<int*>(y + NB);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mw = 2 * mrx + 1, ms = mw * (2 * mry + 1);
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    int xi, yi;
    demorton((uint32_t)morton_of[i], xi, yi);
    for (int j = tid; j < NB; j += nt) pnode[j] = node_at(xi, yi, nbr[j].x, nbr[j].y, L, ncell, unknown_of);
    __syncthreads();
    for (int e = tid; e < NB * NB; e += nt) {
      const int a = e / NB, b = e - a * NB;
      double v = 0.0;
      const int pa = pnode[a], pb = pnode[b];
      if (pa >= 0 && pb >= 0) {
        const int dx = nbr[b].x - nbr[a].x, dy = nbr[b].y - nbr[a].y;
        if (dx >= -mrx && dx <= mrx && dy >= -mry && dy <= mry)
          v = Mst[(int64_t)pa * ms + (dy + mry) * mw + dx + mrx];
      } else if (a == b) {
        v = 1.0;
      }
      Lm[e] = v;
    }
    __syncthreads();
    // right-looking Cholesky, lower triangle
    for (int k = 0; k < NB; ++k) {
      if (tid == 0) {
        double d = Lm[k * NB + k];
        if (!(d > 0)) {
          atomicExch(status, (int)DEV_NOT_SPD);
          d = 1.0;
        }
        Lm[k * NB + k] = sqrt(d);
      }
      __syncthreads();
      const double dk = Lm[k * NB + k];
      for (int r = k + 1 + tid; r < NB; r += nt) Lm[r * NB + k] /= dk;
      __syncthreads();
      const int m = NB - k - 1;
      for (int e = tid; e < m * m; e += nt) {
        const int r = k + 1 + e / m, c = k + 1 + e % m;
        if (c <= r) Lm[r * NB + c] -= Lm[r * NB + k] * Lm[c * NB + k];
      }
      __syncthreads();
    }
    // L z = e_jc, then L^T y = z (serial over k, parallel over rows)
    for (int r = tid; r < NB; r += nt) y[r] = r == jc ? 1.0 : 0.0;
    __syncthreads();
    for (int k = 0; k < NB; ++k) {
      if (tid == 0) y[k] /= Lm[k * NB + k];
      __syncthreads();
      for (int r = k + 1 + tid; r < NB; r += nt) y[r] -= Lm[r * NB + k] * y[k];
      __syncthreads();
    }
    for (int k = NB - 1; k >= 0; --k) {
      if (tid == 0) y[k] /= Lm[k * NB + k];
      __syncthreads();
      for (int r = tid; r < k; r += nt) y[r] -= Lm[k * NB + r] * y[k];
      __syncthreads();
    }
    for (int j = tid; j < NB; j += nt) Minv[(int64_t)i * NB + j] = pnode[j] >= 0 ? y[j] : 0.0;
    __syncthreads();
  }
}

size_t mass_patch_smem_bytes(int NB) {
  return sizeof(double) * ((size_t)NB * NB + NB) + sizeof(int) * (size_t)NB + 16;
}

void launch_mass_patch_inverse(int n, int NB, int jc, const int2* nbr, const double* Mst, int mrx,
                               int mry, const int32_t* morton_of, const int32_t* unknown_of,
                               int L, int64_t ncell, double* Minv, int* status, int num_sms,
                               cudaStream_t s) {
  if (n <= 0) return;
  const size_t smem = mass_patch_smem_bytes(NB);
  cudaFuncSetAttribute(k_mass_patch_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mass_patch_inverse, 64, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > n) grid = n;
  count_launch();
  k_mass_patch_inverse<<<(unsigned)grid, 64, smem, s>>>(n, NB, jc, nbr, Mst, mrx, mry, morton_of,
                                                          unknown_of, L, ncell, Minv, status);
}

// Row i of A^(q),loc = (M^-1,loc)^T A M^-1,loc on the output offsets d:
//   t(w)    = sum_(s, j) in L1_w  A_{node(c_i + w), s} Minv[i][j]   (W_w + A_s = N_j)
//   out[d]  = sum_(j, w) in L2_d  Minv[node(c_i + d)][j] t(w)       (W_w = D_d + N_j)
// One CTA of 128 threads per node.
__global__ void __launch_bounds__(128) k_mass_triple(
    int n, MassTripleGeom g, const double* __restrict__ Ast, const double* __restrict__ Minv,
    const int32_t* __restrict__ morton_of, const int32_t* __restrict__ unknown_of, int L,
    int64_t ncell, double* out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* mi = reinterpret_cast<double*>(smem_raw);  // NB
  double* t = mi + g.NB;                             // nwin
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    int xi, yi;
    demorton((uint32_t)morton_of[i], xi, yi);
    for (int j = threadIdx.x; j < g.NB; j += blockDim.x) mi[j] = Minv[(int64_t)i * g.NB + j];
    __syncthreads();
    for (int w = threadIdx.x; w < g.nwin; w += blockDim.x) {
      const int r = node_at(xi, yi, g.win[w].x, g.win[w].y, L, ncell, unknown_of);
      double acc = 0.0;
      if (r >= 0)
        for (int e = g.l1_ptr[w]; e < g.l1_ptr[w + 1]; ++e) {
          const int2 sj = g.l1[e];
          acc += Ast[(int64_t)r * g.nast + sj.x] * mi[sj.y];
        }
      t[w] = acc;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < g.nout; d += blockDim.x) {
      const int r = node_at(xi, yi, g.out[d].x, g.out[d].y, L, ncell, unknown_of);
      double acc = 0.0;
      if (r >= 0)
        for (int e = g.l2_ptr[d]; e < g.l2_ptr[d + 1]; ++e) {
          const int2 jw = g.l2[e];
          acc += Minv[(int64_t)r * g.NB + jw.x] * t[jw.y];
        }
      out[(int64_t)i * g.nout + d] = acc;
    }
    __syncthreads();
  }
}

void launch_mass_triple(int n, MassTripleGeom g, const double* Ast, const double* Minv,
                        const int32_t* morton_of, const int32_t* unknown_of, int L, int64_t ncell,
                        double* out, cudaStream_t s) {
  if (n <= 0) return;
  const size_t smem = sizeof(double) * ((size_t)g.NB + g.nwin);
  cudaFuncSetAttribute(k_mass_triple, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int grid = n < 65535 * 16 ? n : 65535 * 16;
  count_launch();
  k_mass_triple<<<grid, 128, smem, s>>>(n, g, Ast, Minv, morton_of, unknown_of, L, ncell, out);
}

// Entries per row of the CSR of A^(q),loc: output offsets whose node exists.
__global__ void k_stencil_counts(int n, const int2* __restrict__ off, int noff,
                                 const int32_t* __restrict__ morton_of,
                                 const int32_t* __restrict__ unknown_of, int L, int64_t ncell,
                                 int32_t* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int xi, yi;
  demorton((uint32_t)morton_of[i], xi, yi);
  int c = 0;
  for (int d = 0; d < noff; ++d) c += node_at(xi, yi, off[d].x, off[d].y, L, ncell, unknown_of) >= 0;
  count[i] = c;
}

// CSR fill, symmetrised: value (X_{i,d} + X_{r,-d}) / 2 with r = node(c_i + d)
// and -d at index mirror[d] of the offset list.
__global__ void k_stencil_to_csr(int n, const int2* __restrict__ off, const int* __restrict__ mirror,
                                 int noff, const double* __restrict__ X,
                                 const int32_t* __restrict__ morton_of,
                                 const int32_t* __restrict__ unknown_of, int L, int64_t ncell,
                                 const int32_t* __restrict__ rowptr, int32_t* colind, double* val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int xi, yi;
  demorton((uint32_t)morton_of[i], xi, yi);
  int t = rowptr[i];
  for (int d = 0; d < noff; ++d) {
    const int r = node_at(xi, yi, off[d].x, off[d].y, L, ncell, unknown_of);
    if (r < 0) continue;
    colind[t] = r;
    val[t] = 0.5 * (X[(int64_t)i * noff + d] + X[(int64_t)r * noff + mirror[d]]);
    ++t;
  }
}

void launch_stencil_counts(int n, const int2* off, int noff, const int32_t* morton_of,
                           const int32_t* unknown_of, int L, int64_t ncell, int32_t* count,
                           cudaStream_t s) {
  if (n > 0) { count_launch(); k_stencil_counts<<<(n + 127) / 128, 128, 0, s>>>(n, off, noff, morton_of, unknown_of, L, ncell, count); }
}
void launch_stencil_to_csr(int n, const int2* off, const int* mirror, int noff, const double* X,
                           const int32_t* morton_of, const int32_t* unknown_of, int L,
                           int64_t ncell, const int32_t* rowptr, int32_t* colind, double* val,
                           cudaStream_t s) {
  if (n > 0) { count_launch(); k_stencil_to_csr<<<(n + 127) / 128, 128, 0, s>>>(n, off, mirror, noff, X, morton_of, unknown_of, L, ncell, rowptr, colind, val); }
}

// u_phi[j] = sum_k Minv[r][k] U[r] over the patches that contain node j:
// r = node(c_j - N_k).
__global__ void k_mass_apply(int n, int NB, const int2* __restrict__ nbr,
                             const double* __restrict__ Minv, const double* __restrict__ U,
                             const int32_t* __restrict__ morton_of,
                             const int32_t* __restrict__ unknown_of, int L, int64_t ncell,
                             double* u) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int xj, yj;
  demorton((uint32_t)morton_of[j], xj, yj);
  double acc = 0.0;
  for (int k = 0; k < NB; ++k) {
    const int r = node_at(xj, yj, -nbr[k].x, -nbr[k].y, L, ncell, unknown_of);
    if (r >= 0) acc += Minv[(int64_t)r * NB + k] * U[r];
  }
  u[j] = acc;
}

void launch_mass_apply(int n, int NB, const int2* nbr, const double* Minv, const double* U,
                       const int32_t* morton_of, const int32_t* unknown_of, int L, int64_t ncell,
                       double* u, cudaStream_t s) {
  if (n > 0) { count_launch(); k_mass_apply<<<(n + 127) / 128, 128, 0, s>>>(n, NB, nbr, Minv, U, morton_of, unknown_of, L, ncell, u); }
}

}  // namespace gb
