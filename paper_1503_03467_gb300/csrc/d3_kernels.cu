// d3_kernels.cu - device kernels of the three-dimensional gamblet path.
//
// Hierarchy (Sec. 4.1, Construction defmulires with H = 1/2 in 3-D: a cube
// splits into eight), per-parent Helmert transforms (Sec. 4.6, Lemma
// const0, Construction const2), the localized patch systems of Definition
// defb (Alg. 2 line 11), R = pibar + D W (line 12), the Galerkin product
// A^(k-1) = R A R^T (line 13), the restriction g^(k-1) = R g^(k) (line 15),
// the level systems B^(k) w = W g^(k) (line 8, solved by block-Jacobi CG)
// and the prolongation and sum (lines 10, 17, 18).  The data layout is
// described in d3.cuh.
//
// Work is mapped in groups of eight lanes, one lane per slot of a parent
// (a row of an 8x8 block, an entry of a per-parent vector): a group's loads
// of one block row or one parent vector are 64 contiguous bytes, and the
// per-parent transforms are shuffles within the group.
#include <algorithm>

#include "d3.cuh"

namespace gb {
namespace d3 {

// Index guard: every table-driven index of the setup kernels is checked
// against the size of the buffer it addresses; a violation skips the access
// and records the number of the check in g_guard (first one wins), which the
// host turns into an error.  Never expected to fire; it keeps a corrupted
// plan from reaching memory outside the handle's buffers.
__device__ int g_guard;
__device__ __forceinline__ bool inb(int id, long long idx, long long size) {
  if (idx >= 0 && idx < size) return true;
  atomicCAS(&g_guard, 0, id);
  return false;
}
int guard_take() {
  int v = 0;
  cudaMemcpyFromSymbol(&v, g_guard, sizeof(int));
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_guard, &zero, sizeof(int));
  }
  return v;
}

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double group8_sum(double v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  return v;
}

// Sum of v over the CTA (every thread receives it).  The partial values go
// through shared memory and one warp adds them (eight per lane, then a
// butterfly), so the float64 pipe, the scarce unit of this part, sees 13
// warp instructions per sum instead of 13 for every warp.  red holds
// kRed doubles; all threads of the CTA must call it.
constexpr int kRed = 2 * kThreads + 2;
__device__ __forceinline__ double cta_sum(double v, double* red) {
  const int nt = blockDim.x;
  __syncthreads();  // earlier readers of red are done
  red[threadIdx.x] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0;
    for (int i = threadIdx.x; i < nt; i += 32) s += red[i];
    s = warp_sum(s);
    if (threadIdx.x == 0) red[2 * nt] = s;
  }
  __syncthreads();
  return red[2 * nt];
}

__device__ __forceinline__ void cta_sum2(double& a, double& b, double* red) {
  const int nt = blockDim.x;
  __syncthreads();
  red[threadIdx.x] = a;
  red[nt + threadIdx.x] = b;
  __syncthreads();
  if (threadIdx.x < 32) {
    double sa = 0, sb = 0;
    for (int i = threadIdx.x; i < nt; i += 32) {
      sa += red[i];
      sb += red[nt + i];
    }
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    if (threadIdx.x == 0) {
      red[2 * nt] = sa;
      red[2 * nt + 1] = sb;
    }
  }
  __syncthreads();
  a = red[2 * nt];
  b = red[2 * nt + 1];
}

}  // namespace

// ---------------------------------------------------------------- hierarchy
__global__ void k_cells_to_morton3(const int32_t* __restrict__ cells, int n, int q,
                                   int32_t* morton_of, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = cells[3 * i], y = cells[3 * i + 1], z = cells[3 * i + 2];
  const unsigned L = 1u << q;
  if ((unsigned)x >= L || (unsigned)y >= L || (unsigned)z >= L) {
    atomicExch(flag, 2);
    morton_of[i] = 0;
    return;
  }
  morton_of[i] = (int32_t)morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
}

__global__ void k_scatter3(const int32_t* __restrict__ morton_of, int n, int32_t* unknown_of,
                           uint32_t* pmask_q, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t m = (uint32_t)morton_of[i];
  if (atomicExch(&unknown_of[m], i) != -1) atomicExch(flag, 1);
  atomicOr(&pmask_q[m >> 3], 1u << (m & 7));
}

__global__ void k_coarsen3(const uint32_t* __restrict__ pmask_k, int64_t npar_km1,
                           uint32_t* pmask_km1) {
  const int64_t P = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (P >= npar_km1) return;
  uint32_t m = 0;
  for (int c = 0; c < 8; ++c)
    if (pmask_k[8 * P + c]) m |= 1u << c;
  pmask_km1[P] = m;
}

void launch_cells_to_morton3(const int32_t* cells, int n, int q, int32_t* morton_of, int* flag,
                             cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_cells_to_morton3<<<(n + 255) / 256, 256, 0, s>>>(cells, n, q, morton_of, flag);
}
void launch_scatter3(const int32_t* morton_of, int n, int32_t* unknown_of, uint32_t* pmask_q,
                     int* flag, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_scatter3<<<(n + 255) / 256, 256, 0, s>>>(morton_of, n, unknown_of, pmask_q, flag);
}
void launch_coarsen3(const uint32_t* pmask_k, int64_t npar_km1, uint32_t* pmask_km1,
                     cudaStream_t s) {
  count_launch();
  k_coarsen3<<<(unsigned)((npar_km1 + 255) / 256), 256, 0, s>>>(pmask_k, npar_km1, pmask_km1);
}

// ---------------------------------------------------------------- fine operator
__global__ void k_csr_extent3(int n, const int32_t* __restrict__ rowptr,
                              const int32_t* __restrict__ colind,
                              const int32_t* __restrict__ morton_of, int* ext, int* flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x, y, z;
  demorton3((uint32_t)morton_of[i] >> 3, x, y, z);
  int e = 0;
  for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    const int j = colind[t];
    if ((unsigned)j >= (unsigned)n) {
      atomicExch(flag, 3);
      continue;
    }
    int a, b, c;
    demorton3((uint32_t)morton_of[j] >> 3, a, b, c);
    e = max(e, max(abs(a - x), max(abs(b - y), abs(c - z))));
  }
  atomicMax(ext, e);
}

__global__ void k_csr_to_blocks3(int n, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind,
                                 const double* __restrict__ val,
                                 const int32_t* __restrict__ morton_of, OffLookup lk,
                                 int64_t npar, double* blk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t mi = (uint32_t)morton_of[i];
  int x, y, z;
  demorton3(mi >> 3, x, y, z);
  for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    const uint32_t mj = (uint32_t)morton_of[colind[t]];
    int a, b, c;
    demorton3(mj >> 3, a, b, c);
    const int o = lk.find(a - x, b - y, c - z);
    if (o < 0) continue;  // cannot happen: the set is the box of the measured extent
    if (!inb(1, ((int64_t)o * npar + (mi >> 3)) * 64 + 63, (long long)(2 * lk.R + 1) * (2 * lk.R + 1) * (2 * lk.R + 1) * npar * 64)) continue;
    blk[((int64_t)o * npar + (mi >> 3)) * 64 + (mi & 7) * 8 + (mj & 7)] += val[t];
  }
}

void launch_csr_extent3(int n, const int32_t* rowptr, const int32_t* colind,
                        const int32_t* morton_of, int* ext, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_csr_extent3<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, colind, morton_of, ext, flag);
}
void launch_csr_to_blocks3(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                           const int32_t* morton_of, OffLookup lk, int q, int64_t npar,
                           double* blk, cudaStream_t s) {
  (void)q;
  if (n <= 0) return;
  count_launch();
  k_csr_to_blocks3<<<(n + 255) / 256, 256, 0, s>>>(n, rowptr, colind, val, morton_of, lk, npar,
                                                   blk);
}

// ---------------------------------------------------------------- transforms
// The 8x8 transforms of all 256 masks, row-major, built on the host from
// q8() and uploaded once per handle (qtab[m * 64 + 8 a + c]).
__global__ void k_transform_blocks3(const double* __restrict__ src, double* dst,
                                    const int4* __restrict__ off, const int* __restrict__ mirror,
                                    int noff, int64_t npar, int Lpar,
                                    const uint32_t* __restrict__ pmask,
                                    const double* __restrict__ qtab, int symmetrize) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t blkid = gid >> 3;  // uniform within each group of eight lanes
  const int a = (int)(gid & 7);
  const bool live = blkid < (int64_t)noff * npar;
  int o = 0;
  int64_t p = 0;
  int pn = -1;
  if (live) {
    o = (int)(blkid / npar);
    p = blkid - (int64_t)o * npar;
    int x, y, z;
    demorton3((uint32_t)p, x, y, z);
    const int4 d = off[o];
    pn = shift3(x, y, z, d.x, d.y, d.z, Lpar);
  }
  double row[8];
  const double* sb = src + blkid * 64 + a * 8;
  if (live && pn >= 0 && symmetrize &&
      !inb(2, ((int64_t)mirror[o] * npar + pn) * 64 + 63, (long long)noff * npar * 64))
    pn = -1;
  if (live && pn >= 0) {
#pragma unroll
    for (int b = 0; b < 8; ++b) row[b] = sb[b];
    if (symmetrize) {
      const double* mb = src + ((int64_t)mirror[o] * npar + pn) * 64 + a;
#pragma unroll
      for (int b = 0; b < 8; ++b) row[b] = 0.5 * (row[b] + mb[b * 8]);
    }
  } else {
#pragma unroll
    for (int b = 0; b < 8; ++b) row[b] = 0.0;
  }
  // columns: (A Q'^T)[a][b'] = sum_b A[a][b] Q'[b'][b]
  double t[8];
  const double* Qn = qtab + (int64_t)((pn >= 0 && live) ? pmask[pn] : 0) * 64;
#pragma unroll
  for (int bp = 0; bp < 8; ++bp) {
    double s = 0;
#pragma unroll
    for (int b = 0; b < 8; ++b) s += row[b] * Qn[bp * 8 + b];
    t[bp] = s;
  }
  // rows: out[a'][b'] = sum_a Q[a'][a] t_a[b'] (t_a held by lane a of the group)
  const double* Qp = qtab + (int64_t)(live ? pmask[p] : 0) * 64 + a * 8;
  const int base = threadIdx.x & ~7;
  double out[8];
#pragma unroll
  for (int bp = 0; bp < 8; ++bp) out[bp] = 0.0;
#pragma unroll
  for (int src_lane = 0; src_lane < 8; ++src_lane) {
    const double qa = Qp[src_lane];
#pragma unroll
    for (int bp = 0; bp < 8; ++bp)
      out[bp] += qa * __shfl_sync(0xffffffffu, t[bp], (base + src_lane) & 31);
  }
  if (live) {
    double* db = dst + blkid * 64 + a * 8;
#pragma unroll
    for (int bp = 0; bp < 8; ++bp) db[bp] = out[bp];
  }
}

void launch_transform_blocks3(const double* src, double* dst, const int4* off, const int* mirror,
                              int noff, int64_t npar, int Lpar, const uint32_t* pmask,
                              int symmetrize, const double* qtab, cudaStream_t s) {
  const int64_t threads = (int64_t)noff * npar * 8;
  if (threads <= 0) return;
  count_launch();
  k_transform_blocks3<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      src, dst, off, mirror, noff, npar, Lpar, pmask, qtab, symmetrize);
}

// Block-Jacobi factor of one parent: inverse of the leading (m-1)x(m-1)
// detail block of Ahat(0, p) by Cholesky, one thread per parent.
__global__ void k_detail_inverse3(const double* __restrict__ Ahat, int o0, int64_t npar,
                                  const uint32_t* __restrict__ pmask, double* Dinv, int* status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npar) return;
  double* out = Dinv + p * 64;
  const int nd = max(__popc(pmask[p] & 255u) - 1, 0);
  double L[7][7];
  const double* A = Ahat + ((int64_t)o0 * npar + p) * 64;
  for (int i = 0; i < nd; ++i)
    for (int j = 0; j <= i; ++j) L[i][j] = A[i * 8 + j];
  bool ok = true;
  for (int j = 0; j < nd && ok; ++j) {
    double d = L[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) {
      ok = false;
      break;
    }
    d = sqrt(d);
    L[j][j] = d;
    for (int i = j + 1; i < nd; ++i) {
      double v = L[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / d;
    }
  }
  for (int e = 0; e < 64; ++e) out[e] = 0.0;
  if (!ok) {
    atomicExch(status, (int)DEV_NOT_SPD);
    return;
  }
  // columns of L^-T L^-1: solve L y = e_c, then L^T x = y
  for (int c = 0; c < nd; ++c) {
    double y[7];
    for (int i = 0; i < nd; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
      y[i] = v / L[i][i];
    }
    for (int i = nd - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < nd; ++k) v -= L[k][i] * y[k];
      y[i] = v / L[i][i];
    }
    for (int i = 0; i < nd; ++i) out[i * 8 + c] = y[i];
  }
}

void launch_detail_inverse3(const double* Ahat, int o0, int64_t npar, const uint32_t* pmask,
                            double* Dinv, int* status, cudaStream_t s) {
  if (npar <= 0) return;
  count_launch();
  k_detail_inverse3<<<(unsigned)((npar + 127) / 128), 128, 0, s>>>(Ahat, o0, npar, pmask, Dinv,
                                                                   status);
}

// ---------------------------------------------------------------- patch systems
// One CTA per coarse cell i (parent P_i of level k).  Unknowns: the detail
// slots t <= 6 of the patch parents P_i + N_j, held in shared memory as
// [NB][8] (slot 7 unused).  The matrix is B restricted to the patch: the
// detail-detail part of Ahat(N_b - N_a, P_i + N_a), read through L2.  The
// right-hand side is b_(j,t) = -(W A pibar^T)_((j,t), i)
// = -Ahat(P_i - P_j, P_j)[t][7] / sqrt(m_i).
size_t patch_cg3_smem(int NB) { return (size_t)NB * (5 * 8 * sizeof(double) + 2 * sizeof(int)); }

__global__ void __launch_bounds__(kThreads)
    k_patch_cg3(const double* __restrict__ Ahat, const double* __restrict__ Dinv,
                const uint32_t* __restrict__ pmask_k, Patch3Geom g, double tol, int max_iter,
                double* Rhat, int* iter_stats) {
  extern __shared__ double sm[];
  __shared__ double red[kRed];
  const int NB = g.NB;
  const int NV = NB * 8;
  double* x = sm;
  double* r = x + NV;
  double* z = r + NV;
  double* p = z + NV;
  double* q = p + NV;
  int* pid = reinterpret_cast<int*>(q + NV);
  const int64_t i = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t npar = g.npatch;
  double* Ri = Rhat + i * (int64_t)NV;
  const uint32_t mi = pmask_k[i];
  if (mi == 0) {
    for (int e = tid; e < NV; e += blockDim.x) Ri[e] = 0.0;
    return;
  }
  int cx, cy, cz;
  demorton3((uint32_t)i, cx, cy, cz);
  for (int j = tid; j < NB; j += blockDim.x) {
    const int4 o = g.nbr[j];
    int P = shift3(cx, cy, cz, o.x, o.y, o.z, g.Lpar);
    if (P >= 0 && !inb(3, P, npar)) P = -1;
    pid[j] = (P >= 0 && pmask_k[P] != 0) ? P : -1;
  }
  __syncthreads();
  const double isq = 1.0 / sqrt((double)__popc(mi & 255u));
  double rz = 0, bb = 0;
  for (int e = tid; e < NV; e += blockDim.x) {
    const int j = e >> 3, t = e & 7;
    double b = 0.0;
    const int P = pid[j];
    if (t < 7 && P >= 0) {
      const int o = g.pair_idx[j * NB + g.jc];
      if (o >= 0 && inb(4, o, g.noff)) b = -Ahat[((int64_t)o * npar + P) * 64 + t * 8 + 7] * isq;
    }
    x[e] = 0.0;
    r[e] = b;
  }
  __syncthreads();
  for (int e = tid; e < NV; e += blockDim.x) {
    const int j = e >> 3, t = e & 7;
    const int P = pid[j];
    double v = 0.0;
    if (t < 7 && P >= 0) {
      const double* D = Dinv + (int64_t)P * 64 + t * 8;
      const double* rr = r + j * 8;
#pragma unroll
      for (int u = 0; u < 7; ++u) v += D[u] * rr[u];
    }
    z[e] = v;
    p[e] = v;
    rz += r[e] * v;
    bb += r[e] * r[e];
  }
  cta_sum2(rz, bb, red);
  double rr = bb;
  const double stop = tol * tol * bb;
  int it = 0;
  while (it < max_iter && rr > stop) {
    // q = B p
    for (int e = tid; e < NV; e += blockDim.x) {
      const int j = e >> 3, t = e & 7;
      const int P = pid[j];
      double acc = 0.0;
      if (t < 7 && P >= 0) {
        const int* prow = g.pair_idx + j * NB;
        for (int jb = 0; jb < NB; ++jb) {
          const int o = prow[jb];
          if (o < 0 || pid[jb] < 0 || !inb(5, o, g.noff)) continue;
          const double2* ar =
              reinterpret_cast<const double2*>(Ahat + ((int64_t)o * npar + P) * 64 + t * 8);
          const double* pb = p + jb * 8;
          const double2 a0 = ar[0], a1 = ar[1], a2 = ar[2], a3 = ar[3];
          acc += a0.x * pb[0] + a0.y * pb[1] + a1.x * pb[2] + a1.y * pb[3] + a2.x * pb[4] +
                 a2.y * pb[5] + a3.x * pb[6];
        }
      }
      q[e] = acc;
    }
    __syncthreads();
    double pq = 0.0;
    for (int e = tid; e < NV; e += blockDim.x) pq += p[e] * q[e];
    pq = cta_sum(pq, red);
    if (!(pq > 0.0)) break;
    const double alpha = rz / pq;
    for (int e = tid; e < NV; e += blockDim.x) {
      x[e] += alpha * p[e];
      r[e] -= alpha * q[e];
    }
    __syncthreads();
    double rzn = 0.0, rrn = 0.0;
    for (int e = tid; e < NV; e += blockDim.x) {
      const int j = e >> 3, t = e & 7;
      const int P = pid[j];
      double v = 0.0;
      if (t < 7 && P >= 0) {
        const double* D = Dinv + (int64_t)P * 64 + t * 8;
        const double* rv = r + j * 8;
#pragma unroll
        for (int u = 0; u < 7; ++u) v += D[u] * rv[u];
      }
      z[e] = v;
      rzn += r[e] * v;
      rrn += r[e] * r[e];
    }
    cta_sum2(rzn, rrn, red);
    const double beta = rzn / rz;
    rz = rzn;
    rr = rrn;
    for (int e = tid; e < NV; e += blockDim.x) p[e] = z[e] + beta * p[e];
    __syncthreads();
    ++it;
  }
  for (int e = tid; e < NV; e += blockDim.x) {
    const int j = e >> 3, t = e & 7;
    Ri[e] = (t < 7) ? x[e] : (j == g.jc ? isq : 0.0);
  }
  if (tid == 0) {
    atomicMax(iter_stats, it);
    atomicAdd(iter_stats + 1, it);
    atomicAdd(iter_stats + 2, 1);
  }
}

void launch_patch_cg3(const double* Ahat, const double* Dinv, const uint32_t* pmask_k,
                      Patch3Geom g, double tol, int max_iter, double* Rhat, int* iter_stats,
                      cudaStream_t s) {
  if (g.npatch <= 0) return;
  const size_t smem = patch_cg3_smem(g.NB);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_patch_cg3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch();
  k_patch_cg3<<<(unsigned)g.npatch, kThreads, smem, s>>>(Ahat, Dinv, pmask_k, g, tol, max_iter,
                                                         Rhat, iter_stats);
}

// ---------------------------------------------------------------- Galerkin product
// One CTA per coarse cell i.  Phase 1: T = R_i A^(k) on the dilated parents
// P_i + D_d, T[d][c] = sum over (j, o) with N_j + O_o = D_d of
// sum_a Rhat_i[j][a] Ahat(o, P_i + N_j)[a][c].  Phase 2: for each output
// offset e with i' = i + E_e active, A^(k-1)_(i, i') = sum over (j', d) with
// E_e + N_j' = D_d of T[d] . Rhat_i'[j'] (eight lanes per output).
size_t galerkin3_smem(int NB, int nD) {
  return (size_t)NB * 8 * sizeof(double) + (size_t)nD * 8 * sizeof(double) +
         (size_t)NB * sizeof(int);
}

__global__ void __launch_bounds__(kThreads)
    k_galerkin3(const double* __restrict__ Ahat, const double* __restrict__ Rhat,
                const uint32_t* __restrict__ pmask_k, Galerkin3Geom g, double* out) {
  extern __shared__ double sm[];
  const int NB = g.NB;
  double* Ri = sm;
  double* T = Ri + NB * 8;
  int* pid = reinterpret_cast<int*>(T + g.nD * 8);
  const int64_t i = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t npar = g.npatch;
  if (pmask_k[i] == 0) return;
  int cx, cy, cz;
  demorton3((uint32_t)i, cx, cy, cz);
  for (int e = tid; e < NB * 8; e += blockDim.x) Ri[e] = Rhat[i * NB * 8 + e];
  for (int j = tid; j < NB; j += blockDim.x) {
    const int4 o = g.nbr[j];
    int P = shift3(cx, cy, cz, o.x, o.y, o.z, g.Lpar);
    if (P >= 0 && !inb(6, P, npar)) P = -1;
    pid[j] = (P >= 0 && pmask_k[P] != 0) ? P : -1;
  }
  __syncthreads();
  for (int e = tid; e < g.nD * 8; e += blockDim.x) {
    const int d = e >> 3, c = e & 7;
    double acc = 0.0;
    for (int l = g.l1_ptr[d]; l < g.l1_ptr[d + 1]; ++l) {
      const int2 jo = g.l1[l];
      if (!inb(7, jo.x, NB) || !inb(8, jo.y, g.noff)) continue;
      const int P = pid[jo.x];
      if (P < 0) continue;
      const double* blk = Ahat + ((int64_t)jo.y * npar + P) * 64 + c;
      const double* rj = Ri + jo.x * 8;
#pragma unroll
      for (int a = 0; a < 8; ++a) acc += rj[a] * blk[a * 8];
    }
    T[e] = acc;
  }
  __syncthreads();
  // one group of eight lanes per output (lane c = slot c of the dot
  // products), so the final sum over the slots is three shuffle steps
  const int grp = tid >> 3, c = tid & 7, ngrp = blockDim.x >> 3;
  // level k-1 node i and its parent (a level k-2 cell)
  const int Lout = g.Lpar >> 1;
  int px, py, pz;
  demorton3((uint32_t)(i >> 3), px, py, pz);
  const int nrounds = (g.nE + ngrp - 1) / ngrp;  // every lane runs the same rounds
  for (int rnd = 0; rnd < nrounds; ++rnd) {
    const int e = rnd * ngrp + grp;
    int ip = -1;
    if (e < g.nE) {
      const int4 E = g.E[e];
      ip = shift3(cx, cy, cz, E.x, E.y, E.z, g.Lpar);
      if (ip >= 0 && !inb(9, ip, npar)) ip = -1;
      if (ip >= 0 && pmask_k[ip] == 0) ip = -1;
    }
    double acc = 0.0;
    if (ip >= 0) {
      const double* Rp = Rhat + (int64_t)ip * NB * 8 + c;
      for (int l = g.l2_ptr[e]; l < g.l2_ptr[e + 1]; ++l) {
        const int2 jd = g.l2[l];
        if (!inb(10, jd.y, g.nD) || !inb(11, jd.x, NB)) continue;
        acc += T[jd.y * 8 + c] * Rp[jd.x * 8];
      }
    }
    acc = group8_sum(acc);
    if (ip >= 0 && c == 0) {
      int qx, qy, qz;
      demorton3((uint32_t)ip >> 3, qx, qy, qz);
      const int o = g.out_lk.find(qx - px, qy - py, qz - pz);
      if (o >= 0 && Lout >= 1 && inb(12, o, g.noff_out) && inb(13, i >> 3, g.npar_out))
        out[((int64_t)o * g.npar_out + (i >> 3)) * 64 + (i & 7) * 8 + (ip & 7)] = acc;
    }
  }
}

void launch_galerkin3(const double* Ahat, const double* Rhat, const uint32_t* pmask_k,
                      Galerkin3Geom g, double* out, cudaStream_t s) {
  if (g.npatch <= 0) return;
  const size_t smem = galerkin3_smem(g.NB, g.nD);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(k_galerkin3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch();
  k_galerkin3<<<(unsigned)g.npatch, kThreads, smem, s>>>(Ahat, Rhat, pmask_k, g, out);
}

// ---------------------------------------------------------------- vectors
__global__ void k_transform_vec3(const double* __restrict__ in, double* out, int64_t npar,
                                 const uint32_t* __restrict__ pmask,
                                 const double* __restrict__ qtab, int dir) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t P = gid >> 3;
  const int a = (int)(gid & 7);
  const bool live = P < npar;
  const double v = live ? in[gid] : 0.0;
  const double* Q = qtab + (int64_t)(live ? pmask[P] : 0) * 64;
  const int base = threadIdx.x & ~7;
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const double vb = __shfl_sync(0xffffffffu, v, (base + b) & 31);
    s += (dir > 0 ? Q[a * 8 + b] : Q[b * 8 + a]) * vb;
  }
  if (live) out[gid] = s;
}

void launch_transform_vec3(const double* in, double* out, int64_t npar, const uint32_t* pmask,
                           int dir, const double* qtab, cudaStream_t s) {
  const int64_t threads = npar * 8;
  if (threads <= 0) return;
  count_launch();
  k_transform_vec3<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      in, out, npar, pmask, qtab, dir);
}

// eight lanes per coarse cell, lane c = slot c
__global__ void k_restrict3(const double* __restrict__ Rhat, const double* __restrict__ ghat,
                            const uint32_t* __restrict__ pmask_k, Patch3Geom g, double* gc) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid >> 3;
  const int c = (int)(gid & 7);
  const bool live = i < g.npatch && pmask_k[i] != 0;
  double acc = 0.0;
  if (live) {
    int cx, cy, cz;
    demorton3((uint32_t)i, cx, cy, cz);
    const double* Ri = Rhat + i * (int64_t)g.NB * 8 + c;
    for (int j = 0; j < g.NB; ++j) {
      const int4 o = g.nbr[j];
      const int P = shift3(cx, cy, cz, o.x, o.y, o.z, g.Lpar);
      if (P < 0) continue;
      acc += Ri[j * 8] * ghat[(int64_t)P * 8 + c];
    }
  }
  acc = group8_sum(acc);
  if (i < g.npatch && c == 0) gc[i] = live ? acc : 0.0;
}

void launch_restrict3(const double* Rhat, const double* ghat, const uint32_t* pmask_k,
                      Patch3Geom g, double* gc, cudaStream_t s) {
  const int64_t threads = g.npatch * 8;
  if (threads <= 0) return;
  count_launch();
  k_restrict3<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, s>>>(Rhat, ghat,
                                                                                   pmask_k, g, gc);
}

// eight lanes per parent P of level k, lane c = slot c of v_hat, then
// v = Q^T v_hat through the group
__global__ void k_prolong3(const double* __restrict__ Rhat, const double* __restrict__ vc,
                           const double* __restrict__ w, const uint32_t* __restrict__ pmask_k,
                           Patch3Geom g, const double* __restrict__ qtab, double* v) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t P = gid >> 3;
  const int c = (int)(gid & 7);
  const bool live = P < g.npatch && pmask_k[P] != 0;
  double vh = 0.0;
  if (live) {
    if (w && c < 7) vh = w[P * 8 + c];
    if (vc) {
      int x, y, z;
      demorton3((uint32_t)P, x, y, z);
      for (int j = 0; j < g.NB; ++j) {
        const int4 o = g.nbr[j];
        const int i = shift3(x, y, z, -o.x, -o.y, -o.z, g.Lpar);
        if (i < 0 || pmask_k[i] == 0) continue;
        vh += Rhat[((int64_t)i * g.NB + j) * 8 + c] * vc[i];
      }
    }
  }
  const double* Q = qtab + (int64_t)(live ? pmask_k[P] : 0) * 64;
  const int base = threadIdx.x & ~7;
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 8; ++b) s += Q[b * 8 + c] * __shfl_sync(0xffffffffu, vh, (base + b) & 31);
  if (P < g.npatch) v[gid] = live ? s : 0.0;
}

void launch_prolong3(const double* Rhat, const double* v_coarse, const double* w,
                     const uint32_t* pmask_k, Patch3Geom g, const double* qtab, double* v,
                     cudaStream_t s) {
  const int64_t threads = g.npatch * 8;
  if (threads <= 0) return;
  count_launch();
  k_prolong3<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      Rhat, v_coarse, w, pmask_k, g, qtab, v);
}

// ---------------------------------------------------------------- level CG
// Rows (P, t) of every level in groups of eight lanes, 32 parents per CTA;
// a CTA belongs to one level (the level's CTAs are [blk0, blk0 + nblk)).
namespace {
__device__ __forceinline__ int find_level(const Lcg3Level* lv, int nlev, int b) {
  for (int l = 0; l < nlev; ++l)
    if (b >= lv[l].blk0 && b < lv[l].blk0 + lv[l].nblk) return l;
  return -1;
}
// z = Dinv r for the parent of this group (lane t holds r_t)
__device__ __forceinline__ double precond8(const double* __restrict__ Dinv, int64_t P, int t,
                                           double rt) {
  const int base = threadIdx.x & ~7;
  const double* D = Dinv + P * 64 + t * 8;
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 7; ++u) s += D[u] * __shfl_sync(0xffffffffu, rt, (base + u) & 31);
  return t < 7 ? s : 0.0;
}
}  // namespace

__global__ void k_lcg3_start(const Lcg3Level* __restrict__ lv, int nlev,
                             const double* __restrict__ b, double* x, double* r, double* z,
                             double* p, double* part) {
  __shared__ double red[kRed];
  const int l = find_level(lv, nlev, blockIdx.x);
  const Lcg3Level L = lv[max(l, 0)];
  const int64_t P = (int64_t)(blockIdx.x - L.blk0) * (kThreads / 8) + (threadIdx.x >> 3);
  const int t = threadIdx.x & 7;
  const bool live = l >= 0 && P < L.npar;
  const int64_t e = L.v0 + P * 8 + t;
  const double rt = (live && t < 7) ? b[e] : 0.0;
  const double zt = precond8(L.Dinv, live ? P : 0, t, rt);
  if (live) {
    x[e] = 0.0;
    r[e] = rt;
    z[e] = zt;
    p[e] = zt;
  }
  double rz = rt * zt, bb = rt * rt;
  cta_sum2(rz, bb, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 0] = rz;
    part[blockIdx.x * 3 + 1] = bb;
  }
}

// one CTA per level: sum the level's partials (fixed order)
__device__ __forceinline__ double level_sum(const Lcg3Level& L, const double* part, int slot,
                                            double* red) {
  double s = 0.0;
  for (int b = threadIdx.x; b < L.nblk; b += blockDim.x) s += part[(L.blk0 + b) * 3 + slot];
  return cta_sum(s, red);
}

__global__ void k_lcg3_init_scalars(const Lcg3Level* __restrict__ lv, const double* part,
                                    Lcg3Scalars* sc, double tol) {
  __shared__ double red[kRed];
  const Lcg3Level L = lv[blockIdx.x];
  const double rz = level_sum(L, part, 0, red);
  const double bb = level_sum(L, part, 1, red);
  if (threadIdx.x == 0) {
    Lcg3Scalars s{};
    s.rz = rz;
    s.bb = bb;
    s.active = bb > 0.0 ? 1 : 0;
    s.iters = 0;
    (void)tol;
    sc[blockIdx.x] = s;
  }
}

__global__ void k_lcg3_spmv(const Lcg3Level* __restrict__ lv, int nlev,
                            const Lcg3Scalars* __restrict__ sc, const double* __restrict__ p,
                            double* Ap, double* part) {
  __shared__ double red[kRed];
  const int l = find_level(lv, nlev, blockIdx.x);
  if (l < 0 || sc[l].active != 1) return;
  const Lcg3Level L = lv[l];
  const int64_t P = (int64_t)(blockIdx.x - L.blk0) * (kThreads / 8) + (threadIdx.x >> 3);
  const int t = threadIdx.x & 7;
  const bool live = P < L.npar;
  double acc = 0.0;
  if (live && t < 7) {
    int x, y, z;
    demorton3((uint32_t)P, x, y, z);
    for (int o = 0; o < L.noff; ++o) {
      const int4 d = L.off[o];
      const int Pn = shift3(x, y, z, d.x, d.y, d.z, L.Lpar);
      if (Pn < 0) continue;
      const double2* ar = reinterpret_cast<const double2*>(L.A + ((int64_t)o * L.npar + P) * 64 + t * 8);
      const double* pb = p + L.v0 + (int64_t)Pn * 8;
      const double2 a0 = ar[0], a1 = ar[1], a2 = ar[2], a3 = ar[3];
      acc += a0.x * pb[0] + a0.y * pb[1] + a1.x * pb[2] + a1.y * pb[3] + a2.x * pb[4] +
             a2.y * pb[5] + a3.x * pb[6];
    }
  }
  const int64_t e = L.v0 + P * 8 + t;
  if (live) Ap[e] = acc;
  double pq = live ? p[e] * acc : 0.0;
  pq = cta_sum(pq, red);
  if (threadIdx.x == 0) part[blockIdx.x * 3 + 0] = pq;
}

__global__ void k_lcg3_alpha(const Lcg3Level* __restrict__ lv, const double* part,
                             Lcg3Scalars* sc) {
  __shared__ double red[kRed];
  const Lcg3Level L = lv[blockIdx.x];
  if (sc[blockIdx.x].active != 1) return;
  const double pq = level_sum(L, part, 0, red);
  if (threadIdx.x == 0) {
    Lcg3Scalars& s = sc[blockIdx.x];
    if (pq > 0.0) {
      s.alpha = s.rz / pq;
    } else {
      s.alpha = 0.0;
      s.active = 0;
    }
  }
}

__global__ void k_lcg3_update(const Lcg3Level* __restrict__ lv, int nlev,
                              const Lcg3Scalars* __restrict__ sc, const double* __restrict__ p,
                              const double* __restrict__ Ap, double* x, double* r, double* z,
                              double* part) {
  __shared__ double red[kRed];
  const int l = find_level(lv, nlev, blockIdx.x);
  if (l < 0 || sc[l].active != 1) return;
  const Lcg3Level L = lv[l];
  const double alpha = sc[l].alpha;
  const int64_t P = (int64_t)(blockIdx.x - L.blk0) * (kThreads / 8) + (threadIdx.x >> 3);
  const int t = threadIdx.x & 7;
  const bool live = P < L.npar;
  const int64_t e = L.v0 + P * 8 + t;
  double rt = 0.0;
  if (live) {
    x[e] += alpha * p[e];
    rt = r[e] - alpha * Ap[e];
    r[e] = rt;
  }
  const double zt = precond8(L.Dinv, live ? P : 0, t, rt);
  if (live) z[e] = zt;
  double rz = rt * zt, rr = rt * rt;
  cta_sum2(rz, rr, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x * 3 + 1] = rz;
    part[blockIdx.x * 3 + 2] = rr;
  }
}

__global__ void k_lcg3_beta(const Lcg3Level* __restrict__ lv, const double* part,
                            Lcg3Scalars* sc, double tol, int max_iter) {
  __shared__ double red[kRed];
  const Lcg3Level L = lv[blockIdx.x];
  if (sc[blockIdx.x].active != 1) return;
  const double rz = level_sum(L, part, 1, red);
  const double rr = level_sum(L, part, 2, red);
  if (threadIdx.x == 0) {
    Lcg3Scalars& s = sc[blockIdx.x];
    s.beta = rz / s.rz;
    s.rz = rz;
    s.iters += 1;
    if (rr <= tol * tol * s.bb) s.active = 0;
    else if (s.iters >= max_iter) s.active = -1;  // capped, not converged
  }
}

__global__ void k_lcg3_direction(const Lcg3Level* __restrict__ lv, int nlev,
                                 const Lcg3Scalars* __restrict__ sc, const double* __restrict__ z,
                                 double* p) {
  const int l = find_level(lv, nlev, blockIdx.x);
  if (l < 0 || sc[l].active != 1) return;
  const Lcg3Level L = lv[l];
  const double beta = sc[l].beta;
  const int64_t P = (int64_t)(blockIdx.x - L.blk0) * (kThreads / 8) + (threadIdx.x >> 3);
  if (P >= L.npar) return;
  const int64_t e = L.v0 + P * 8 + (threadIdx.x & 7);
  p[e] = z[e] + beta * p[e];
}

void launch_lcg3_start(const Lcg3Level* lv, int nlev, int nblk, const double* b, double* x,
                       double* r, double* z, double* p, double* part, cudaStream_t s) {
  count_launch();
  k_lcg3_start<<<nblk, kThreads, 0, s>>>(lv, nlev, b, x, r, z, p, part);
}
void launch_lcg3_init_scalars(const Lcg3Level* lv, int nlev, const double* part,
                              Lcg3Scalars* sc, double tol, cudaStream_t s) {
  count_launch();
  k_lcg3_init_scalars<<<nlev, kThreads, 0, s>>>(lv, part, sc, tol);
}
void launch_lcg3_spmv(const Lcg3Level* lv, int nlev, int nblk, const Lcg3Scalars* sc,
                      const double* p, double* Ap, double* part, cudaStream_t s) {
  count_launch();
  k_lcg3_spmv<<<nblk, kThreads, 0, s>>>(lv, nlev, sc, p, Ap, part);
}
void launch_lcg3_alpha(const Lcg3Level* lv, int nlev, const double* part, Lcg3Scalars* sc,
                       cudaStream_t s) {
  count_launch();
  k_lcg3_alpha<<<nlev, kThreads, 0, s>>>(lv, part, sc);
}
void launch_lcg3_update(const Lcg3Level* lv, int nlev, int nblk, const Lcg3Scalars* sc,
                        const double* p, const double* Ap, double* x, double* r, double* z,
                        double* part, cudaStream_t s) {
  count_launch();
  k_lcg3_update<<<nblk, kThreads, 0, s>>>(lv, nlev, sc, p, Ap, x, r, z, part);
}
void launch_lcg3_beta(const Lcg3Level* lv, int nlev, const double* part, Lcg3Scalars* sc,
                      double tol, int max_iter, cudaStream_t s) {
  count_launch();
  k_lcg3_beta<<<nlev, kThreads, 0, s>>>(lv, part, sc, tol, max_iter);
}
void launch_lcg3_direction(const Lcg3Level* lv, int nlev, int nblk, const Lcg3Scalars* sc,
                           const double* z, double* p, cudaStream_t s) {
  count_launch();
  k_lcg3_direction<<<nblk, kThreads, 0, s>>>(lv, nlev, sc, z, p);
}

// ---------------------------------------------------------------- coarsest level
// Dense Cholesky of the active part (details 0..m-2 and slot 7) of the one
// level-1 block, one thread.
__global__ void k_coarsest3(const double* __restrict__ A1, uint32_t mask,
                            const double* __restrict__ g1, const double* __restrict__ qtab,
                            double* U1, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int cnt = __popc(mask & 255u);
  int idx[8];
  int n = 0;
  for (int a = 0; a < cnt - 1; ++a) idx[n++] = a;
  if (cnt > 0) idx[n++] = 7;
  const double* Q = qtab + (int64_t)mask * 64;
  double gh[8];
  for (int a = 0; a < 8; ++a) {
    double s = 0.0;
    for (int c = 0; c < 8; ++c) s += Q[a * 8 + c] * g1[c];
    gh[a] = s;
  }
  double L[8][8];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) L[i][j] = A1[idx[i] * 8 + idx[j]];
  for (int j = 0; j < n; ++j) {
    double d = L[j][j];
    for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
    if (!(d > 0.0)) {
      atomicExch(status, (int)DEV_NOT_SPD);
      for (int c = 0; c < 8; ++c) U1[c] = 0.0;
      return;
    }
    d = sqrt(d);
    L[j][j] = d;
    for (int i = j + 1; i < n; ++i) {
      double v = L[i][j];
      for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
      L[i][j] = v / d;
    }
  }
  double y[8];
  for (int i = 0; i < n; ++i) {
    double v = gh[idx[i]];
    for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
    y[i] = v / L[i][i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double v = y[i];
    for (int k = i + 1; k < n; ++k) v -= L[k][i] * y[k];
    y[i] = v / L[i][i];
  }
  double uh[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int i = 0; i < n; ++i) uh[idx[i]] = y[i];
  for (int c = 0; c < 8; ++c) {
    double s = 0.0;
    for (int a = 0; a < 8; ++a) s += Q[a * 8 + c] * uh[a];
    U1[c] = s;
  }
}

void launch_coarsest3(const double* A1hat, uint32_t mask, const double* g1, const double* qtab,
                      double* U1, int* status, cudaStream_t s) {
  count_launch();
  k_coarsest3<<<1, 32, 0, s>>>(A1hat, mask, g1, qtab, U1, status);
}

// ---------------------------------------------------------------- fine level
__global__ void k_gather3(const double* __restrict__ in, const int32_t* __restrict__ unknown_of,
                          int64_t ncell, double* out) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ncell) return;
  const int u = unknown_of[m];
  out[m] = u >= 0 ? in[u] : 0.0;
}
__global__ void k_scatter_unknown3(const double* __restrict__ in_m,
                                   const int32_t* __restrict__ morton_of, int n, double* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = in_m[morton_of[i]];
}
void launch_gather3(const double* in, const int32_t* unknown_of, int64_t ncell, double* out,
                    cudaStream_t s) {
  if (ncell <= 0) return;
  count_launch();
  k_gather3<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(in, unknown_of, ncell, out);
}
void launch_scatter_unknown3(const double* in_m, const int32_t* morton_of, int n, double* out,
                             cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_scatter_unknown3<<<(n + 255) / 256, 256, 0, s>>>(in_m, morton_of, n, out);
}

// eight lanes per row
__global__ void k_csr_spmv3(int n, const int32_t* __restrict__ rowptr,
                            const int32_t* __restrict__ colind, const double* __restrict__ val,
                            const double* __restrict__ x, double* y) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = gid >> 3;
  const int lane = (int)(gid & 7);
  double acc = 0.0;
  if (i < n)
    for (int t = rowptr[i] + lane; t < rowptr[i + 1]; t += 8) acc += val[t] * x[colind[t]];
  acc = group8_sum(acc);
  if (i < n && lane == 0) y[i] = acc;
}
void launch_csr_spmv3(int n, const int32_t* rowptr, const int32_t* colind, const double* val,
                      const double* x, double* y, cudaStream_t s) {
  const int64_t threads = (int64_t)n * 8;
  if (threads <= 0) return;
  count_launch();
  k_csr_spmv3<<<(unsigned)((threads + kThreads - 1) / kThreads), kThreads, 0, s>>>(
      n, rowptr, colind, val, x, y);
}

int dot3_blocks(int64_t n) {
  const int64_t b = (n + kThreads - 1) / kThreads;
  return (int)std::min<int64_t>(std::max<int64_t>(b, 1), 1024);
}
__global__ void k_dot3(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                       const double* __restrict__ w, double* part) {
  __shared__ double red[kRed];
  double a = 0.0, b = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    a += x[i] * y[i];
    if (w) b += x[i] * w[i];
  }
  cta_sum2(a, b, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = a;
    part[gridDim.x + blockIdx.x] = b;
  }
}
__global__ void k_dot3_finish(const double* __restrict__ part, int nb, int nout, double* out) {
  __shared__ double red[kRed];
  for (int o = 0; o < nout; ++o) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[o * nb + b];
    s = cta_sum(s, red);
    if (threadIdx.x == 0) out[o] = s;
  }
}
void launch_dot3(int64_t n, const double* x, const double* y, const double* w, double* part,
                 cudaStream_t s) {
  count_launch();
  k_dot3<<<dot3_blocks(n), kThreads, 0, s>>>(n, x, y, w, part);
}
void launch_dot3_finish(const double* part, int nb, int nout, double* out, cudaStream_t s) {
  count_launch();
  k_dot3_finish<<<1, kThreads, 0, s>>>(part, nb, nout, out);
}

__global__ void k_axpby3(int64_t n, double a, const double* __restrict__ x, double b, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i] + b * y[i];
}
void launch_axpby3(int64_t n, double a, const double* x, double b, double* y, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_axpby3<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, b, y);
}

}  // namespace d3
}  // namespace gb
