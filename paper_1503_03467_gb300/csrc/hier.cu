// hier.cu - measurement hierarchy, fine-operator import and per-parent
// Helmert transforms.
//
// Sec. 4.1 (Definition defindextree, Construction defmulires): the level-k
// subdomain of a fine unknown is its level-q cell shifted by q-k bits; with
// Morton indexing the parent of cell s is s >> 2 and pi^(k-1,k) needs no
// storage.  Sec. 4.6 (Lemma const0, Construction const2): W^(k) is built
// from the orthonormal Helmert rows of each parent, applied through the
// per-parent transform evaluated by qmat (common.cuh).
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

// ---------------------------------------------------------------- hierarchy
// Morton code of every unknown's level-q cell; flag[0] = 2 for a cell
// outside the lattice, flag[1] = largest code (sizes the stored prefix).
__global__ void k_cells_to_morton(const int32_t* __restrict__ cells, int n, int q,
                                  int32_t* morton_of, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int x = cells[2 * i], y = cells[2 * i + 1];
  int L = 1 << q;
  if ((unsigned)x >= (unsigned)L || (unsigned)y >= (unsigned)L) {
    atomicExch(flag, 2);
    morton_of[i] = 0;
    return;
  }
  uint32_t s = morton((uint32_t)x, (uint32_t)y);
  morton_of[i] = (int32_t)s;
  atomicMax(flag + 1, (int)s);
}

// unknown_of (cell -> unknown) and the level-q child masks; flag[0] = 1 when
// two unknowns share a cell.
__global__ void k_scatter_cells(const int32_t* __restrict__ morton_of, int n,
                                int32_t* unknown_of, uint32_t* pmask_q, int* flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t s = (uint32_t)morton_of[i];
  int old = atomicExch(&unknown_of[s], i);
  if (old != -1) atomicExch(flag, 1);
  atomicOr(&pmask_q[s >> 2], 1u << (s & 3));
}

void launch_cells_to_morton(const int32_t* cells, int n, int q, int32_t* morton_of, int* flag,
                            cudaStream_t s) {
  if (n <= 0) return;
  { count_launch(); k_cells_to_morton<<<(n + 255) / 256, 256, 0, s>>>(cells, n, q, morton_of, flag); }
}
void launch_scatter_cells(const int32_t* morton_of, int n, int32_t* unknown_of,
                          uint32_t* pmask_q, int* flag, cudaStream_t s) {
  if (n <= 0) return;
  { count_launch(); k_scatter_cells<<<(n + 255) / 256, 256, 0, s>>>(morton_of, n, unknown_of, pmask_q, flag); }
}

// Parent P of level k-1 has child c active iff level-k parent 4P + c exists
// (4P + c < npar_k) and has any active child.
__global__ void k_coarsen_masks(const uint32_t* __restrict__ pmask_k, int64_t npar_k,
                                int64_t npar_km1, uint32_t* pmask_km1) {
  int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (P >= npar_km1) return;
  uint32_t m = 0;
  for (int c = 0; c < 4; ++c)
    if (4 * P + c < npar_k && pmask_k[4 * P + c]) m |= 1u << c;
  pmask_km1[P] = m;
}

void launch_coarsen_masks(const uint32_t* pmask_k, int64_t npar_k, uint32_t* pmask_km1,
                          int64_t npar_km1, cudaStream_t s) {
  if (npar_km1 <= 0) return;
  { count_launch(); k_coarsen_masks<<<(unsigned)((npar_km1 + 255) / 256), 256, 0, s>>>(pmask_k, npar_k, npar_km1, pmask_km1); }
}

// ---------------------------------------------------------------- batched problems
// Problem owning combined row i (or entry t): the last segment starting at
// or before it (segments are in row order).
__device__ __forceinline__ int find_seg_row(const BatchSeg* seg, int nprob, int64_t i) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg[mid].row0 <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
__device__ __forceinline__ int find_seg_nnz(const BatchSeg* seg, int nprob, int64_t t) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (seg[mid].nnz0 <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void k_batch_rows(int nprob, const BatchSeg* __restrict__ seg, int64_t n,
                             int32_t* rowptr, int32_t* cells, int* flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BatchSeg b = seg[find_seg_row(seg, nprob, i)];
  rowptr[i] += (int32_t)b.nnz0;
  const int x = cells[2 * i], y = cells[2 * i + 1], L = 1 << b.q;
  if ((unsigned)x >= (unsigned)L || (unsigned)y >= (unsigned)L) {
    atomicExch(flag, 2);
    cells[2 * i] = b.x0;  // any cell of the problem; the setup fails on the flag
    cells[2 * i + 1] = b.y0;
    return;
  }
  cells[2 * i] = x + b.x0;
  cells[2 * i + 1] = y + b.y0;
}

__global__ void k_batch_cols(int nprob, const BatchSeg* __restrict__ seg, int64_t nnz,
                             int32_t* colind, int* flag) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nnz) return;
  const BatchSeg b = seg[find_seg_nnz(seg, nprob, t)];
  const int c = colind[t];
  if ((unsigned)c >= (unsigned)b.n) {
    atomicExch(flag, 1);
    colind[t] = (int32_t)b.row0;
    return;
  }
  colind[t] = c + (int32_t)b.row0;
}

void launch_batch_fixup(int nprob, const BatchSeg* seg, int64_t n, int64_t nnz, int32_t* rowptr,
                        int32_t* colind, int32_t* cells, int* flag, cudaStream_t s) {
  if (n > 0) { count_launch(); k_batch_rows<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(nprob, seg, n, rowptr, cells, flag); }
  if (nnz > 0) { count_launch(); k_batch_cols<<<(unsigned)((nnz + 255) / 256), 256, 0, s>>>(nprob, seg, nnz, colind, flag); }
}

// ---------------------------------------------------------------- fine operator
__global__ void k_csr_extent(int n, const int32_t* __restrict__ rowptr,
                             const int32_t* __restrict__ colind,
                             const int32_t* __restrict__ morton_of, int* ext, int* bad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int si = morton_of[i];
  int xi, yi;
  demorton((uint32_t)si >> 2, xi, yi);
  int mx = 0, my = 0;
  int b = rowptr[i], e = rowptr[i + 1];
  if (e < b) {
    atomicExch(bad, 1);
    return;
  }
  for (int t = b; t < e; ++t) {
    int j = colind[t];
    if ((unsigned)j >= (unsigned)n) {
      atomicExch(bad, 1);
      continue;
    }
    int xj, yj;
    demorton((uint32_t)morton_of[j] >> 2, xj, yj);
    mx = max(mx, abs(xj - xi));
    my = max(my, abs(yj - yi));
  }
  atomicMax(&ext[0], mx);
  atomicMax(&ext[1], my);
}

void launch_csr_offset_extent(int n, const int32_t* rowptr, const int32_t* colind,
                              const int32_t* morton_of, int* ext, int* bad_flag,
                              cudaStream_t s) {
  if (n <= 0) return;
  { count_launch(); k_csr_extent<<<(n + 127) / 128, 128, 0, s>>>(n, rowptr, colind, morton_of, ext, bad_flag); }
}

__global__ void k_csr_to_blocks(int n, const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colind,
                                const double* __restrict__ val,
                                const int32_t* __restrict__ morton_of, int rx, int ry,
                                int64_t npar, double* blk) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t si = (uint32_t)morton_of[i];
  int xi, yi;
  demorton(si >> 2, xi, yi);
  int a = si & 3;
  for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    int j = colind[t];
    if ((unsigned)j >= (unsigned)n) continue;
    uint32_t sj = (uint32_t)morton_of[j];
    int xj, yj;
    demorton(sj >> 2, xj, yj);
    int o = (yj - yi + ry) * (2 * rx + 1) + (xj - xi + rx);
    atomicAdd(&blk[((int64_t)o * npar + (si >> 2)) * 16 + a * 4 + (sj & 3)], val[t]);
  }
}

void launch_csr_to_blocks(int n, const int32_t* rowptr, const int32_t* colind,
                          const double* val, const int32_t* morton_of, int rx, int ry,
                          int64_t npar, double* blk, cudaStream_t s) {
  if (n <= 0) return;
  { count_launch(); k_csr_to_blocks<<<(n + 127) / 128, 128, 0, s>>>(n, rowptr, colind, val, morton_of, rx, ry,
                                                  npar, blk); }
}

// ---------------------------------------------------------------- transforms
__global__ void k_transform_blocks(double* blk, const int2* __restrict__ off, int noff,
                                   int64_t npar, int Lpar, const uint32_t* __restrict__ pmask) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  int o = (int)(t / npar);
  int64_t p = t - (int64_t)o * npar;
  double* B = blk + t * 16;
  int x, y;
  demorton((uint32_t)p, x, y);
  int pp = shift_cell(x, y, off[o].x, off[o].y, Lpar, npar);
  int mr = (int)pmask[p] & 15;
  int mc = pp >= 0 ? (int)pmask[pp] & 15 : 0;
  double M[16], Tm[16], Qr[16], Qc[16];
  qmat<double>(mr, Qr);
  qmat<double>(mc, Qc);
#pragma unroll
  for (int e = 0; e < 16; ++e) M[e] = B[e];
  // Tm = Q_r M
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      double acc = 0;
#pragma unroll
      for (int r = 0; r < 4; ++r) acc += Qr[a * 4 + r] * M[r * 4 + c];
      Tm[a * 4 + c] = acc;
    }
  // B = Tm Q_c^T
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double acc = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc += Tm[a * 4 + c] * Qc[b * 4 + c];
      B[a * 4 + b] = acc;
    }
}

void launch_transform_blocks(double* blk, const int2* off, int noff, int64_t npar, int Lpar,
                             const uint32_t* pmask, cudaStream_t s) {
  int64_t n = (int64_t)noff * npar;
  if (n <= 0) return;
  { count_launch(); k_transform_blocks<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blk, off, noff, npar, Lpar,
                                                                pmask); }
}

// Fine CSR -> node stencil in Morton order: St[s][c] = A_{i, j} with c the
// level-q cell of unknown i and c + S_s that of j (S: the (2 rx + 1) x
// (2 ry + 1) box, row-major in (dy, dx)); cells without an unknown stay 0.
// St must be zeroed; each (s, c) is written by the thread of its row only.
__global__ void k_csr_to_mstencil(int n, const int32_t* __restrict__ rowptr,
                                  const int32_t* __restrict__ colind,
                                  const double* __restrict__ val,
                                  const int32_t* __restrict__ morton_of, int rx, int ry,
                                  int64_t ncell, double* St) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ci = morton_of[i];
  int xi, yi;
  demorton((uint32_t)ci, xi, yi);
  for (int t = rowptr[i]; t < rowptr[i + 1]; ++t) {
    const int j = colind[t];
    if ((unsigned)j >= (unsigned)n) continue;
    int xj, yj;
    demorton((uint32_t)morton_of[j], xj, yj);
    const int dx = xj - xi, dy = yj - yi;
    if (dx < -rx || dx > rx || dy < -ry || dy > ry) continue;
    St[(int64_t)((dy + ry) * (2 * rx + 1) + dx + rx) * ncell + ci] += val[t];
  }
}
void launch_csr_to_mstencil(int n, const int32_t* rowptr, const int32_t* colind,
                            const double* val, const int32_t* morton_of, int rx, int ry,
                            int64_t ncell, double* St, cudaStream_t s) {
  if (n > 0) {
    count_launch();
    k_csr_to_mstencil<<<(n + 127) / 128, 128, 0, s>>>(n, rowptr, colind, val, morton_of, rx, ry,
                                                      ncell, St);
  }
}

// out(o, p) = Q_{mask p} blk(o, p) Q_{mask p+off_o}^T in float32 arithmetic
// from an untransformed float64 block stencil: the level-q operator of the
// mixed path without a float64 transform (the float64 pipe is the slow one).
__global__ void k_transform_blocks_f32(const double* __restrict__ blk, float* out,
                                       const int2* __restrict__ off, int noff, int64_t npar,
                                       int Lpar, const uint32_t* __restrict__ pmask) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t p = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)p, x, y);
  const int pp = shift_cell(x, y, off[o].x, off[o].y, Lpar, npar);
  const int mr = (int)pmask[p] & 15;
  const int mc = pp >= 0 ? (int)pmask[pp] & 15 : 0;
  float M[16], Tm[16], Qr[16], Qc[16];
  qmat<float>(mr, Qr);
  qmat<float>(mc, Qc);
  const double2* B2 = reinterpret_cast<const double2*>(blk + t * 16);
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const double2 v = B2[e];
    M[2 * e] = (float)v.x;
    M[2 * e + 1] = (float)v.y;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float acc = 0.f;
#pragma unroll
      for (int r = 0; r < 4; ++r) acc += Qr[a * 4 + r] * M[r * 4 + c];
      Tm[a * 4 + c] = acc;
    }
  float4* O4 = reinterpret_cast<float4*>(out + t * 16);
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float v[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float acc = 0.f;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc += Tm[a * 4 + c] * Qc[b * 4 + c];
      v[b] = acc;
    }
    O4[a] = make_float4(v[0], v[1], v[2], v[3]);
  }
}
void launch_transform_blocks_f32(const double* blk, float* out, const int2* off, int noff,
                                 int64_t npar, int Lpar, const uint32_t* pmask, cudaStream_t s) {
  const int64_t n = (int64_t)noff * npar;
  if (n > 0) {
    count_launch();
    k_transform_blocks_f32<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blk, out, off, noff, npar,
                                                                        Lpar, pmask);
  }
}

__global__ void k_f64_to_f32(const double* __restrict__ in, float* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}
__global__ void k_f32_to_f64(const float* __restrict__ in, double* out, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = (double)in[i];
}
void launch_convert_f64_f32(const double* in, float* out, int64_t n, cudaStream_t s) {
  if (n > 0) { count_launch(); k_f64_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n); }
}
void launch_convert_f32_f64(const float* in, double* out, int64_t n, cudaStream_t s) {
  if (n > 0) { count_launch(); k_f32_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n); }
}

template <typename T>
__global__ void k_transform_vec(const T* __restrict__ in, T* out, int64_t npar,
                                const uint32_t* __restrict__ pmask, int dir) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npar) return;
  int m = (int)pmask[p] & 15;
  T v[4], o[4], Q[16];
  qmat<T>(m, Q);
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = in[4 * p + c];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T acc = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) acc += (dir > 0 ? Q[a * 4 + c] : Q[c * 4 + a]) * v[c];
    o[a] = acc;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) out[4 * p + a] = o[a];
}

template <typename T>
void launch_transform_vec(const T* in, T* out, int64_t npar, const uint32_t* pmask, int dir,
                          cudaStream_t s) {
  if (npar <= 0) return;
  { count_launch(); k_transform_vec<T><<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(in, out, npar, pmask, dir); }
}
template void launch_transform_vec<double>(const double*, double*, int64_t, const uint32_t*,
                                           int, cudaStream_t);
template void launch_transform_vec<float>(const float*, float*, int64_t, const uint32_t*, int,
                                          cudaStream_t);

__global__ void k_gather_morton(const double* __restrict__ in, const int32_t* __restrict__ unk,
                                int64_t ncell, double* out) {
  int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (s >= ncell) return;
  int i = unk[s];
  out[s] = i >= 0 ? in[i] : 0.0;
}
__global__ void k_scatter_unknown(const double* __restrict__ in, const int32_t* __restrict__ mo,
                                  int n, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[mo[i]];
}
void launch_gather_morton(const double* in_unknown, const int32_t* unknown_of, int64_t ncell,
                          double* out_morton, cudaStream_t s) {
  if (ncell > 0)
    { count_launch(); k_gather_morton<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(in_unknown, unknown_of,
                                                                    ncell, out_morton); }
}
void launch_scatter_unknown(const double* in_morton, const int32_t* morton_of, int n,
                            double* out_unknown, cudaStream_t s) {
  if (n > 0)
    { count_launch(); k_scatter_unknown<<<(n + 255) / 256, 256, 0, s>>>(in_morton, morton_of, n, out_unknown); }
}

}  // namespace gb
