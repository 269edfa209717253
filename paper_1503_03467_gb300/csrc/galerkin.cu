// galerkin.cu - Galerkin coarsening A^(k-1) = R^(k-1,k) A^(k) R^(k,k-1)
// (Theorem thmhggfees5, Eq. eqhuhiuv; Algorithm 2, line 13).
//
// Everything is evaluated in the transformed basis: with Rhat = R Q^T and
// Ahat = Q A^(k) Q^T (Q block-orthonormal), R A R^T = Rhat Ahat Rhat^T.
// For a coarse cell i the row Rhat_i lives on the patch i + N_j; the product
// t_i = Ahat Rhat_i^T lives on the window i + WIN_w (WIN = N + O_k), and
//   A^(k-1)_{i, i+S_d} = Rhat_{i+S_d} . t_i   (WIN_w = S_d + N_j).
// The index lists (j, o) per window position and (j, w) per output offset
// are built once per level on the host from the offset sets.  A^(k-1) is
// symmetric, so only the offsets of one half-plane S+ are computed; the
// conversion to blocks reads the other half as A_{i, i+d} = A_{i+d, i}.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

// 16-element block / 4-element row loads as 128-bit transactions
__device__ __forceinline__ void load_block16(const float* p, float* b) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float4 v = __ldg(q + k);
    b[4 * k] = v.x;
    b[4 * k + 1] = v.y;
    b[4 * k + 2] = v.z;
    b[4 * k + 3] = v.w;
  }
}
__device__ __forceinline__ void load_block16(const double* p, double* b) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const double2 v = __ldg(q + k);
    b[2 * k] = v.x;
    b[2 * k + 1] = v.y;
  }
}
__device__ __forceinline__ void load_vec4(const float* p, float* b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  b[0] = v.x;
  b[1] = v.y;
  b[2] = v.z;
  b[3] = v.w;
}
__device__ __forceinline__ void load_vec4(const double* p, double* b) {
  const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  b[0] = v0.x;
  b[1] = v0.y;
  b[2] = v1.x;
  b[3] = v1.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_galerkin(const T* __restrict__ Ahat,
                                                  const T* __restrict__ Rhat,
                                                  const uint32_t* __restrict__ pmask,
                                                  GalerkinGeom g, T* __restrict__ Aout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rrow = reinterpret_cast<T*>(smem_raw);
  T* t = rrow + 4 * g.NB;
  const int64_t nrow = g.nrow;
  for (int64_t i = blockIdx.x; i < nrow; i += gridDim.x) {
    if ((pmask[i] & 15u) == 0) {
      for (int d = threadIdx.x; d < g.nout; d += blockDim.x) Aout[(int64_t)d * nrow + i] = T(0);
      continue;
    }
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    for (int idx = threadIdx.x; idx < 4 * g.NB; idx += blockDim.x)
      rrow[idx] = Rhat[i * 4 * g.NB + idx];
    __syncthreads();
    // t_i = Ahat Rhat_i^T on the window
    for (int w = threadIdx.x; w < g.nwin; w += blockDim.x) {
      T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
      const int p = shift_cell(xi, yi, g.win[w].x, g.win[w].y, g.Lpar);
      if (p >= 0) {
        for (int e = g.l1_ptr[w]; e < g.l1_ptr[w + 1]; ++e) {
          const int2 jo = g.l1_pairs[e];
          const T* blk = Ahat + ((int64_t)jo.y * nrow + p) * 16;
          T b[16];
          load_block16(blk, b);
          const T r0 = rrow[4 * jo.x], r1 = rrow[4 * jo.x + 1];
          const T r2 = rrow[4 * jo.x + 2], r3 = rrow[4 * jo.x + 3];
          acc0 += b[0] * r0 + b[1] * r1 + b[2] * r2 + b[3] * r3;
          acc1 += b[4] * r0 + b[5] * r1 + b[6] * r2 + b[7] * r3;
          acc2 += b[8] * r0 + b[9] * r1 + b[10] * r2 + b[11] * r3;
          acc3 += b[12] * r0 + b[13] * r1 + b[14] * r2 + b[15] * r3;
        }
      }
      t[4 * w] = acc0;
      t[4 * w + 1] = acc1;
      t[4 * w + 2] = acc2;
      t[4 * w + 3] = acc3;
    }
    __syncthreads();
    // A_{i, i+S_d} = Rhat_{i+S_d} . t_i
    for (int d = threadIdx.x; d < g.nout; d += blockDim.x) {
      T acc = 0;
      const int ip = shift_cell(xi, yi, g.out[d].x, g.out[d].y, g.Lpar);
      if (ip >= 0 && (pmask[ip] & 15u)) {
        const T* rrow_ip = Rhat + (int64_t)ip * 4 * g.NB;
        for (int e = g.l2_ptr[d]; e < g.l2_ptr[d + 1]; ++e) {
          const int2 jw = g.l2_pairs[e];
          const T* tw = t + 4 * jw.y;
          T rv[4];
          load_vec4(rrow_ip + 4 * jw.x, rv);
#pragma unroll
          for (int c = 0; c < 4; ++c) acc += rv[c] * tw[c];
        }
      }
      Aout[(int64_t)d * nrow + i] = acc;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_galerkin(const T* Ahat, const T* Rhat, const uint32_t* pmask_k, GalerkinGeom g,
                     T* Aout, cudaStream_t s) {
  if (g.nrow <= 0) return;
  size_t smem = sizeof(T) * 4 * ((size_t)g.NB + (size_t)g.nwin);
  cudaFuncSetAttribute(k_galerkin<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int64_t grid = g.nrow < 65535 * 16 ? g.nrow : 65535 * 16;
  { count_launch(); k_galerkin<T><<<(unsigned)grid, 256, smem, s>>>(Ahat, Rhat, pmask_k, g, Aout); }
}
template void launch_galerkin<float>(const float*, const float*, const uint32_t*, GalerkinGeom,
                                     float*, cudaStream_t);
template void launch_galerkin<double>(const double*, const double*, const uint32_t*,
                                      GalerkinGeom, double*, cudaStream_t);

// Cell stencil of level k-1 -> transformed block stencil of level k-1.
template <typename T>
__global__ void k_cells_to_blocks(const T* __restrict__ Acell, int64_t ncell,
                                  const int* __restrict__ map, int nO,
                                  const int2* __restrict__ Ooff, int Lpar, int64_t npar,
                                  const uint32_t* __restrict__ pmask, T* __restrict__ blk) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nO * npar) return;
  const int o = (int)(t / npar);
  const int64_t P = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)P, x, y);
  const int PP = shift_cell(x, y, Ooff[o].x, Ooff[o].y, Lpar);
  const int mr = (int)pmask[P] & 15;
  const int mc = PP >= 0 ? (int)pmask[PP] & 15 : 0;
  double M[16], Tm[16], Qr[16], Qc[16];
  qmat<double>(mr, Qr);
  qmat<double>(mc, Qc);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int d = map[o * 16 + c * 4 + cc];
      double v = 0.0;
      if (PP >= 0 && d >= 0) v = (double)Acell[(int64_t)d * ncell + 4 * P + c];
      else if (PP >= 0 && d <= -2) v = (double)Acell[(int64_t)(-d - 2) * ncell + 4 * PP + cc];
      M[c * 4 + cc] = v;
    }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      double acc = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc += Qr[a * 4 + c] * M[c * 4 + cc];
      Tm[a * 4 + cc] = acc;
    }
  T* out = blk + t * 16;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double acc = 0;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) acc += Tm[a * 4 + cc] * Qc[b * 4 + cc];
      out[a * 4 + b] = (T)acc;
    }
}

template <typename T>
void launch_cells_to_blocks(const T* Acell, int64_t ncell, const int* map, int nO,
                            const int2* Ooff, int Lpar, int64_t npar, const uint32_t* pmask,
                            T* blk, cudaStream_t s) {
  int64_t n = (int64_t)nO * npar;
  if (n <= 0) return;
  { count_launch(); k_cells_to_blocks<T><<<(unsigned)((n + 127) / 128), 128, 0, s>>>(Acell, ncell, map, nO, Ooff,
                                                                   Lpar, npar, pmask, blk); }
}
template void launch_cells_to_blocks<float>(const float*, int64_t, const int*, int, const int2*,
                                            int, int64_t, const uint32_t*, float*, cudaStream_t);
template void launch_cells_to_blocks<double>(const double*, int64_t, const int*, int,
                                             const int2*, int, int64_t, const uint32_t*, double*,
                                             cudaStream_t);

}  // namespace gb

namespace gb {

// ---------------------------------------------------------------------------
// Tiled Galerkin product: one CTA per TR x TR tile of coarse rows i.  Every
// block Ahat[o][p'] and every interpolation row Rhat_{i'} the tile touches is
// read from L2 once and applied to all rows of the tile, with the products
// accumulated in registers:
//   phase 1  thread per window parent p':  t_i[p' - i] = sum_o Ahat[o][p'] Rhat_i[j],
//            N_j = p' + O_o - i, for every tile row i;
//   phase 2  thread per output neighbour i': A_{i, i'} = sum_j Rhat_{i'}[j] . t_i[i' + N_j - i]
//            for every tile row i with i' - i in the half-plane S+.
// Offsets are located through small dense lookup tables held in shared memory.
template <typename T, int TR>
__global__ void __launch_bounds__(256) k_galerkin_tiled(const T* __restrict__ Ahat,
                                                        const T* __restrict__ Rhat,
                                                        const uint32_t* __restrict__ pmask,
                                                        GalerkinTileGeom g, T* __restrict__ Aout) {
  constexpr int NR = TR * TR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = g.NB;
  T* rr = reinterpret_cast<T*>(smem_raw);           // NR x 4 NB
  T* t = rr + NR * 4 * NB;                          // NR x nwin x 4
  int* nmap = reinterpret_cast<int*>(t + (size_t)NR * g.nwin * 4);
  const int DN = 2 * g.RN + 1, DW = 2 * g.RW + 1, DS = 2 * g.RS + 1;
  int* wmap = nmap + DN * DN;
  int* smap = wmap + DW * DW;
  for (int e = threadIdx.x; e < DN * DN; e += blockDim.x) nmap[e] = g.nmap[e];
  for (int e = threadIdx.x; e < DW * DW; e += blockDim.x) wmap[e] = g.wmap[e];
  for (int e = threadIdx.x; e < DS * DS; e += blockDim.x) smap[e] = g.smap[e];
  int bx, by;
  demorton((uint32_t)blockIdx.x, bx, by);
  const int x0 = bx * TR, y0 = by * TR;
  int64_t irow[NR];
  bool ract[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int rx = x0 + r % TR, ry = y0 + r / TR;
    irow[r] = morton((uint32_t)rx, (uint32_t)ry);
    ract[r] = (pmask[irow[r]] & 15u) != 0;
  }
  for (int e = threadIdx.x; e < NR * 4 * NB; e += blockDim.x) {
    const int r = e / (4 * NB), q = e - r * 4 * NB;
    rr[e] = ract[r] ? Rhat[irow[r] * 4 * NB + q] : T(0);
  }
  // window parents outside the lattice are never written below; their Rhat
  // partners are zero, so they must read as zero too
  for (int e = threadIdx.x; e < NR * g.nwin * 4; e += blockDim.x) t[e] = T(0);
  __syncthreads();

  // ---- phase 1: t_i = Ahat Rhat_i^T on the window of every tile row
  const int BW = TR + 2 * g.RW;
  for (int c = threadIdx.x; c < BW * BW; c += blockDim.x) {
    const int px = x0 - g.RW + c % BW, py = y0 - g.RW + c / BW;
    if ((unsigned)px >= (unsigned)g.Lpar || (unsigned)py >= (unsigned)g.Lpar) continue;
    int wr[NR];
    bool any = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int wx = px - (x0 + r % TR), wy = py - (y0 + r / TR);
      int w = -1;
      if (ract[r] && abs(wx) <= g.RW && abs(wy) <= g.RW) w = wmap[(wy + g.RW) * DW + wx + g.RW];
      wr[r] = w;
      any |= w >= 0;
    }
    if (!any) continue;
    const int64_t pp = morton((uint32_t)px, (uint32_t)py);
    T acc[NR][4];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[r][b] = T(0);
    for (int o = 0; o < g.noff; ++o) {
      const int2 d = g.off[o];
      int jr[NR];
      bool use = false;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        const int nx = px + d.x - (x0 + r % TR), ny = py + d.y - (y0 + r / TR);
        int j = -1;
        if (wr[r] >= 0 && abs(nx) <= g.RN && abs(ny) <= g.RN) j = nmap[(ny + g.RN) * DN + nx + g.RN];
        jr[r] = j;
        use |= j >= 0;
      }
      if (!use) continue;
      T blk[16];
      load_block16(Ahat + ((int64_t)o * g.nrow + pp) * 16, blk);
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (jr[r] < 0) continue;
        const T* rv = rr + r * 4 * NB + 4 * jr[r];
        const T r0 = rv[0], r1 = rv[1], r2 = rv[2], r3 = rv[3];
#pragma unroll
        for (int b = 0; b < 4; ++b)
          acc[r][b] += blk[4 * b] * r0 + blk[4 * b + 1] * r1 + blk[4 * b + 2] * r2 + blk[4 * b + 3] * r3;
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (wr[r] < 0) continue;
      T* tw = t + ((size_t)r * g.nwin + wr[r]) * 4;
#pragma unroll
      for (int b = 0; b < 4; ++b) tw[b] = acc[r][b];
    }
  }
  __syncthreads();

  // ---- phase 2: A_{i, i'} = Rhat_{i'} . t_i for i' - i in S+
  const int BS = TR + 2 * g.RS;
  for (int c = threadIdx.x; c < BS * BS; c += blockDim.x) {
    const int ix = x0 - g.RS + c % BS, iy = y0 - g.RS + c / BS;
    if ((unsigned)ix >= (unsigned)g.Lpar || (unsigned)iy >= (unsigned)g.Lpar) continue;
    const int64_t ip = morton((uint32_t)ix, (uint32_t)iy);
    if (!(pmask[ip] & 15u)) continue;
    int sr[NR], dxr[NR], dyr[NR];
    bool any = false;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      dxr[r] = ix - (x0 + r % TR);
      dyr[r] = iy - (y0 + r / TR);
      int si = -1;
      if (ract[r] && abs(dxr[r]) <= g.RS && abs(dyr[r]) <= g.RS)
        si = smap[(dyr[r] + g.RS) * DS + dxr[r] + g.RS];
      sr[r] = si;
      any |= si >= 0;
    }
    if (!any) continue;
    T acc2[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc2[r] = T(0);
    const T* rowp = Rhat + ip * 4 * NB;
    for (int j = 0; j < NB; ++j) {
      T rv[4];
      load_vec4(rowp + 4 * j, rv);
      const int2 nj = g.nbr[j];
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        if (sr[r] < 0) continue;
        const int wx = dxr[r] + nj.x, wy = dyr[r] + nj.y;
        if (abs(wx) > g.RW || abs(wy) > g.RW) continue;
        const int w = wmap[(wy + g.RW) * DW + wx + g.RW];
        if (w < 0) continue;
        const T* tw = t + ((size_t)r * g.nwin + w) * 4;
        acc2[r] += rv[0] * tw[0] + rv[1] * tw[1] + rv[2] * tw[2] + rv[3] * tw[3];
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (sr[r] >= 0) Aout[(int64_t)sr[r] * g.nrow + irow[r]] = acc2[r];
  }
}

size_t galerkin_tiled_smem(const GalerkinTileGeom& g, int tr, size_t elem) {
  const int nr = tr * tr;
  size_t b = elem * ((size_t)nr * 4 * g.NB + (size_t)nr * g.nwin * 4);
  b += sizeof(int) * ((size_t)(2 * g.RN + 1) * (2 * g.RN + 1) + (size_t)(2 * g.RW + 1) * (2 * g.RW + 1) +
                      (size_t)(2 * g.RS + 1) * (2 * g.RS + 1));
  return (b + 15) & ~(size_t)15;
}

template <typename T, int TR>
static void launch_tiled(const T* Ahat, const T* Rhat, const uint32_t* pmask, GalerkinTileGeom g,
                         T* Aout, cudaStream_t s) {
  const size_t smem = galerkin_tiled_smem(g, TR, sizeof(T));
  cudaFuncSetAttribute(k_galerkin_tiled<T, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  const int64_t tiles = (int64_t)(g.Lpar / TR) * (g.Lpar / TR);
  { count_launch(); k_galerkin_tiled<T, TR><<<(unsigned)tiles, 256, smem, s>>>(Ahat, Rhat, pmask, g, Aout); }
}

template <typename T>
void launch_galerkin_tiled(const T* Ahat, const T* Rhat, const uint32_t* pmask_k,
                           GalerkinTileGeom g, int tr, T* Aout, cudaStream_t s) {
  if (g.nrow <= 0) return;
  cudaMemsetAsync(Aout, 0, sizeof(T) * (size_t)g.nout * (size_t)g.nrow, s);
  if (tr >= 4) launch_tiled<T, 4>(Ahat, Rhat, pmask_k, g, Aout, s);
  else if (tr == 2) launch_tiled<T, 2>(Ahat, Rhat, pmask_k, g, Aout, s);
  else launch_tiled<T, 1>(Ahat, Rhat, pmask_k, g, Aout, s);
}
template void launch_galerkin_tiled<float>(const float*, const float*, const uint32_t*,
                                           GalerkinTileGeom, int, float*, cudaStream_t);
template void launch_galerkin_tiled<double>(const double*, const double*, const uint32_t*,
                                            GalerkinTileGeom, int, double*, cudaStream_t);

}  // namespace gb
