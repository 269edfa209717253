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

// 4-element row loads as 128-bit transactions
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

// A whole 4x4 block (64 bytes float, 128 bytes double) as 32-byte loads: two
// (float) or four (double) instead of four or eight 16-byte loads, so each
// 32-byte sector of a block is looked up once by the L1 instead of twice.
// Blocks start at multiples of 16 elements from the base; load_block takes
// this path when the base is 32-byte aligned (the library's allocations are)
// and the 16-byte one otherwise.
__device__ __forceinline__ void load_blk16(const float* p, float* b) {
#pragma unroll
  for (int h = 0; h < 2; ++h)
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(b[8 * h]), "=f"(b[8 * h + 1]), "=f"(b[8 * h + 2]), "=f"(b[8 * h + 3]),
                   "=f"(b[8 * h + 4]), "=f"(b[8 * h + 5]), "=f"(b[8 * h + 6]), "=f"(b[8 * h + 7])
                 : "l"(p + 8 * h));
}
__device__ __forceinline__ void load_blk16(const double* p, double* b) {
#pragma unroll
  for (int h = 0; h < 4; ++h)
    asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
                 : "=d"(b[4 * h]), "=d"(b[4 * h + 1]), "=d"(b[4 * h + 2]), "=d"(b[4 * h + 3])
                 : "l"(p + 4 * h));
}

template <typename T>
__device__ __forceinline__ void load_block(const T* p, T* b, bool wide) {
  if (wide) {
    load_blk16(p, b);
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q) load_vec4(p + 4 * q, b + 4 * q);
  }
}

// 4-element rows (shared or global memory) as single 16-byte (float) or two 16-byte
// (double) accesses: lanes that touch consecutive rows then hit distinct
// banks, where four scalar accesses at a 16-byte stride collide four ways.
__device__ __forceinline__ void sld4(const float* p, float* v) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void sld4(const double* p, double* v) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void sst4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void sst4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// One CTA per coarse row i, one thread per window position (phase 1: the
// thread reads whole 4x4 blocks, 64 bytes, and keeps four accumulators) and
// one thread per output offset (phase 2).  Fewer instructions per block
// product than k_galerkin_warp; better when the block lists per window
// position are short (the finest level's 9-point stencil).
template <typename T>
__global__ void __launch_bounds__(256) k_galerkin_rows(const T* __restrict__ Ahat,
                                                       const T* __restrict__ Rhat,
                                                       const uint32_t* __restrict__ pmask,
                                                       GalerkinGeom g, T* __restrict__ Aout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rrow = reinterpret_cast<T*>(smem_raw);
  T* t = rrow + 4 * g.NB;
  const int64_t nrow = g.nrow;
  const bool wide = (reinterpret_cast<uintptr_t>(Ahat) & 31) == 0;
  for (int64_t i = g.i_begin + blockIdx.x; i < g.i_end; i += gridDim.x) {
    if ((pmask[i] & 15u) == 0) {
      for (int d = threadIdx.x; d < g.nout; d += blockDim.x) Aout[(int64_t)d * nrow + i] = T(0);
      continue;
    }
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    for (int idx = threadIdx.x; idx < 4 * g.NB; idx += blockDim.x)
      rrow[idx] = Rhat[i * 4 * g.NB + idx];
    __syncthreads();
    for (int w = threadIdx.x; w < g.nwin; w += blockDim.x) {
      T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
      const int p = shift_cell(xi, yi, g.win[w].x, g.win[w].y, g.Lpar, nrow);
      if (p >= 0) {
        for (int e = g.l1_ptr[w]; e < g.l1_ptr[w + 1]; ++e) {
          const int2 jo = g.l1_pairs[e];
          const T* blk = Ahat + ((int64_t)jo.y * nrow + p) * 16;
          T b[16];
          load_block(blk, b, wide);
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
    for (int d = threadIdx.x; d < g.nout; d += blockDim.x) {
      T acc = 0;
      const int ip = shift_cell(xi, yi, g.out[d].x, g.out[d].y, g.Lpar, nrow);
      if (ip >= 0 && (pmask[ip] & 15u)) {
        const T* rr = Rhat + (int64_t)ip * 4 * g.NB;
        for (int e = g.l2_ptr[d]; e < g.l2_ptr[d + 1]; ++e) {
          const int2 jw = g.l2_pairs[e];
          const T* tw = t + 4 * jw.y;
          T rv[4];
          load_vec4(rr + 4 * jw.x, rv);
          acc += rv[0] * tw[0] + rv[1] * tw[1] + rv[2] * tw[2] + rv[3] * tw[3];
        }
      }
      Aout[(int64_t)d * nrow + i] = acc;
    }
    __syncthreads();
  }
}

// Four coarse rows per CTA: the 2 x 2 cells i0..i0+3 of one level-(k-2)
// parent (row r at (r & 1, r >> 1) from the tile origin).  Phase 1: for each
// position u of the tile's window box that phase 2 reads, a thread walks u's
// block list (host list t1; positions in t1_items): each block
// Ahat[o][origin+u] is loaded once and applied to every row whose patch
// reaches it (the neighbour index j of each row), accumulating t_r(u) for
// the four rows.
// Phase 2: LPT lanes per output target cell c (host list t2), or per
// horizontal pair of targets (host list t3, variants 6-8), walk the list of
// window positions u = c + N_j, reading Rhat_c(j) from global memory and
// t_r(u) from shared memory, and form the dot products of every row r for
// which c - r is an output offset.  Compared with a row per CTA this reads
// each block and each Rhat row up to four times less often.
size_t galerkin_tile_smem_bytes(const GalerkinGeom& g, size_t elem) {
  return elem * (16 * (size_t)g.NB + 16 * (size_t)g.nt1u);
}

// Phase 2 of the tile kernel over horizontal pairs of targets (c, c + (1, 0)):
// one list of window positions u per pair (the union of the two targets'
// lists), so each t_r(u) read from shared memory serves both targets and the
// list bookkeeping is shared; a target without partner has d = -1 in its
// second record and ja / jb = 0xff where its patch does not reach u.  The
// eight sums (two targets x four rows) are reduce-scattered over the LPT
// lanes: lanes that differ in bit 0 trade four of them, in bit 1 two, in bit
// 2 one, and higher bits add whole values.
template <typename T, int LPT>
__device__ __forceinline__ void galerkin_tile_pairs(const GalerkinGeom& g, const T* __restrict__ Rhat,
                                                    const uint32_t* __restrict__ pmask,
                                                    const T* tt, int NT, int x0, int y0, int64_t i0,
                                                    const bool (&live)[4], T* __restrict__ Aout) {
  constexpr int TPW = 32 / LPT;
  constexpr int H = LPT >= 8 ? 1 : 2;  // values a lane holds after the reduce-scatter
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int sub = lane & (LPT - 1), grp = lane / LPT;
  const int NB = g.NB;
  const int64_t nrow = g.nrow;
  // pairs by decreasing length, dealt to the warps in alternating direction
  // so that no warp takes the longest lists of every round
  const int per_round = TPW * nwarp;
  for (int round = 0; round * per_round < g.nt3; ++round) {
    const int slot = TPW * warp + grp;
    const int e = round * per_round + ((round & 1) ? per_round - 1 - slot : slot);
    const bool ok = e < g.nt3;
    const int4 ta = ok ? g.t3[2 * e] : make_int4(0, 0, -1, -1);
    const int4 tb = ok ? g.t3[2 * e + 1] : make_int4(0, 0, -1, -1);
    int d[8] = {(int)(short)(ta.z & 0xffff), ta.z >> 16, (int)(short)(ta.w & 0xffff), ta.w >> 16,
                (int)(short)(tb.z & 0xffff), tb.z >> 16, (int)(short)(tb.w & 0xffff), tb.w >> 16};
    const bool any_b = d[4] >= 0 || d[5] >= 0 || d[6] >= 0 || d[7] >= 0;
    const int ipa = ok ? shift_cell(x0, y0, ta.x, ta.y, g.Lpar, nrow) : -1;
    const int ipb = ok && any_b ? shift_cell(x0, y0, tb.x, tb.y, g.Lpar, nrow) : -1;
    const bool ha = ipa >= 0 && (pmask[ipa] & 15u);
    const bool hb = ipb >= 0 && (pmask[ipb] & 15u);
    bool need[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) need[r] = d[r] >= 0 || d[4 + r] >= 0;
    T v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = T(0);
    if (ha || hb) {
      const T* ra = Rhat + (int64_t)(ha ? ipa : 0) * 4 * NB;
      const T* rb = Rhat + (int64_t)(hb ? ipb : 0) * 4 * NB;
      const int q1 = g.t3p_ptr[e + 1];
      for (int q = g.t3p_ptr[e] + sub; q < q1; q += LPT) {
        const uint32_t pu = __ldg(g.t3p + q);
        const int cu = (int)(pu & 0xffffu), ja = (int)((pu >> 16) & 0xffu), jb = (int)(pu >> 24);
        T va[4] = {T(0), T(0), T(0), T(0)}, vb[4] = {T(0), T(0), T(0), T(0)};
        if (ha && ja != 0xff) load_vec4(ra + 4 * ja, va);
        if (hb && jb != 0xff) load_vec4(rb + 4 * jb, vb);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (!need[r]) continue;
          T tv[4];
          sld4(tt + ((size_t)r * NT + cu) * 4, tv);
          v[r] += va[0] * tv[0] + va[1] * tv[1] + va[2] * tv[2] + va[3] * tv[3];
          v[4 + r] += vb[0] * tv[0] + vb[1] * tv[1] + vb[2] * tv[2] + vb[3] * tv[3];
        }
      }
    }
    int base = 0;
#pragma unroll
    for (int h = 4, bit = 1; h >= H && bit < LPT; h >>= 1, bit <<= 1) {
      const bool upper = (sub & bit) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const T send = upper ? v[i] : v[i + h];
        const T keep = upper ? v[i + h] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
      }
      if (upper) base += h;
    }
#pragma unroll
    for (int bit = 8; bit < LPT; bit <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], bit);
    if (sub < 8 / H && ok) {
#pragma unroll
      for (int t = 0; t < H; ++t) {
        const int idx = base + t, r = idx & 3;
        int dv = -1;
#pragma unroll
        for (int c = 0; c < 8; ++c)
          if (c == idx) dv = d[c];
        const bool lr = r == 0 ? live[0] : (r == 1 ? live[1] : (r == 2 ? live[2] : live[3]));
        if (dv >= 0 && i0 + r >= g.i_begin && i0 + r < g.i_end)
          Aout[(int64_t)dv * nrow + i0 + r] = lr ? v[t] : T(0);
      }
    }
  }
}

template <typename T, int LPT, bool PAIRS>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1) k_galerkin_tile(const T* __restrict__ Ahat,
                                                       const T* __restrict__ Rhat,
                                                       const uint32_t* __restrict__ pmask,
                                                       GalerkinGeom g, T* __restrict__ Aout) {
  static_assert(LPT >= 4 && LPT <= 32 && (LPT & (LPT - 1)) == 0, "lanes per target");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = g.NB, W = g.tile_W, NT = g.nt1u, wmin = g.tile_wmin;
  T* rr = reinterpret_cast<T*>(smem_raw);  // [4][NB][4]
  T* tt = rr + 16 * NB;                    // [4][NT][4]: t_r at the positions phase 2 reads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int64_t nrow = g.nrow;
  const bool wide = (reinterpret_cast<uintptr_t>(Ahat) & 31) == 0;
  const int64_t t0 = g.i_begin >> 2, t1 = (g.i_end + 3) >> 2;
  for (int64_t tile = t0 + blockIdx.x; tile < t1; tile += gridDim.x) {
    const int64_t i0 = tile << 2;
    int x0, y0;
    demorton((uint32_t)i0, x0, y0);
    bool live[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
      live[r] = i0 + r >= g.i_begin && i0 + r < g.i_end && (pmask[i0 + r] & 15u);
    for (int idx = threadIdx.x; idx < 4 * NB; idx += blockDim.x) {
      const int r = idx / NB, j = idx - r * NB;
      T v[4] = {T(0), T(0), T(0), T(0)};
      if (live[r]) load_vec4(Rhat + ((i0 + r) * NB + j) * 4, v);
      sst4(rr + (r * NB + j) * 4, v);
    }
    __syncthreads();
    // phase 1: t_r(u) = sum over stored blocks of the window, for the
    // positions that phase 2 reads (longest lists first, dealt in
    // alternating direction so that the threads' totals even out)
    const int nthr = blockDim.x;
    for (int round = 0; round * nthr < g.nitems; ++round) {
      const int iw = round * nthr + ((round & 1) ? nthr - 1 - (int)threadIdx.x : (int)threadIdx.x);
      if (iw >= g.nitems) continue;
      const int4 item = __ldg(g.t1_items + iw);
      const int u = item.x & 0xffff, cu = item.x >> 16;
      const int uy = u / W, ux = u - uy * W;
      const int p = shift_cell(x0, y0, ux + wmin, uy + wmin, g.Lpar, nrow);
      T acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = T(0);
      if (p >= 0) {
        for (int e = item.y; e < item.z; ++e) {
          const int2 ent = g.t1[e];
          const T* blk = Ahat + ((int64_t)ent.x * nrow + p) * 16;
          T b[16];
          load_block(blk, b, wide);
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int j = ((unsigned)ent.y >> (8 * r)) & 0xffu;
            if (j == 0xff) continue;
            T rv[4];
            sld4(rr + (r * NB + j) * 4, rv);
#pragma unroll
            for (int a = 0; a < 4; ++a)
              acc[r][a] += b[4 * a] * rv[0] + b[4 * a + 1] * rv[1] + b[4 * a + 2] * rv[2] +
                           b[4 * a + 3] * rv[3];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) sst4(tt + ((size_t)r * NT + cu) * 4, acc[r]);
    }
    __syncthreads();
    // phase 2: outputs A_{i0+r, c} for every target cell c.  LPT lanes per
    // target or pair of targets (4, 8 or 16, chosen per level by the
    // launch-shape tuner) stride over its list of window positions; the
    // partial sums are reduce-scattered over the lanes.
    if constexpr (PAIRS) {
      galerkin_tile_pairs<T, LPT>(g, Rhat, pmask, tt, NT, x0, y0, i0, live, Aout);
    } else {
      constexpr int TPW = 32 / LPT;
      const int sub = lane & (LPT - 1), grp = lane / LPT;
      for (int e0 = TPW * warp; e0 < g.nt2; e0 += TPW * nwarp) {
        const int e = e0 + grp;
        const bool ok = e < g.nt2;
        const int4 tg = ok ? g.t2[e] : make_int4(0, 0, -1, -1);
        const int d[4] = {(int)(short)(tg.z & 0xffff), tg.z >> 16, (int)(short)(tg.w & 0xffff),
                          tg.w >> 16};
        const int ip = ok ? shift_cell(x0, y0, tg.x, tg.y, g.Lpar, nrow) : -1;
        const bool have = ip >= 0 && (pmask[ip] & 15u);
        T acc[4] = {T(0), T(0), T(0), T(0)};
        if (have) {
          const T* rc = Rhat + (int64_t)ip * 4 * NB;
          const int q1 = g.t2p_ptr[e + 1];
          for (int q = g.t2p_ptr[e] + sub; q < q1; q += LPT) {
            const int pu = __ldg(g.t2p + q);
            const int j = pu & 0xff, cu = pu >> 8;
            T rv[4];
            load_vec4(rc + 4 * j, rv);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              if (d[r] < 0) continue;
              T tv[4];
              sld4(tt + ((size_t)r * NT + cu) * 4, tv);
              acc[r] += rv[0] * tv[0] + rv[1] * tv[1] + rv[2] * tv[2] + rv[3] * tv[3];
            }
          }
        }
        // Reduce-scatter of the four row sums over the LPT lanes: the lanes
        // that differ in bit 0 trade two of the four partial sums, those that
        // differ in bit 1 trade one, and the remaining bits add whole values,
        // so lane `sub` < 4 ends with row r = 2 (sub & 1) + (sub >> 1 & 1):
        // 3 + log2(LPT / 4) shuffles instead of 4 log2(LPT).
        const bool b0 = (sub & 1) != 0, b1 = (sub & 2) != 0;
        T k0 = b0 ? acc[2] : acc[0], k1 = b0 ? acc[3] : acc[1];
        k0 += __shfl_xor_sync(0xffffffffu, b0 ? acc[0] : acc[2], 1);
        k1 += __shfl_xor_sync(0xffffffffu, b0 ? acc[1] : acc[3], 1);
        T v = (b1 ? k1 : k0) + __shfl_xor_sync(0xffffffffu, b1 ? k0 : k1, 2);
#pragma unroll
        for (int o = 4; o < LPT; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int r = 2 * (int)b0 + (int)b1;
        const int dr = r == 0 ? d[0] : (r == 1 ? d[1] : (r == 2 ? d[2] : d[3]));
        const bool lr = r == 0 ? live[0] : (r == 1 ? live[1] : (r == 2 ? live[2] : live[3]));
        if (sub < 4 && ok && dr >= 0 && i0 + r >= g.i_begin && i0 + r < g.i_end)
          Aout[(int64_t)dr * nrow + i0 + r] = lr ? v : T(0);
      }
    }
    __syncthreads();
  }
}

// One warp per coarse row, the work split as in k_galerkin_rows (lanes over
// window positions, then over output offsets) but synchronised per warp
// only: each warp keeps its own Rhat row and window in shared memory, so the
// rows of a CTA proceed independently and no warp idles at a CTA barrier
// while another finishes a phase.  Suited to short rows (the finest level).
template <typename T>
__global__ void __launch_bounds__(256) k_galerkin_warprow(const T* __restrict__ Ahat,
                                                          const T* __restrict__ Rhat,
                                                          const uint32_t* __restrict__ pmask,
                                                          GalerkinGeom g, T* __restrict__ Aout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int per = 4 * (g.NB + g.nwin);  // T per warp
  T* rrow = reinterpret_cast<T*>(smem_raw) + (size_t)warp * per;
  T* t = rrow + 4 * g.NB;
  const int64_t nrow = g.nrow;
  const bool wide = (reinterpret_cast<uintptr_t>(Ahat) & 31) == 0;
  for (int64_t i = g.i_begin + (int64_t)blockIdx.x * nwarp + warp; i < g.i_end;
       i += (int64_t)gridDim.x * nwarp) {
    if ((pmask[i] & 15u) == 0) {
      for (int d = lane; d < g.nout; d += 32) Aout[(int64_t)d * nrow + i] = T(0);
      continue;
    }
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    for (int j = lane; j < g.NB; j += 32) {
      T v[4];
      load_vec4(Rhat + (i * g.NB + j) * 4, v);
#pragma unroll
      for (int c = 0; c < 4; ++c) rrow[4 * j + c] = v[c];
    }
    __syncwarp();
    for (int w = lane; w < g.nwin; w += 32) {
      T acc0 = 0, acc1 = 0, acc2 = 0, acc3 = 0;
      const int p = shift_cell(xi, yi, g.win[w].x, g.win[w].y, g.Lpar, nrow);
      if (p >= 0) {
        for (int e = g.l1_ptr[w]; e < g.l1_ptr[w + 1]; ++e) {
          const int2 jo = g.l1_pairs[e];
          const T* blk = Ahat + ((int64_t)jo.y * nrow + p) * 16;
          T b[16];
          load_block(blk, b, wide);
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
    __syncwarp();
    for (int d = lane; d < g.nout; d += 32) {
      T acc = 0;
      const int ip = shift_cell(xi, yi, g.out[d].x, g.out[d].y, g.Lpar, nrow);
      if (ip >= 0 && (pmask[ip] & 15u)) {
        const T* rr = Rhat + (int64_t)ip * 4 * g.NB;
        for (int e = g.l2_ptr[d]; e < g.l2_ptr[d + 1]; ++e) {
          const int2 jw = g.l2_pairs[e];
          const T* tw = t + 4 * jw.y;
          T rv[4];
          load_vec4(rr + 4 * jw.x, rv);
          acc += rv[0] * tw[0] + rv[1] * tw[1] + rv[2] * tw[2] + rv[3] * tw[3];
        }
      }
      Aout[(int64_t)d * nrow + i] = acc;
    }
    __syncwarp();  // rrow and t are rewritten by the warp's next row
  }
}

// One CTA per coarse row i.  Phase 1: a half-warp per window position w;
// its 16 lanes hold the 16 entries of a 4x4 block, so every block of Ahat is
// one coalesced 64-byte (float) read, multiplied by the matching entry of
// Rhat_i from shared memory and reduced over the block's columns by two
// shuffles.  Phase 2: a warp per output offset d; its lanes walk the (j, w)
// pairs of d, reading the row Rhat_{i+S_d} with unit stride, and the dot
// product ends in a warp reduction.
template <typename T>
__global__ void __launch_bounds__(256) k_galerkin_warp(const T* __restrict__ Ahat,
                                                  const T* __restrict__ Rhat,
                                                  const uint32_t* __restrict__ pmask,
                                                  GalerkinGeom g, T* __restrict__ Aout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rrow = reinterpret_cast<T*>(smem_raw);
  T* t = rrow + 4 * g.NB;
  const int64_t nrow = g.nrow;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int half = threadIdx.x >> 4, nhalf = blockDim.x >> 4;
  const int e = threadIdx.x & 15, cb = e & 3;  // block entry (a = e >> 2, column cb)
  const unsigned hmask = 0xffffu << (16 * (half & 1));
  for (int64_t i = g.i_begin + blockIdx.x; i < g.i_end; i += gridDim.x) {
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
    for (int w = half; w < g.nwin; w += nhalf) {
      const int p = shift_cell(xi, yi, g.win[w].x, g.win[w].y, g.Lpar, nrow);
      T acc = 0;
      if (p >= 0) {
        const int e0 = g.l1_ptr[w], e1 = g.l1_ptr[w + 1];
        for (int q = e0; q < e1; ++q) {
          const int2 jo = g.l1_pairs[q];
          acc += __ldg(Ahat + ((int64_t)jo.y * nrow + p) * 16 + e) * rrow[4 * jo.x + cb];
        }
      }
      acc += __shfl_xor_sync(hmask, acc, 1);
      acc += __shfl_xor_sync(hmask, acc, 2);
      if (cb == 0) t[4 * w + (e >> 2)] = acc;
    }
    __syncthreads();
    // A_{i, i+S_d} = Rhat_{i+S_d} . t_i
    for (int d = warp; d < g.nout; d += nwarp) {
      const int ip = shift_cell(xi, yi, g.out[d].x, g.out[d].y, g.Lpar, nrow);
      T acc = 0;
      if (ip >= 0 && (pmask[ip] & 15u)) {
        const T* rr = Rhat + (int64_t)ip * 4 * g.NB;
        const int e1 = g.l2_ptr[d + 1];
        for (int q = g.l2_ptr[d] + lane; q < e1; q += 32) {
          const int2 jw = g.l2_pairs[q];
          T rv[4];
          load_vec4(rr + 4 * jw.x, rv);
          const T* tw = t + 4 * jw.y;
          acc += rv[0] * tw[0] + rv[1] * tw[1] + rv[2] * tw[2] + rv[3] * tw[3];
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) Aout[(int64_t)d * nrow + i] = acc;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_galerkin(const T* Ahat, const T* Rhat, const uint32_t* pmask_k, GalerkinGeom g,
                     T* Aout, cudaStream_t s) {
  const int64_t nrows = g.i_end - g.i_begin;
  if (nrows <= 0) return;
  size_t smem = sizeof(T) * 4 * ((size_t)g.NB + (size_t)g.nwin);
  int64_t grid = nrows < 65535 * 16 ? nrows : 65535 * 16;
  count_launch();
  if (g.variant >= 3) {
    // 3, 4, 5: the tile kernel with 8, 4 or 16 lanes per output target;
    // 6, 7, 8: the same with 4, 8 or 16 lanes per horizontal pair of targets
    const size_t st = galerkin_tile_smem_bytes(g, sizeof(T));
    void (*kern)(const T*, const T*, const uint32_t*, GalerkinGeom, T*) =
        g.variant == 4   ? k_galerkin_tile<T, 4, false>
        : g.variant == 5 ? k_galerkin_tile<T, 16, false>
        : g.variant == 6 ? k_galerkin_tile<T, 4, true>
        : g.variant == 7 ? k_galerkin_tile<T, 8, true>
        : g.variant == 8 ? k_galerkin_tile<T, 16, true>
                         : k_galerkin_tile<T, 8, false>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st);
    const int64_t nt = ((g.i_end + 3) >> 2) - (g.i_begin >> 2);
    const int threads = g.tile_threads == 128 ? 128 : 256;
    kern<<<(unsigned)(nt < 65535 * 16 ? nt : 65535 * 16), threads, st, s>>>(Ahat, Rhat, pmask_k,
                                                                           g, Aout);
  } else if (g.variant == 2) {
    const size_t smem8 = 8 * smem;  // eight warps, one row each
    cudaFuncSetAttribute(k_galerkin_warprow<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem8);
    const int64_t g8 = (nrows + 7) / 8;
    k_galerkin_warprow<T><<<(unsigned)(g8 < 65535 * 16 ? g8 : 65535 * 16), 256, smem8, s>>>(
        Ahat, Rhat, pmask_k, g, Aout);
  } else if (g.variant == 1) {
    cudaFuncSetAttribute(k_galerkin_warp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_galerkin_warp<T><<<(unsigned)grid, 256, smem, s>>>(Ahat, Rhat, pmask_k, g, Aout);
  } else {
    cudaFuncSetAttribute(k_galerkin_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_galerkin_rows<T><<<(unsigned)grid, 256, smem, s>>>(Ahat, Rhat, pmask_k, g, Aout);
  }
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
  const int PP = shift_cell(x, y, Ooff[o].x, Ooff[o].y, Lpar, npar);
  const int mr = (int)pmask[P] & 15;
  const int mc = PP >= 0 ? (int)pmask[PP] & 15 : 0;
  // the transform runs in the working precision: float64 arithmetic would
  // make this memory-bound kernel wait on the float64 pipe in the mixed path
  T M[16], Tm[16], Qr[16], Qc[16];
  qmat<T>(mr, Qr);
  qmat<T>(mc, Qc);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int d = map[o * 16 + c * 4 + cc];
      T v = T(0);
      // only existing cells are read (the last parent of a prefix may have
      // children beyond the ncell rows of Acell)
      if (PP >= 0 && ((mr >> c) & 1) && ((mc >> cc) & 1)) {
        if (d >= 0) v = Acell[(int64_t)d * ncell + 4 * P + c];
        else if (d <= -2) v = Acell[(int64_t)(-d - 2) * ncell + 4 * PP + cc];
      }
      M[c * 4 + cc] = v;
    }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      T acc = 0;
#pragma unroll
      for (int c = 0; c < 4; ++c) acc += Qr[a * 4 + c] * M[c * 4 + cc];
      Tm[a * 4 + cc] = acc;
    }
  T* out = blk + t * 16;  // 16-byte aligned: one vector store per output row
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    T row[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      T acc = 0;
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) acc += Tm[a * 4 + cc] * Qc[b * 4 + cc];
      row[b] = acc;
    }
    sst4(out + 4 * a, row);
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

