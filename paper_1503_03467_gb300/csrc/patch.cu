// patch.cu - localized patch solves (Sec. 5.3, Definition defb; Algorithm 2,
// line 11) and the interpolation rows they define (Eq. eqhuhiddeuv).
//
// For each coarse cell i of level k-1 the patch i^rho holds NB neighbour
// parents p_j = i + N_j (level-(k-1) cells, i.e. level-k parents).  In the
// transformed basis Ahat = Q A^(k) Q^T the patch matrix is
//   B^(i,rho)[(j,t),(j',t')] = Ahat[(p_j, t), (p_j', t')],  t, t' < 3,
// the right-hand side is
//   b_(j,t) = -(W A pibar^T)_{(j,t), i} = -Ahat[(p_j, t), (i, 3)] / sqrt(m_i),
// and the solution y gives the interpolation row in the transformed basis:
//   Rhat[i][(p_j, t)] = y_(j,t),  Rhat[i][(i, 3)] = 1 / sqrt(m_i)
// (R = pibar + D^T W with pibar Q^T = e_(i,3) / sqrt(m_i) and W Q^T = [I 0]).
//
// Factorisation: the system is padded to n = 3 NB unknowns (unknowns whose
// parent lies outside the lattice or has fewer children are decoupled
// identity rows) and bordered by the right-hand side as the last row of
// [[B, b], [b^T, c]] with c large, so the Cholesky factor's last row is
// z = L^-1 b (the forward substitution comes free).  The lower triangle is
// stored as 8 x 8 tiles (column-major inside a tile, tile stride padded to
// an XOR swizzle against bank conflicts) and factored right-looking one tile
// column at a time: one warp factors the diagonal tile, all threads solve
// the tiles below it, then pairs of threads update the trailing tiles with
// rank-8 products held in registers (4 x 8 accumulators each; small enough
// for three float32 patches per SM).  One warp finishes
// with the tile-blocked back substitution L^T y = z.  One CTA per patch,
// persistent over the patches of the level.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

constexpr int kTile = 8;
constexpr int kTileStride = 64;
constexpr int kPatchThreads = 256;

// Element idx = 8 c + r of tile t sits at t * 64 + (idx ^ swz(t)): the XOR on
// bits 2..4 spreads equal offsets of different tiles over different bank
// groups while keeping every aligned group of four elements contiguous.
__host__ __device__ __forceinline__ int swz(int t) { return (t & 7) << 2; }

__host__ __device__ __forceinline__ int patch_rows(int NB) {
  return ((3 * NB + 1 + kTile - 1) / kTile) * kTile;  // unknowns + rhs row, padded
}
__host__ __device__ __forceinline__ int tri_tiles(int nt) { return nt * (nt + 1) / 2; }
__host__ __device__ __forceinline__ int tile_index(int I, int K) { return I * (I + 1) / 2 + K; }

template <typename T>
size_t patch_smem_bytes(int NB) {
  const int nt = patch_rows(NB) / kTile;
  size_t b = sizeof(T) * (size_t)tri_tiles(nt) * kTileStride;  // factor tiles
  b += sizeof(T) * (size_t)patch_rows(NB);                      // solution vector
  b += sizeof(T) * kTile;                                       // reciprocal pivots
  b += sizeof(int) * 2 * (size_t)NB;                            // parent index, child count
  b += sizeof(int) * (size_t)patch_rows(NB);                    // row descriptors
  return (b + 15) & ~(size_t)15;
}
template size_t patch_smem_bytes<float>(int);
template size_t patch_smem_bytes<double>(int);

template <typename T>
__device__ __forceinline__ T dev_sqrt(T v);
template <>
__device__ __forceinline__ float dev_sqrt<float>(float v) { return sqrtf(v); }
template <>
__device__ __forceinline__ double dev_sqrt<double>(double v) { return sqrt(v); }

template <typename T>
__device__ __forceinline__ T big_corner();
template <>
__device__ __forceinline__ float big_corner<float>() { return 1e30f; }
template <>
__device__ __forceinline__ double big_corner<double>() { return 1e200; }

// element (r, c), r >= c, of the tiled lower triangle
template <typename T>
__device__ __forceinline__ T& tel(T* M, int r, int c) {
  const int t = tile_index(r / kTile, c / kTile);
  return M[t * kTileStride + (((c % kTile) * kTile + (r % kTile)) ^ swz(t))];
}

// float32: three CTAs per SM (registers <= 85); float64 is ALU-bound anyway.
template <typename T>
struct PatchOcc {
  static constexpr int kMinBlocks = 1;
};
template <>
struct PatchOcc<float> {
  static constexpr int kMinBlocks = 3;
};

template <typename T>
__global__ void __launch_bounds__(kPatchThreads, PatchOcc<T>::kMinBlocks)
    k_patch_solve(const T* __restrict__ Ahat,
                                                               const uint32_t* __restrict__ pmask,
                                                               PatchGeom g, T* __restrict__ Rhat,
                                                               int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = g.NB;
  const int n = 3 * NB;               // patch unknowns (padded layout)
  const int N1 = patch_rows(NB);      // rows incl. padding and the rhs row
  const int NT = N1 / kTile;
  const int rhs = N1 - 1;             // the bordering row
  T* M = reinterpret_cast<T*>(smem_raw);
  T* y = M + tri_tiles(NT) * kTileStride;
  T* rinv = y + N1;
  int* pj = reinterpret_cast<int*>(rinv + kTile);
  int* mj = pj + NB;
  int* rowd = mj + NB;  // (j << 2 | t) of an active unknown, -1 otherwise
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarp = kPatchThreads / 32;
  const int64_t np = g.npatch;

  for (int64_t i = blockIdx.x; i < np; i += gridDim.x) {
    const uint32_t mi = pmask[i] & 15u;
    if (mi == 0) {  // empty coarse cell: no gamblet
      for (int idx = tid; idx < NB * 4; idx += kPatchThreads) Rhat[i * 4 * NB + idx] = T(0);
      continue;
    }
    const T inv_sqrt_mi = T(1) / dev_sqrt<T>(T(__popc(mi)));
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    for (int j = tid; j < NB; j += kPatchThreads) {
      const int p = shift_cell(xi, yi, g.nbr[j].x, g.nbr[j].y, g.Lpar, g.npatch);
      pj[j] = p;
      mj[j] = p >= 0 ? __popc(pmask[p] & 15u) : 0;
    }
    __syncthreads();

    for (int r = tid; r < N1; r += kPatchThreads) {
      int d = -1;
      if (r < n) {
        const int j = r / 3, t = r - 3 * j;
        if (pj[j] >= 0 && t < mj[j] - 1) d = (j << 2) | t;
      }
      rowd[r] = d;
    }
    __syncthreads();

    // ---- gather [B b; b^T c] into the tiles (lower triangle)
    for (int r = warp; r < N1; r += nwarp) {
      const int da = rowd[r];
      if (r < n) {
        const int ja = da >> 2, ta = da & 3;
        const int pa = da >= 0 ? pj[ja] : 0;
        const int* prow = g.pair_idx + ja * NB;
        for (int c = lane; c <= r; c += 32) {
          const int db = rowd[c];
          T v;
          if (da >= 0 && db >= 0) {
            const int o = prow[db >> 2];
            v = o >= 0 ? Ahat[((int64_t)o * np + pa) * 16 + ta * 4 + (db & 3)] : T(0);
          } else {
            v = (r == c) ? T(1) : T(0);
          }
          tel(M, r, c) = v;
        }
      } else if (r < rhs) {  // padding rows: identity
        for (int c = lane; c <= r; c += 32) tel(M, r, c) = (r == c) ? T(1) : T(0);
      } else {  // bordering row b^T and the corner
        for (int c = lane; c <= r; c += 32) {
          T v = T(0);
          const int db = c < n ? rowd[c] : -1;
          if (db >= 0) {
            const int jb = db >> 2;
            const int o = g.pair_idx[jb * NB + g.jc];
            if (o >= 0) v = -inv_sqrt_mi * Ahat[((int64_t)o * np + pj[jb]) * 16 + (db & 3) * 4 + 3];
          } else if (c == rhs) {
            v = big_corner<T>();
          }
          tel(M, r, c) = v;
        }
      }
    }
    __syncthreads();

    // ---- right-looking tiled Cholesky
    for (int J = 0; J < NT; ++J) {
      const int tJ = tile_index(J, J);
      T* D = M + tJ * kTileStride;
      const int sJ = swz(tJ);
      // (1) diagonal tile, one warp; lane l < 8 owns row l during the sweep
      if (warp == 0) {
        for (int c = 0; c < kTile; ++c) {
          T d = D[(c * kTile + c) ^ sJ];
          if (!(d > T(0))) {
            if (lane == 0) atomicExch(status, (int)DEV_NOT_SPD);
            d = T(1);
          }
          const T s = dev_sqrt<T>(d);
          const T is = T(1) / s;
          __syncwarp();
          if (lane == 0) {
            D[(c * kTile + c) ^ sJ] = s;
            rinv[c] = is;
          }
          if (lane > c && lane < kTile) D[(c * kTile + lane) ^ sJ] *= is;
          __syncwarp();
          // rank-1 update of the remaining lower part: lanes cover (r, cc), c < cc <= r < 8
          for (int e = lane; e < kTile * kTile; e += 32) {
            const int r = e % kTile, cc = e / kTile;
            if (cc > c && r >= cc)
              D[(cc * kTile + r) ^ sJ] -= D[(c * kTile + r) ^ sJ] * D[(c * kTile + cc) ^ sJ];
          }
          __syncwarp();
        }
      }
      __syncthreads();
      // (2) tiles below: L_IJ = A_IJ L_JJ^-T, one thread per row
      const int below = (NT - 1 - J) * kTile;
      for (int t = tid; t < below; t += kPatchThreads) {
        const int I = J + 1 + t / kTile, rr = t % kTile;
        const int tI = tile_index(I, J), sI = swz(tI);
        T* A = M + tI * kTileStride;
        T x[kTile];
#pragma unroll
        for (int c = 0; c < kTile; ++c) {
          T v = A[(c * kTile + rr) ^ sI];
#pragma unroll
          for (int cp = 0; cp < c; ++cp) v -= D[(cp * kTile + c) ^ sJ] * x[cp];
          x[c] = v * rinv[c];
        }
#pragma unroll
        for (int c = 0; c < kTile; ++c) A[(c * kTile + rr) ^ sI] = x[c];
      }
      __syncthreads();
      // (3) trailing update: A_IK -= L_IJ L_KJ^T for J < K <= I; two threads
      //     per tile, each owning 4 rows x 8 columns in registers
      const int m = NT - 1 - J;
      const int count = m * (m + 1) / 2;
      for (int t2 = tid; t2 < 2 * count; t2 += kPatchThreads) {
        const int t = t2 >> 1, half = t2 & 1;
        int ii = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
        while (ii * (ii + 1) / 2 > t) --ii;
        while ((ii + 1) * (ii + 2) / 2 <= t) ++ii;
        const int kk = t - ii * (ii + 1) / 2;
        const int I = J + 1 + ii, K = J + 1 + kk;
        const int tI = tile_index(I, J), tK = tile_index(K, J), tC = tile_index(I, K);
        const int sI = swz(tI), sK = swz(tK), sC = swz(tC);
        const T* LI = M + tI * kTileStride;
        const T* LK = M + tK * kTileStride;
        T* C = M + tC * kTileStride;
        const int h4 = 4 * half;
        T acc[4][kTile];
#pragma unroll
        for (int c = 0; c < kTile; ++c) {
          const T* cp = C + ((c * kTile + h4) ^ sC);
#pragma unroll
          for (int r = 0; r < 4; ++r) acc[r][c] = cp[r];
        }
#pragma unroll
        for (int q = 0; q < kTile; ++q) {
          T a[4], b[kTile];
          const T* ap = LI + ((q * kTile + h4) ^ sI);
          const T* b0 = LK + ((q * kTile) ^ sK);
          const T* b1 = LK + ((q * kTile + 4) ^ sK);
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = ap[r];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            b[c] = b0[c];
            b[c + 4] = b1[c];
          }
#pragma unroll
          for (int c = 0; c < kTile; ++c)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r][c] -= a[r] * b[c];
        }
#pragma unroll
        for (int c = 0; c < kTile; ++c) {
          T* cp = C + ((c * kTile + h4) ^ sC);
#pragma unroll
          for (int r = 0; r < 4; ++r) cp[r] = acc[r][c];
        }
      }
      __syncthreads();
    }

    // ---- back substitution L^T y = z (z = bordering row), one warp
    if (warp == 0) {
      for (int c = lane; c < rhs; c += 32) y[c] = tel(M, rhs, c);
      __syncwarp();
      for (int I = NT - 1; I >= 0; --I) {
        const int r0 = I * kTile;
        const int r1 = min(r0 + kTile, rhs);  // exclusive; skips the bordering row
        const int tD = tile_index(I, I), sD = swz(tD);
        const T* Dt = M + tD * kTileStride;
        if (lane == 0) {
          for (int r = r1 - 1; r >= r0; --r) {
            T v = y[r];
            for (int rp = r + 1; rp < r1; ++rp) v -= Dt[((r - r0) * kTile + (rp - r0)) ^ sD] * y[rp];
            y[r] = v / Dt[((r - r0) * kTile + (r - r0)) ^ sD];
          }
        }
        __syncwarp();
        // subtract block I's contribution from the rows above it
        for (int c = lane; c < r0; c += 32) {
          const int tL = tile_index(I, c / kTile), sL = swz(tL);
          const T* Lt = M + tL * kTileStride;
          const int cb = (c % kTile) * kTile;
          T v = y[c];
          for (int r = r0; r < r1; ++r) v -= Lt[(cb + r - r0) ^ sL] * y[r];
          y[c] = v;
        }
        __syncwarp();
      }
    }
    __syncthreads();

    // ---- interpolation row of coarse cell i (row-contiguous [j][slot])
    for (int idx = tid; idx < NB * 4; idx += kPatchThreads) {
      const int j = idx >> 2, c = idx & 3;
      T v = T(0);
      if (c < 3) {
        if (pj[j] >= 0 && c < mj[j] - 1) v = y[3 * j + c];
      } else if (j == g.jc) {
        v = inv_sqrt_mi;
      }
      Rhat[i * 4 * NB + idx] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Block-Jacobi preconditioned CG on the patch system (the iterative solve
// Sec. 5.4 proposes for Alg. 2 line 11, to the accuracy Thm tmdiscreteaccuracy
// allows).  The preconditioner inverts each neighbour parent's 3x3 diagonal
// detail block; for rough coefficients this leaves a condition number of a
// few units, so a handful of iterations reach the tolerance.
//
// The patch matrix is stored as its nonzero 3x3 blocks: one block per
// neighbour pair (ja >= jb) whose offset N_jb - N_ja lies in O_k (host list
// `half`), so the finest level, where A^(q) is a 9-point operator, keeps ~8x
// fewer entries than the dense patch.  Thread j owns neighbour parent j: its
// three unknowns, their residuals and its 3x3 block-Jacobi inverse live in
// registers, so the preconditioner needs no communication; the block row of
// j is walked through a compact adjacency list (stored block, other
// neighbour, transposed flag) staged once per CTA in shared memory, split
// over `spp` adjacent lanes when block rows are long (dense coarse levels).
// Reductions run in the working precision (float32 in the mixed path, where
// the patch factorisations accumulate in float32).
template <typename T>
size_t patch_pcg_smem_bytes(const PatchPcgGeom& pg) {
  const int nadj = pg.nadj;
  size_t b = sizeof(T) * 9 * (size_t)pg.nhalf;           // stored blocks (slots)
  b += sizeof(T) * 3 * (size_t)pg.NB;                     // shared direction vector
  b += sizeof(int) * ((size_t)nadj + pg.NB + 1);          // adjacency (packed) + row pointers
  b += sizeof(int) * 2 * (size_t)pg.NB;                   // parent index, active unknowns
  b += sizeof(double) * 24 + 16;                          // reduction slots
  return (b + 15) & ~(size_t)15;
}
template size_t patch_pcg_smem_bytes<float>(const PatchPcgGeom&);
template size_t patch_pcg_smem_bytes<double>(const PatchPcgGeom&);

// One 4-entry row of a 4x4 block (16-byte aligned) as vector loads.
__device__ __forceinline__ void load_row4(const float* p, float* r) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}
__device__ __forceinline__ void load_row4(const double* p, double* r) {
  const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  r[0] = v0.x;
  r[1] = v0.y;
  r[2] = v1.x;
  r[3] = v1.y;
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block sums for at most eight warps.  Each warp's lane 0 writes its partial
// into a slot array that is zero past the warp count, and every thread then
// reads the whole array as 16-byte broadcasts (two to eight loads instead of
// one per warp and value).  Consecutive reductions alternate between two slot
// arrays, so one barrier per reduction suffices: a thread writes a slot array
// again only after the barrier of the reduction in between, which every
// thread reaches after reading it.
__device__ __forceinline__ float sum8(const float* r) {
  const float4 u = *reinterpret_cast<const float4*>(r);
  const float4 v = *reinterpret_cast<const float4*>(r + 4);
  return ((u.x + u.y) + (u.z + u.w)) + ((v.x + v.y) + (v.z + v.w));
}
__device__ __forceinline__ double sum8(const double* r) {
  double t = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const double2 u = reinterpret_cast<const double2*>(r)[w];
    t += u.x + u.y;
  }
  return t;
}
// slots (a_w, b_w) interleaved, 16 entries
__device__ __forceinline__ void sum8x2(const float* r, float& a, float& b) {
  a = 0;
  b = 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const float4 u = reinterpret_cast<const float4*>(r)[w];
    a += u.x + u.z;
    b += u.y + u.w;
  }
}
__device__ __forceinline__ void sum8x2(const double* r, double& a, double& b) {
  a = 0;
  b = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const double2 u = reinterpret_cast<const double2*>(r)[w];
    a += u.x;
    b += u.y;
  }
}

// sum over the block of a (every thread gets it); red1: 8 slots
template <typename T>
__device__ __forceinline__ T block_sum1(T a, T* red1) {
  a = warp_sum_t(a);
  if ((threadIdx.x & 31) == 0) red1[threadIdx.x >> 5] = a;
  __syncthreads();
  return sum8(red1);
}
// sum over the block of a and b (every thread gets both); red2: 16 slots
template <typename T>
__device__ __forceinline__ void block_sum2(T& a, T& b, T* red2) {
  a = warp_sum_t(a);
  b = warp_sum_t(b);
  if ((threadIdx.x & 31) == 0) {
    red2[2 * (threadIdx.x >> 5)] = a;
    red2[2 * (threadIdx.x >> 5) + 1] = b;
  }
  __syncthreads();
  sum8x2(red2, a, b);
}

// kAdj: the same patch systems with the right-hand side b_i read from
// adj_rhs ([i][NB][4], detail slots) and the solution written to Rhat's
// layout with a zero average slot (the adjoint solves of the reverse pass).
template <typename T, int kGather, bool kAdj>
__global__ void __launch_bounds__(256, 3) k_patch_pcg(const T* __restrict__ Ahat,
                                                   const uint32_t* __restrict__ pmask,
                                                   PatchPcgGeom g, T* __restrict__ Rhat,
                                                   double tol2, int max_iter, int* iter_stats,
                                                   const T* __restrict__ adj_rhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = g.NB;
  const int nadj = g.nadj;
  T* blk = reinterpret_cast<T*>(smem_raw);
  T* sv = blk + 9 * g.nhalf;
  int* sadj = reinterpret_cast<int*>(sv + 3 * NB);
  int* sptr = sadj + nadj;
  int* pj = sptr + NB + 1;
  int* mj = pj + NB;
  T* red = reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(mj + NB) + 15) & ~(uintptr_t)15);
  T* red1 = red;       // 8 slots: p.q
  T* red2 = red + 8;   // 16 slots: (r.z, r.r)
  const int tid = threadIdx.x;
  if (tid < 24) red[tid] = T(0);  // slots of absent warps stay zero
  const int64_t np = g.npatch;
  const int S = g.spp;  // threads per neighbour parent (lanes of one warp)
  // patch structure, identical for every patch of the level
  for (int e = tid; e < nadj; e += blockDim.x) {
    const int4 ad = g.adj[e];  // (stored block, other neighbour, transposed, -)
    sadj[e] = (ad.x << 9) | (ad.y << 1) | ad.z;
  }
  for (int j = tid; j <= NB; j += blockDim.x) sptr[j] = g.adj_ptr[j];
  __syncthreads();
  const int j = tid / S, sub = tid - (tid / S) * S;
  const bool own = j < NB;
  const bool lead = own && sub == 0;  // writes and reductions
  const int e0 = own ? sptr[j] : 0, e1 = own ? sptr[j + 1] : 0;
  int it_max = 0, it_sum = 0, done = 0;

  for (int64_t i = g.i_begin + blockIdx.x; i < g.i_end; i += gridDim.x) {
    const uint32_t mi = pmask[i] & 15u;
    if (mi == 0) {
      for (int idx = tid; idx < NB * 4; idx += blockDim.x) Rhat[i * 4 * NB + idx] = T(0);
      continue;
    }
    const T inv_sqrt_mi = T(1) / dev_sqrt<T>(T(__popc(mi)));
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    int na = 0, pjj = -1;
    if (own) {
      pjj = shift_cell(xi, yi, g.nbr[j].x, g.nbr[j].y, g.Lpar, g.npatch);
      const int m = pjj >= 0 ? __popc(pmask[pjj] & 15u) : 0;
      na = m > 1 ? m - 1 : 0;  // active detail unknowns of neighbour j
      if (lead) {
        pj[j] = pjj;
        mj[j] = na;
      }
    }
    __syncthreads();
    // ---- gather the stored blocks (identity on inactive diagonal entries).
    // kGather 0: a thread per block with nine scalar reads (many reads in
    // flight per thread, one L1 wavefront per scattered sector); 1: a
    // half-warp per block, lane (a, b) reading entry (a, b), one coalesced
    // read per block; 2: four lanes per block, one 16-byte row each, four
    // blocks in flight per group.
    if (kGather == 2) {
      // four lanes per block, lane a loading row a as one 16-byte vector;
      // each group of four lanes keeps four blocks in flight
      const int grp = tid >> 2, ngrp = blockDim.x >> 2, a = tid & 3;
      for (int h0 = grp; h0 < g.nhalf; h0 += 4 * ngrp) {
        T row[4][4];
        int4 ent[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int h = h0 + u * ngrp;
          ent[u] = h < g.nhalf ? g.half[h] : make_int4(-1, -1, 0, 0);
          const int nra = ent[u].x >= 0 ? mj[ent[u].x] : 0;
          const int nrb = ent[u].x >= 0 ? mj[ent[u].y] : 0;
#pragma unroll
          for (int b = 0; b < 4; ++b) row[u][b] = T(0);
          if (a < nra && nrb > 0)
            load_row4(Ahat + ((int64_t)ent[u].z * np + pj[ent[u].x]) * 16 + 4 * a, row[u]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int h = h0 + u * ngrp;
          if (h >= g.nhalf || ent[u].x < 0 || a >= 3) continue;
          const int nra = mj[ent[u].x], nrb = mj[ent[u].y];
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            T v = (a < nra && b < nrb) ? row[u][b] : T(0);
            if (ent[u].x == ent[u].y && a == b && a >= nra) v = T(1);
            blk[9 * h + 3 * a + b] = v;
          }
        }
      }
    } else if (kGather == 0) {
      for (int h = tid; h < g.nhalf; h += blockDim.x) {
        const int4 e = g.half[h];  // (ja, jb, o, -); ja < 0 marks a padding slot
        if (e.x < 0) continue;
        const int nra = mj[e.x], nrb = mj[e.y];
        const T* src = Ahat + ((int64_t)e.z * np + (nra > 0 ? pj[e.x] : 0)) * 16;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            T v = (a < nra && b < nrb) ? __ldg(src + 4 * a + b) : T(0);
            if (e.x == e.y && a == b && a >= nra) v = T(1);
            blk[9 * h + 3 * a + b] = v;
          }
      }
    } else {
      const int hw = tid >> 4, nhw = blockDim.x >> 4;
      const int a = (tid >> 2) & 3, b = tid & 3;
      for (int h = hw; h < g.nhalf; h += nhw) {
        const int4 e = g.half[h];  // (ja, jb, o, -); ja < 0 marks a padding slot
        if (e.x < 0) continue;
        const int nra = mj[e.x], nrb = mj[e.y];
        if (a < 3 && b < 3) {
          T v = T(0);
          if (a < nra && b < nrb) v = __ldg(Ahat + ((int64_t)e.z * np + pj[e.x]) * 16 + 4 * a + b);
          else if (e.x == e.y && a == b) v = T(1);
          blk[9 * h + 3 * a + b] = v;
        }
      }
    }
    // ---- right-hand side of neighbour j
    T rv[3] = {T(0), T(0), T(0)};
    if (kAdj) {
      if (own && na > 0) {
        const T* b = adj_rhs + i * 4 * NB + 4 * j;
#pragma unroll
        for (int t = 0; t < 3; ++t) rv[t] = t < na ? b[t] : T(0);
      }
    } else if (own && na > 0) {
      const int o = g.pair_idx[j * NB + g.jc];
      if (o >= 0) {
        const T* bl = Ahat + ((int64_t)o * np + pjj) * 16;
#pragma unroll
        for (int t = 0; t < 3; ++t) rv[t] = t < na ? -inv_sqrt_mi * bl[4 * t + 3] : T(0);
      }
    }
    __syncthreads();
    // ---- block-Jacobi inverse of j's diagonal block (Gauss-Jordan, registers)
    T Di[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Di[q] = (q % 4 == 0) ? T(1) : T(0);
    if (own) {
      T Mm[9];
      const T* D = blk + 9 * g.diag_h[j];
#pragma unroll
      for (int q = 0; q < 9; ++q) Mm[q] = D[q];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const T d = Mm[4 * c] > T(0) ? Mm[4 * c] : T(1);
        const T id = T(1) / d;
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) {
          Mm[3 * c + b2] *= id;
          Di[3 * c + b2] *= id;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a == c) continue;
          const T f = Mm[3 * a + c];
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2) {
            Mm[3 * a + b2] -= f * Mm[3 * c + b2];
            Di[3 * a + b2] -= f * Di[3 * c + b2];
          }
        }
      }
    }
    // ---- PCG
    T xv[3] = {T(0), T(0), T(0)}, zv[3], pv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) zv[a] = Di[3 * a] * rv[0] + Di[3 * a + 1] * rv[1] + Di[3 * a + 2] * rv[2];
    T rz = lead ? rv[0] * zv[0] + rv[1] * zv[1] + rv[2] * zv[2] : T(0);
    T rr0 = lead ? rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2] : T(0);
    block_sum2<T>(rz, rr0, red2);
#pragma unroll
    for (int a = 0; a < 3; ++a) pv[a] = zv[a];
    int it = 0;
    if (rr0 > T(0)) {
      for (it = 1; it <= max_iter; ++it) {
        if (lead) {
          sv[3 * j] = pv[0];
          sv[3 * j + 1] = pv[1];
          sv[3 * j + 2] = pv[2];
        }
        __syncthreads();
        T q0 = 0, q1 = 0, q2 = 0;
        for (int e = e0 + sub; e < e1; e += S) {
          const int ad = sadj[e];
          const T* B = blk + 9 * (ad >> 9);
          const T* ps = sv + 3 * ((ad >> 1) & 255);
          const T p0 = ps[0], p1 = ps[1], p2 = ps[2];
          if (ad & 1) {
            q0 += B[0] * p0 + B[3] * p1 + B[6] * p2;
            q1 += B[1] * p0 + B[4] * p1 + B[7] * p2;
            q2 += B[2] * p0 + B[5] * p1 + B[8] * p2;
          } else {
            q0 += B[0] * p0 + B[1] * p1 + B[2] * p2;
            q1 += B[3] * p0 + B[4] * p1 + B[5] * p2;
            q2 += B[6] * p0 + B[7] * p1 + B[8] * p2;
          }
        }
        for (int o = 1; o < S; o <<= 1) {  // combine the S partial products
          q0 += __shfl_xor_sync(0xffffffffu, q0, o);
          q1 += __shfl_xor_sync(0xffffffffu, q1, o);
          q2 += __shfl_xor_sync(0xffffffffu, q2, o);
        }
        const T pq = block_sum1<T>(lead ? pv[0] * q0 + pv[1] * q1 + pv[2] * q2 : T(0), red1);
        const T alpha = pq > T(0) ? rz / pq : T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) xv[a] += alpha * pv[a];
        rv[0] -= alpha * q0;
        rv[1] -= alpha * q1;
        rv[2] -= alpha * q2;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          zv[a] = Di[3 * a] * rv[0] + Di[3 * a + 1] * rv[1] + Di[3 * a + 2] * rv[2];
        T rz_new = lead ? rv[0] * zv[0] + rv[1] * zv[1] + rv[2] * zv[2] : T(0);
        T rr = lead ? rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2] : T(0);
        block_sum2<T>(rz_new, rr, red2);
        if ((double)rr <= tol2 * (double)rr0 || !(rz_new > T(0))) break;
        const T beta = rz_new / rz;
        rz = rz_new;
#pragma unroll
        for (int a = 0; a < 3; ++a) pv[a] = zv[a] + beta * pv[a];
      }
      if (it > max_iter) it = max_iter;
    }
    it_max = max(it_max, it);
    it_sum += it;
    ++done;
    // ---- interpolation row: detail coefficients of neighbour j and the average slot
    if (lead) {
      T* row = Rhat + i * 4 * NB + 4 * j;
#pragma unroll
      for (int t = 0; t < 3; ++t) row[t] = t < na ? xv[t] : T(0);
      row[3] = (!kAdj && j == g.jc) ? inv_sqrt_mi : T(0);
    }
    __syncthreads();
  }
  if (tid == 0 && iter_stats) {
    atomicMax(&iter_stats[0], it_max);
    atomicAdd(&iter_stats[1], it_sum);
    atomicAdd(&iter_stats[2], done);
  }
}

template <typename T>
void launch_patch_pcg(const T* Ahat, const uint32_t* pmask_k, PatchPcgGeom g, T* Rhat, double tol,
                      int max_iter, int* iter_stats, int num_sms, cudaStream_t s) {
  const int64_t nsolve = g.i_end - g.i_begin;
  if (nsolve <= 0) return;
  const size_t smem = patch_pcg_smem_bytes<T>(g);
  auto kern = g.gather == 2 ? k_patch_pcg<T, 2, false>
                            : (g.gather == 1 ? k_patch_pcg<T, 1, false> : k_patch_pcg<T, 0, false>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int threads = ((g.NB * g.spp + 31) / 32) * 32;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > nsolve) grid = nsolve;
  {
    count_launch();
    kern<<<(unsigned)grid, threads, smem, s>>>(Ahat, pmask_k, g, Rhat, tol * tol, max_iter,
                                               iter_stats, nullptr);
  }
}

template <typename T>
void launch_patch_pcg_adjoint(const T* Ahat, const uint32_t* pmask_k, PatchPcgGeom g,
                              const T* rhs, T* out, double tol, int max_iter, int* iter_stats,
                              int num_sms, cudaStream_t s) {
  const int64_t nsolve = g.i_end - g.i_begin;
  if (nsolve <= 0) return;
  const size_t smem = patch_pcg_smem_bytes<T>(g);
  auto kern = g.gather == 2 ? k_patch_pcg<T, 2, true>
                            : (g.gather == 1 ? k_patch_pcg<T, 1, true> : k_patch_pcg<T, 0, true>);
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int threads = ((g.NB * g.spp + 31) / 32) * 32;
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > nsolve) grid = nsolve;
  count_launch();
  kern<<<(unsigned)grid, threads, smem, s>>>(Ahat, pmask_k, g, out, tol * tol, max_iter,
                                             iter_stats, rhs);
}
template void launch_patch_pcg_adjoint<float>(const float*, const uint32_t*, PatchPcgGeom,
                                              const float*, float*, double, int, int*, int,
                                              cudaStream_t);
template void launch_patch_pcg_adjoint<double>(const double*, const uint32_t*, PatchPcgGeom,
                                               const double*, double*, double, int, int*, int,
                                               cudaStream_t);
template void launch_patch_pcg<float>(const float*, const uint32_t*, PatchPcgGeom, float*, double,
                                      int, int*, int, cudaStream_t);
template void launch_patch_pcg<double>(const double*, const uint32_t*, PatchPcgGeom, double*,
                                       double, int, int*, int, cudaStream_t);

template <typename T>
void launch_patch_solve(const T* Ahat, const uint32_t* pmask_k, PatchGeom g, T* Rhat,
                        int* status, int num_sms, cudaStream_t s) {
  if (g.npatch <= 0) return;
  size_t smem = patch_smem_bytes<T>(g.NB);
  cudaFuncSetAttribute(k_patch_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_solve<T>, kPatchThreads, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > g.npatch) grid = g.npatch;
  { count_launch(); k_patch_solve<T><<<(unsigned)grid, kPatchThreads, smem, s>>>(Ahat, pmask_k, g, Rhat, status); }
}
template void launch_patch_solve<float>(const float*, const uint32_t*, PatchGeom, float*, int*,
                                        int, cudaStream_t);
template void launch_patch_solve<double>(const double*, const uint32_t*, PatchGeom, double*,
                                         int*, int, cudaStream_t);

}  // namespace gb
