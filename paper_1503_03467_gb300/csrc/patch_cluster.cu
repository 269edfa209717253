// patch_cluster.cu - localized patch solves (Sec. 5.3, Definition defb;
// Algorithm 2, line 11) for patches whose blocks exceed one CTA's shared
// memory: larger radii rho (the localization error decays with rho, Sec. 4.10
// Theorem thmerrorpropagation, so rho has to grow like ln(1/eps)), and the
// float64 path from rho = 4 on.
//
// A thread-block cluster of cs CTAs (cs = 2, 4, 8 or 16 on one GPU) solves
// one patch at a time.  The neighbour parents j of the patch are split into cs
// contiguous ranges; CTA c keeps, in its own shared memory, every nonzero 3x3
// block (j, jb) of the patch matrix for the rows j it owns (both orientations,
// read straight from the block stencil Ahat, which stores every offset), and
// one warp per owned row computes that row of each matrix product.  Every CTA
// holds a full copy of the CG direction vector: after each update the owner
// of row j writes p_j into the copies of all cs CTAs (distributed shared
// memory).  Inner products are summed per CTA, the cs partial sums are
// exchanged the same way and added in rank order, so every CTA takes the
// same decisions.  The iteration is the block-Jacobi preconditioned CG of the
// single-CTA kernel (patch.cu), with the same stopping rule.
#include <cooperative_groups.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace gb {

namespace {

template <typename T>
__device__ __forceinline__ T warp_sum_c(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T csqrt(T v);
template <>
__device__ __forceinline__ float csqrt<float>(float v) { return sqrtf(v); }
template <>
__device__ __forceinline__ double csqrt<double>(double v) { return sqrt(v); }

struct ClusterLayout {
  size_t blk, pall, pj, mj, sadj, slots, red, total;
};

__host__ __device__ __forceinline__ size_t take_bytes(size_t& off, size_t bytes) {
  const size_t at = off;
  off = (off + bytes + 15) & ~(size_t)15;
  return at;
}

template <typename T>
__host__ __device__ ClusterLayout cluster_layout(const PatchClusterGeom& c) {
  ClusterLayout L{};
  size_t off = 0;
  auto take = [&off](size_t bytes) { return take_bytes(off, bytes); };
  const int NB = c.pg.NB;
  L.blk = take(sizeof(T) * 9 * (size_t)c.max_blocks);
  L.pall = take(sizeof(T) * 3 * (size_t)NB);
  L.pj = take(sizeof(int) * (size_t)NB);
  L.mj = take(sizeof(int) * (size_t)NB);
  L.sadj = take(sizeof(int) * (size_t)c.max_blocks);
  L.slots = take(sizeof(T) * 2 * 16 * 4);
  L.red = take(sizeof(T) * 32 * 4);
  L.total = off;
  return L;
}

}  // namespace

template <typename T>
size_t patch_cluster_smem_bytes(const PatchClusterGeom& c) {
  return cluster_layout<T>(c).total;
}
template size_t patch_cluster_smem_bytes<float>(const PatchClusterGeom&);
template size_t patch_cluster_smem_bytes<double>(const PatchClusterGeom&);

// Sum over the cluster of V values that lane 0 of every warp holds (zero
// elsewhere): warp partials -> CTA partial (thread 0) -> written into slot
// [rank] of every CTA's slot array `buf` -> cluster barrier -> every thread
// adds the cs slots in rank order.
template <typename T, int V>
__device__ __forceinline__ void cluster_sums(T (&v)[V], T* red, T* slots_buf, int cs, int rank,
                                             cg::cluster_group& cl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < V; ++a) red[warp * 4 + a] = v[a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T s[V];
#pragma unroll
    for (int a = 0; a < V; ++a) s[a] = T(0);
    for (int w = 0; w < nwarp; ++w)
#pragma unroll
      for (int a = 0; a < V; ++a) s[a] += red[w * 4 + a];
    for (int r = 0; r < cs; ++r) {
      T* dst = cl.map_shared_rank(slots_buf, r);
#pragma unroll
      for (int a = 0; a < V; ++a) dst[rank * 4 + a] = s[a];
    }
  }
  cl.sync();
#pragma unroll
  for (int a = 0; a < V; ++a) v[a] = T(0);
  for (int r = 0; r < cs; ++r)
#pragma unroll
    for (int a = 0; a < V; ++a) v[a] += slots_buf[r * 4 + a];
}

template <typename T>
__global__ void __launch_bounds__(1024, 1)
    k_patch_pcg_cluster(const T* __restrict__ Ahat, const uint32_t* __restrict__ pmask,
                        PatchClusterGeom c, T* __restrict__ Rhat, double tol2, int max_iter,
                        int* iter_stats) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cg::cluster_group cl = cg::this_cluster();
  const PatchPcgGeom& g = c.pg;
  const ClusterLayout Ly = cluster_layout<T>(c);
  T* blk = reinterpret_cast<T*>(smem_raw + Ly.blk);
  T* pall = reinterpret_cast<T*>(smem_raw + Ly.pall);
  int* pj = reinterpret_cast<int*>(smem_raw + Ly.pj);
  int* mj = reinterpret_cast<int*>(smem_raw + Ly.mj);
  int* sadj = reinterpret_cast<int*>(smem_raw + Ly.sadj);
  T* slots = reinterpret_cast<T*>(smem_raw + Ly.slots);
  T* red = reinterpret_cast<T*>(smem_raw + Ly.red);
  const int NB = g.NB;
  const int cs = c.cs;
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int j0 = c.jsplit[rank], j1 = c.jsplit[rank + 1];
  const int j = j0 + warp;  // this warp's row (when j < j1)
  const bool own = j < j1;
  const int eb = __ldg(g.adj_ptr + j0);  // first adjacency entry of this CTA
  const int er0 = own ? __ldg(g.adj_ptr + j) : 0, er1 = own ? __ldg(g.adj_ptr + j + 1) : 0;
  const int64_t np = g.npatch;
  const int64_t cid = blockIdx.x / cs, ncl = gridDim.x / cs;
  int it_max = 0, it_sum = 0, done = 0;

  for (int64_t i = g.i_begin + cid; i < g.i_end; i += ncl) {
    const uint32_t mi = pmask[i] & 15u;
    if (mi == 0) {
      if (own && lane < 4) Rhat[(i * NB + j) * 4 + lane] = T(0);
      continue;
    }
    const T inv_sqrt_mi = T(1) / csqrt<T>(T(__popc(mi)));
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    for (int jj = tid; jj < NB; jj += blockDim.x) {
      const int p = shift_cell(xi, yi, g.nbr[jj].x, g.nbr[jj].y, g.Lpar, np);
      const int m = p >= 0 ? __popc(pmask[p] & 15u) : 0;
      pj[jj] = p;
      mj[jj] = m > 1 ? m - 1 : 0;
    }
    __syncthreads();
    // ---- this CTA's rows of the patch matrix (identity on inactive diagonal entries)
    const int na = own ? mj[j] : 0;
    const int pjj = own ? pj[j] : -1;
    for (int e = er0 + lane; e < er1; e += 32) {
      const int jb = __ldg(&g.adj[e].y);
      const int nb = mj[jb];
      const int o = __ldg(g.pair_idx + (size_t)j * NB + jb);
      T* B = blk + 9 * (e - eb);
      const T* src = Ahat + ((int64_t)(o >= 0 ? o : 0) * np + (pjj >= 0 ? pjj : 0)) * 16;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          T v = (o >= 0 && a < na && b < nb) ? __ldg(src + 4 * a + b) : T(0);
          if (jb == j && a == b && a >= na) v = T(1);
          B[3 * a + b] = v;
        }
      sadj[e - eb] = jb;
    }
    // ---- right-hand side and block-Jacobi inverse of row j (lane 0)
    T rv[3] = {T(0), T(0), T(0)}, Di[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Di[q] = (q % 4 == 0) ? T(1) : T(0);
    if (own && lane == 0 && na > 0) {
      const int o = __ldg(g.pair_idx + (size_t)j * NB + g.jc);
      if (o >= 0) {
        const T* bl = Ahat + ((int64_t)o * np + pjj) * 16;
#pragma unroll
        for (int t = 0; t < 3; ++t) rv[t] = t < na ? -inv_sqrt_mi * bl[4 * t + 3] : T(0);
      }
      const int od = __ldg(g.pair_idx + (size_t)j * NB + j);
      const T* dg = Ahat + ((int64_t)od * np + pjj) * 16;
      T Mm[9];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) Mm[3 * a + b] = (a < na && b < na) ? dg[4 * a + b] : T(a == b);
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) {
        const T d = Mm[4 * cc] > T(0) ? Mm[4 * cc] : T(1);
        const T id = T(1) / d;
#pragma unroll
        for (int b2 = 0; b2 < 3; ++b2) {
          Mm[3 * cc + b2] *= id;
          Di[3 * cc + b2] *= id;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          if (a == cc) continue;
          const T f = Mm[3 * a + cc];
#pragma unroll
          for (int b2 = 0; b2 < 3; ++b2) {
            Mm[3 * a + b2] -= f * Mm[3 * cc + b2];
            Di[3 * a + b2] -= f * Di[3 * cc + b2];
          }
        }
      }
    }
    // ---- block-Jacobi PCG; row j's iterates live in lane 0 of its warp
    T xv[3] = {T(0), T(0), T(0)}, zv[3], pv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) zv[a] = Di[3 * a] * rv[0] + Di[3 * a + 1] * rv[1] + Di[3 * a + 2] * rv[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) pv[a] = zv[a];
    // p into every CTA's copy of the direction vector (lane 0 holds it; lanes
    // 0..cs-1 write it into the cs copies)
    {
      T pb[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) pb[a] = __shfl_sync(0xffffffffu, pv[a], 0);
      if (own && lane < cs) {
        T* dst = cl.map_shared_rank(pall, lane);
#pragma unroll
        for (int a = 0; a < 3; ++a) dst[3 * j + a] = pb[a];
      }
    }
    T s2[2] = {own && lane == 0 ? rv[0] * zv[0] + rv[1] * zv[1] + rv[2] * zv[2] : T(0),
               own && lane == 0 ? rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2] : T(0)};
    cluster_sums<T, 2>(s2, red, slots + 64, cs, rank, cl);  // also publishes p
    T rz = s2[0];
    const T rr0 = s2[1];
    int it = 0;
    if (rr0 > T(0)) {
      for (it = 1; it <= max_iter; ++it) {
        // q_j = sum over the row's blocks of B_(j, jb) p_jb
        T q0 = 0, q1 = 0, q2 = 0;
        for (int e = er0 + lane; e < er1; e += 32) {
          const T* B = blk + 9 * (e - eb);
          const T* ps = pall + 3 * sadj[e - eb];
          const T p0 = ps[0], p1 = ps[1], p2 = ps[2];
          q0 += B[0] * p0 + B[1] * p1 + B[2] * p2;
          q1 += B[3] * p0 + B[4] * p1 + B[5] * p2;
          q2 += B[6] * p0 + B[7] * p1 + B[8] * p2;
        }
        q0 = warp_sum_c(q0);
        q1 = warp_sum_c(q1);
        q2 = warp_sum_c(q2);
        T s1[1] = {own && lane == 0 ? pv[0] * q0 + pv[1] * q1 + pv[2] * q2 : T(0)};
        cluster_sums<T, 1>(s1, red, slots, cs, rank, cl);
        const T pq = s1[0];
        const T alpha = pq > T(0) ? rz / pq : T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) xv[a] += alpha * pv[a];
        rv[0] -= alpha * q0;
        rv[1] -= alpha * q1;
        rv[2] -= alpha * q2;
#pragma unroll
        for (int a = 0; a < 3; ++a)
          zv[a] = Di[3 * a] * rv[0] + Di[3 * a + 1] * rv[1] + Di[3 * a + 2] * rv[2];
        T s3[2] = {own && lane == 0 ? rv[0] * zv[0] + rv[1] * zv[1] + rv[2] * zv[2] : T(0),
                   own && lane == 0 ? rv[0] * rv[0] + rv[1] * rv[1] + rv[2] * rv[2] : T(0)};
        cluster_sums<T, 2>(s3, red, slots + 64, cs, rank, cl);
        const T rz_new = s3[0], rr = s3[1];
        if ((double)rr <= tol2 * (double)rr0 || !(rz_new > T(0))) break;
        const T beta = rz_new / rz;
        rz = rz_new;
#pragma unroll
        for (int a = 0; a < 3; ++a) pv[a] = zv[a] + beta * pv[a];
        // lane 0 holds the new p_j; lanes 0..cs-1 write it into the cs copies
        T pb[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) pb[a] = __shfl_sync(0xffffffffu, pv[a], 0);
        if (own && lane < cs) {
          T* dst = cl.map_shared_rank(pall, lane);
#pragma unroll
          for (int a = 0; a < 3; ++a) dst[3 * j + a] = pb[a];
        }
        cl.sync();
      }
      if (it > max_iter) it = max_iter;
    }
    it_max = max(it_max, it);
    it_sum += it;
    ++done;
    // ---- interpolation row: detail coefficients of neighbour j and the average slot
    if (own && lane == 0) {
      T* row = Rhat + (i * NB + j) * 4;
#pragma unroll
      for (int t = 0; t < 3; ++t) row[t] = t < na ? xv[t] : T(0);
      row[3] = j == g.jc ? inv_sqrt_mi : T(0);
    }
    // no CTA writes into another's slots or direction copy for the next patch
    // before every CTA has finished reading them for this one
    cl.sync();
  }
  if (tid == 0 && rank == 0 && iter_stats) {
    atomicMax(&iter_stats[0], it_max);
    atomicAdd(&iter_stats[1], it_sum);
    atomicAdd(&iter_stats[2], done);
  }
}

template <typename T>
cudaError_t launch_patch_pcg_cluster(const T* Ahat, const uint32_t* pmask_k,
                                     const PatchClusterGeom& c, T* Rhat, double tol,
                                     int max_iter, int* iter_stats, cudaStream_t s) {
  const int64_t nsolve = c.pg.i_end - c.pg.i_begin;
  if (nsolve <= 0) return cudaSuccess;
  const size_t smem = patch_cluster_smem_bytes<T>(c);
  auto kern = k_patch_pcg_cluster<T>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (c.cs > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = c.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.blockDim = dim3(32 * c.max_rows, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.gridDim = dim3(c.cs, 1, 1);
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaErrorInvalidConfiguration;
  int64_t ncl = nclusters;
  if (ncl > nsolve) ncl = nsolve;
  cfg.gridDim = dim3((unsigned)(ncl * c.cs), 1, 1);
  count_launch();
  return cudaLaunchKernelEx(&cfg, kern, Ahat, pmask_k, c, Rhat, tol * tol, max_iter, iter_stats);
}
template cudaError_t launch_patch_pcg_cluster<float>(const float*, const uint32_t*,
                                                     const PatchClusterGeom&, float*, double,
                                                     int, int*, cudaStream_t);
template cudaError_t launch_patch_pcg_cluster<double>(const double*, const uint32_t*,
                                                      const PatchClusterGeom&, double*, double,
                                                      int, int*, cudaStream_t);

}  // namespace gb
