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
// Layout: the patch system is padded to n = 3 NB unknowns; unknowns whose
// parent lies outside the lattice or has fewer children are decoupled
// identity rows with zero right-hand side.  The right-hand side is carried
// as row n of a packed lower-triangular augmented matrix, so the Cholesky
// elimination also performs the forward substitution; one warp finishes
// with the back substitution.  One CTA per patch, persistent over patches.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

__host__ __device__ __forceinline__ int packed_size(int n) { return (n + 1) * (n + 2) / 2; }

template <typename T>
size_t patch_smem_bytes(int NB) {
  int n = 3 * NB;
  size_t b = sizeof(T) * (size_t)packed_size(n);     // augmented packed matrix
  b += sizeof(T) * (size_t)(n + 1);                   // column buffer / solution
  b += sizeof(int) * 2 * (size_t)NB;                  // parent index, child count
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
__global__ void __launch_bounds__(256) k_patch_solve(const T* __restrict__ Ahat,
                                                     const uint32_t* __restrict__ pmask,
                                                     PatchGeom g, T* __restrict__ Rhat,
                                                     int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NB = g.NB;
  const int n = 3 * NB;
  T* M = reinterpret_cast<T*>(smem_raw);
  T* col = M + packed_size(n);
  int* pj = reinterpret_cast<int*>(col + (n + 1));
  int* mj = pj + NB;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  const int nwarp = blockDim.x >> 5;
  const int64_t np = g.npatch;

  for (int64_t i = blockIdx.x; i < np; i += gridDim.x) {
    const uint32_t mi = pmask[i] & 15u;
    if (mi == 0) {  // empty coarse cell: no gamblet
      for (int idx = tid; idx < NB * 4; idx += blockDim.x) Rhat[(int64_t)idx * np + i] = T(0);
      continue;
    }
    const T inv_sqrt_mi = T(1) / dev_sqrt<T>(T(__popc(mi)));
    int xi, yi;
    demorton((uint32_t)i, xi, yi);
    for (int j = tid; j < NB; j += blockDim.x) {
      int p = shift_cell(xi, yi, g.nbr[j].x, g.nbr[j].y, g.Lpar);
      pj[j] = p;
      mj[j] = p >= 0 ? __popc(pmask[p] & 15u) : 0;
    }
    __syncthreads();

    // ---- gather the augmented packed matrix [B b; b^T *]
    for (int r = warp; r <= n; r += nwarp) {
      const int base = r * (r + 1) / 2;
      if (r < n) {
        const int ja = r / 3, ta = r - 3 * ja;
        const int pa = pj[ja];
        const bool acta = pa >= 0 && ta < mj[ja] - 1;
        for (int c = lane; c <= r; c += 32) {
          const int jb = c / 3, tb = c - 3 * jb;
          const bool actb = pj[jb] >= 0 && tb < mj[jb] - 1;
          T v;
          if (acta && actb) {
            const int o = g.pair_idx[ja * NB + jb];
            v = o >= 0 ? Ahat[((int64_t)o * np + pa) * 16 + ta * 4 + tb] : T(0);
          } else {
            v = (r == c) ? T(1) : T(0);
          }
          M[base + c] = v;
        }
      } else {
        for (int c = lane; c <= n; c += 32) {
          T v = T(0);
          if (c < n) {
            const int jb = c / 3, tb = c - 3 * jb;
            const int pb = pj[jb];
            if (pb >= 0 && tb < mj[jb] - 1) {
              const int o = g.pair_idx[jb * NB + g.jc];
              if (o >= 0) v = -inv_sqrt_mi * Ahat[((int64_t)o * np + pb) * 16 + tb * 4 + 3];
            }
          } else {
            v = T(1);
          }
          M[base + c] = v;
        }
      }
    }
    __syncthreads();

    // ---- right-looking Cholesky on the first n columns of the augmented matrix
    for (int j = 0; j < n; ++j) {
      const int jj = j * (j + 1) / 2 + j;
      T d = M[jj];
      if (!(d > T(0))) {  // non-positive or NaN pivot
        if (tid == 0) atomicExch(status, (int)DEV_NOT_SPD);
        d = T(1);
      }
      const T s = dev_sqrt<T>(d);
      const T inv = T(1) / s;
      for (int r = j + 1 + tid; r <= n; r += blockDim.x) {
        const int idx = r * (r + 1) / 2 + j;
        const T l = M[idx] * inv;
        M[idx] = l;
        col[r] = l;
      }
      __syncthreads();
      if (tid == 0) M[jj] = s;
      for (int r = j + 1 + warp; r <= n; r += nwarp) {
        const T lr = col[r];
        if (lr == T(0)) continue;
        const int base = r * (r + 1) / 2;
        const int cmax = r < n ? r : n - 1;
        for (int c = j + 1 + lane; c <= cmax; c += 32) M[base + c] -= lr * col[c];
      }
      __syncthreads();
    }

    // ---- back substitution L^T y = z, z = row n (one warp)
    if (warp == 0) {
      const int zb = n * (n + 1) / 2;
      for (int c = lane; c < n; c += 32) col[c] = M[zb + c];
      __syncwarp();
      for (int j = n - 1; j >= 0; --j) {
        const int rb = j * (j + 1) / 2;
        const T yj = col[j] / M[rb + j];
        __syncwarp();
        for (int c = lane; c < j; c += 32) col[c] -= M[rb + c] * yj;
        if (lane == 0) col[j] = yj;
        __syncwarp();
      }
    }
    __syncthreads();

    // ---- interpolation row of coarse cell i (SoA over [j][slot])
    for (int idx = tid; idx < NB * 4; idx += blockDim.x) {
      const int j = idx >> 2, c = idx & 3;
      T v = T(0);
      if (c < 3) {
        if (pj[j] >= 0 && c < mj[j] - 1) v = col[3 * j + c];
      } else if (j == g.jc) {
        v = inv_sqrt_mi;
      }
      Rhat[(int64_t)idx * np + i] = v;
    }
    __syncthreads();
  }
}

template <typename T>
void launch_patch_solve(const T* Ahat, const uint32_t* pmask_k, PatchGeom g, T* Rhat,
                        int* status, int num_sms, cudaStream_t s) {
  if (g.npatch <= 0) return;
  size_t smem = patch_smem_bytes<T>(g.NB);
  cudaFuncSetAttribute(k_patch_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_solve<T>, 256, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > g.npatch) grid = g.npatch;
  { count_launch(); k_patch_solve<T><<<(unsigned)grid, 256, smem, s>>>(Ahat, pmask_k, g, Rhat, status); }
}
template void launch_patch_solve<float>(const float*, const uint32_t*, PatchGeom, float*, int*,
                                        int, cudaStream_t);
template void launch_patch_solve<double>(const double*, const uint32_t*, PatchGeom, double*,
                                         int*, int, cudaStream_t);

}  // namespace gb
