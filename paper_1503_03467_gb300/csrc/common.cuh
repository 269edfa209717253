// common.cuh - shared device helpers of the gamblet library.
//
// Data layout used by every kernel (all levels, all phases):
//  * A level-k vector is indexed by the Morton code of its lattice cell
//    (x, y), 0 <= x, y < 2^k: bits of x in the even positions, bits of y in
//    the odd ones.  The four children of a level-(k-1) cell p are then the
//    contiguous entries 4p + c, with slot c = (y & 1) * 2 + (x & 1) - the
//    row-major (y, x) sibling order of the detail basis W^(k) (Sec. 4.6).
//  * A level stores the Morton prefix of its lattice that holds cells:
//    npar_k parents (level-(k-1) cells) and ncell_k = 4 npar_k cells, with
//    npar_(k-1) = ceil(npar_k / 4).  A single square problem fills the
//    lattice (npar_k = 4^(k-1)); independent problems packed into aligned
//    subtrees of one lattice fill a prefix of it.  Cells beyond the prefix
//    do not exist: every neighbour lookup (shift_cell) rejects them.
//  * Each parent p carries a 4-bit mask of its non-empty children (holes
//    occur where the fine grid has no node, and in the last parents of a
//    prefix).  Its orthonormal 4x4
//    transform Q_p (rows: detail t = 0..m-2, unused rows, and row 3 =
//    1/sqrt(m) on the children) is the Helmert matrix Ubar^(m) of Lemma
//    const0 (Construction const2) embedded on the active slots; it is
//    evaluated from the mask (qv / qmat below).  x_hat = Q x splits a level vector into
//    W^(k) x (slots 0..2) and sqrt(m) * pibar x (slot 3).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

// Counts every kernel launch issued by the library (reported by
// gamblet_kernel_launches() so a caller can attribute GPU work to it).
void count_launch();

__host__ __device__ __forceinline__ int __popc_portable(unsigned v) {
#ifdef __CUDA_ARCH__
  return __popc(v);
#else
  return __builtin_popcount(v);
#endif
}

// Status codes written by device code into a status word (never traps).
enum DevStatus : int {
  DEV_OK = 0,
  DEV_NOT_SPD = 1,   // non-positive pivot in a factorisation
  DEV_TIMEOUT = 2,   // a bounded wait on an asynchronous unit (tensor-core
                     // completion barrier) gave up; the kernel returned early
};

// ---------------------------------------------------------------- Morton
__host__ __device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
  v &= 0x0000ffffu;
  v = (v | (v << 8)) & 0x00ff00ffu;
  v = (v | (v << 4)) & 0x0f0f0f0fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
__host__ __device__ __forceinline__ uint32_t compact_bits(uint32_t v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0f0f0f0fu;
  v = (v | (v >> 4)) & 0x00ff00ffu;
  v = (v | (v >> 8)) & 0x0000ffffu;
  return v;
}
__host__ __device__ __forceinline__ uint32_t morton(uint32_t x, uint32_t y) {
  return spread_bits(x) | (spread_bits(y) << 1);
}
__host__ __device__ __forceinline__ void demorton(uint32_t m, int& x, int& y) {
  x = (int)compact_bits(m);
  y = (int)compact_bits(m >> 1);
}
// Morton index of (x + dx, y + dy) on a side-L lattice whose stored cells
// are the Morton prefix [0, n) (n = L * L for a full square), or -1 when the
// shifted cell is outside the lattice or beyond the prefix.
__host__ __device__ __forceinline__ int shift_cell(int x, int y, int dx, int dy, int L,
                                                   int64_t n) {
  int nx = x + dx, ny = y + dy;
  if ((unsigned)nx >= (unsigned)L || (unsigned)ny >= (unsigned)L) return -1;
  const uint32_t m = morton((uint32_t)nx, (uint32_t)ny);
  return (int64_t)m < n ? (int)m : -1;
}

// Entry (a, c) of the per-parent transform Q for child mask m: with
// cnt = popcount(m) active children and c the j-th of them (j = number of
// active slots below c), row 3 is 1/sqrt(cnt) and row t < cnt - 1 is the
// normalised Helmert row t + 1 of Lemma const0:
//   U^(n)_{t+1, .} = (1, ..., 1 [t+1 times], -(t+1), 0, ...) / sqrt((t+1)(t+2)).
// 1 / sqrt(n) for the six n that occur (cnt = 1..4 and (t + 1)(t + 2) =
// 2, 6, 12) as literal constants: float64 square roots and divisions per
// element are slow on this part's float64 pipe.
template <typename T>
__host__ __device__ __forceinline__ T inv_sqrt_q(int n) {
  switch (n) {
    case 1: return T(1);
    case 2: return T(0.70710678118654752440);   // 1/sqrt(2)
    case 3: return T(0.57735026918962576451);   // 1/sqrt(3)
    case 4: return T(0.5);
    case 6: return T(0.40824829046386301637);   // 1/sqrt(6)
    case 12: return T(0.28867513459481288225);  // 1/sqrt(12)
    default: return T(1) / sqrt(T(n));
  }
}

template <typename T>
__host__ __device__ __forceinline__ T qv(int m, int a, int c) {
  if (!((m >> c) & 1)) return T(0);
  const int cnt = __popc_portable(m & 15);
  const int j = __popc_portable(m & ((1 << c) - 1));
  if (a == 3) return inv_sqrt_q<T>(cnt);
  if (a >= cnt - 1) return T(0);
  const T nrm = inv_sqrt_q<T>((a + 1) * (a + 2));
  if (j <= a) return nrm;
  if (j == a + 1) return -T(a + 1) * nrm;
  return T(0);
}

// Full 4x4 transform of mask m, row-major Q[a * 4 + c].
template <typename T>
__host__ __device__ __forceinline__ void qmat(int m, T* Q) {
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) Q[a * 4 + c] = qv<T>(m, a, c);
}

__device__ __forceinline__ int popc4(int m) { return __popc(m & 15); }

// Warp reduction of a double.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace gb
