// patch_mma.cu - localized patch solves (Sec. 5.3, Definition defb; Algorithm
// 2, line 11) on the tensor cores, for the float32 (mixed) path.
//
// The patches of a G x G group of neighbouring coarse cells (a "window", G = 1
// or 2) are principal submatrices of one matrix: B^(k) restricted to the union
// U of their neighbourhoods i^rho.  One CTA gathers that union matrix once and
// runs the G^2 conjugate-gradient solves together: their direction vectors,
// each zero outside its own patch, are the columns of one dense product
// B_U [p_1 .. p_G^2], issued as tcgen05.mma from shared memory into a tensor
// memory accumulator, and each patch reads back only its own rows.
//
// Arithmetic.  The union matrix is scaled symmetrically by the inverse
// Cholesky factors of its 3x3 diagonal blocks, Btilde = L^-1 B L^-T with
// L = blockdiag(L_u), D_u = L_u L_u^T.  CG on Btilde with the right-hand side
// L^-1 b is block-Jacobi preconditioned CG on B (the preconditioner of the
// float32 SIMT kernel), and Btilde has a unit diagonal, so every entry has
// |Btilde_ij| <= 1 and is stored as float16 (kind::f16): the same 10-bit
// significand as TF32 at half the shared memory.  Rounding each entry to
// float16 perturbs Btilde element by element by at most 2^-11 relative, so the
// solution moves by about 2^-11 times the condition number of Btilde (the
// block-Jacobi scaled patch matrix, a few units to tens for rough
// coefficients) - the order of the 1e-3 patch tolerance of the mixed path,
// which Theorem tmdiscreteaccuracy allows and the float64 outer iteration
// removes.  The direction vectors carry float32 accuracy into the product:
// each is scaled by a power of two to O(1) and split into float16 high and low
// parts, which occupy separate columns of the product (accumulated in
// float32) and are added in the epilogue.
//
// Iteration: the Chronopoulos-Gear form of CG (the same iterates as CG in
// exact arithmetic), whose matrix product is applied to the residual and
// whose two inner products per iteration, (r, r) and (A r, r), are summed in
// one block reduction, so an iteration costs one tensor-core product and two
// barriers.  Each M-tile's products are issued by its own thread.
//
// Shared memory: Btilde as Mt * 128 rows x Kp columns of float16 (n = 3 |U|
// unknowns, Kp = n rounded up to 16, Mt M-tiles of 128 rows) in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices, core matrix
// (r / 8, k / 8) at ((r / 8) * Kp / 8 + k / 8) * 128 bytes), the B operand (16
// rows: high parts, low parts, zeros) in the same layout, and per-union-parent
// factors.  Tensor memory: 16 float32 columns per M-tile.  One thread owns one
// row of the union system: its entries of the G^2 iterates x, r, p live in
// registers.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace gb {

namespace {

constexpr int kMmaN = 16;  // columns of one accumulator
// Each M-tile's product is split over kAccSplit accumulators (k-steps dealt
// round-robin, summed in the epilogue) so that consecutive tensor-core
// instructions do not wait on one accumulator; kIssuers threads per M-tile
// issue them (each owns the accumulators j with j % kIssuers equal to its
// index).
constexpr int kAccSplit = 2;
constexpr int kIssuers = 2;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major tile without swizzle: start
// address, byte distance between core matrices adjacent in K (lbo) and in
// M or N (sbo), descriptor version 1 (bit 46), no base offset, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::f16: float32 accumulator, float16 A and B,
// both K-major, shape M x N.
__host__ __device__ constexpr uint32_t umma_idesc_f16(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (r, k) in a K-major core-matrix tile with Kp columns
__device__ __forceinline__ int kmaj_off(int r, int k, int Kp) {
  return (((r >> 3) * (Kp >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1);
}

// Entries (r, k0), (r, k0 + 1), (r, k0 + 2) as one aligned pair and one
// single store: an even column and its successor always share a core-matrix
// row (16 bytes, 8 columns), so the pair is one 4-byte store.
__device__ __forceinline__ void store_run3(unsigned char* tile, int r, int k0, int Kp, float a,
                                           float b, float c) {
  if ((k0 & 1) == 0) {
    *reinterpret_cast<__half2*>(tile + kmaj_off(r, k0, Kp)) = __floats2half2_rn(a, b);
    *reinterpret_cast<__half*>(tile + kmaj_off(r, k0 + 2, Kp)) = __float2half_rn(c);
  } else {
    *reinterpret_cast<__half*>(tile + kmaj_off(r, k0, Kp)) = __float2half_rn(a);
    *reinterpret_cast<__half2*>(tile + kmaj_off(r, k0 + 1, Kp)) = __floats2half2_rn(b, c);
  }
}

// Bounded wait for phase `phase` of an mbarrier; false after the limit.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < (1 << 22); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Power of two 2^(3 - e) with 2^e <= x < 2^(e+1) (x > 0, normal): scales a
// vector whose largest entry is about x to entries of at most 16.  With
// squared = true, x is the square of that size (2^(2e) <= x < 2^(2e+2)).
__device__ __forceinline__ void pow2_scale(float x, bool squared, float& sc, float& isc) {
  int e = ((__float_as_int(x) >> 23) & 255) - 127;
  if (squared) e >>= 1;
  const int a = max(min(3 - e, 120), -120);
  sc = __int_as_float((127 + a) << 23);
  isc = __int_as_float((127 - a) << 23);
}

// Sums over the block of V values per thread (every thread gets them).  A
// warp first reduces and scatters the V values over its lanes (each halving
// step trades half of the values with the partner lane: V - 1 shuffles in
// all), sums the remaining lane groups, and lanes 0..V-1 write the warp's V
// partial sums into its row of red (row stride kRedStride floats); after
// one barrier every thread adds the NW rows as float4 vectors.  Callers
// alternate between two slot arrays so that one barrier per reduction
// suffices.
constexpr int kRedStride = 8;
template <int V, int NW>
__device__ __forceinline__ void block_sums(float (&v)[V], float* red) {
  static_assert(V <= kRedStride && V % 4 == 0 && (V & (V - 1)) == 0, "slot layout");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int idx = 0;  // value index this lane ends up holding
#pragma unroll
  for (int h = V / 2, bit = 1; h >= 1; h >>= 1, bit <<= 1) {
    const bool upper = (lane & bit) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = upper ? v[i] : v[i + h];
      const float keep = upper ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
    }
    if (upper) idx += h;
  }
#pragma unroll
  for (int bit = V; bit < 32; bit <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], bit);
  if (lane < V) red[warp * kRedStride + idx] = v[0];
  __syncthreads();
#pragma unroll
  for (int c = 0; c < V; ++c) v[c] = 0.f;
#pragma unroll
  for (int w = 0; w < NW; ++w)
#pragma unroll
    for (int c = 0; c < V; c += 4) {
      const float4 t = *reinterpret_cast<const float4*>(red + w * kRedStride + c);
      v[c] += t.x;
      v[c + 1] += t.y;
      v[c + 2] += t.z;
      v[c + 3] += t.w;
    }
}

}  // namespace

size_t patch_mma_smem_bytes(const PatchMmaGeom& g) {
  const int rows = g.Mt * 128;
  size_t b = (size_t)rows * g.Kp * 2;            // Btilde (float16)
  b += (size_t)kMmaN * g.Kp * 2;                 // B operand (float16)
  b += sizeof(float) * 9 * (size_t)g.nU;         // inverse Cholesky factors
  b += sizeof(float) * (size_t)g.NP * rows;      // right-hand sides, then solutions
  b += sizeof(int) * 2 * (size_t)g.nU;           // parent index, active unknowns
  b += sizeof(float) * 2 * 12 * kRedStride;      // reduction slots (two arrays, 12 warps)
  b += sizeof(float) * 4 + 32;                   // right-hand-side maxima, mbarrier, TMEM address
  return (b + 127) & ~(size_t)127;
}

// NP patches per window (1 or 4), MT M-tiles of 128 rows (4 MT warps).
template <int NP, int MT>
__global__ void __launch_bounds__(128 * MT, 1)
    k_patch_mma(const float* __restrict__ Ahat, const uint32_t* __restrict__ pmask,
                PatchMmaGeom g, float* __restrict__ Rhat, float tol2, int max_iter,
                int* iter_stats, int* status) {
  constexpr int NW = 4 * MT;
  constexpr int rows = 128 * MT;
  constexpr int V = NP == 1 ? 4 : 8;  // reduction values: (r.r, w.r) per patch, padded
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const int Kp = g.Kp, n = g.n, nU = g.nU, NB = g.NB;
  unsigned char* As = smem_raw;
  unsigned char* Bs = As + (size_t)rows * Kp * 2;
  float* Linv = reinterpret_cast<float*>(Bs + (size_t)kMmaN * Kp * 2);
  float* vec = Linv + 9 * nU;                 // [NP][rows]
  int* pu = reinterpret_cast<int*>(vec + NP * rows);
  int* nau = pu + nU;
  float* red = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(nau + nU) + 15) & ~(uintptr_t)15);  // 2 x [12][kRedStride]
  unsigned* bmax = reinterpret_cast<unsigned*>(red + 2 * 12 * kRedStride);
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(bmax + 4) + 7) & ~(uintptr_t)7);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t np = g.npatch;
  const uint32_t bar_a = smem_addr(bar);

  // ---- one-time set-up: mbarrier (one arrival per M-tile issuer), tensor
  // memory (16 columns per M-tile)
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_a), "r"(MT * kIssuers));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  constexpr int kCols = MT * kAccSplit * kMmaN;
  constexpr uint32_t ncols = kCols <= 32 ? 32u : (kCols <= 64 ? 64u : (kCols <= 128 ? 128u : 256u));
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(tslot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t sbo = (uint32_t)Kp * 16;  // one 8-row group across all Kp columns
  const uint32_t idesc = umma_idesc_f16(128, kMmaN);
  const int ksteps = Kp / 16;
  // this thread's row, M-tile and tensor-memory lane block; lane 0 of warp
  // 4 m + ii (ii < kIssuers) issues part of the products of M-tile m
  const int row = tid;
  const int mt = warp >> 2;
  const int issuer_idx = (warp & 3);
  const bool issuer = (tid & 31) == 0 && issuer_idx < kIssuers;
  const uint32_t taddr =
      tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(mt * kAccSplit * kMmaN);
  const int ru = row / 3, rt = row - 3 * (row / 3);
  const int rbits = row < n ? g.ubits[ru] : 0;
  uint32_t phase = 0;
  int it_max = 0, it_sum = 0, done_cnt = 0, nprod = 0;
  bool fault = false;

  for (int64_t w = g.w_begin + blockIdx.x; w < g.w_end && !fault; w += gridDim.x) {
    const int64_t i0 = w * NP;  // coarse cells i0 .. i0 + NP - 1 (Morton)
    int x0, y0;
    demorton((uint32_t)i0, x0, y0);
    if (tid < 4) bmax[tid] = 0u;
    // ---- union parents and the inverse Cholesky factors of their diagonal blocks
    for (int u = tid; u < nU; u += blockDim.x) {
      const int2 o = g.U[u];
      const int p = shift_cell(x0, y0, o.x, o.y, g.Lpar, np);
      const int m = p >= 0 ? __popc(pmask[p] & 15u) : 0;
      const int na = m > 1 ? m - 1 : 0;
      pu[u] = p;
      nau[u] = na;
      float d[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) d[q] = (q % 4 == 0) ? 1.f : 0.f;
      if (na > 0) {
        const float* src = Ahat + ((int64_t)g.diag_o * np + p) * 16;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            if (a < na && b < na) d[3 * a + b] = __ldg(src + 4 * a + b);
      }
      float l11 = d[0], l21, l31, l22, l32, l33;
      bool spd = l11 > 0.f;
      l11 = sqrtf(spd ? l11 : 1.f);
      l21 = d[3] / l11;
      l31 = d[6] / l11;
      float t = d[4] - l21 * l21;
      spd = spd && t > 0.f;
      l22 = sqrtf(t > 0.f ? t : 1.f);
      l32 = (d[7] - l31 * l21) / l22;
      t = d[8] - l31 * l31 - l32 * l32;
      spd = spd && t > 0.f;
      l33 = sqrtf(t > 0.f ? t : 1.f);
      if (!spd) atomicExch(status, (int)DEV_NOT_SPD);
      const float i11 = 1.f / l11, i22 = 1.f / l22, i33 = 1.f / l33;
      const float i21 = -l21 * i11 * i22;
      const float i32 = -l32 * i22 * i33;
      const float i31 = -(l31 * i11 + l32 * i21) * i33;
      float* Li = Linv + 9 * u;
      Li[0] = i11; Li[1] = 0.f; Li[2] = 0.f;
      Li[3] = i21; Li[4] = i22; Li[5] = 0.f;
      Li[6] = i31; Li[7] = i32; Li[8] = i33;
    }
    // ---- zero the matrix tile and the B operand (16-byte stores)
    {
      uint4* z = reinterpret_cast<uint4*>(As);
      const int nz = (int)(((size_t)rows * Kp * 2 + (size_t)kMmaN * Kp * 2) >> 4);
      const uint4 zero = make_uint4(0, 0, 0, 0);
      for (int i = tid; i < nz; i += blockDim.x) z[i] = zero;
    }
    __syncthreads();
    // ---- scaled blocks Btilde_ab = L_a^-1 B_ab L_b^-T (a > b) and their
    // transposes, four blocks in flight per thread; unit diagonal
    for (int e0 = tid; e0 < g.npair; e0 += 4 * blockDim.x) {
      float4 rw[4][3];
      int4 pr[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int e = e0 + v * blockDim.x;
        pr[v] = e < g.npair ? g.pairs[e] : make_int4(0, 0, -1, 0);
        const bool live = pr[v].z >= 0 && nau[pr[v].x] > 0 && nau[pr[v].y] > 0;
        if (!live) pr[v].z = -1;
        const float* src = Ahat + ((int64_t)(live ? pr[v].z : 0) * np + (live ? pu[pr[v].x] : 0)) * 16;
#pragma unroll
        for (int r = 0; r < 3; ++r)
          rw[v][r] = live ? __ldg(reinterpret_cast<const float4*>(src + 4 * r))
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        if (pr[v].z < 0) continue;
        const int a = pr[v].x, b = pr[v].y;
        const int naa = nau[a], nab = nau[b];
        float B[9];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          B[3 * r] = (r < naa && 0 < nab) ? rw[v][r].x : 0.f;
          B[3 * r + 1] = (r < naa && 1 < nab) ? rw[v][r].y : 0.f;
          B[3 * r + 2] = (r < naa && 2 < nab) ? rw[v][r].z : 0.f;
        }
        const float* La = Linv + 9 * a;
        const float* Lb = Linv + 9 * b;
        float X[9], T[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            X[3 * r + c] = La[3 * r] * B[c] + La[3 * r + 1] * B[3 + c] + La[3 * r + 2] * B[6 + c];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c)
            T[3 * r + c] = X[3 * r] * Lb[3 * c] + X[3 * r + 1] * Lb[3 * c + 1] +
                           X[3 * r + 2] * Lb[3 * c + 2];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          store_run3(As, 3 * a + r, 3 * b, Kp, T[3 * r], T[3 * r + 1], T[3 * r + 2]);
          store_run3(As, 3 * b + r, 3 * a, Kp, T[r], T[3 + r], T[6 + r]);
        }
      }
    }
    for (int r = tid; r < n; r += blockDim.x)
      *reinterpret_cast<__half*>(As + kmaj_off(r, r, Kp)) = __float2half_rn(1.f);
    // ---- right-hand sides b~ = L_u^-1 b_u of the window's patches and their
    // largest entries
    for (int e = tid; e < NP * nU; e += blockDim.x) {
      const int c = e / nU, u = e - c * nU;
      float bv[3] = {0.f, 0.f, 0.f};
      const int na = nau[u];
      const uint32_t mi = pmask[i0 + c] & 15u;
      const int o = g.rhs_o[c * nU + u];
      if (mi != 0 && na > 0 && ((g.ubits[u] >> c) & 1) && o >= 0) {
        const float sgn = -inv_sqrt_q<float>(__popc(mi));
        const float* src = Ahat + ((int64_t)o * np + pu[u]) * 16;
        float braw[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) braw[t] = t < na ? sgn * __ldg(src + 4 * t + 3) : 0.f;
        const float* Li = Linv + 9 * u;
#pragma unroll
        for (int t = 0; t < 3; ++t)
          bv[t] = Li[3 * t] * braw[0] + Li[3 * t + 1] * braw[1] + Li[3 * t + 2] * braw[2];
        const float am = fmaxf(fabsf(bv[0]), fmaxf(fabsf(bv[1]), fabsf(bv[2])));
        if (am > 0.f) atomicMax(bmax + c, __float_as_uint(am));
      }
#pragma unroll
      for (int t = 0; t < 3; ++t) vec[c * rows + 3 * u + t] = bv[t];
    }
    __syncthreads();
    // ---- Chronopoulos-Gear CG on the NP patch systems (this thread: row `row`).
    // Iteration i: w = A r_i (tensor cores), gamma_i = (r_i, r_i),
    // delta_i = (w, r_i) in one reduction; stop when gamma_i <= tol^2 gamma_0;
    // beta_i = gamma_i / gamma_(i-1), alpha_i = gamma_i / (delta_i - beta_i
    // gamma_i / alpha_(i-1)); p = r + beta p, s = w + beta s (s = A p);
    // x += alpha p, r -= alpha s.
    float xv[NP], rv[NP], pv[NP], sv[NP], gam[NP], gam0[NP], alp[NP], nrm[NP];
    bool act[NP], done[NP];
    int its[NP];
    int any = 0;
#pragma unroll
    for (int c = 0; c < NP; ++c) {
      const bool cell = (pmask[i0 + c] & 15u) != 0;
      act[c] = cell && row < n && ((rbits >> c) & 1) && pu[ru] >= 0 && rt < nau[ru];
      xv[c] = 0.f;
      rv[c] = act[c] ? vec[c * rows + row] : 0.f;
      pv[c] = 0.f;
      sv[c] = 0.f;
      gam[c] = 0.f;
      gam0[c] = 0.f;
      alp[c] = 1.f;
      nrm[c] = __uint_as_float(bmax[c]);
      done[c] = !(nrm[c] > 0.f);
      any |= !done[c];
      its[c] = 0;
    }
    int rb = 0;  // reduction slot array in use next
    for (int it = 0; any; ++it) {
      // B operand: the residuals scaled by powers of two to entries of O(1),
      // split into high and low float16 parts (rows c and NP + c)
      float isc[NP];
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        float sc = 0.f;
        isc[c] = 0.f;
        if (!done[c]) pow2_scale(nrm[c], it > 0, sc, isc[c]);
        if (row < n) {
          const float v = rv[c] * sc;
          const __half hi = __float2half_rn(v);
          const __half lo = __float2half_rn(v - __half2float(hi));
          *reinterpret_cast<__half*>(Bs + kmaj_off(c, row, Kp)) = hi;
          *reinterpret_cast<__half*>(Bs + kmaj_off(NP + c, row, Kp)) = lo;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (issuer) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_addr(As) + (uint32_t)mt * 16u * sbo, b0 = smem_addr(Bs);
        for (int ks = 0; ks < ksteps; ++ks) {
          const int j = ks % kAccSplit;
          if (j % kIssuers != issuer_idx) continue;
          const uint32_t dcol = tmem + (uint32_t)((mt * kAccSplit + j) * kMmaN);
          const uint64_t da = umma_desc(a0 + (uint32_t)ks * 256u, 128u, sbo);
          const uint64_t db = umma_desc(b0 + (uint32_t)ks * 256u, 128u, sbo);
          const uint32_t acc = ks >= kAccSplit;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
              "l"(da), "l"(db), "r"(idesc), "r"(acc));
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                bar_a)
            : "memory");
      }
      const bool ok = mbar_wait(bar_a, phase);
      phase ^= 1u;
      ++nprod;
      if (__syncthreads_or(!ok)) {
        fault = true;
        if (tid == 0) atomicExch(status, (int)DEV_TIMEOUT);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float dsum[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) dsum[q] = 0.f;
#pragma unroll
      for (int j = 0; j < kAccSplit; ++j) {
        if (j >= ksteps) break;  // an accumulator that no k-step wrote holds stale values
        uint32_t d[8];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]),
              "=r"(d[7])
            : "r"(taddr + (uint32_t)(j * kMmaN)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 8; ++q) dsum[q] += __uint_as_float(d[q]);
      }
      float wv[NP], sums[V];
#pragma unroll
      for (int c = 0; c < V; ++c) sums[c] = 0.f;
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        const float q = dsum[c] + dsum[NP + c];
        wv[c] = (act[c] && !done[c]) ? q * isc[c] : 0.f;
        sums[2 * c] = rv[c] * rv[c];
        sums[2 * c + 1] = wv[c] * rv[c];
      }
      block_sums<V, NW>(sums, red + rb * 12 * kRedStride);
      rb ^= 1;
      any = 0;
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        if (done[c]) continue;
        const float gi = sums[2 * c], di = sums[2 * c + 1];
        if (it == 0) gam0[c] = gi;
        if (gi <= tol2 * gam0[c] || it >= max_iter || !(gi > 0.f)) {
          done[c] = true;
          continue;
        }
        const float beta = it == 0 ? 0.f : __fdividef(gi, gam[c]);
        const float den = di - (it == 0 ? 0.f : __fdividef(beta * gi, alp[c]));
        if (!(den > 0.f)) {
          done[c] = true;
          continue;
        }
        const float alpha = __fdividef(gi, den);
        pv[c] = rv[c] + beta * pv[c];
        sv[c] = wv[c] + beta * sv[c];
        xv[c] += alpha * pv[c];
        rv[c] -= alpha * sv[c];
        gam[c] = gi;
        alp[c] = alpha;
        nrm[c] = gi;  // squared size of the next residual's scale
        its[c] = it + 1;
        any = 1;
      }
    }
    if (fault) break;
    // ---- solutions y_u = L_u^-T x~_u into the interpolation rows
#pragma unroll
    for (int c = 0; c < NP; ++c) vec[c * rows + row] = act[c] ? xv[c] : 0.f;
    if (tid == 0) {
#pragma unroll
      for (int c = 0; c < NP; ++c) {
        if (!(pmask[i0 + c] & 15u)) continue;
        it_max = max(it_max, its[c]);
        it_sum += its[c];
        ++done_cnt;
      }
    }
    __syncthreads();
    for (int e = tid; e < NP * NB; e += blockDim.x) {
      const int c = e / NB, j = e - c * NB;
      const int64_t i = i0 + c;
      const uint32_t mi = pmask[i] & 15u;
      float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
      if (mi != 0) {
        const int u = g.outmap[c * NB + j];
        const int na = nau[u];
        const float* Li = Linv + 9 * u;
        const float* xs = vec + c * rows + 3 * u;
        const float x0v = xs[0], x1v = xs[1], x2v = xs[2];
        const float y0 = Li[0] * x0v + Li[3] * x1v + Li[6] * x2v;
        const float y1 = Li[4] * x1v + Li[7] * x2v;
        const float y2 = Li[8] * x2v;
        out.x = na > 0 ? y0 : 0.f;
        out.y = na > 1 ? y1 : 0.f;
        out.z = na > 2 ? y2 : 0.f;
        out.w = j == g.jc ? inv_sqrt_q<float>(__popc(mi)) : 0.f;
      }
      *reinterpret_cast<float4*>(Rhat + (i * NB + j) * 4) = out;
    }
    __syncthreads();
  }
  if (tid == 0 && iter_stats) {
    atomicMax(&iter_stats[0], it_max);
    atomicAdd(&iter_stats[1], it_sum);
    atomicAdd(&iter_stats[2], done_cnt);
    atomicAdd(&iter_stats[3], nprod);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
  }
}

template <int NP, int MT>
void launch_mma_kernel(const float* Ahat, const uint32_t* pmask_k, const PatchMmaGeom& g,
                       float* Rhat, double tol, int max_iter, int* iter_stats, int* status,
                       int num_sms, cudaStream_t s) {
  const int64_t nwin = g.w_end - g.w_begin;
  const size_t smem = patch_mma_smem_bytes(g);
  auto kern = k_patch_mma<NP, MT>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 128 * MT, smem);
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)num_sms * per_sm;
  if (grid > nwin) grid = nwin;
  count_launch();
  kern<<<(unsigned)grid, 128 * MT, smem, s>>>(Ahat, pmask_k, g, Rhat, (float)(tol * tol),
                                               max_iter, iter_stats, status);
}

void launch_patch_mma(const float* Ahat, const uint32_t* pmask_k, PatchMmaGeom g, float* Rhat,
                      double tol, int max_iter, int* iter_stats, int* status, int num_sms,
                      cudaStream_t s) {
  if (g.w_end - g.w_begin <= 0) return;
  if (g.NP == 4) {
    if (g.Mt == 1) launch_mma_kernel<4, 1>(Ahat, pmask_k, g, Rhat, tol, max_iter, iter_stats, status, num_sms, s);
    else if (g.Mt == 2) launch_mma_kernel<4, 2>(Ahat, pmask_k, g, Rhat, tol, max_iter, iter_stats, status, num_sms, s);
    else launch_mma_kernel<4, 3>(Ahat, pmask_k, g, Rhat, tol, max_iter, iter_stats, status, num_sms, s);
  } else {
    if (g.Mt == 1) launch_mma_kernel<1, 1>(Ahat, pmask_k, g, Rhat, tol, max_iter, iter_stats, status, num_sms, s);
    else if (g.Mt == 2) launch_mma_kernel<1, 2>(Ahat, pmask_k, g, Rhat, tol, max_iter, iter_stats, status, num_sms, s);
    else launch_mma_kernel<1, 3>(Ahat, pmask_k, g, Rhat, tol, max_iter, iter_stats, status, num_sms, s);
  }
}

}  // namespace gb
