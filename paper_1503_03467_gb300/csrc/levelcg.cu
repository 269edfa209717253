// levelcg.cu - the independent level systems B^(k) w^(k) = W g^(k)
// (Eq. eqsdjoejddi1), k = 2..q, solved by conjugate gradients (Sec. 4.9) for
// all levels at once: every launch covers every level still iterating, one
// CTA per 16 x 16 Morton tile of parents (the paper's "parallel in
// subscale", Sec. 5.4, as one grid).
//
// B^(k) is the 3x3 detail block of the transformed block stencil; for the
// CG it is kept as a separate coalesced copy Bd[o][e][p] (e = 3a + b).  Each
// CTA stages the direction vector of its tile plus a halo of R cells (R =
// largest offset of the level) in shared memory, so the inner loop over
// offsets reads the matrix with unit stride and the vector from shared
// memory.  The CG is preconditioned by the inverse of each parent's 3x3
// diagonal detail block (block Jacobi).  Dots accumulate in float64.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace gb {

__device__ __forceinline__ int find_level(const CgLevel* lv, int nlev, int b) {
  int l = 0;
  while (l + 1 < nlev && lv[l + 1].block_begin <= b) ++l;
  return l;
}
__device__ __forceinline__ int find_level_spmv(const CgLevel* lv, int nlev, int b) {
  int l = 0;
  while (l + 1 < nlev && lv[l + 1].spmv_begin <= b) ++l;
  return l;
}

__device__ __forceinline__ void block_sum_add(double v, double* dst, double* red) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0 && v != 0.0) atomicAdd(dst, v);
  }
  __syncthreads();
}

// The same for per-thread partials in the working precision T: the warp
// reduces in T (float shuffles and adds on the mixed path, so the float64
// pipe sees only the per-warp values), the warps and the blocks in float64.
// Two sums (a -> *da, b -> *db) share one pair of barriers; red needs 16.
template <typename T>
__device__ __forceinline__ T warp_sum_w(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ void block_sum2_add(T a, T b, double* da, double* db, double* red) {
  a = warp_sum_w(a);
  b = warp_sum_w(b);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp] = (double)a;
    red[8 + warp] = (double)b;
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (int)(blockDim.x >> 5);
    double va = lane < nw ? red[lane] : 0.0;
    double vb = lane < nw ? red[8 + lane] : 0.0;
    va = warp_sum(va);
    vb = warp_sum(vb);
    if (lane == 0) {
      if (va != 0.0) atomicAdd(da, va);
      if (vb != 0.0) atomicAdd(db, vb);
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void block_sum1_add(T a, double* da, double* red) {
  a = warp_sum_w(a);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = (double)a;
  __syncthreads();
  if (warp == 0) {
    double va = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    va = warp_sum(va);
    if (lane == 0 && va != 0.0) atomicAdd(da, va);
  }
  __syncthreads();
}

// z = Dinv r for one parent (3 active slots at most)
template <typename T>
__device__ __forceinline__ void apply_dinv(const T* __restrict__ Dinv, int64_t npar, int64_t p,
                                           const T r[3], T z[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T acc = 0;
#pragma unroll
    for (int b = 0; b < 3; ++b) acc += Dinv[(int64_t)(3 * a + b) * npar + p] * r[b];
    z[a] = acc;
  }
}

// r = b, x = 0, z = Dinv r, p = z; rz = r.z, rr = r.r
template <typename T>
__global__ void __launch_bounds__(256) k_cg_init(const CgLevel* __restrict__ lv, int nlev,
                                                 CgScalars* sc) {
  __shared__ double red[8];
  const int l = find_level(lv, nlev, blockIdx.x);
  const CgLevel L = lv[l];
  const int64_t p = (int64_t)(blockIdx.x - L.block_begin) * blockDim.x + threadIdx.x;
  double rz = 0, rr = 0;
  if (p < L.npar) {
    const T* b = (const T*)L.b;
    T rv[3], zv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rv[a] = b[4 * p + a];
    apply_dinv<T>((const T*)L.Dinv, L.npar, p, rv, zv);
    T* x = (T*)L.x;
    T* r = (T*)L.r;
    T* z = (T*)L.z;
    T* pp = (T*)L.p;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[4 * p + a] = 0;
      r[4 * p + a] = rv[a];
      z[4 * p + a] = zv[a];
      pp[4 * p + a] = zv[a];
      rz += (double)rv[a] * (double)zv[a];
      rr += (double)rv[a] * (double)rv[a];
    }
    x[4 * p + 3] = 0;
    pp[4 * p + 3] = 0;
  }
  block_sum_add(rz, &sc[l].rz, red);
  block_sum_add(rr, &sc[l].rr, red);
}

// Levels l >= nlev_on stay inactive (truncated solves stop below them).
__global__ void k_cg_start(CgScalars* sc, int nlev, int nlev_on, double tol2, int* any_active) {
  if (threadIdx.x != 0) return;
  int act = 0;
  for (int l = 0; l < nlev; ++l) {
    CgScalars s = sc[l];
    s.rr0 = s.rr;
    s.active = l < nlev_on && s.rr > 0.0 && s.rz > 0.0;
    s.iters = 0;
    s.pAp = 0;
    s.rz_new = 0;
    s.rr_new = 0;
    act |= s.active;
    sc[l] = s;
  }
  *any_active = act;
}

// Entries 0..8 of a 32-byte float16 block record (two 16-byte words).
template <typename T>
__device__ __forceinline__ void unpack9(const uint4& u0, const uint4& u1, T* b) {
  const __half2* h0 = reinterpret_cast<const __half2*>(&u0);
  const __half2* h1 = reinterpret_cast<const __half2*>(&u1);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(h0[i]);
    b[2 * i] = (T)f.x;
    b[2 * i + 1] = (T)f.y;
  }
  b[8] = (T)__low2float(h1[0]);
}

// Ap = B p over the 3x3 detail blocks; pAp += p.Ap.  One CTA = one tile of
// T x T parents (T = 16, or 8 with four threads per parent splitting the
// offsets when the stencil is wide; or the whole lattice when smaller).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 0) k_cg_spmv(const CgLevel* __restrict__ lv, int nlev,
                                                 CgScalars* sc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const int l = find_level_spmv(lv, nlev, blockIdx.x);
  if (!sc[l].active) return;
  const CgLevel L = lv[l];
  const int spp = L.spp;
  const int tmax = cg_tile_side(spp);
  const int tile = L.Lpar < tmax ? L.Lpar : tmax;
  const int R = L.R;
  const int TS = tile + 2 * R;
  T* xs = reinterpret_cast<T*>(smem_raw);  // 3 planes of TS x TS
  const int64_t base = (int64_t)(blockIdx.x - L.spmv_begin) * (tmax * tmax);
  int x0, y0;
  demorton((uint32_t)base, x0, y0);
  const T* pv = (const T*)L.p;
  for (int c = threadIdx.x; c < TS * TS; c += blockDim.x) {
    const int gx = x0 - R + c % TS, gy = y0 - R + c / TS;
    T v0 = 0, v1 = 0, v2 = 0;
    if ((unsigned)gx < (unsigned)L.Lpar && (unsigned)gy < (unsigned)L.Lpar) {
      const int64_t q = morton((uint32_t)gx, (uint32_t)gy);
      if (q < L.npar) {
        v0 = pv[4 * q];
        v1 = pv[4 * q + 1];
        v2 = pv[4 * q + 2];
      }
    }
    xs[c] = v0;
    xs[TS * TS + c] = v1;
    xs[2 * TS * TS + c] = v2;
  }
  __syncthreads();
  const int pl = threadIdx.x / spp, sub = threadIdx.x - (threadIdx.x / spp) * spp;
  const int64_t p = base + pl;
  const bool own = pl < tile * tile && p < L.npar;
  T y0v = 0, y1v = 0, y2v = 0;
  int lx = 0, ly = 0;
  if (own) {
    int px, py;
    demorton((uint32_t)p, px, py);
    lx = px - x0 + R;
    ly = py - y0 + R;
    const int64_t np = L.npar;
    if (L.Bq) {
      // 32-byte float16 records of the half-plane offsets (two 16-byte loads
      // per block): the record of d at p gives B(p, p + d), the record of d
      // at p - d gives B(p, p - d) as its transpose, so each stored block is
      // read from DRAM once per product and serves both of its rows
      const uint4* Bq = reinterpret_cast<const uint4*>(L.Bq);
      for (int hh = sub; hh < L.nhoff; hh += spp) {
        const int2 d = L.hoff[hh];
        const int qn = (d.x | d.y) ? shift_cell(px, py, -d.x, -d.y, L.Lpar, np) : -1;
        const uint4 u0 = __ldg(Bq + ((int64_t)hh * np + p) * 2);
        const uint4 u1 = __ldg(Bq + ((int64_t)hh * np + p) * 2 + 1);
        uint4 w0 = make_uint4(0, 0, 0, 0), w1 = make_uint4(0, 0, 0, 0);
        if (qn >= 0) {
          w0 = __ldg(Bq + ((int64_t)hh * np + qn) * 2);
          w1 = __ldg(Bq + ((int64_t)hh * np + qn) * 2 + 1);
        }
        T b[9], b2[9];
        unpack9<T>(u0, u1, b);
        unpack9<T>(w0, w1, b2);
        const int c = (ly + d.y) * TS + lx + d.x;
        const int c2 = (ly - d.y) * TS + lx - d.x;
        const T a0 = xs[c], a1 = xs[TS * TS + c], a2 = xs[2 * TS * TS + c];
        const T e0 = xs[c2], e1 = xs[TS * TS + c2], e2 = xs[2 * TS * TS + c2];
        y0v += b[0] * a0 + b[1] * a1 + b[2] * a2 + b2[0] * e0 + b2[3] * e1 + b2[6] * e2;
        y1v += b[3] * a0 + b[4] * a1 + b[5] * a2 + b2[1] * e0 + b2[4] * e1 + b2[7] * e2;
        y2v += b[6] * a0 + b[7] * a1 + b[8] * a2 + b2[2] * e0 + b2[5] * e1 + b2[8] * e2;
      }
      const T si = (T)*L.bq_inv_scale;  // a power of two: exact
      y0v *= si;
      y1v *= si;
      y2v *= si;
    } else {
      const T* Bd = (const T*)L.Bd;
      // two offsets per pass: their 18 matrix loads are in flight together
      for (int o = sub; o < L.noff; o += 2 * spp) {
        const int o2 = o + spp;
        const bool two = o2 < L.noff;
        const int2 d = L.off[o];
        const int2 d2 = L.off[two ? o2 : o];
        const T* B = Bd + (int64_t)o * 9 * np + p;
        const T* B2 = Bd + (int64_t)(two ? o2 : o) * 9 * np + p;
        T b[9], b2[9];
#pragma unroll
        for (int e = 0; e < 9; ++e) b[e] = B[e * np];
#pragma unroll
        for (int e = 0; e < 9; ++e) b2[e] = two ? B2[e * np] : T(0);
        const int c = (ly + d.y) * TS + lx + d.x;
        const int c2 = (ly + d2.y) * TS + lx + d2.x;
        const T a0 = xs[c], a1 = xs[TS * TS + c], a2 = xs[2 * TS * TS + c];
        const T e0 = xs[c2], e1 = xs[TS * TS + c2], e2 = xs[2 * TS * TS + c2];
        y0v += b[0] * a0 + b[1] * a1 + b[2] * a2 + b2[0] * e0 + b2[1] * e1 + b2[2] * e2;
        y1v += b[3] * a0 + b[4] * a1 + b[5] * a2 + b2[3] * e0 + b2[4] * e1 + b2[5] * e2;
        y2v += b[6] * a0 + b[7] * a1 + b[8] * a2 + b2[6] * e0 + b2[7] * e1 + b2[8] * e2;
      }
    }
  }
  for (int o = 1; o < spp; o <<= 1) {
    y0v += __shfl_xor_sync(0xffffffffu, y0v, o);
    y1v += __shfl_xor_sync(0xffffffffu, y1v, o);
    y2v += __shfl_xor_sync(0xffffffffu, y2v, o);
  }
  T part = 0;
  if (own && sub == 0) {
    T* Ap = (T*)L.Ap;
    Ap[4 * p] = y0v;
    Ap[4 * p + 1] = y1v;
    Ap[4 * p + 2] = y2v;
    const int c0 = ly * TS + lx;
    part = xs[c0] * y0v + xs[TS * TS + c0] * y1v + xs[2 * TS * TS + c0] * y2v;
  }
  block_sum1_add<T>(part, &sc[l].pAp, red);
}

// x += alpha p, r -= alpha Ap, z = Dinv r; rz_new += r.z, rr_new += r.r
template <typename T>
__global__ void __launch_bounds__(256) k_cg_update(const CgLevel* __restrict__ lv, int nlev,
                                                   CgScalars* sc) {
  __shared__ double red[16];
  __shared__ T salpha;
  const int l = find_level(lv, nlev, blockIdx.x);
  if (!sc[l].active) return;
  const CgLevel L = lv[l];
  // alpha once per block: a float64 division per element would hold this
  // memory-bound kernel on the float64 pipe
  if (threadIdx.x == 0) {
    const double pAp = sc[l].pAp;
    salpha = pAp > 0 ? (T)(sc[l].rz / pAp) : T(0);
  }
  __syncthreads();
  const int64_t p = (int64_t)(blockIdx.x - L.block_begin) * blockDim.x + threadIdx.x;
  T rz = 0, rr = 0;
  if (p < L.npar) {
    const T alpha = salpha;
    T* x = (T*)L.x;
    T* r = (T*)L.r;
    T* z = (T*)L.z;
    const T* pv = (const T*)L.p;
    const T* Ap = (const T*)L.Ap;
    T rv[3], zv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[4 * p + a] += alpha * pv[4 * p + a];
      rv[a] = r[4 * p + a] - alpha * Ap[4 * p + a];
      r[4 * p + a] = rv[a];
    }
    apply_dinv<T>((const T*)L.Dinv, L.npar, p, rv, zv);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      z[4 * p + a] = zv[a];
      rz += rv[a] * zv[a];
      rr += rv[a] * rv[a];
    }
  }
  block_sum2_add<T>(rz, rr, &sc[l].rz_new, &sc[l].rr_new, red);
}

// beta, convergence on |r|_2, counters; one thread so any_active is exact
__global__ void k_cg_scalars(CgScalars* sc, int nlev, double tol2, int max_iter,
                             int* any_active, cudaGraphConditionalHandle cond, int use_cond,
                             int* loop_count, int loop_limit) {
  if (threadIdx.x != 0) return;
  int act = 0;
  for (int l = 0; l < nlev; ++l) {
    CgScalars s = sc[l];
    if (!s.active) continue;
    s.iters += 1;
    s.beta = s.rz > 0 ? s.rz_new / s.rz : 0.0;
    s.rz = s.rz_new;
    s.rr = s.rr_new;
    s.rz_new = 0;
    s.rr_new = 0;
    s.pAp = 0;
    if (s.rr <= tol2 * s.rr0 || s.iters >= max_iter || !(s.rr == s.rr) || !(s.rz > 0))
      s.active = 0;
    else
      act = 1;
    sc[l] = s;
  }
  *any_active = act;
  if (use_cond) {
    // body of a device-side while loop: continue while a level iterates;
    // the per-level caps end it, the pass counter bounds it regardless
    const int c = ++(*loop_count);
    cudaGraphSetConditional(cond, (act && c < loop_limit) ? 1u : 0u);
  }
}

// p = z + beta p
template <typename T>
__global__ void __launch_bounds__(256) k_cg_dir(const CgLevel* __restrict__ lv, int nlev,
                                                CgScalars* sc) {
  const int l = find_level(lv, nlev, blockIdx.x);
  if (!sc[l].active) return;
  const CgLevel L = lv[l];
  const int64_t p = (int64_t)(blockIdx.x - L.block_begin) * blockDim.x + threadIdx.x;
  if (p >= L.npar) return;
  const T beta = (T)sc[l].beta;
  T* pv = (T*)L.p;
  const T* z = (const T*)L.z;
#pragma unroll
  for (int a = 0; a < 3; ++a) pv[4 * p + a] = z[4 * p + a] + beta * pv[4 * p + a];
}

size_t cg_spmv_smem_bytes(int max_ts, size_t elem) { return 3 * elem * (size_t)max_ts * max_ts; }

template <typename T>
void launch_cg_init(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc,
                    cudaStream_t s) {
  if (total_blocks <= 0) return;
  { count_launch(); k_cg_init<T><<<total_blocks, 256, 0, s>>>(lv, nlev, sc); }
}

void launch_cg_start(CgScalars* sc, int nlev, int nlev_on, double tol2, int* any_active,
                     cudaStream_t s) {
  { count_launch(); k_cg_start<<<1, 32, 0, s>>>(sc, nlev, nlev_on, tol2, any_active); }
}

// Iteration counts of one level-CG call added to stats[k] (level k = l + 2)
// and stats[32] set when a solved level (k <= kmax) missed the tolerance, so
// that the host reads them once per solve instead of after every call.
// stats[33] accumulates the passes of the device-side loop (loop_count, may
// be NULL), each of which launched the four kernels of one CG iteration.
__global__ void k_cg_collect(const CgScalars* __restrict__ sc, int nlev, int kmax, double tol2,
                             const int* loop_count, int* stats) {
  const int l = threadIdx.x;
  if (l == 0 && loop_count) stats[33] += *loop_count;
  if (l >= nlev || l + 2 > 31) return;
  stats[l + 2] += sc[l].iters;
  if (l + 2 <= kmax && sc[l].rr > tol2 * sc[l].rr0) stats[32] = 1;
}

void launch_cg_collect(const CgScalars* sc, int nlev, int kmax, double tol2,
                       const int* loop_count, int* stats, cudaStream_t s) {
  if (nlev <= 0) return;
  count_launch();
  k_cg_collect<<<1, 32, 0, s>>>(sc, nlev, kmax, tol2, loop_count, stats);
}

template <typename T>
void prepare_cg_spmv(int max_ts) {
  const size_t smem = cg_spmv_smem_bytes(max_ts, sizeof(T));
  cudaFuncSetAttribute(k_cg_spmv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}
template void prepare_cg_spmv<float>(int);
template void prepare_cg_spmv<double>(int);

template <typename T>
void launch_cg_spmv(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc, int max_ts,
                    cudaStream_t s) {
  if (total_blocks <= 0) return;
  const size_t smem = cg_spmv_smem_bytes(max_ts, sizeof(T));
  { count_launch(); k_cg_spmv<T><<<total_blocks, 256, smem, s>>>(lv, nlev, sc); }
}

template <typename T>
void launch_cg_rest(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc, double tol2,
                    int max_iter, int* any_active, cudaStream_t s,
                    cudaGraphConditionalHandle cond, int use_cond, int* loop_count,
                    int loop_limit) {
  if (total_blocks <= 0) return;
  { count_launch(); k_cg_update<T><<<total_blocks, 256, 0, s>>>(lv, nlev, sc); }
  { count_launch(); k_cg_scalars<<<1, 32, 0, s>>>(sc, nlev, tol2, max_iter, any_active, cond, use_cond, loop_count, loop_limit); }
  { count_launch(); k_cg_dir<T><<<total_blocks, 256, 0, s>>>(lv, nlev, sc); }
}

template void launch_cg_init<float>(const CgLevel*, int, int, CgScalars*, cudaStream_t);
template void launch_cg_init<double>(const CgLevel*, int, int, CgScalars*, cudaStream_t);
template void launch_cg_spmv<float>(const CgLevel*, int, int, CgScalars*, int, cudaStream_t);
template void launch_cg_spmv<double>(const CgLevel*, int, int, CgScalars*, int, cudaStream_t);
template void launch_cg_rest<float>(const CgLevel*, int, int, CgScalars*, double, int, int*,
                                    cudaStream_t, cudaGraphConditionalHandle, int, int*, int);
template void launch_cg_rest<double>(const CgLevel*, int, int, CgScalars*, double, int, int*,
                                     cudaStream_t, cudaGraphConditionalHandle, int, int*, int);

// ---------------------------------------------------------------- set-up helpers
// Bd[o][3a+b][p] = Ahat[o][p][4a+b] (detail block, coalesced copy).
// One 4-entry row of a 4x4 block (16-byte aligned) as vector loads.
__device__ __forceinline__ void ldrow4(const float* p, float* r) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  r[0] = v.x;
  r[1] = v.y;
  r[2] = v.z;
  r[3] = v.w;
}
__device__ __forceinline__ void ldrow4(const double* p, double* r) {
  const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  r[0] = v0.x;
  r[1] = v0.y;
  r[2] = v1.x;
  r[3] = v1.y;
}

template <typename T>
__global__ void k_extract_detail(const T* __restrict__ Ahat, int noff, int64_t npar, T* Bd) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t p = t - (int64_t)o * npar;
  const T* A = Ahat + t * 16;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T row[4];
    ldrow4(A + 4 * a, row);  // one 16-byte load per block row
#pragma unroll
    for (int b = 0; b < 3; ++b) Bd[((int64_t)o * 9 + 3 * a + b) * npar + p] = row[b];
  }
}

// Dinv[e][p] = inverse of the active leading block of the diagonal detail
// block (zeros outside it), in the working precision (a 3x3 SPD block; the
// float64 pipe would make this kernel wait in the mixed path).  Fixed trip
// counts with predicates keep every array in registers.
// With amax, also the largest active diagonal entry of the level (atomicMax on
// its bits): B^(k) is symmetric positive definite, so |B_ij| <=
// sqrt(B_ii B_jj) and that entry bounds every entry of every block.
template <typename T>
__global__ void k_detail_dinv(const T* __restrict__ Ahat, int o0, int64_t npar,
                              const uint32_t* __restrict__ pmask, T* Dinv, unsigned* amax) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (amax) {  // warp-uniform: every lane reaches the shuffles
    float dm = 0.f;
    if (p < npar) {
      const int mm = __popc(pmask[p] & 15u);
      const int nn = mm > 0 ? mm - 1 : 0;
      const T* A = Ahat + ((int64_t)o0 * npar + p) * 16;
      for (int a = 0; a < nn; ++a) dm = fmaxf(dm, fabsf((float)A[5 * a]));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if ((threadIdx.x & 31) == 0 && dm > 0.f) atomicMax(amax, __float_as_uint(dm));
  }
  if (p >= npar) return;
  const int m = __popc(pmask[p] & 15u);
  const int na = m > 0 ? m - 1 : 0;
  T M[9], Inv[9];
  const T* A = Ahat + ((int64_t)o0 * npar + p) * 16;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T row[4];
    ldrow4(A + 4 * a, row);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      M[3 * a + b] = (a < na && b < na) ? row[b] : T(0);
      Inv[3 * a + b] = (a == b && a < na) ? T(1) : T(0);
    }
  }
  // Gauss-Jordan on the na x na SPD block (no pivoting needed)
  bool ok = true;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (c >= na) continue;
    const T d = M[4 * c];
    ok = ok && d > T(0);
    const T id = d > T(0) ? T(1) / d : T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      M[3 * c + b] *= id;
      Inv[3 * c + b] *= id;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a == c || a >= na) continue;
      const T f = M[3 * a + c];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        M[3 * a + b] -= f * M[3 * c + b];
        Inv[3 * a + b] -= f * Inv[3 * c + b];
      }
    }
  }
#pragma unroll
  for (int e = 0; e < 9; ++e) Dinv[(int64_t)e * npar + p] = ok ? Inv[e] : T(0);
}

template <typename T>
void launch_extract_detail(const T* Ahat, int noff, int64_t npar, T* Bd, cudaStream_t s) {
  const int64_t n = (int64_t)noff * npar;
  if (n > 0) {
    count_launch();
    k_extract_detail<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Ahat, noff, npar, Bd);
  }
}
template void launch_extract_detail<float>(const float*, int, int64_t, float*, cudaStream_t);
template void launch_extract_detail<double>(const double*, int, int64_t, double*, cudaStream_t);

template <typename T>
void launch_cg_level_setup(const T* Ahat, int noff, int o0, int64_t npar, const uint32_t* pmask,
                           T* Bd, T* Dinv, unsigned* amax, cudaStream_t s) {
  if (Bd) launch_extract_detail<T>(Ahat, noff, npar, Bd, s);
  if (amax) cudaMemsetAsync(amax, 0, sizeof(unsigned), s);
  if (npar > 0) {
    count_launch();
    k_detail_dinv<T><<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(Ahat, o0, npar, pmask, Dinv,
                                                                   amax);
  }
}
template void launch_cg_level_setup<float>(const float*, int, int, int64_t, const uint32_t*,
                                           float*, float*, unsigned*, cudaStream_t);

// One thread per block (h, p): the 3x3 detail block of offset hidx[h] at
// parent p as one 32-byte record.
__global__ void k_block_records(const float* __restrict__ Ahat, const int* __restrict__ hidx,
                                int nh, int64_t npar, const unsigned* __restrict__ amax, uint4* Bq,
                                float* inv_scale) {
  const float m = __uint_as_float(*amax);
  // 2^e <= m < 2^(e+1); the scale 2^(14 - e) puts the largest entry in [2^14, 2^15)
  const int e = m > 0.f ? ((__float_as_int(m) >> 23) & 255) - 127 : 0;
  const int a = max(min(14 - e, 100), -100);
  const float sc = ldexpf(1.f, a);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t == 0) *inv_scale = ldexpf(1.f, -a);
  if (t >= (int64_t)nh * npar) return;
  const int64_t hh = t / npar;
  const float* A = Ahat + ((int64_t)hidx[hh] * npar + (t - hh * npar)) * 16;
  float v[16];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float4 row = __ldg(reinterpret_cast<const float4*>(A + 4 * r));
    v[3 * r] = row.x * sc;
    v[3 * r + 1] = row.y * sc;
    v[3 * r + 2] = row.z * sc;
  }
#pragma unroll
  for (int i = 9; i < 16; ++i) v[i] = 0.f;
  uint4 w[2];
  __half2* h = reinterpret_cast<__half2*>(w);
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
  Bq[2 * t] = w[0];
  Bq[2 * t + 1] = w[1];
}

void launch_cg_block_records(const float* Ahat, const int* hidx, int nh, int64_t npar,
                             const unsigned* amax, void* Bq, float* inv_scale, cudaStream_t s) {
  if (nh <= 0 || npar <= 0) return;
  const int64_t nr = (int64_t)nh * npar;
  count_launch();
  k_block_records<<<(unsigned)((nr + 255) / 256), 256, 0, s>>>(Ahat, hidx, nh, npar, amax,
                                                               reinterpret_cast<uint4*>(Bq),
                                                               inv_scale);
}
template void launch_cg_level_setup<double>(const double*, int, int, int64_t, const uint32_t*,
                                            double*, double*, unsigned*, cudaStream_t);

// ---------------------------------------------------------------- diagnostics
// y = B^(k) x on the detail slots (thread per parent, float64 vectors): the
// plain operator of the level system, for the Lanczos estimate of its
// extreme eigenvalues.
template <typename T>
__global__ void k_detail_spmv(const T* __restrict__ Bd, const int2* __restrict__ off, int noff,
                              int Lpar, int64_t npar, const double* __restrict__ x, double* y) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npar) return;
  int px, py;
  demorton((uint32_t)p, px, py);
  double y0 = 0, y1 = 0, y2 = 0;
  for (int o = 0; o < noff; ++o) {
    const int qn = shift_cell(px, py, off[o].x, off[o].y, Lpar, npar);
    if (qn < 0) continue;
    const double a0 = x[4 * (int64_t)qn], a1 = x[4 * (int64_t)qn + 1], a2 = x[4 * (int64_t)qn + 2];
    const T* B = Bd + (int64_t)o * 9 * npar + p;
    y0 += (double)B[0] * a0 + (double)B[npar] * a1 + (double)B[2 * npar] * a2;
    y1 += (double)B[3 * npar] * a0 + (double)B[4 * npar] * a1 + (double)B[5 * npar] * a2;
    y2 += (double)B[6 * npar] * a0 + (double)B[7 * npar] * a1 + (double)B[8 * npar] * a2;
  }
  y[4 * p] = y0;
  y[4 * p + 1] = y1;
  y[4 * p + 2] = y2;
  y[4 * p + 3] = 0.0;
}

// Deterministic start vector on the active detail slots, zero elsewhere: the
// SplitMix64 output function (Steele, Lea and Flood, 2014) of the slot
// index, mapped to [-1, 1).
__global__ void k_detail_start(int64_t npar, const uint32_t* __restrict__ pmask, double* v) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npar) return;
  const int na = __popc(pmask[p] & 15u) - 1;
  for (int a = 0; a < 4; ++a) {
    uint64_t z = (uint64_t)(4 * p + a) + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    v[4 * p + a] = a < na ? (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0 : 0.0;
  }
}

template <typename T>
void launch_detail_spmv(const T* Bd, const int2* off, int noff, int Lpar, int64_t npar,
                        const double* x, double* y, cudaStream_t s) {
  if (npar > 0) { count_launch(); k_detail_spmv<T><<<(unsigned)((npar + 127) / 128), 128, 0, s>>>(Bd, off, noff, Lpar, npar, x, y); }
}
void launch_detail_start(int64_t npar, const uint32_t* pmask, double* v, cudaStream_t s) {
  if (npar > 0) { count_launch(); k_detail_start<<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(npar, pmask, v); }
}
template void launch_detail_spmv<float>(const float*, const int2*, int, int, int64_t,
                                        const double*, double*, cudaStream_t);
template void launch_detail_spmv<double>(const double*, const int2*, int, int, int64_t,
                                         const double*, double*, cudaStream_t);

// ---------------------------------------------------------------- several right-hand sides
template <typename T>
__global__ void __launch_bounds__(256) k_cgm_init(const CgLevel* __restrict__ lv, int nlev,
                                                  CgScalars* sc, int nrhs) {
  __shared__ double red[8];
  const int l = find_level(lv, nlev, blockIdx.x);
  const int rh = blockIdx.y;
  const CgLevel L = lv[l];
  const int64_t off = rh * L.rstride;
  const int64_t p = (int64_t)(blockIdx.x - L.block_begin) * blockDim.x + threadIdx.x;
  double rz = 0, rr = 0;
  if (p < L.npar) {
    const T* b = (const T*)L.b + off;
    T rv[3], zv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) rv[a] = b[4 * p + a];
    apply_dinv<T>((const T*)L.Dinv, L.npar, p, rv, zv);
    T* x = (T*)L.x + off;
    T* r = (T*)L.r + off;
    T* z = (T*)L.z + off;
    T* pp = (T*)L.p + off;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[4 * p + a] = 0;
      r[4 * p + a] = rv[a];
      z[4 * p + a] = zv[a];
      pp[4 * p + a] = zv[a];
      rz += (double)rv[a] * (double)zv[a];
      rr += (double)rv[a] * (double)rv[a];
    }
    x[4 * p + 3] = 0;
    pp[4 * p + 3] = 0;
  }
  block_sum_add(rz, &sc[l * nrhs + rh].rz, red);
  block_sum_add(rr, &sc[l * nrhs + rh].rr, red);
}

__global__ void k_cgm_start(CgScalars* sc, int n, double tol2, int* any_active) {
  if (threadIdx.x != 0) return;
  int act = 0;
  for (int i = 0; i < n; ++i) {
    CgScalars s = sc[i];
    s.rr0 = s.rr;
    s.active = s.rr > 0.0 && s.rz > 0.0;
    s.iters = 0;
    s.pAp = 0;
    s.rz_new = 0;
    s.rr_new = 0;
    act |= s.active;
    sc[i] = s;
  }
  *any_active = act;
}

// Ap = B p for every active right-hand side of the tile's level: the halo
// of each right-hand side is staged in shared memory and each 3x3 block is
// read once for all of them.
template <typename T>
__global__ void __launch_bounds__(256) k_cgm_spmv(const CgLevel* __restrict__ lv, int nlev,
                                                  CgScalars* sc, int nrhs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[8];
  const int l = find_level_spmv(lv, nlev, blockIdx.x);
  int act = 0;
  for (int r = 0; r < nrhs; ++r) act |= sc[l * nrhs + r].active << r;
  if (!act) return;
  const CgLevel L = lv[l];
  const int spp = L.spp;
  const int tmax = cg_tile_side(spp);
  const int tile = L.Lpar < tmax ? L.Lpar : tmax;
  const int R = L.R;
  const int TS = tile + 2 * R;
  const int plane = TS * TS;
  T* xs = reinterpret_cast<T*>(smem_raw);  // [nrhs][3][TS * TS]
  const int64_t base = (int64_t)(blockIdx.x - L.spmv_begin) * (tmax * tmax);
  int x0, y0;
  demorton((uint32_t)base, x0, y0);
  for (int c = threadIdx.x; c < plane; c += blockDim.x) {
    const int gx = x0 - R + c % TS, gy = y0 - R + c / TS;
    int64_t q = -1;
    if ((unsigned)gx < (unsigned)L.Lpar && (unsigned)gy < (unsigned)L.Lpar) {
      q = morton((uint32_t)gx, (uint32_t)gy);
      if (q >= L.npar) q = -1;
    }
    for (int r = 0; r < nrhs; ++r) {
      const T* pv = (const T*)L.p + r * L.rstride;
      const bool on = q >= 0 && ((act >> r) & 1);
      xs[(r * 3) * plane + c] = on ? pv[4 * q] : T(0);
      xs[(r * 3 + 1) * plane + c] = on ? pv[4 * q + 1] : T(0);
      xs[(r * 3 + 2) * plane + c] = on ? pv[4 * q + 2] : T(0);
    }
  }
  __syncthreads();
  const int pl = threadIdx.x / spp, sub = threadIdx.x - (threadIdx.x / spp) * spp;
  const int64_t p = base + pl;
  const bool own = pl < tile * tile && p < L.npar;
  T yv[kMaxRhs][3];
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r) yv[r][0] = yv[r][1] = yv[r][2] = T(0);
  int lx = 0, ly = 0;
  if (own) {
    int px, py;
    demorton((uint32_t)p, px, py);
    lx = px - x0 + R;
    ly = py - y0 + R;
    const T* Bd = (const T*)L.Bd;
    const uint4* Bq = reinterpret_cast<const uint4*>(L.Bq);
    const int64_t np = L.npar;
    if (Bq) {
      // the half-plane block records of the single-right-hand-side CG: the
      // record of d at p and, transposed, the record of d at p - d
      for (int hh = sub; hh < L.nhoff; hh += spp) {
        const int2 d = L.hoff[hh];
        const int qn = (d.x | d.y) ? shift_cell(px, py, -d.x, -d.y, L.Lpar, np) : -1;
        const int c = (ly + d.y) * TS + lx + d.x;
        const int c2 = (ly - d.y) * TS + lx - d.x;
        T b[9], bt[9];
        unpack9<T>(__ldg(Bq + ((int64_t)hh * np + p) * 2),
                   __ldg(Bq + ((int64_t)hh * np + p) * 2 + 1), b);
        if (qn >= 0) {
          unpack9<T>(__ldg(Bq + ((int64_t)hh * np + qn) * 2),
                     __ldg(Bq + ((int64_t)hh * np + qn) * 2 + 1), bt);
        } else {
#pragma unroll
          for (int e = 0; e < 9; ++e) bt[e] = T(0);
        }
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r) {
          if (r < nrhs) {
            const T a0 = xs[(r * 3) * plane + c], a1 = xs[(r * 3 + 1) * plane + c],
                    a2 = xs[(r * 3 + 2) * plane + c];
            const T e0 = xs[(r * 3) * plane + c2], e1 = xs[(r * 3 + 1) * plane + c2],
                    e2 = xs[(r * 3 + 2) * plane + c2];
            yv[r][0] += b[0] * a0 + b[1] * a1 + b[2] * a2 + bt[0] * e0 + bt[3] * e1 + bt[6] * e2;
            yv[r][1] += b[3] * a0 + b[4] * a1 + b[5] * a2 + bt[1] * e0 + bt[4] * e1 + bt[7] * e2;
            yv[r][2] += b[6] * a0 + b[7] * a1 + b[8] * a2 + bt[2] * e0 + bt[5] * e1 + bt[8] * e2;
          }
        }
      }
    } else {
      for (int o = sub; o < L.noff; o += spp) {
        const int2 d = L.off[o];
        const int c = (ly + d.y) * TS + lx + d.x;
        T b[9];
        const T* B = Bd + (int64_t)o * 9 * np + p;
#pragma unroll
        for (int e = 0; e < 9; ++e) b[e] = B[e * np];
#pragma unroll
        for (int r = 0; r < kMaxRhs; ++r) {
          if (r < nrhs) {
            const T a0 = xs[(r * 3) * plane + c], a1 = xs[(r * 3 + 1) * plane + c],
                    a2 = xs[(r * 3 + 2) * plane + c];
            yv[r][0] += b[0] * a0 + b[1] * a1 + b[2] * a2;
            yv[r][1] += b[3] * a0 + b[4] * a1 + b[5] * a2;
            yv[r][2] += b[6] * a0 + b[7] * a1 + b[8] * a2;
          }
        }
      }
    }
  }
  if (own && L.Bq) {
    const T si = (T)*L.bq_inv_scale;  // a power of two: exact
#pragma unroll
    for (int r = 0; r < kMaxRhs; ++r)
#pragma unroll
      for (int a = 0; a < 3; ++a) yv[r][a] *= si;
  }
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r)
    for (int o = 1; o < spp; o <<= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) yv[r][a] += __shfl_xor_sync(0xffffffffu, yv[r][a], o);
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r) {
    if (r >= nrhs) break;
    T part = 0;
    if (own && sub == 0 && ((act >> r) & 1)) {
      T* Ap = (T*)L.Ap + r * L.rstride;
      Ap[4 * p] = yv[r][0];
      Ap[4 * p + 1] = yv[r][1];
      Ap[4 * p + 2] = yv[r][2];
      const int c0 = ly * TS + lx;
      part = xs[(r * 3) * plane + c0] * yv[r][0] + xs[(r * 3 + 1) * plane + c0] * yv[r][1] +
             xs[(r * 3 + 2) * plane + c0] * yv[r][2];
    }
    block_sum1_add<T>(part, &sc[l * nrhs + r].pAp, red);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_cgm_update(const CgLevel* __restrict__ lv, int nlev,
                                                    CgScalars* sc, int nrhs) {
  __shared__ double red[16];
  const int l = find_level(lv, nlev, blockIdx.x);
  const int rh = blockIdx.y;
  CgScalars* S = &sc[l * nrhs + rh];
  if (!S->active) return;
  const CgLevel L = lv[l];
  const int64_t off = rh * L.rstride;
  __shared__ T salpha;  // once per block, as in k_cg_update
  if (threadIdx.x == 0) {
    const double pAp = S->pAp;
    salpha = pAp > 0 ? (T)(S->rz / pAp) : T(0);
  }
  __syncthreads();
  const int64_t p = (int64_t)(blockIdx.x - L.block_begin) * blockDim.x + threadIdx.x;
  T rz = 0, rr = 0;
  if (p < L.npar) {
    const T alpha = salpha;
    T* x = (T*)L.x + off;
    T* r = (T*)L.r + off;
    T* z = (T*)L.z + off;
    const T* pv = (const T*)L.p + off;
    const T* Ap = (const T*)L.Ap + off;
    T rv[3], zv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      x[4 * p + a] += alpha * pv[4 * p + a];
      rv[a] = r[4 * p + a] - alpha * Ap[4 * p + a];
      r[4 * p + a] = rv[a];
    }
    apply_dinv<T>((const T*)L.Dinv, L.npar, p, rv, zv);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      z[4 * p + a] = zv[a];
      rz += rv[a] * zv[a];
      rr += rv[a] * rv[a];
    }
  }
  block_sum2_add<T>(rz, rr, &S->rz_new, &S->rr_new, red);
}

__global__ void k_cgm_scalars(CgScalars* sc, int n, double tol2, int max_iter, int* any_active) {
  if (threadIdx.x != 0) return;
  int act = 0;
  for (int i = 0; i < n; ++i) {
    CgScalars s = sc[i];
    if (!s.active) continue;
    s.iters += 1;
    s.beta = s.rz > 0 ? s.rz_new / s.rz : 0.0;
    s.rz = s.rz_new;
    s.rr = s.rr_new;
    s.rz_new = 0;
    s.rr_new = 0;
    s.pAp = 0;
    if (s.rr <= tol2 * s.rr0 || s.iters >= max_iter || !(s.rr == s.rr) || !(s.rz > 0))
      s.active = 0;
    else
      act = 1;
    sc[i] = s;
  }
  *any_active = act;
}

template <typename T>
__global__ void __launch_bounds__(256) k_cgm_dir(const CgLevel* __restrict__ lv, int nlev,
                                                 CgScalars* sc, int nrhs) {
  const int l = find_level(lv, nlev, blockIdx.x);
  const int rh = blockIdx.y;
  const CgScalars* S = &sc[l * nrhs + rh];
  if (!S->active) return;
  const CgLevel L = lv[l];
  const int64_t p = (int64_t)(blockIdx.x - L.block_begin) * blockDim.x + threadIdx.x;
  if (p >= L.npar) return;
  const T beta = (T)S->beta;
  T* pv = (T*)L.p + rh * L.rstride;
  const T* z = (const T*)L.z + rh * L.rstride;
#pragma unroll
  for (int a = 0; a < 3; ++a) pv[4 * p + a] = z[4 * p + a] + beta * pv[4 * p + a];
}

size_t cgm_spmv_smem_bytes(int max_ts, size_t elem, int nrhs) {
  return 3 * elem * (size_t)max_ts * max_ts * (size_t)nrhs;
}

template <typename T>
void launch_cgm_init(const CgLevel* lv, int nlev, int total_blocks, CgScalars* sc, int nrhs,
                     cudaStream_t s) {
  if (total_blocks <= 0) return;
  count_launch();
  k_cgm_init<T><<<dim3(total_blocks, nrhs), 256, 0, s>>>(lv, nlev, sc, nrhs);
}
void launch_cgm_start(CgScalars* sc, int n, double tol2, int* any_active, cudaStream_t s) {
  count_launch();
  k_cgm_start<<<1, 32, 0, s>>>(sc, n, tol2, any_active);
}
template <typename T>
void launch_cgm_iteration(const CgLevel* lv, int nlev, int spmv_blocks, int total_blocks,
                          CgScalars* sc, int nrhs, int max_ts, double tol2, int max_iter,
                          int* any_active, cudaStream_t s) {
  if (total_blocks <= 0) return;
  const size_t smem = cgm_spmv_smem_bytes(max_ts, sizeof(T), nrhs);
  cudaFuncSetAttribute(k_cgm_spmv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  count_launch();
  k_cgm_spmv<T><<<spmv_blocks, 256, smem, s>>>(lv, nlev, sc, nrhs);
  count_launch();
  k_cgm_update<T><<<dim3(total_blocks, nrhs), 256, 0, s>>>(lv, nlev, sc, nrhs);
  count_launch();
  k_cgm_scalars<<<1, 32, 0, s>>>(sc, nlev * nrhs, tol2, max_iter, any_active);
  count_launch();
  k_cgm_dir<T><<<dim3(total_blocks, nrhs), 256, 0, s>>>(lv, nlev, sc, nrhs);
}
template void launch_cgm_init<float>(const CgLevel*, int, int, CgScalars*, int, cudaStream_t);
template void launch_cgm_init<double>(const CgLevel*, int, int, CgScalars*, int, cudaStream_t);
template void launch_cgm_iteration<float>(const CgLevel*, int, int, int, CgScalars*, int, int,
                                          double, int, int*, cudaStream_t);
template void launch_cgm_iteration<double>(const CgLevel*, int, int, int, CgScalars*, int, int,
                                           double, int, int*, cudaStream_t);

}  // namespace gb
