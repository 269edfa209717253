// solve.cu - the solve phase: restriction g^(k-1) = R g^(k) (Eq. eqyguugy6t),
// the independent level systems B^(k) w^(k) = W g^(k) solved by CG
// (Eq. eqsdjoejddi1, Sec. 4.9), the coarsest system A^(1) U^(1) = g^(1)
// (Eq. eqsdjoejddi2), prolongation and summation of the components
// (Theorem thddwedmgugyug), and the float64 outer operations.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

// 4-element loads as 128-bit transactions (rows of Rhat / RT and level
// vectors are 16-byte aligned: 4 T per neighbour or cell)
__device__ __forceinline__ void ld4(const float* p, float* b) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  b[0] = v.x;
  b[1] = v.y;
  b[2] = v.z;
  b[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* b) {
  const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
  b[0] = v0.x;
  b[1] = v0.y;
  b[2] = v1.x;
  b[3] = v1.y;
}

__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}

// ---------------------------------------------------------------- restriction
// Sixteen lanes per coarse row i (lanes over the neighbours j, so the row of
// R-hat is read with unit stride; four neighbours per lane, their loads
// issued before use), two rows per warp; the eight rows of a CTA are the
// children of two level-(k-2) parents, whose transforms Q^(k-1) are applied
// through shared memory before the write.
template <typename T>
__global__ void __launch_bounds__(128) k_restrict(const T* __restrict__ Rhat, int NB,
                                                  const int2* __restrict__ nbr, int Lpar,
                                                  int64_t nrow, const T* __restrict__ ghat, T* out,
                                                  const uint32_t* __restrict__ pmask_km1) {
  __shared__ T vals[8];
  const int l16 = threadIdx.x & 15, hr = threadIdx.x >> 4;
  const int64_t base = (int64_t)blockIdx.x * 8;
  const int64_t i = base + hr;
  T acc = 0;
  if (i < nrow) {
    int x, y;
    demorton((uint32_t)i, x, y);
    const T* row = Rhat + i * 4 * NB;
    for (int j0 = l16; j0 < NB; j0 += 64) {
      T r[4][4], gv[4][4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int j = j0 + 16 * v;
        const int p = j < NB ? shift_cell(x, y, nbr[j].x, nbr[j].y, Lpar, nrow) : -1;
#pragma unroll
        for (int c = 0; c < 4; ++c) r[v][c] = gv[v][c] = T(0);
        if (p >= 0) {
          ld4(row + 4 * j, r[v]);
          ld4(ghat + 4 * (int64_t)p, gv[v]);
        }
      }
#pragma unroll
      for (int v = 0; v < 4; ++v)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc += r[v][c] * gv[v][c];
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (pmask_km1 == nullptr) {
    if (l16 == 0 && i < nrow) out[i] = acc;
    return;
  }
  if (l16 == 0) vals[hr] = acc;
  __syncthreads();
  if (threadIdx.x < 8) {
    // all four slots of a parent are written: in the last parent of a prefix
    // the rows >= nrow are absent children (zero), but the slots of the
    // transformed vector are not
    const int q = threadIdx.x >> 2, a = threadIdx.x & 3;
    const int64_t pb = base + 4 * q;
    if (pb < nrow) {
      const int m = (int)pmask_km1[pb >> 2] & 15;
      const T* v = vals + 4 * q;
      out[pb + a] = qv<T>(m, a, 0) * v[0] + qv<T>(m, a, 1) * v[1] + qv<T>(m, a, 2) * v[2] +
                    qv<T>(m, a, 3) * v[3];
    }
  }
}

template <typename T>
void launch_restrict(const T* Rhat, int NB, const int2* nbr, int Lpar, int64_t nrow,
                     const T* ghat_k, T* g_km1, const uint32_t* pmask_km1, cudaStream_t s) {
  if (nrow <= 0) return;
  { count_launch(); k_restrict<T><<<(unsigned)((nrow + 7) / 8), 128, 0, s>>>(Rhat, NB, nbr, Lpar, nrow, ghat_k, g_km1, pmask_km1); }
}
template void launch_restrict<float>(const float*, int, const int2*, int, int64_t, const float*,
                                     float*, const uint32_t*, cudaStream_t);
template void launch_restrict<double>(const double*, int, const int2*, int, int64_t,
                                      const double*, double*, const uint32_t*, cudaStream_t);

// ---------------------------------------------------------------- prolongation
// RT[p][j][a] = Rhat[p - N_j][j][a]: the interpolation rows regrouped by the
// parent they reach, so the prolongation reads them with unit stride.
template <typename T>
__global__ void k_transpose_rhat(const T* __restrict__ Rhat, int NB, const int2* __restrict__ nbr,
                                 int Lpar, int64_t npar, T* RT) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npar * NB) return;
  const int64_t p = t / NB;
  const int j = (int)(t - p * NB);
  int x, y;
  demorton((uint32_t)p, x, y);
  const int i = shift_cell(x, y, -nbr[j].x, -nbr[j].y, Lpar, npar);
  // one 16-byte load and store per entry (slot 3 of RT is zero)
  T v[4] = {T(0), T(0), T(0), T(0)};
  if (i >= 0) ld4(Rhat + (int64_t)i * 4 * NB + 4 * j, v);
  v[3] = T(0);
  st4(RT + t * 4, v);
}

template <typename T>
void launch_transpose_rhat(const T* Rhat, int NB, const int2* nbr, int Lpar, int64_t npar, T* RT,
                           cudaStream_t s) {
  const int64_t n = npar * NB;
  if (n > 0) { count_launch(); k_transpose_rhat<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Rhat, NB, nbr, Lpar, npar, RT); }
}
template void launch_transpose_rhat<float>(const float*, int, const int2*, int, int64_t, float*,
                                           cudaStream_t);
template void launch_transpose_rhat<double>(const double*, int, const int2*, int, int64_t,
                                            double*, cudaStream_t);

// Sixteen lanes per parent p (two parents per warp, four neighbours' loads
// in flight per lane): vhat = [w; v_p / sqrt(m)] + sum_j RT[p][j] v[p - N_j],
// then (inverse) v = Q^T vhat.
template <typename T>
__global__ void __launch_bounds__(128) k_prolong(const T* __restrict__ RT, int NB,
                                                 const int2* __restrict__ nbr, int Lpar,
                                                 int64_t npar, const T* __restrict__ v,
                                                 const T* __restrict__ w,
                                                 const uint32_t* __restrict__ pmask, int inverse,
                                                 T* out) {
  const int l16 = threadIdx.x & 15;
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
  const bool valid = p < npar;  // no early exit: every lane takes part in the shuffles
  const int m = valid ? (int)pmask[p] & 15 : 0;
  T h0 = 0, h1 = 0, h2 = 0;
  if (m) {
    int x, y;
    demorton((uint32_t)p, x, y);
    const T* row = RT + p * 4 * NB;
    for (int j0 = l16; j0 < NB; j0 += 64) {
      T r[4][4], vv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = j0 + 16 * t;
        const int i = j < NB ? shift_cell(x, y, -nbr[j].x, -nbr[j].y, Lpar, npar) : -1;
#pragma unroll
        for (int c = 0; c < 4; ++c) r[t][c] = T(0);
        vv[t] = T(0);
        if (i >= 0) {
          ld4(row + 4 * j, r[t]);
          vv[t] = v[i];
        }
      }
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        h0 += r[t][0] * vv[t];
        h1 += r[t][1] * vv[t];
        h2 += r[t][2] * vv[t];
      }
    }
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    h0 += __shfl_xor_sync(0xffffffffu, h0, o);
    h1 += __shfl_xor_sync(0xffffffffu, h1, o);
    h2 += __shfl_xor_sync(0xffffffffu, h2, o);
  }
  if (l16 != 0 || !valid) return;
  T h3 = 0;
  if (m) {
    h3 = v[p] * inv_sqrt_q<T>(__popc(m));
    if (w) {
      h0 += w[4 * p];
      h1 += w[4 * p + 1];
      h2 += w[4 * p + 2];
    }
  }
  if (inverse) {
    T Q[16];
    qmat<T>(m, Q);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      out[4 * p + c] = Q[c] * h0 + Q[4 + c] * h1 + Q[8 + c] * h2 + Q[12 + c] * h3;
  } else {
    out[4 * p] = h0;
    out[4 * p + 1] = h1;
    out[4 * p + 2] = h2;
    out[4 * p + 3] = h3;
  }
}

template <typename T>
void launch_prolong(const T* RT, int NB, const int2* nbr, int Lpar, int64_t npar,
                    const T* v_km1, const T* w_k, const uint32_t* pmask_k, int inverse, T* out,
                    cudaStream_t s) {
  if (npar <= 0) return;
  { count_launch(); k_prolong<T><<<(unsigned)((npar * 16 + 127) / 128), 128, 0, s>>>(RT, NB, nbr, Lpar, npar, v_km1, w_k, pmask_k, inverse, out); }
}
template void launch_prolong<float>(const float*, int, const int2*, int, int64_t, const float*,
                                    const float*, const uint32_t*, int, float*, cudaStream_t);
template void launch_prolong<double>(const double*, int, const int2*, int, int64_t,
                                     const double*, const double*, const uint32_t*, int, double*,
                                     cudaStream_t);

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ void block_atomic_add(double v, double* dst) {
  __shared__ double red[32];
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0 && v != 0.0) atomicAdd(dst, v);
  }
  __syncthreads();  // red[] may be reused by the next call
}

// ---------------------------------------------------------------- coarsest level
// A^(1) (4 x 4, float64) from the level-1 cell stencil; Cholesky in place.
// Acell holds the nrow <= 4 level-1 cells that exist ([d][i], stride nrow).
template <typename T>
__global__ void k_level1_factor(const T* __restrict__ Acell, int nrow,
                                const int* __restrict__ map, double* A1, int* status) {
  if (threadIdx.x != 0) return;
  double M[16];
  for (int e = 0; e < 16; ++e) {
    const int i = e / 4, j = e % 4;
    const int d = map[e];
    double v = 0.0;
    if (i < nrow && j < nrow) {
      if (d >= 0) v = (double)Acell[(int64_t)d * nrow + i];
      else if (d <= -2) v = (double)Acell[(int64_t)(-d - 2) * nrow + j];
    }
    M[e] = v;
  }
  // inactive cells (zero row and column) become identity rows
  for (int i = 0; i < 4; ++i) {
    bool zero = true;
    for (int j = 0; j < 4; ++j) zero = zero && M[i * 4 + j] == 0.0;
    if (zero) M[i * 4 + i] = 1.0;
  }
  for (int j = 0; j < 4; ++j) {
    double d = M[j * 4 + j];
    for (int k = 0; k < j; ++k) d -= M[j * 4 + k] * M[j * 4 + k];
    if (!(d > 0)) {
      atomicExch(status, (int)DEV_NOT_SPD);
      d = 1.0;
    }
    d = sqrt(d);
    M[j * 4 + j] = d;
    for (int i = j + 1; i < 4; ++i) {
      double v = M[i * 4 + j];
      for (int k = 0; k < j; ++k) v -= M[i * 4 + k] * M[j * 4 + k];
      M[i * 4 + j] = v / d;
    }
  }
  for (int e = 0; e < 16; ++e) A1[e] = M[e];
}

template <typename T>
void launch_level1_factor(const T* Acell, int nrow, const int* map, double* A1, int* status,
                          cudaStream_t s) {
  { count_launch(); k_level1_factor<T><<<1, 32, 0, s>>>(Acell, nrow, map, A1, status); }
}
template void launch_level1_factor<float>(const float*, int, const int*, double*, int*,
                                          cudaStream_t);
template void launch_level1_factor<double>(const double*, int, const int*, double*, int*,
                                           cudaStream_t);

template <typename T>
__global__ void k_level1_solve(const double* __restrict__ L, const T* __restrict__ g, T* U) {
  if (threadIdx.x != 0) return;
  double z[4];
  for (int i = 0; i < 4; ++i) {
    double v = (double)g[i];
    for (int k = 0; k < i; ++k) v -= L[i * 4 + k] * z[k];
    z[i] = v / L[i * 4 + i];
  }
  for (int i = 3; i >= 0; --i) {
    double v = z[i];
    for (int k = i + 1; k < 4; ++k) v -= L[k * 4 + i] * z[k];
    z[i] = v / L[i * 4 + i];
  }
  for (int i = 0; i < 4; ++i) U[i] = (T)z[i];
}

template <typename T>
void launch_level1_solve(const double* L, const T* g, T* U, cudaStream_t s) {
  { count_launch(); k_level1_solve<T><<<1, 32, 0, s>>>(L, g, U); }
}
template void launch_level1_solve<float>(const double*, const float*, float*, cudaStream_t);
template void launch_level1_solve<double>(const double*, const double*, double*, cudaStream_t);

// ---------------------------------------------------------------- outer float64
// yhat = Q (A x) on the float64 level-q vectors: x untransformed (Morton
// order), A the node stencil St[s][c] over the cell offsets off[s].  One
// thread per parent: per offset its four cells' stencil values are 32
// contiguous bytes (one coalesced stream across the warp), then the
// parent's Q (rows unrolled, so its constants fold) transforms the result.
// With yhat = Q A Q^T xhat this is the transformed operator at 9 stored
// values per node instead of 36 per node in 4 x 4 transformed blocks.
__global__ void __launch_bounds__(256) k_stencil_spmv_q(const double* __restrict__ St,
                                                        const int2* __restrict__ off, int ns,
                                                        int L, int64_t ncell, int64_t npar,
                                                        const uint32_t* __restrict__ pmask,
                                                        const double* __restrict__ x,
                                                        double* yhat) {
  const int64_t P = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (P >= npar) return;
  int xc[4], yc[4];
  bool in[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    in[a] = 4 * P + a < ncell;
    demorton((uint32_t)(4 * P + a), xc[a], yc[a]);
  }
  double y[4] = {0.0, 0.0, 0.0, 0.0};
  for (int t = 0; t < ns; ++t) {
    const int2 o = off[t];
    const double2* s2 = reinterpret_cast<const double2*>(St + (int64_t)t * ncell + 4 * P);
    const double2 s01 = __ldg(s2), s23 = __ldg(s2 + 1);
    const double sv[4] = {s01.x, s01.y, s23.x, s23.y};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int nb = in[a] ? shift_cell(xc[a], yc[a], o.x, o.y, L, ncell) : -1;
      if (nb >= 0) y[a] += sv[a] * x[nb];
    }
  }
  const int m = (int)pmask[P] & 15;
#pragma unroll
  for (int a = 0; a < 4; ++a)
    yhat[4 * P + a] = qv<double>(m, a, 0) * y[0] + qv<double>(m, a, 1) * y[1] +
                      qv<double>(m, a, 2) * y[2] + qv<double>(m, a, 3) * y[3];
}

void launch_stencil_spmv_q(const double* St, const int2* off, int ns, int L, int64_t ncell,
                           int64_t npar, const uint32_t* pmask, const double* x, double* yhat,
                           cudaStream_t s) {
  if (npar <= 0) return;
  count_launch();
  k_stencil_spmv_q<<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(St, off, ns, L, ncell, npar,
                                                                  pmask, x, yhat);
}

__global__ void k_dots(int64_t n, const double* __restrict__ a0, const double* __restrict__ b0,
                       const double* __restrict__ a1, const double* __restrict__ b1,
                       const double* __restrict__ a2, const double* __restrict__ b2,
                       double* dots) {
  double s0 = 0, s1 = 0, s2 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (a0) s0 += a0[i] * b0[i];
    if (a1) s1 += a1[i] * b1[i];
    if (a2) s2 += a2[i] * b2[i];
  }
  if (a0) block_atomic_add(s0, &dots[0]);
  if (a1) block_atomic_add(s1, &dots[1]);
  if (a2) block_atomic_add(s2, &dots[2]);
}

void launch_dots(int64_t n, const double* a0, const double* b0, const double* a1,
                 const double* b1, const double* a2, const double* b2, double* dots,
                 cudaStream_t s) {
  if (n <= 0) return;
  // at most four blocks per SM: every block adds its partial sums to the
  // same three words, and those atomics serialise
  static thread_local int dev_cached = -1, sms = 152;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    dev_cached = dev;
  }
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4 * (int64_t)sms) blocks = 4 * (int64_t)sms;
  { count_launch(); k_dots<<<(unsigned)blocks, 256, 0, s>>>(n, a0, b0, a1, b1, a2, b2, dots); }
}

// Grid of a reduction kernel: at most four blocks per SM (every block adds
// its partial sums to the same words, and those atomics serialise).
static int64_t reduction_blocks(int64_t n) {
  static thread_local int dev_cached = -1, sms = 152;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != dev_cached) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    dev_cached = dev;
  }
  const int64_t blocks = (n + 255) / 256;
  return blocks > 4 * (int64_t)sms ? 4 * (int64_t)sms : blocks;
}

// One step of the outer flexible CG in one pass: u += (num / den) p,
// r -= (num / den) q, and *rr += r.r of the updated r.
__global__ void k_update_ur(int64_t n, const double* __restrict__ num,
                            const double* __restrict__ den, const double* __restrict__ p,
                            const double* __restrict__ q, double* u, double* r, double* rr) {
  __shared__ double sa;  // once per block, as in k_axpy
  if (threadIdx.x == 0) {
    const double d = *den;
    sa = d != 0.0 ? (*num) / d : 0.0;
  }
  __syncthreads();
  const double a = sa;
  double s0 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    u[i] += a * p[i];
    const double ri = r[i] - a * q[i];
    r[i] = ri;
    s0 += ri * ri;
  }
  block_atomic_add(s0, rr);
}
void launch_update_ur(int64_t n, const double* num, const double* den, const double* p,
                      const double* q, double* u, double* r, double* rr, cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_update_ur<<<(unsigned)reduction_blocks(n), 256, 0, s>>>(n, num, den, p, q, u, r, rr);
}

// z = (double) zf and *zq += z.q in one pass.
__global__ void k_widen_dot(int64_t n, const float* __restrict__ zf, double* z,
                            const double* __restrict__ q, double* zq) {
  double s0 = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double zi = (double)zf[i];
    z[i] = zi;
    s0 += zi * q[i];
  }
  block_atomic_add(s0, zq);
}
void launch_widen_dot(int64_t n, const float* zf, double* z, const double* q, double* zq,
                      cudaStream_t s) {
  if (n <= 0) return;
  count_launch();
  k_widen_dot<<<(unsigned)reduction_blocks(n), 256, 0, s>>>(n, zf, z, q, zq);
}

// y += sign * (num / den) * x
// (the scalar is formed once per block: a float64 division per element
// would hold this memory-bound kernel on the float64 pipe)
__global__ void k_axpy(int64_t n, const double* __restrict__ num, const double* __restrict__ den,
                       double sign, const double* __restrict__ x, double* y) {
  __shared__ double sa;
  if (threadIdx.x == 0) {
    const double d = *den;
    sa = d != 0.0 ? sign * (*num) / d : 0.0;
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] += sa * x[i];
}
void launch_axpy(int64_t n, const double* alpha_num, const double* alpha_den, double sign,
                 const double* x, double* y, cudaStream_t s) {
  if (n > 0)
    { count_launch(); k_axpy<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, alpha_num, alpha_den, sign, x, y); }
}
// p = x + sign * (num / den) * p
__global__ void k_xpby(int64_t n, const double* __restrict__ x, const double* __restrict__ num,
                       const double* __restrict__ den, double sign, double* p) {
  __shared__ double sb;  // once per block, as in k_axpy
  if (threadIdx.x == 0) {
    const double d = *den;
    sb = d != 0.0 ? sign * (*num) / d : 0.0;
  }
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = x[i] + sb * p[i];
}
void launch_xpby(int64_t n, const double* x, const double* beta_num, const double* beta_den,
                 double sign, double* p, cudaStream_t s) {
  if (n > 0)
    { count_launch(); k_xpby<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, beta_num, beta_den, sign, p); }
}

// ---------------------------------------------------------------- adjoint contraction
__constant__ double c_Kref[16];

void launch_set_kref(const double* K_ref_host) {
  cudaMemcpyToSymbol(c_Kref, K_ref_host, 16 * sizeof(double));
}

__global__ void k_adjoint_contract(int ncell, const int32_t* __restrict__ cn,
                                   const double* __restrict__ a, const double* __restrict__ lam,
                                   const double* __restrict__ u, double* dJ) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  double lv[4], uv[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const int nd = cn[4 * c + p];
    lv[p] = nd >= 0 ? lam[nd] : 0.0;
    uv[p] = nd >= 0 ? u[nd] : 0.0;
  }
  double s = 0;
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int r = 0; r < 4; ++r) s += lv[p] * c_Kref[p * 4 + r] * uv[r];
  dJ[c] = -a[c] * s;
}

// A values from the cell coefficients: each cell adds exp(log_a) K_ref on
// its interior corner pairs; the CSR position is found by binary search.
__global__ void k_assemble_cells(int n, const int32_t* __restrict__ rowptr,
                                 const int32_t* __restrict__ colind, int ncell,
                                 const int32_t* __restrict__ cn, const double* __restrict__ log_a,
                                 double* val, double* cell_a, int* missing) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const double a = exp(log_a[c]);
  if (cell_a) cell_a[c] = a;
  int nd[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) nd[p] = cn[4 * c + p];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    if (nd[p] < 0 || nd[p] >= n) continue;
    const int b = rowptr[nd[p]], e = rowptr[nd[p] + 1];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (nd[r] < 0 || nd[r] >= n) continue;
      int lo = b, hi = e - 1, pos = -1;
      while (lo <= hi) {
        const int mid = (lo + hi) >> 1;
        const int cm = colind[mid];
        if (cm == nd[r]) {
          pos = mid;
          break;
        }
        if (cm < nd[r]) lo = mid + 1;
        else hi = mid - 1;
      }
      if (pos < 0) {
        atomicExch(missing, 1);
        continue;
      }
      atomicAdd(&val[pos], a * c_Kref[p * 4 + r]);
    }
  }
}

void launch_assemble_cells(int n, const int32_t* rowptr, const int32_t* colind, int ncell,
                           const int32_t* cell_nodes, const double* log_a, double* val,
                           double* cell_a, int* missing, cudaStream_t s) {
  if (ncell > 0) {
    count_launch();
    k_assemble_cells<<<(ncell + 255) / 256, 256, 0, s>>>(n, rowptr, colind, ncell, cell_nodes,
                                                         log_a, val, cell_a, missing);
  }
}

void launch_adjoint_contract(int ncell, const int32_t* cell_nodes, const double* cell_a,
                             const double* lam, const double* u, double* dJ, cudaStream_t s) {
  if (ncell > 0)
    { count_launch(); k_adjoint_contract<<<(ncell + 255) / 256, 256, 0, s>>>(ncell, cell_nodes, cell_a, lam, u, dJ); }
}

// ---------------------------------------------------------------- compression
// Normalised detail coefficients c = w^(k)_j sqrt(B^(k)_jj) (||chi_j||_a),
// B_jj being entry (a, a) of the diagonal detail block Bd[o0][4a][p].
template <typename T>
__device__ __forceinline__ double coef_norm(const T* __restrict__ w, const T* __restrict__ Bd,
                                            int o0, int64_t npar, int64_t p, int a) {
  const double b = (double)Bd[((int64_t)o0 * 9 + 4 * a) * npar + p];
  return fabs((double)w[4 * p + a]) * sqrt(b > 0 ? b : 0.0);
}

template <typename T>
__global__ void k_coef_max(const T* __restrict__ w, const T* __restrict__ Bd, int o0,
                           int64_t npar, const uint32_t* __restrict__ pmask,
                           unsigned long long* cmax) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double m = 0;
  if (p < npar) {
    const int na = __popc(pmask[p] & 15u) - 1;
    for (int a = 0; a < na; ++a) m = fmax(m, coef_norm(w, Bd, o0, npar, p, a));
  }
  // non-negative doubles order as their bit patterns
  if (m > 0) atomicMax(cmax, (unsigned long long)__double_as_longlong(m));
}

template <typename T>
__global__ void k_coef_threshold(T* w, const T* __restrict__ Bd, int o0, int64_t npar,
                                 const uint32_t* __restrict__ pmask, double thr,
                                 unsigned long long* kept) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npar) return;
  const int na = __popc(pmask[p] & 15u) - 1;
  int k = 0;
  for (int a = 0; a < na; ++a) {
    if (coef_norm(w, Bd, o0, npar, p, a) >= thr) ++k;
    else w[4 * p + a] = T(0);
  }
  if (k) atomicAdd(kept, (unsigned long long)k);
}

template <typename T>
void launch_coef_max(const T* w, const T* Bd, int o0, int64_t npar, const uint32_t* pmask,
                     unsigned long long* cmax, cudaStream_t s) {
  if (npar > 0) { count_launch(); k_coef_max<T><<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(w, Bd, o0, npar, pmask, cmax); }
}
template <typename T>
void launch_coef_threshold(T* w, const T* Bd, int o0, int64_t npar, const uint32_t* pmask,
                           double thr, unsigned long long* kept, cudaStream_t s) {
  if (npar > 0) { count_launch(); k_coef_threshold<T><<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(w, Bd, o0, npar, pmask, thr, kept); }
}
template void launch_coef_max<float>(const float*, const float*, int, int64_t, const uint32_t*,
                                     unsigned long long*, cudaStream_t);
template void launch_coef_max<double>(const double*, const double*, int, int64_t,
                                      const uint32_t*, unsigned long long*, cudaStream_t);
template void launch_coef_threshold<float>(float*, const float*, int, int64_t, const uint32_t*,
                                           double, unsigned long long*, cudaStream_t);
template void launch_coef_threshold<double>(double*, const double*, int, int64_t,
                                            const uint32_t*, double, unsigned long long*,
                                            cudaStream_t);

// out = a x + b y + c z (y, z may be NULL); out may alias x.
__global__ void k_lanczos_step(int64_t n, double a, const double* x, const double* y, double b,
                               const double* z, double c, double* out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = a * x[i];
  if (y) v += b * y[i];
  if (z) v += c * z[i];
  out[i] = v;
}
void launch_lanczos_step(int64_t n, double a, const double* x, const double* y, double b,
                         const double* z, double c, double* out, cudaStream_t s) {
  if (n > 0) { count_launch(); k_lanczos_step<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, x, y, b, z, c, out); }
}

// Change of detail basis on transformed level vectors, per parent with
// cnt active children: out = M in (transpose = 0) or M^T in (1), with
// M = W1 W2^T the matrix taking the orthonormal Helmert rows W2 (the stored
// basis) to the consecutive differences W1 of Construction const1 (row t:
// child t minus child t + 1, in the order of the active children).  Then
// W1 A W1^T = M B M^T.  Slot 3 and inactive slots are zero on output.
// in and out may be the same array: a thread reads its parent's slots
// before it writes them, and parents do not overlap.
__global__ void k_detail_basis(int64_t npar, const uint32_t* __restrict__ pmask,
                               const double* in, double* out, int transpose) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= npar) return;
  const int m = (int)pmask[p] & 15;
  const int cnt = __popc(m);
  int cidx[4] = {0, 0, 0, 0};  // slot of the j-th active child
  for (int c = 0, j = 0; c < 4; ++c)
    if ((m >> c) & 1) cidx[j++] = c;
  double M[3][3];
  for (int t = 0; t < 3; ++t)
    for (int a = 0; a < 3; ++a) {
      M[t][a] = 0.0;
      if (t < cnt - 1 && a < cnt - 1)
        M[t][a] = qv<double>(m, a, cidx[t]) - qv<double>(m, a, cidx[t + 1]);
    }
  const double x0 = in[4 * p], x1 = in[4 * p + 1], x2 = in[4 * p + 2];
  for (int t = 0; t < 3; ++t) {
    const double v = transpose ? M[0][t] * x0 + M[1][t] * x1 + M[2][t] * x2
                               : M[t][0] * x0 + M[t][1] * x1 + M[t][2] * x2;
    out[4 * p + t] = t < cnt - 1 ? v : 0.0;
  }
  out[4 * p + 3] = 0.0;
}
void launch_detail_basis(int64_t npar, const uint32_t* pmask, const double* in, double* out,
                         int transpose, cudaStream_t s) {
  if (npar > 0) {
    count_launch();
    k_detail_basis<<<(unsigned)((npar + 255) / 256), 256, 0, s>>>(npar, pmask, in, out, transpose);
  }
}

// ---------------------------------------------------------------- several right-hand sides
// Restriction of nrhs vectors: the row of Rhat is read once per lane and
// applied to the neighbours' slots of every right-hand side.
template <typename T>
__global__ void __launch_bounds__(128) k_restrict_m(const T* __restrict__ Rhat, int NB,
                                                    const int2* __restrict__ nbr, int Lpar,
                                                    int64_t nrow, const T* __restrict__ ghat,
                                                    int64_t gstride, T* out, int64_t ostride,
                                                    const uint32_t* __restrict__ pmask_km1,
                                                    int nrhs) {
  __shared__ T vals[kMaxRhs][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * 4 + w;
  T acc[kMaxRhs];
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r) acc[r] = T(0);
  if (i < nrow) {
    int x, y;
    demorton((uint32_t)i, x, y);
    const T* row = Rhat + i * 4 * NB;
    for (int j = lane; j < NB; j += 32) {
      const int p = shift_cell(x, y, nbr[j].x, nbr[j].y, Lpar, nrow);
      if (p < 0) continue;
      T rv[4];
      ld4(row + 4 * j, rv);
#pragma unroll
      for (int r = 0; r < kMaxRhs; ++r) {
        if (r < nrhs) {
          T gv[4];
          ld4(ghat + r * gstride + 4 * (int64_t)p, gv);
          acc[r] += rv[0] * gv[0] + rv[1] * gv[1] + rv[2] * gv[2] + rv[3] * gv[3];
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
  if (pmask_km1 == nullptr) {
    if (lane == 0 && i < nrow)
      for (int r = 0; r < nrhs; ++r) out[r * ostride + i] = acc[r];
    return;
  }
  if (lane == 0)
#pragma unroll
    for (int r = 0; r < kMaxRhs; ++r) vals[r][w] = acc[r];
  __syncthreads();
  if (threadIdx.x < 4 * nrhs) {
    const int r = threadIdx.x >> 2, a = threadIdx.x & 3;
    const int64_t base = (int64_t)blockIdx.x * 4;
    const int m = (int)pmask_km1[base >> 2] & 15;
    out[r * ostride + base + a] = qv<T>(m, a, 0) * vals[r][0] + qv<T>(m, a, 1) * vals[r][1] +
                                  qv<T>(m, a, 2) * vals[r][2] + qv<T>(m, a, 3) * vals[r][3];
  }
}

template <typename T>
void launch_restrict_m(const T* Rhat, int NB, const int2* nbr, int Lpar, int64_t nrow,
                       const T* ghat_k, int64_t gstride, T* g_km1, int64_t ostride,
                       const uint32_t* pmask_km1, int nrhs, cudaStream_t s) {
  if (nrow <= 0) return;
  count_launch();
  k_restrict_m<T><<<(unsigned)((nrow + 3) / 4), 128, 0, s>>>(Rhat, NB, nbr, Lpar, nrow, ghat_k,
                                                             gstride, g_km1, ostride, pmask_km1,
                                                             nrhs);
}
template void launch_restrict_m<float>(const float*, int, const int2*, int, int64_t, const float*,
                                       int64_t, float*, int64_t, const uint32_t*, int,
                                       cudaStream_t);
template void launch_restrict_m<double>(const double*, int, const int2*, int, int64_t,
                                        const double*, int64_t, double*, int64_t, const uint32_t*,
                                        int, cudaStream_t);

// Prolongation of nrhs vectors with the rows of RT read once.
template <typename T>
__global__ void __launch_bounds__(128) k_prolong_m(const T* __restrict__ RT, int NB,
                                                   const int2* __restrict__ nbr, int Lpar,
                                                   int64_t npar, const T* __restrict__ v,
                                                   int64_t vstride, const T* __restrict__ w,
                                                   int64_t wstride,
                                                   const uint32_t* __restrict__ pmask, int inverse,
                                                   T* out, int64_t ostride, int nrhs) {
  const int lane = threadIdx.x & 31;
  const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (p >= npar) return;
  const int m = (int)pmask[p] & 15;
  T h[kMaxRhs][3];
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r) h[r][0] = h[r][1] = h[r][2] = T(0);
  if (m) {
    int x, y;
    demorton((uint32_t)p, x, y);
    const T* row = RT + p * 4 * NB;
    for (int j = lane; j < NB; j += 32) {
      const int i = shift_cell(x, y, -nbr[j].x, -nbr[j].y, Lpar, npar);
      if (i < 0) continue;
      T rv[4];
      ld4(row + 4 * j, rv);
#pragma unroll
      for (int r = 0; r < kMaxRhs; ++r) {
        if (r < nrhs) {
          const T vi = v[r * vstride + i];
          h[r][0] += rv[0] * vi;
          h[r][1] += rv[1] * vi;
          h[r][2] += rv[2] * vi;
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int a = 0; a < 3; ++a) h[r][a] += __shfl_xor_sync(0xffffffffu, h[r][a], o);
  if (lane >= nrhs) return;
  // lane r writes right-hand side r
  T hh[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int r = 0; r < kMaxRhs; ++r)
    if (r == lane) {
      hh[0] = h[r][0];
      hh[1] = h[r][1];
      hh[2] = h[r][2];
    }
  const int r = lane;
  if (m) {
    hh[3] = v[r * vstride + p] * (T(1) / sqrt(T(__popc(m))));
    if (w) {
      hh[0] += w[r * wstride + 4 * p];
      hh[1] += w[r * wstride + 4 * p + 1];
      hh[2] += w[r * wstride + 4 * p + 2];
    }
  }
  T* o = out + r * ostride + 4 * p;
  if (inverse) {
    T Q[16];
    qmat<T>(m, Q);
#pragma unroll
    for (int c = 0; c < 4; ++c)
      o[c] = Q[c] * hh[0] + Q[4 + c] * hh[1] + Q[8 + c] * hh[2] + Q[12 + c] * hh[3];
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = hh[c];
  }
}

template <typename T>
void launch_prolong_m(const T* RT, int NB, const int2* nbr, int Lpar, int64_t npar,
                      const T* v_km1, int64_t vstride, const T* w_k, int64_t wstride,
                      const uint32_t* pmask_k, int inverse, T* out, int64_t ostride, int nrhs,
                      cudaStream_t s) {
  if (npar <= 0) return;
  count_launch();
  k_prolong_m<T><<<(unsigned)((npar * 32 + 127) / 128), 128, 0, s>>>(
      RT, NB, nbr, Lpar, npar, v_km1, vstride, w_k, wstride, pmask_k, inverse, out, ostride, nrhs);
}
template void launch_prolong_m<float>(const float*, int, const int2*, int, int64_t, const float*,
                                      int64_t, const float*, int64_t, const uint32_t*, int,
                                      float*, int64_t, int, cudaStream_t);
template void launch_prolong_m<double>(const double*, int, const int2*, int, int64_t,
                                       const double*, int64_t, const double*, int64_t,
                                       const uint32_t*, int, double*, int64_t, int, cudaStream_t);


}  // namespace gb
