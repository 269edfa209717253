// dense.cu - dense float64 kernels of the exact (non-localized) transform,
// Algorithm 1 of Sec. 5.2: B^(k) = W A^(k) W^T factored once per level,
// D^(k,k-1) = -B^-1 W A pibar^T for every coarse column at once, and the
// Galerkin product R A R^T as two dense products.  Used for small problems
// (every level held densely); the localized path never calls them.
#include "common.cuh"
#include "kernels.cuh"

namespace gb {

// Dense matrix (nslot x nslot, row-major) from a transformed block stencil.
__global__ void k_dense_from_blocks(const double* __restrict__ blk, const int2* __restrict__ off,
                                    int noff, int Lpar, int64_t npar, double* D) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)noff * npar) return;
  const int o = (int)(t / npar);
  const int64_t p = t - (int64_t)o * npar;
  int x, y;
  demorton((uint32_t)p, x, y);
  const int pp = shift_cell(x, y, off[o].x, off[o].y, Lpar, npar);
  if (pp < 0) return;
  const int64_t ld = 4 * npar;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) D[(4 * p + a) * ld + 4 * pp + b] = blk[t * 16 + a * 4 + b];
}

void launch_dense_from_blocks(const double* blk, const int2* off, int noff, int Lpar,
                              int64_t npar, double* D, cudaStream_t s) {
  const int64_t n = (int64_t)noff * npar;
  if (n > 0)
    { count_launch(); k_dense_from_blocks<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(blk, off, noff, Lpar, npar, D); }
}

// Blockwise transform of a dense level matrix: D <- Qblk D Qblk^T.
__global__ void k_dense_transform(const double* __restrict__ in, int64_t npar,
                                  const uint32_t* __restrict__ pmask, double* out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= npar * npar) return;
  const int64_t P = t / npar, PP = t - P * npar;
  const int mr = (int)pmask[P] & 15, mc = (int)pmask[PP] & 15;
  const int64_t ld = 4 * npar;
  double M[16], Tm[16], Qr[16], Qc[16];
  qmat<double>(mr, Qr);
  qmat<double>(mc, Qc);
  for (int c = 0; c < 4; ++c)
    for (int cc = 0; cc < 4; ++cc) M[c * 4 + cc] = in[(4 * P + c) * ld + 4 * PP + cc];
  for (int a = 0; a < 4; ++a)
    for (int cc = 0; cc < 4; ++cc) {
      double acc = 0;
      for (int c = 0; c < 4; ++c) acc += Qr[a * 4 + c] * M[c * 4 + cc];
      Tm[a * 4 + cc] = acc;
    }
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) {
      double acc = 0;
      for (int cc = 0; cc < 4; ++cc) acc += Tm[a * 4 + cc] * Qc[b * 4 + cc];
      out[(4 * P + a) * ld + 4 * PP + b] = acc;
    }
}

void launch_dense_transform(const double* in, int64_t npar, const uint32_t* pmask, double* out,
                            cudaStream_t s) {
  const int64_t n = npar * npar;
  if (n > 0) { count_launch(); k_dense_transform<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(in, npar, pmask, out); }
}

// C = alpha op(A) op(B) + beta C, row-major, 16 x 16 shared-memory tiles.
template <int TA, int TB>
__global__ void k_dgemm(int m, int n, int kk, double alpha, const double* __restrict__ A,
                        const double* __restrict__ B, double beta, double* C) {
  __shared__ double As[16][17], Bs[16][17];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int row = blockIdx.y * 16 + ty, colx = blockIdx.x * 16 + tx;
  double acc = 0;
  for (int k0 = 0; k0 < kk; k0 += 16) {
    {  // A tile: rows blockIdx.y*16.., cols k0..
      const int r = blockIdx.y * 16 + ty, c = k0 + tx;
      double v = 0;
      if (r < m && c < kk) v = TA ? A[(int64_t)c * m + r] : A[(int64_t)r * kk + c];
      As[ty][tx] = v;
    }
    {  // B tile: rows k0.., cols blockIdx.x*16..
      const int r = k0 + ty, c = blockIdx.x * 16 + tx;
      double v = 0;
      if (r < kk && c < n) v = TB ? B[(int64_t)c * kk + r] : B[(int64_t)r * n + c];
      Bs[ty][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < 16; ++e) acc += As[ty][e] * Bs[e][tx];
    __syncthreads();
  }
  if (row < m && colx < n) {
    double* cp = C + (int64_t)row * n + colx;
    *cp = alpha * acc + (beta != 0.0 ? beta * *cp : 0.0);
  }
}

void launch_dgemm_t(int m, int n, int kk, double alpha, const double* A, int transA,
                    const double* B, int transB, double beta, double* C, cudaStream_t s) {
  if (m <= 0 || n <= 0) return;
  dim3 blk(16, 16), grd((n + 15) / 16, (m + 15) / 16);
  if (!transA && !transB) { count_launch(); k_dgemm<0, 0><<<grd, blk, 0, s>>>(m, n, kk, alpha, A, B, beta, C); }
  else if (!transA && transB) { count_launch(); k_dgemm<0, 1><<<grd, blk, 0, s>>>(m, n, kk, alpha, A, B, beta, C); }
  else if (transA && !transB) { count_launch(); k_dgemm<1, 0><<<grd, blk, 0, s>>>(m, n, kk, alpha, A, B, beta, C); }
  else { count_launch(); k_dgemm<1, 1><<<grd, blk, 0, s>>>(m, n, kk, alpha, A, B, beta, C); }
}

void launch_dgemm(int m, int n, int kk, double alpha, const double* A, const double* B,
                  int transB, double beta, double* C, cudaStream_t s) {
  launch_dgemm_t(m, n, kk, alpha, A, 0, B, transB, beta, C, s);
}

// In-place lower Cholesky (single CTA, right-looking); upper part untouched.
__global__ void k_dpotrf(double* A, int n, int* status) {
  __shared__ double s_inv;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x == 0) {
      double d = A[(int64_t)j * n + j];
      if (!(d > 0)) {
        atomicExch(status, (int)DEV_NOT_SPD);
        d = 1.0;
      }
      d = sqrt(d);
      A[(int64_t)j * n + j] = d;
      s_inv = 1.0 / d;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int r = j + 1 + threadIdx.x; r < n; r += blockDim.x) A[(int64_t)r * n + j] *= inv;
    __syncthreads();
    const int64_t m = n - j - 1;
    for (int64_t e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int r = j + 1 + (int)(e / m), c = j + 1 + (int)(e % m);
      if (c <= r) A[(int64_t)r * n + c] -= A[(int64_t)r * n + j] * A[(int64_t)c * n + j];
    }
    __syncthreads();
  }
}

void launch_dpotrf(double* A, int n, int* status, cudaStream_t s) {
  if (n > 0) { count_launch(); k_dpotrf<<<1, 1024, 0, s>>>(A, n, status); }
}

// Solve L L^T x = b for column `col` of B (n x nrhs row-major); one warp per column.
__global__ void k_dpotrs(const double* __restrict__ L, int n, double* B, int nrhs) {
  extern __shared__ double z[];
  const int col = blockIdx.x;
  const int lane = threadIdx.x;
  for (int i = lane; i < n; i += 32) z[i] = B[(int64_t)i * nrhs + col];
  __syncwarp();
  for (int i = 0; i < n; ++i) {  // forward: z_i = (b_i - L_i. z) / L_ii
    double acc = 0;
    for (int k = lane; k < i; k += 32) acc += L[(int64_t)i * n + k] * z[k];
    acc = warp_sum(acc);
    if (lane == 0) z[i] = (z[i] - acc) / L[(int64_t)i * n + i];
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {  // backward, row-oriented on L
    const double yi = z[i] / L[(int64_t)i * n + i];
    __syncwarp();
    for (int k = lane; k < i; k += 32) z[k] -= L[(int64_t)i * n + k] * yi;
    if (lane == 0) z[i] = yi;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) B[(int64_t)i * nrhs + col] = z[i];
}

void launch_dpotrs(const double* L, int n, double* B, int nrhs, cudaStream_t s) {
  if (n <= 0 || nrhs <= 0) return;
  size_t smem = sizeof(double) * (size_t)n;
  cudaFuncSetAttribute(k_dpotrs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  { count_launch(); k_dpotrs<<<nrhs, 32, smem, s>>>(L, n, B, nrhs); }
}

// out[a][b] = D[rows[a]][cols[b]] * alpha * (col_scale ? col_scale[b] : 1)
__global__ void k_gather_rc(const double* __restrict__ D, int ld, const int32_t* __restrict__ rows,
                            int nr, const int32_t* __restrict__ cols, int nc, double alpha,
                            const double* __restrict__ col_scale, double* out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)nr * nc) return;
  const int a = (int)(t / nc), b = (int)(t % nc);
  double v = D[(int64_t)rows[a] * ld + cols[b]] * alpha;
  if (col_scale) v *= col_scale[b];
  out[t] = v;
}

void launch_gather_rows_cols(const double* D, int ld, const int32_t* rows, int nr,
                             const int32_t* cols, int nc, double alpha_scale,
                             const double* col_scale, double* out, cudaStream_t s) {
  const int64_t n = (int64_t)nr * nc;
  if (n > 0)
    { count_launch(); k_gather_rc<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(D, ld, rows, nr, cols, nc, alpha_scale,
                                                            col_scale, out); }
}

// Rhat dense (npar x nslot): Rhat[par_b][det_a] = Y[a][b], Rhat[p][4p+3] = 1/sqrt(m_p).
__global__ void k_dense_rhat(const double* __restrict__ Y, const int32_t* __restrict__ det, int nJ,
                             const int32_t* __restrict__ par, int nA,
                             const uint32_t* __restrict__ pmask, int64_t npar, double* Rh) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t nslot = 4 * npar;
  if (t < (int64_t)nJ * nA) {
    const int a = (int)(t / nA), b = (int)(t % nA);
    Rh[(int64_t)par[b] * nslot + det[a]] = Y[t];
  }
  if (t < npar) {
    const int m = __popc(pmask[t] & 15u);
    if (m) Rh[t * nslot + 4 * t + 3] = 1.0 / sqrt((double)m);
  }
}

void launch_dense_rhat(const double* Y, const int32_t* det, int nJ, const int32_t* par, int nA,
                       const uint32_t* pmask, int64_t npar, double* Rh, cudaStream_t s) {
  int64_t n = (int64_t)nJ * nA;
  if (n < npar) n = npar;
  if (n > 0)
    { count_launch(); k_dense_rhat<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Y, det, nJ, par, nA, pmask, npar, Rh); }
}

// Scatter a compact detail vector into AoS4 slots (others 0) and gather back.
__global__ void k_scatter_det(const double* __restrict__ wc, const int32_t* __restrict__ det,
                              int nJ, double* w) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < nJ) w[det[a]] = wc[a];
}
void launch_scatter_det(const double* wc, const int32_t* det, int nJ, double* w, cudaStream_t s) {
  if (nJ > 0) { count_launch(); k_scatter_det<<<(nJ + 255) / 256, 256, 0, s>>>(wc, det, nJ, w); }
}
__global__ void k_gather_det(const double* __restrict__ w, const int32_t* __restrict__ det, int nJ,
                             double* wc) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  if (a < nJ) wc[a] = w[det[a]];
}
void launch_gather_det(const double* w, const int32_t* det, int nJ, double* wc, cudaStream_t s) {
  if (nJ > 0) { count_launch(); k_gather_det<<<(nJ + 255) / 256, 256, 0, s>>>(w, det, nJ, wc); }
}

// Level-1 factor from a dense 4 x 4 (float64); zero rows become identity.
__global__ void k_level1_factor_dense(const double* __restrict__ A, double* L, int* status) {
  if (threadIdx.x != 0) return;
  double M[16];
  for (int e = 0; e < 16; ++e) M[e] = A[e];
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
  for (int e = 0; e < 16; ++e) L[e] = M[e];
}
void launch_level1_factor_dense(const double* A, double* L, int* status, cudaStream_t s) {
  { count_launch(); k_level1_factor_dense<<<1, 32, 0, s>>>(A, L, status); }
}

}  // namespace gb
