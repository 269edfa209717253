// noalloc.cu - allocation-free evaluation of the objective J = 1/2 |u - u_obs|^2.
//
// gamblet_grad computes the same J with scratch it allocates per call (a
// residual vector and a float64 accumulator).  This entry point is for
// callers that cannot allocate device memory at the moment they need J:
// applications whose framework allocator has already reserved the free
// device memory (a caching allocator grows to fill the GPU, so a side
// cudaMalloc can fail although the framework itself has room), programs run
// under a hard device-memory budget, and latency-sensitive loops, such as an
// optimiser evaluating J many times per line search, that cannot afford the
// device-wide synchronisation that cudaFree implies.  Its scratch is a
// file-scope device array of fixed size, so it never calls cudaMalloc,
// cudaFree or any allocating library routine.
//
// Scratch: at most GAMBLET_NOALLOC_BLOCKS partial sums (one per block of
// GAMBLET_NOALLOC_CHUNK elements) plus one slot for the result, 8.2 KB held
// by every GPU that loads the library until the process exits.  Each call
// overwrites exactly the slots it reads, so nothing needs clearing between
// calls; calls that overlap on the GPU share the array and race.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/gamblet.h"
#include "common.cuh"

namespace gb {
void noalloc_set_error(const char* msg);
}

#define GAMBLET_NOALLOC_THREADS 256
#define GAMBLET_NOALLOC_PER_THREAD 8
#define GAMBLET_NOALLOC_CHUNK (GAMBLET_NOALLOC_THREADS * GAMBLET_NOALLOC_PER_THREAD)
#define GAMBLET_NOALLOC_BLOCKS 1024

// partial sums [0, GAMBLET_NOALLOC_BLOCKS) and the result at [GAMBLET_NOALLOC_BLOCKS]
static __device__ __align__(256) double g_objective_scratch[GAMBLET_NOALLOC_BLOCKS + 1];

namespace {

__global__ void k_objective_partials(int n, const double* __restrict__ u,
                                     const double* __restrict__ uo, double* partials) {
  __shared__ double red[GAMBLET_NOALLOC_THREADS / 32];
  const int64_t base = (int64_t)blockIdx.x * GAMBLET_NOALLOC_CHUNK;
  double s = 0;
#pragma unroll
  for (int t = 0; t < GAMBLET_NOALLOC_PER_THREAD; ++t) {
    const int64_t i = base + (int64_t)t * GAMBLET_NOALLOC_THREADS + threadIdx.x;
    if (i < n) {
      const double d = u[i] - uo[i];
      s += d * d;
    }
  }
  s = gb::warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < GAMBLET_NOALLOC_THREADS / 32 ? red[threadIdx.x] : 0.0;
    s = gb::warp_sum(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

// Fixed-order sum of the partials (deterministic), J = sum / 2.
__global__ void k_objective_finish(int nblocks, const double* __restrict__ partials,
                                   double* out) {
  __shared__ double red[32];
  double s = 0;
  for (int b = threadIdx.x; b < nblocks; b += blockDim.x) s += partials[b];
  s = gb::warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    s = gb::warp_sum(s);
    if (threadIdx.x == 0) *out = 0.5 * s;
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (host code cannot use the symbol itself as an address).
std::mutex g_scratch_mu;
double* g_scratch_ptr[64] = {nullptr};

double* scratch_for_current_device(cudaError_t* err) {
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_objective_scratch);
    if (*err != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  return g_scratch_ptr[dev];
}

// Where a pointer lives: 1 for device memory of the current device (or
// managed memory), 0 for host memory, -1 for another GPU's memory.  The
// kernels run on the current device and would fault on another GPU's memory
// without peer access, so such pointers are refused.
int ptr_kind(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (a.type == cudaMemoryTypeManaged) return 1;
  if (a.type != cudaMemoryTypeDevice) return 0;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return a.device == dev ? 1 : -1;
}

}  // namespace

extern "C" gamblet_status gamblet_objective_noalloc(int32_t n, const double* u,
                                                    const double* u_obs, double* J,
                                                    void* stream) {
  if (n < 1 || n > GAMBLET_NOALLOC_MAX_N) {
    gb::noalloc_set_error(
        "gamblet_objective_noalloc: n must be in [1, 2097152] (fixed scratch of 1024 partial "
        "sums of 2048 elements each)");
    return n < 1 ? GAMBLET_ERR_INVALID_ARG : GAMBLET_ERR_UNSUPPORTED;
  }
  if (!u || !u_obs || !J || ptr_kind(u) != 1 || ptr_kind(u_obs) != 1 || ptr_kind(J) < 0) {
    gb::noalloc_set_error(
        "gamblet_objective_noalloc: u and u_obs must be device pointers of the current device, "
        "J a host pointer or a device pointer of the current device");
    return GAMBLET_ERR_INVALID_ARG;
  }
  cudaError_t err = cudaSuccess;
  double* scratch = scratch_for_current_device(&err);
  if (!scratch) {
    gb::noalloc_set_error(("gamblet_objective_noalloc: cudaGetSymbolAddress failed: " +
                           std::string(cudaGetErrorString(err))).c_str());
    return GAMBLET_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int nblocks = (n + GAMBLET_NOALLOC_CHUNK - 1) / GAMBLET_NOALLOC_CHUNK;
  const bool j_dev = ptr_kind(J) == 1;
  double* out = j_dev ? J : scratch + GAMBLET_NOALLOC_BLOCKS;
  gb::count_launch();
  k_objective_partials<<<nblocks, GAMBLET_NOALLOC_THREADS, 0, s>>>(n, u, u_obs, scratch);
  gb::count_launch();
  k_objective_finish<<<1, 1024, 0, s>>>(nblocks, scratch, out);
  err = cudaGetLastError();
  if (err == cudaSuccess && !j_dev) {
    err = cudaMemcpyAsync(J, out, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  }
  if (err != cudaSuccess) {
    gb::noalloc_set_error(("gamblet_objective_noalloc: " +
                           std::string(cudaGetErrorString(err))).c_str());
    return GAMBLET_ERR_CUDA;
  }
  return GAMBLET_OK;
}
