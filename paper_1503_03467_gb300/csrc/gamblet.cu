// gamblet.cu - host orchestration behind the C ABI of include/gamblet.h.
//
// Setup (Algorithm 2 of Sec. 5.3 for rho > 0, Algorithm 1 of Sec. 5.2 for
// rho <= 0), fine to coarse, k = q..2:
//   import A^(q) -> transformed block stencil Ahat^(q) = Q A Q^T
//   patch solves (Definition defb)            -> Rhat^(k-1,k)
//   Galerkin product R A R^T (Eq. eqhuhiuv)   -> A^(k-1) -> Ahat^(k-1)
// Solve: restriction chain, all level CGs batched in one launch sequence,
// coarsest Cholesky, prolongation and summation; optionally as the
// preconditioner of a float64 flexible CG on A^(q).
//
// Host work is limited to symbolic offset sets (a few thousand integers per
// level), launch sequencing and one read-back per outer iteration / CG chunk.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <functional>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "../../include/gamblet.h"
#include "common.cuh"
#include "kernels.cuh"

namespace gb {
// declared in dense.cu / solve.cu
void launch_dense_transform(const double* in, int64_t npar, const uint32_t* pmask, double* out,
                            cudaStream_t s);
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
// Kernels launched by replays of a captured graph are counted per replay;
// the counts taken while capturing are removed again.
long long launches_now() { return g_launches.load(std::memory_order_relaxed); }
void uncount_launches(long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace gb

using namespace gb;

namespace {

thread_local std::string g_last_error;

struct GbError {
  gamblet_status st;
  std::string msg;
};

[[noreturn]] void fail(gamblet_status st, const std::string& msg) { throw GbError{st, msg}; }

#define CK(x)                                                                           \
  do {                                                                                  \
    cudaError_t e_ = (x);                                                               \
    if (e_ != cudaSuccess) {                                                            \
      if (e_ == cudaErrorMemoryAllocation)                                              \
        fail(GAMBLET_ERR_OUT_OF_MEMORY, std::string(#x) + ": " + cudaGetErrorString(e_)); \
      fail(GAMBLET_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_));          \
    }                                                                                   \
  } while (0)

// ---------------------------------------------------------------- device memory
// Stream-ordered allocations from a memory pool that the library owns, one
// per device.  Its release threshold is unlimited, so freed blocks stay
// cached for the next handle and a repeated setup does not pay for
// cudaMalloc; the device's default pool, which the caller's own allocators
// may share, keeps its settings.  The cached memory is returned when the
// process exits.
cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(GAMBLET_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t mp = nullptr;
    CK(cudaMemPoolCreate(&mp, &props));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &thr));
    pools[dev] = mp;
  }
  return pools[dev];
}

struct Pool {
  std::vector<void*> ptrs;
  int64_t bytes = 0;
  cudaStream_t s = nullptr;
  cudaMemPool_t mp = nullptr;
  template <typename T>
  T* alloc(int64_t n) {
    if (n <= 0) n = 1;
    if (!mp) mp = library_pool();
    void* p = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&p, sizeof(T) * (size_t)n, mp, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(GAMBLET_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(sizeof(T) * n) + " bytes");
    }
    ptrs.push_back(p);
    bytes += (int64_t)sizeof(T) * n;
    return static_cast<T*>(p);
  }
  template <typename T>
  T* zeros(int64_t n, cudaStream_t s) {
    T* p = alloc<T>(n);
    CK(cudaMemsetAsync(p, 0, sizeof(T) * (size_t)std::max<int64_t>(n, 1), s));
    return p;
  }
  template <typename T>
  T* upload(const std::vector<T>& v, cudaStream_t s) {
    T* p = alloc<T>((int64_t)v.size());
    if (!v.empty()) CK(cudaMemcpyAsync(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
    return p;
  }
  void release() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
    ptrs.clear();
    bytes = 0;
  }
  ~Pool() { release(); }
};

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy n elements from caller memory (host or device) into a device buffer.
template <typename T>
void to_device(Pool& pool, T*& dst, const T* src, int64_t n, cudaStream_t s) {
  if (!dst) dst = pool.alloc<T>(n);
  if (n > 0) CK(cudaMemcpyAsync(dst, src, sizeof(T) * (size_t)n, cudaMemcpyDefault, s));
}

// Caller memory as a device pointer: device memory is read in place (the
// calls that use this finish with a stream synchronisation), host memory is
// copied into a pool buffer.
template <typename T>
const T* as_device(Pool& pool, const T* src, int64_t n, cudaStream_t s) {
  if (is_device_ptr(src)) return src;
  T* dst = nullptr;
  to_device(pool, dst, src, n, s);
  return dst;
}

// ---------------------------------------------------------------- offset sets
using Off = std::pair<int, int>;  // (dx, dy)

struct OffSet {
  std::vector<int2> v;
  std::map<Off, int> idx;
  void add(int dx, int dy) {
    Off k{dx, dy};
    if (idx.count(k)) return;
    idx[k] = (int)v.size();
    v.push_back(make_int2(dx, dy));
  }
  int find(int dx, int dy) const {
    auto it = idx.find(Off{dx, dy});
    return it == idx.end() ? -1 : it->second;
  }
  int size() const { return (int)v.size(); }
};

// i^rho offsets of Sec. 4.10 in cell units, row-major (dy, dx).
OffSet neighbour_offsets(double rho, int rule) {
  OffSet N;
  const int R = (int)std::floor(rho) + 1;
  for (int dy = -R; dy <= R; ++dy)
    for (int dx = -R; dx <= R; ++dx) {
      bool ok;
      if (rule == 0) {
        const double ex = std::max(std::abs(dx) - 1, 0), ey = std::max(std::abs(dy) - 1, 0);
        ok = ex * ex + ey * ey <= rho * rho * (1 + 1e-12);
      } else {
        ok = std::max(std::abs(dx), std::abs(dy)) <= rho + 1e-12;
      }
      if (ok) N.add(dx, dy);
    }
  return N;
}

// Symbolic data of one localized level k (patch, Galerkin, conversion).
struct SymLevel {
  OffSet O;                       // block offsets of Ahat^(k) (level k-1 cell units)
  std::vector<int> pair_idx;      // NB x NB
  OffSet WIN, S;                  // window and output cell offsets
  OffSet Sp;                      // the half-plane of S that is computed
  std::vector<int> l1_ptr, l2_ptr;
  std::vector<int2> l1_pairs, l2_pairs;
  std::vector<int> map_next;      // conversion map to level k-1 blocks (or level-1 map)
  // 2 x 2 row tiles (k_galerkin_tile): window positions u of the tile as a
  // box [wmin, wmin + W)^2 relative to the tile origin; per u the offsets o
  // with, for each of the four rows, the neighbour index j (0xff = none);
  // output targets c with the index d in Sp of c - row, per row (-1 = none)
  int tile_wmin = 0, tile_W = 0;
  std::vector<int> t1_ptr;
  std::vector<int2> t1;           // (o, j of rows 0..3 packed in bytes)
  std::vector<int4> t2;           // (c.x, c.y, d0 | d1 << 16, d2 | d3 << 16)
  // per target e, the pairs (j, u) whose window position u = c + N_j lies in
  // the window of some row of the tile (packed j | u << 8, ranges t2p_ptr);
  // targets are sorted by decreasing pair count so that the targets that a
  // warp handles together have about the same work
  std::vector<int> t2p_ptr, t2p;
};

// ---------------------------------------------------------------- handle
struct LevelDev {
  int k = 0;
  int L = 0;          // 2^k
  int64_t ncell = 0;  // stored cells, 4 npar (4^k for a full square)
  int64_t npar = 0;   // stored level-(k-1) cells (4^(k-1) for a full square)
  std::vector<uint32_t> pmask_h;
  uint32_t* pmask = nullptr;
  int n_active = 0, nJ = 0;
  // localized
  const int2* off = nullptr;
  int noff = 0;
  std::vector<int2> off_h;
  void* Ahat = nullptr;      // T
  double* Ahat64 = nullptr;  // level q float64 copy (mixed) or alias
  void* Rhat = nullptr;      // T, npar rows
  void* RT = nullptr;        // T, Rhat regrouped by parent (prolongation)
  const int* pair_idx = nullptr;
  int shape[4] = {0, 0, 0, 0};  // launch shapes used: patch spp, patch gather, Galerkin variant, CG spp
  // exact (dense)
  double* D = nullptr;       // transformed dense Ahat^(k)
  double* Bc = nullptr;      // Cholesky factor of B^(k)
  double* Rh = nullptr;      // dense Rhat (npar x ncell)
  int32_t* det = nullptr;
  int32_t* par = nullptr;
  std::vector<int32_t> det_h, par_h;
  // solve buffers (T)
  void* ghat = nullptr;  // ncell
  void* v = nullptr;     // ncell
  void* w = nullptr;     // ncell
  void* cr = nullptr;
  void* cz = nullptr;
  void* cp = nullptr;
  void* cAp = nullptr;
  double* wc = nullptr;  // compact detail vector (exact path)
  // level CG operator (localized path)
  void* Bd = nullptr;    // [noff][9][npar]
  void* Bq = nullptr;    // 32-byte float16 block records of the level CG (mixed path), or NULL
  float* bq_scale = nullptr;  // device: inverse scale of Bq
  void* Dinv = nullptr;  // [9][npar]
  int R = 0;             // halo radius
  int o0 = -1;           // index of the zero offset in O_k (diagonal blocks)
};

// Per-kernel CUDA-event timing on the library's stream (opts.profile).
struct Prof {
  struct Stat {
    std::string name;
    long long launches = 0;
    double ms = 0, bytes = 0, flops = 0;
  };
  struct Pend {
    int id;
    cudaEvent_t a, b;
    double bytes, flops;
  };
  bool on = false;
  std::vector<Stat> stats;
  std::vector<Pend> pend;
  std::vector<cudaEvent_t> pool;
  int id(const std::string& name) {
    for (size_t i = 0; i < stats.size(); ++i)
      if (stats[i].name == name) return (int)i;
    stats.push_back(Stat{name});
    return (int)stats.size() - 1;
  }
  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    return e;
  }
  // returns a token for end(); -1 when profiling is off
  int begin(const std::string& name, double bytes, double flops, cudaStream_t s) {
    if (!on) return -1;
    Pend p{id(name), ev(), ev(), bytes, flops};
    CK(cudaEventRecord(p.a, s));
    pend.push_back(p);
    return (int)pend.size() - 1;
  }
  void end(int tok, cudaStream_t s) {
    if (tok < 0) return;
    CK(cudaEventRecord(pend[tok].b, s));
  }
  // call after the stream has been synchronised
  void resolve() {
    for (Pend& p : pend) {
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, p.a, p.b));
      Stat& st = stats[p.id];
      st.launches += 1;
      st.ms += ms;
      st.bytes += p.bytes;
      st.flops += p.flops;
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pend.clear();
  }
  void add(const std::string& name, double bytes, double flops) {
    if (!on) return;
    Stat& st = stats[id(name)];
    st.bytes += bytes;
    st.flops += flops;
  }
  ~Prof() {
    for (Pend& p : pend) {
      cudaEventDestroy(p.a);
      cudaEventDestroy(p.b);
    }
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
  }
};

struct Plan;  // symbolic plan of a geometry (defined with the setup code)

}  // namespace

struct gamblet_ctx {
  Prof prof;
  std::shared_ptr<const Plan> plan;
  gamblet_opts opts;
  cudaStream_t s = nullptr;
  int q = 0;
  int n = 0;           // fine unknowns
  int nprob = 1;       // independent problems packed in the hierarchy
  int kmax = 0;        // finest level whose detail component a solve adds (q = all)
  // level-q initialisation by the mass matrix: nodal coefficients are
  // u_phi = M^-1,loc U (Minv[i][j] on the patch offsets nbrq)
  bool mass = false;
  double* Minv = nullptr;
  int2* nbrq = nullptr;
  int NBq = 0;
  bool exact = false;
  bool mixed = false;
  int num_sms = 1;
  Pool pool;
  int32_t* morton_of = nullptr;   // n
  int32_t* unknown_of = nullptr;  // 4^q
  std::vector<int32_t> morton_of_h;
  std::vector<LevelDev> lv;       // index k (0 unused)
  OffSet N;                       // neighbour offsets
  int jc = 0;
  int2* nbr = nullptr;
  // level 1
  double* A1 = nullptr;      // plain 4 x 4 (copy, for getters)
  double* A1L = nullptr;     // Cholesky factor
  void* g1 = nullptr;        // T, 4
  void* U1 = nullptr;        // T, 4
  const int* l1map = nullptr;
  // CG batch
  CgLevel* cg_lv = nullptr;
  CgLevel* cg_lv_h = nullptr;  // pinned staging copy (the upload does not wait for the setup)
  CgScalars* cg_sc = nullptr;
  int* any_active = nullptr;
  int* any_active_h = nullptr;  // pinned
  int cg_blocks = 0;
  int cg_spmv_blocks = 0;
  int cg_nlev = 0;
  int cg_max_ts = 1;
  cudaGraphExec_t cg_exec = nullptr;
  bool cg_while = false;           // cg_exec is a device-side while loop
  int* cg_loop_count = nullptr;    // passes of that loop
  int* cg_stats = nullptr;         // device: level-CG iterations per level, [32] not converged,
                                   // [33] passes of the device-side loop
  // per level and CG iteration: algorithmic traffic and flops of the SpMV and
  // of the vector kernels
  std::vector<double> cg_bytes_spmv, cg_flops_spmv, cg_bytes_vec, cg_flops_vec;
  // outer: the fine operator as a Morton node stencil (float64), its cell
  // offsets, and a scratch vector for the untransformed SpMV input
  double* qst = nullptr;
  const int2* qoff = nullptr;
  int qns = 0;
  double* xplain = nullptr;
  double* u64 = nullptr;
  double* r64 = nullptr;
  double* z64 = nullptr;
  double* p64 = nullptr;
  double* q64 = nullptr;
  double* g64 = nullptr;
  void* rT = nullptr;
  void* zT = nullptr;
  double* dots = nullptr;
  double* dots_h = nullptr;  // pinned
  int* status = nullptr;
  int* status_h = nullptr;   // pinned
  double setup_ms = 0;
  double patch_tol = 0;         // resolved patch tolerance (< 0: Cholesky)
  int* patch_stats = nullptr;   // device: max, sum, count over all levels
  int patch_iters_max = 0;
  double patch_iters_mean = 0;
  std::vector<double> patch_flops_iter_k;  // per level: flops of one iteration of one patch
  std::vector<double> patch_mma_flops_k;   // per level: tensor-core flops of one window product
  std::vector<bool> patch_cluster_k;        // per level: patch CG over a thread-block cluster
  int level_iters_acc[32];
  bool level_not_conv = false;
  const char* dplan = nullptr;  // device copy of the plan tables (localized setup)
};

namespace {

template <typename T>
constexpr bool is_f32() {
  return sizeof(T) == 4;
}

void check_status(gamblet_ctx* h, const char* where) {
  CK(cudaMemcpyAsync(h->status_h, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (*h->status_h == DEV_NOT_SPD)
    fail(GAMBLET_ERR_NOT_SPD, std::string("non-positive pivot in ") + where);
  if (*h->status_h == DEV_TIMEOUT)
    fail(GAMBLET_ERR_CUDA, std::string("a tensor-core completion wait gave up in ") + where);
}

// ------------------------------------------------------------ symbolic build
SymLevel build_sym(const OffSet& O_k, const OffSet& N, int k) {
  SymLevel S;
  S.O = O_k;
  const int NB = N.size();
  const int Lpar = 1 << (k - 1);  // level k-1 lattice side
  S.pair_idx.assign((size_t)NB * NB, -1);
  for (int a = 0; a < NB; ++a)
    for (int b = 0; b < NB; ++b)
      S.pair_idx[(size_t)a * NB + b] = O_k.find(N.v[b].x - N.v[a].x, N.v[b].y - N.v[a].y);
  // window: positions p' = i + WIN_w reachable from the patch through O_k
  for (int j = 0; j < NB; ++j)
    for (const int2& o : O_k.v) {
      const int wx = N.v[j].x - o.x, wy = N.v[j].y - o.y;  // row parent p' with p - p' = o
      if (std::abs(wx) <= Lpar - 1 && std::abs(wy) <= Lpar - 1) S.WIN.add(wx, wy);
    }
  S.l1_ptr.assign(S.WIN.size() + 1, 0);
  std::vector<std::vector<int2>> l1(S.WIN.size());
  for (int j = 0; j < NB; ++j)
    for (int o = 0; o < O_k.size(); ++o) {
      const int w = S.WIN.find(N.v[j].x - O_k.v[o].x, N.v[j].y - O_k.v[o].y);
      if (w >= 0) l1[w].push_back(make_int2(j, o));
    }
  for (int w = 0; w < S.WIN.size(); ++w) {
    S.l1_ptr[w + 1] = S.l1_ptr[w] + (int)l1[w].size();
    S.l1_pairs.insert(S.l1_pairs.end(), l1[w].begin(), l1[w].end());
  }
  // outputs d with WIN_w = d + N_j
  for (int w = 0; w < S.WIN.size(); ++w)
    for (int j = 0; j < NB; ++j) {
      const int dx = S.WIN.v[w].x - N.v[j].x, dy = S.WIN.v[w].y - N.v[j].y;
      if (std::abs(dx) <= Lpar - 1 && std::abs(dy) <= Lpar - 1) S.S.add(dx, dy);
    }
  for (const int2& d : S.S.v)
    if (d.y > 0 || (d.y == 0 && d.x >= 0)) S.Sp.add(d.x, d.y);
  std::vector<std::vector<int2>> l2(S.Sp.size());
  for (int d = 0; d < S.Sp.size(); ++d)
    for (int j = 0; j < NB; ++j) {
      const int w = S.WIN.find(S.Sp.v[d].x + N.v[j].x, S.Sp.v[d].y + N.v[j].y);
      if (w >= 0) l2[d].push_back(make_int2(j, w));
    }
  S.l2_ptr.assign(S.Sp.size() + 1, 0);
  for (int d = 0; d < S.Sp.size(); ++d) {
    S.l2_ptr[d + 1] = S.l2_ptr[d] + (int)l2[d].size();
    S.l2_pairs.insert(S.l2_pairs.end(), l2[d].begin(), l2[d].end());
  }
  // 2 x 2 tiles: row r sits at (r & 1, r >> 1) from the tile origin
  int wmin = 0, wmax = 0;
  for (const int2& w : S.WIN.v) {
    wmin = std::min(wmin, std::min(w.x, w.y));
    wmax = std::max(wmax, std::max(w.x, w.y));
  }
  const int W = wmax - wmin + 2;
  S.tile_wmin = wmin;
  S.tile_W = W;
  S.t1_ptr.assign((size_t)W * W + 1, 0);
  for (int uy = 0; uy < W; ++uy)
    for (int ux = 0; ux < W; ++ux) {
      const int u = uy * W + ux;
      for (int o = 0; o < O_k.size(); ++o) {
        uint32_t packed = 0;
        bool any = false;
        for (int r = 0; r < 4; ++r) {
          // t_i(w) gathers A_hat[o][i + w] R_hat_i[j] with N_j = w + O_o
          const int wx = ux + wmin - (r & 1), wy = uy + wmin - (r >> 1);
          int j = S.WIN.find(wx, wy) >= 0 ? N.find(wx + O_k.v[o].x, wy + O_k.v[o].y) : -1;
          if (j > 254) fail(GAMBLET_ERR_UNSUPPORTED, "neighbourhood too large for tiled Galerkin");
          if (j >= 0) any = true;
          packed |= (uint32_t)(j >= 0 ? j : 0xff) << (8 * r);
        }
        if (any) S.t1.push_back(make_int2(o, (int)packed));
      }
      S.t1_ptr[u + 1] = (int)S.t1.size();
    }
  std::set<std::pair<int, int>> targets;
  for (int r = 0; r < 4; ++r)
    for (const int2& d : S.Sp.v) targets.insert({d.y + (r >> 1), d.x + (r & 1)});
  // window positions holding a nonzero t_r(u) for some row r of the tile
  std::set<std::pair<int, int>> win4;
  for (int r = 0; r < 4; ++r)
    for (const int2& w : S.WIN.v) win4.insert({w.y + (r >> 1), w.x + (r & 1)});
  struct Target {
    int4 t;
    std::vector<int> pairs;
  };
  std::vector<Target> tl;
  for (const auto& c : targets) {
    const int cx = c.second, cy = c.first;
    int dr[4];
    for (int r = 0; r < 4; ++r) dr[r] = S.Sp.find(cx - (r & 1), cy - (r >> 1));
    if (S.Sp.size() > 32767) fail(GAMBLET_ERR_UNSUPPORTED, "output stencil too large for tiled Galerkin");
    auto pack = [](int lo, int hi) {
      return (int)(((uint32_t)lo & 0xffffu) | ((uint32_t)hi << 16));
    };
    Target t;
    t.t = make_int4(cx, cy, pack(dr[0], dr[1]), pack(dr[2], dr[3]));
    for (int j = 0; j < NB; ++j) {
      const int wx = cx + N.v[j].x, wy = cy + N.v[j].y;
      if (!win4.count({wy, wx})) continue;
      const int u = (wy - wmin) * W + (wx - wmin);  // inside the box: win4 lies in it
      if (u < 0 || u >= W * W || (u >> 23) != 0)
        fail(GAMBLET_ERR_UNSUPPORTED, "window too large for tiled Galerkin");
      t.pairs.push_back(j | (u << 8));
    }
    tl.push_back(std::move(t));
  }
  std::stable_sort(tl.begin(), tl.end(), [](const Target& a, const Target& b) {
    return a.pairs.size() > b.pairs.size();
  });
  S.t2p_ptr.assign(1, 0);
  for (const Target& t : tl) {
    S.t2.push_back(t.t);
    S.t2p.insert(S.t2p.end(), t.pairs.begin(), t.pairs.end());
    S.t2p_ptr.push_back((int)S.t2p.size());
  }
  return S;
}

// Where A_{i, i+d} lives in the half-plane output: index of d in Sp, or
// -2 - (index of -d) for the mirrored half, or -1 when d is outside S.
int half_code(const OffSet& Sp, int dx, int dy) {
  const int a = Sp.find(dx, dy);
  if (a >= 0) return a;
  const int b = Sp.find(-dx, -dy);
  return b >= 0 ? -2 - b : -1;
}

// Block offsets of level k-1 (level k-2 cell units) from the level k-1 cell
// offsets S, and the conversion map [o][c*4+c'] (half_code of the offset).
OffSet blocks_from_cells(const OffSet& S, const OffSet& Sp, int km1, std::vector<int>& map) {
  OffSet O;
  const int Lp = 1 << (km1 - 1);
  for (const int2& d : S.v)
    for (int c = 0; c < 4; ++c)
      for (int cc = 0; cc < 4; ++cc) {
        const int ex = d.x - ((cc & 1) - (c & 1)), ey = d.y - ((cc >> 1) - (c >> 1));
        if ((ex & 1) || (ey & 1)) continue;
        const int Dx = ex / 2, Dy = ey / 2;
        if (std::abs(Dx) <= Lp - 1 && std::abs(Dy) <= Lp - 1) O.add(Dx, Dy);
      }
  map.assign((size_t)O.size() * 16, -1);
  for (int o = 0; o < O.size(); ++o)
    for (int c = 0; c < 4; ++c)
      for (int cc = 0; cc < 4; ++cc)
        map[(size_t)o * 16 + c * 4 + cc] =
            half_code(Sp, 2 * O.v[o].x + (cc & 1) - (c & 1), 2 * O.v[o].y + (cc >> 1) - (c >> 1));
  return O;
}

// ------------------------------------------------------------ hierarchy
// Level sizes follow the stored Morton prefix: npar_q = ceil((largest cell
// code + 1) / 4), npar_(k-1) = ceil(npar_k / 4), and level 1 always has the
// single root parent.  One square problem gives npar_k = 4^(k-1).
void build_hierarchy(gamblet_ctx* h, const int32_t* cells_user) {
  const int q = h->q;
  cudaStream_t s = h->s;
  Pool& P = h->pool;
  const int32_t* cells = as_device(P, cells_user, 2 * (int64_t)h->n, s);
  h->morton_of = P.alloc<int32_t>(h->n);
  int* flag = P.zeros<int>(4, s);
  launch_cells_to_morton(cells, h->n, q, h->morton_of, flag, s);
  CK(cudaGetLastError());
  int flag_h[4];
  CK(cudaMemcpyAsync(flag_h, flag, sizeof(flag_h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flag_h[0] == 2) fail(GAMBLET_ERR_INVALID_ARG, "a cell lies outside [0, 2^q)");
  h->lv.assign(q + 1, LevelDev());
  // the dense exact transform keeps the full square
  int64_t npar = h->exact ? ((int64_t)1 << (2 * (q - 1))) : ((int64_t)flag_h[1] + 1 + 3) / 4;
  for (int k = q; k >= 1; --k) {
    LevelDev& L = h->lv[k];
    L.k = k;
    L.L = 1 << k;
    L.npar = k == 1 ? 1 : npar;
    L.ncell = 4 * L.npar;
    L.pmask = P.zeros<uint32_t>(L.npar, s);
    npar = (npar + 3) / 4;
  }
  h->unknown_of = P.alloc<int32_t>(h->lv[q].ncell);
  CK(cudaMemsetAsync(h->unknown_of, 0xff, sizeof(int32_t) * h->lv[q].ncell, s));
  CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
  launch_scatter_cells(h->morton_of, h->n, h->unknown_of, h->lv[q].pmask, flag, s);
  for (int k = q; k >= 2; --k)
    launch_coarsen_masks(h->lv[k].pmask, h->lv[k].npar, h->lv[k - 1].pmask, h->lv[k - 1].npar, s);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(flag_h, flag, sizeof(flag_h), cudaMemcpyDeviceToHost, s));
  for (int k = 1; k <= q; ++k) {
    h->lv[k].pmask_h.resize(h->lv[k].npar);
    CK(cudaMemcpyAsync(h->lv[k].pmask_h.data(), h->lv[k].pmask, sizeof(uint32_t) * h->lv[k].npar,
                       cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  if (flag_h[0] == 1) fail(GAMBLET_ERR_INVALID_ARG, "two unknowns share a level-q cell");
  for (int k = 1; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    int na = 0, nJ = 0;
    for (uint32_t m : L.pmask_h) {
      const int c = __builtin_popcount(m & 15u);
      na += c;
      nJ += c > 0 ? c - 1 : 0;
    }
    L.n_active = na;
    L.nJ = nJ;
  }
}

// Fine CSR -> transformed block stencil of level q (float64).
void import_fine(gamblet_ctx* h, const gamblet_csr* A) {
  cudaStream_t s = h->s;
  Pool& P = h->pool;
  const int n = h->n;
  const int32_t* rowptr = as_device(P, A->rowptr, (int64_t)n + 1, s);
  int32_t rp_last[2];
  CK(cudaMemcpyAsync(rp_last, rowptr, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(rp_last + 1, rowptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (rp_last[0] != 0 || (int64_t)rp_last[1] != A->nnz)
    fail(GAMBLET_ERR_INVALID_ARG, "rowptr[0] must be 0 and rowptr[n] must equal nnz");
  const int32_t* colind = as_device(P, A->colind, A->nnz, s);
  const double* val = as_device(P, A->val, A->nnz, s);
  int* ext = P.zeros<int>(4, s);
  launch_csr_offset_extent(n, rowptr, colind, h->morton_of, ext, ext + 2, s);
  CK(cudaGetLastError());
  int ext_h[4];
  CK(cudaMemcpyAsync(ext_h, ext, sizeof(ext_h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (ext_h[2]) fail(GAMBLET_ERR_INVALID_ARG, "CSR column index out of range or rowptr decreasing");
  const int q = h->q;
  LevelDev& L = h->lv[q];
  const int Lpar = 1 << (q - 1);
  const int rx = std::min(ext_h[0], Lpar - 1), ry = std::min(ext_h[1], Lpar - 1);
  L.off_h.clear();
  for (int dy = -ry; dy <= ry; ++dy)
    for (int dx = -rx; dx <= rx; ++dx) L.off_h.push_back(make_int2(dx, dy));
  L.noff = (int)L.off_h.size();
  L.off = P.upload(L.off_h, s);
  double* blk = P.zeros<double>((int64_t)L.noff * L.npar * 16, s);
  launch_csr_to_blocks(n, rowptr, colind, val, h->morton_of, rx, ry, L.npar, blk, s);
  if (h->mixed) {
    // the working copy is transformed in float32 straight from the float64
    // blocks; the outer float64 iteration applies the node stencil instead
    float* a32 = P.alloc<float>((int64_t)L.noff * L.npar * 16);
    launch_transform_blocks_f32(blk, a32, L.off, L.noff, L.npar, Lpar, L.pmask, s);
    L.Ahat = a32;
    L.Ahat64 = nullptr;
  } else {
    launch_transform_blocks(blk, L.off, L.noff, L.npar, Lpar, L.pmask, s);
    L.Ahat64 = blk;
  }
  CK(cudaGetLastError());
  // node stencil of A^(q) in Morton order for the outer float64 SpMV
  int* next = P.zeros<int>(4, s);
  launch_csr_node_extent(n, rowptr, colind, h->morton_of, next, next + 2, s);
  int next_h[4];
  CK(cudaMemcpyAsync(next_h, next, sizeof(next_h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int nrx = next_h[0], nry = next_h[1];
  std::vector<int2> qoff;
  for (int dy = -nry; dy <= nry; ++dy)
    for (int dx = -nrx; dx <= nrx; ++dx) qoff.push_back(make_int2(dx, dy));
  h->qns = (int)qoff.size();
  h->qoff = P.upload(qoff, s);
  h->qst = P.zeros<double>((int64_t)h->qns * L.ncell, s);
  launch_csr_to_mstencil(n, rowptr, colind, val, h->morton_of, nrx, nry, L.ncell, h->qst, s);
  CK(cudaGetLastError());
}

// yhat = Ahat^(q) xhat = Q A Q^T xhat in float64 on transformed level-q
// vectors: untransform, node-stencil SpMV, transform (the last two fused).
void outer_spmv(gamblet_ctx* h, const double* xhat, double* yhat) {
  LevelDev& Lq = h->lv[h->q];
  launch_transform_vec<double>(xhat, h->xplain, Lq.npar, Lq.pmask, -1, h->s);
  launch_stencil_spmv_q(h->qst, h->qoff, h->qns, 1 << h->q, Lq.ncell, Lq.npar, Lq.pmask,
                        h->xplain, yhat, h->s);
}

// ------------------------------------------------------------ symbolic plan
// Everything the localized setup derives from the geometry alone (q, rho,
// neighbour rule and the fine operator's block offsets): offset sets, the
// patch block lists and the Galerkin pair lists of every level.  It does not
// depend on coefficient values, so it is built once per geometry and kept in
// a process-wide cache (like an FFT plan).
// Tables of the tensor-core patch solves (patch_mma.cu) for windows of G x G
// coarse cells, G = 1 and 2: the union of the windows' neighbourhoods, which
// patches each union parent belongs to, the stored blocks between union
// parents, the right-hand-side blocks and the union index of every patch
// neighbour.  All are offsets, so one table serves every window of the level.
struct MmaWin {
  bool ok = false;  // fits one CTA (at most three M-tiles and the shared memory)
  int NP = 0, nU = 0, n = 0, Kp = 0, Mt = 0, diag_o = -1;
  std::vector<int2> U;
  std::vector<int> ubits, rhs_o, outmap;
  std::vector<int4> pairs;
  size_t off[5] = {};  // U, ubits, pairs, rhs_o, outmap in Plan::packed
};

struct PlanLevel {
  SymLevel S;
  MmaWin mwin[2];  // G = 1, G = 2
  std::vector<int4> half, adj;   // patch CG: stored blocks and per-row adjacency
  std::vector<int> adj_ptr, diag_h;
  int spp = 1;
  double flops_iter = 0;
  std::vector<int> map_next;          // block conversion map (or the level-1 map)
  OffSet O_next;
  // byte offsets of this level's tables in Plan::packed
  enum { kPairIdx, kHalf, kAdjPtr, kAdj, kDiagH, kWin, kL1Ptr, kL1Pairs, kOut, kL2Ptr, kL2Pairs,
         kT1Ptr, kT1, kT2, kT2pPtr, kT2p, kOffNext, kMapNext, kNumTables };
  size_t table_off[kNumTables] = {};
};
struct Plan {
  std::vector<PlanLevel> lv;  // index k
  std::string key;            // geometry key of the process-wide cache
  // every table of every level in one 16-byte aligned buffer, so that a setup
  // moves the whole plan to the device with one copy
  std::vector<char> packed;
};

// Device address of table t of level k in a device copy of Plan::packed.
template <typename E>
const E* plan_table(const char* dev, const PlanLevel& pl, int t) {
  return reinterpret_cast<const E*>(dev + pl.table_off[t]);
}

int half_code(const OffSet& Sp, int dx, int dy);
OffSet blocks_from_cells(const OffSet& S, const OffSet& Sp, int km1, std::vector<int>& map);

// Shared-memory slots of the stored patch blocks, chosen so that the lanes
// of a warp that read blocks in the same CG step hit distinct banks.  Thread
// (j, sub) of the patch CG walks entries sub, sub + S, ... of row j's
// adjacency list (S = pl.spp lanes per neighbour parent), so the blocks read
// together are those of one (warp, step) group.  A block's words sit at
// 9 * slot + q, and 9 is invertible modulo 32, so blocks whose slots differ
// modulo 32 never share a bank.  Each block is greedily given a residue
// (colour) unused in its two groups (the row of ja and, transposed, of jb);
// when all 32 are taken the least used one is reused.  Slots are colour +
// 32 * rank; unused slots are padding (ja = -1).  Only the layout changes,
// not the arithmetic.
void assign_bank_slots(PlanLevel& pl, int NB) {
  const int nb = (int)pl.half.size();
  const int S = pl.spp;
  std::vector<std::vector<int>> groups_of(nb);
  std::map<std::pair<int, int>, int> gid;
  for (int j = 0; j < NB; ++j)
    for (int e = pl.adj_ptr[j]; e < pl.adj_ptr[j + 1]; ++e) {
      const int kpos = e - pl.adj_ptr[j];
      const int thread = j * S + kpos % S;
      const std::pair<int, int> key{thread / 32, kpos / S};
      auto it = gid.find(key);
      const int g = it == gid.end() ? (gid[key] = (int)gid.size()) : it->second;
      groups_of[pl.adj[e].x].push_back(g);
    }
  std::vector<uint32_t> used(gid.size(), 0u);           // colours taken per group
  std::vector<std::array<int, 32>> use_count(gid.size());
  for (auto& a : use_count) a.fill(0);
  std::vector<int> colour(nb, 0), count(32, 0);
  for (int b = 0; b < nb; ++b) {
    uint32_t taken = 0;
    for (int g : groups_of[b]) taken |= used[g];
    int c = -1;
    for (int t = 0; t < 32; ++t) {
      const int cand = (b + t) & 31;  // rotate the start to balance the classes
      if (!((taken >> cand) & 1u)) {
        c = cand;
        break;
      }
    }
    if (c < 0) {  // every residue taken: the least used in these groups
      int best = 1 << 30;
      for (int cand = 0; cand < 32; ++cand) {
        int u = 0;
        for (int g : groups_of[b]) u += use_count[g][cand];
        if (u < best) {
          best = u;
          c = cand;
        }
      }
    }
    colour[b] = c;
    for (int g : groups_of[b]) {
      used[g] |= 1u << c;
      ++use_count[g][c];
    }
  }
  std::vector<int> rank(nb);
  for (int b = 0; b < nb; ++b) rank[b] = count[colour[b]]++;
  const int per = *std::max_element(count.begin(), count.end());
  std::vector<int> slot(nb);
  std::vector<int4> half(32 * (size_t)per, make_int4(-1, -1, 0, 0));
  for (int b = 0; b < nb; ++b) {
    slot[b] = colour[b] + 32 * rank[b];
    half[slot[b]] = pl.half[b];
  }
  pl.half.swap(half);
  for (int4& a : pl.adj) a.x = slot[a.x];
  for (int& d : pl.diag_h) d = slot[d];
}

size_t patch_mma_smem_bytes_of(const MmaWin& W, int NB) {
  PatchMmaGeom g{};
  g.NP = W.NP;
  g.nU = W.nU;
  g.n = W.n;
  g.Kp = W.Kp;
  g.Mt = W.Mt;
  g.NB = NB;
  return patch_mma_smem_bytes(g);
}

void build_mma_window(MmaWin& W, int G, const OffSet& O, const OffSet& N) {
  const int NB = N.size();
  W.NP = G * G;
  std::vector<int2> cell(W.NP);
  for (int c = 0; c < W.NP; ++c) cell[c] = make_int2(c & 1, c >> 1);
  std::map<std::pair<int, int>, int> bits;  // (dy, dx) -> patch bits, row-major order
  for (int c = 0; c < W.NP; ++c)
    for (const int2& o : N.v) bits[{cell[c].y + o.y, cell[c].x + o.x}] |= 1 << c;
  OffSet U;
  W.U.clear();
  W.ubits.clear();
  for (const auto& kv : bits) {
    U.add(kv.first.second, kv.first.first);
    W.U.push_back(make_int2(kv.first.second, kv.first.first));
    W.ubits.push_back(kv.second);
  }
  W.nU = U.size();
  W.n = 3 * W.nU;
  W.Kp = (W.n + 15) / 16 * 16;
  W.Mt = (W.n + 127) / 128;
  W.diag_o = O.find(0, 0);
  W.pairs.clear();
  for (int a = 0; a < W.nU; ++a)
    for (int b = 0; b < a; ++b) {
      const int o = O.find(W.U[b].x - W.U[a].x, W.U[b].y - W.U[a].y);
      if (o >= 0) W.pairs.push_back(make_int4(a, b, o, 0));
    }
  W.rhs_o.assign((size_t)W.NP * W.nU, -1);
  for (int c = 0; c < W.NP; ++c)
    for (int u = 0; u < W.nU; ++u)
      W.rhs_o[(size_t)c * W.nU + u] = O.find(cell[c].x - W.U[u].x, cell[c].y - W.U[u].y);
  W.outmap.assign((size_t)W.NP * NB, 0);
  for (int c = 0; c < W.NP; ++c)
    for (int j = 0; j < NB; ++j)
      W.outmap[(size_t)c * NB + j] = U.find(cell[c].x + N.v[j].x, cell[c].y + N.v[j].y);
  W.ok = W.diag_o >= 0 && W.Mt <= 3 && patch_mma_smem_bytes_of(W, NB) <= 227 * 1024;
}

std::shared_ptr<const Plan> build_plan(int q, const OffSet& Oq, const OffSet& N,
                                       const std::string& key) {
  auto plan = std::make_shared<Plan>();
  plan->key = key;
  plan->lv.resize(q + 1);
  const int NB = N.size();
  OffSet O = Oq;
  for (int k = q; k >= 2; --k) {
    PlanLevel& pl = plan->lv[k];
    pl.S = build_sym(O, N, k);
    // patch blocks: pairs (ja >= jb) coupled through O_k
    std::vector<std::vector<int4>> rows(NB);
    pl.adj_ptr.assign(NB + 1, 0);
    pl.diag_h.assign(NB, -1);
    for (int ja = 0; ja < NB; ++ja)
      for (int jb = 0; jb <= ja; ++jb) {
        const int o = pl.S.pair_idx[(size_t)ja * NB + jb];
        if (o < 0) continue;
        const int hidx = (int)pl.half.size();
        pl.half.push_back(make_int4(ja, jb, o, 0));
        rows[ja].push_back(make_int4(hidx, jb, 0, 0));
        if (jb != ja) rows[jb].push_back(make_int4(hidx, ja, 1, 0));
        else pl.diag_h[ja] = hidx;
      }
    for (int j = 0; j < NB; ++j) {
      if (pl.diag_h[j] < 0) fail(GAMBLET_ERR_INVALID_ARG, "patch block without diagonal");
      pl.adj_ptr[j + 1] = pl.adj_ptr[j] + (int)rows[j].size();
      pl.adj.insert(pl.adj.end(), rows[j].begin(), rows[j].end());
    }
    const double row_len = (double)pl.adj.size() / NB;
    pl.spp = row_len > 24 ? 4 : (row_len > 12 ? 2 : 1);
    while (pl.spp > 1 && NB * pl.spp > 256) pl.spp >>= 1;
    pl.flops_iter = 18.0 * (2.0 * pl.half.size() - NB) + 60.0 * NB;
    assign_bank_slots(pl, NB);
    for (int gi = 0; gi < 2; ++gi) build_mma_window(pl.mwin[gi], gi + 1, pl.S.O, N);
    if (k - 1 >= 2) {
      pl.O_next = blocks_from_cells(pl.S.S, pl.S.Sp, k - 1, pl.map_next);
      O = pl.O_next;
    } else {
      pl.map_next.assign(16, -1);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
          pl.map_next[i * 4 + j] = half_code(pl.S.Sp, (j & 1) - (i & 1), (j >> 1) - (i >> 1));
    }
  }
  std::vector<char>& buf = plan->packed;
  auto put = [&buf](const void* src, size_t bytes) {
    const size_t off = buf.size();
    buf.resize(off + std::max<size_t>((bytes + 15) & ~(size_t)15, 16), 0);
    if (bytes) std::memcpy(buf.data() + off, src, bytes);
    return off;
  };
  auto put_v = [&put](const auto& v) { return put(v.data(), v.size() * sizeof(v[0])); };
  for (int k = q; k >= 2; --k) {
    PlanLevel& pl = plan->lv[k];
    const SymLevel& S = pl.S;
    pl.table_off[PlanLevel::kPairIdx] = put_v(S.pair_idx);
    pl.table_off[PlanLevel::kHalf] = put_v(pl.half);
    pl.table_off[PlanLevel::kAdjPtr] = put_v(pl.adj_ptr);
    pl.table_off[PlanLevel::kAdj] = put_v(pl.adj);
    pl.table_off[PlanLevel::kDiagH] = put_v(pl.diag_h);
    pl.table_off[PlanLevel::kWin] = put_v(S.WIN.v);
    pl.table_off[PlanLevel::kL1Ptr] = put_v(S.l1_ptr);
    pl.table_off[PlanLevel::kL1Pairs] = put_v(S.l1_pairs);
    pl.table_off[PlanLevel::kOut] = put_v(S.Sp.v);
    pl.table_off[PlanLevel::kL2Ptr] = put_v(S.l2_ptr);
    pl.table_off[PlanLevel::kL2Pairs] = put_v(S.l2_pairs);
    pl.table_off[PlanLevel::kT1Ptr] = put_v(S.t1_ptr);
    pl.table_off[PlanLevel::kT1] = put_v(S.t1);
    pl.table_off[PlanLevel::kT2] = put_v(S.t2);
    pl.table_off[PlanLevel::kT2pPtr] = put_v(S.t2p_ptr);
    pl.table_off[PlanLevel::kT2p] = put_v(S.t2p);
    pl.table_off[PlanLevel::kOffNext] = put_v(pl.O_next.v);
    pl.table_off[PlanLevel::kMapNext] = put_v(pl.map_next);
    for (MmaWin& W : pl.mwin) {
      W.off[0] = put_v(W.U);
      W.off[1] = put_v(W.ubits);
      W.off[2] = put_v(W.pairs);
      W.off[3] = put_v(W.rhs_o);
      W.off[4] = put_v(W.outmap);
    }
  }
  return plan;
}

std::shared_ptr<const Plan> cached_plan(int q, double rho, int rule, const OffSet& Oq,
                                        const OffSet& N) {
  static std::mutex mu;
  static std::map<std::string, std::shared_ptr<const Plan>> cache;
  std::string key = std::to_string(q) + "/" + std::to_string(rho) + "/" + std::to_string(rule);
  for (const int2& o : Oq.v) key += "/" + std::to_string(o.x) + "," + std::to_string(o.y);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
  }
  auto plan = build_plan(q, Oq, N, key);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = plan;
  return plan;
}

// ------------------------------------------------------------ autotuner
// Launch shapes chosen by timing the candidates on the device, once per
// geometry key, level and working precision in a process, then reused by
// every later setup of that geometry (the results depend on the shape only
// through summation order).  Levels smaller than kTuneMinParents keep the
// fixed rule: their kernels are too short for the choice to matter.
constexpr int64_t kTuneMinParents = 16384;
constexpr int64_t kTuneSample = 4096;  // a 64 x 64 Morton block of coarse cells
// Galerkin rows are cheap and one variant packs eight rows per CTA: a larger
// sample keeps every candidate's grid larger than the GPU
constexpr int64_t kTuneSampleRows = 16384;

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;

bool tune_lookup(const std::string& key, int* v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) return false;
  *v = it->second;
  return true;
}
void tune_store(const std::string& key, int v) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune[key] = v;
}

// Best of two timed runs after one warm-up run, CUDA events on stream s.
template <typename F>
float time_on_stream(cudaStream_t s, F&& launch) {
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  launch();
  float best = 1e30f;
  for (int r = 0; r < 2; ++r) {
    CK(cudaEventRecord(a, s));
    launch();
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, a, b));
    best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  CK(cudaGetLastError());
  return best;
}

// Algorithmic flops of the level-k patch solves: for a patch with n active
// unknowns, n^3/3 (Cholesky, right-hand side carried along) + 2 n^2 (the two
// triangular sweeps), multiply-adds counted as two flops.
double patch_flops(gamblet_ctx* h, int k) {
  const LevelDev& L = h->lv[k];
  const int Lpar = 1 << (k - 1);
  double f = 0;
  for (int64_t i = 0; i < L.npar; ++i) {
    if (!(L.pmask_h[i] & 15u)) continue;
    int x, y;
    demorton((uint32_t)i, x, y);
    double na = 0;
    for (const int2& o : h->N.v) {
      const int p = shift_cell(x, y, o.x, o.y, Lpar, L.npar);
      if (p < 0) continue;
      const int m = __builtin_popcount(L.pmask_h[p] & 15u);
      na += m > 0 ? m - 1 : 0;
    }
    f += 2.0 * (na * na * na / 6.0 + na * na / 2.0) + 2.0 * 2.0 * na * na / 2.0;
  }
  return f;
}

// Cluster split of the patch CG of level k for patches beyond one CTA's
// shared memory: the smallest cluster (2, 4, 8, 16 CTAs) whose CTAs each hold
// at most 32 block rows and fit their blocks into shared memory, the rows cut
// into contiguous ranges of at most B blocks for the smallest feasible B.
template <typename T>
bool cluster_geometry(const PatchPcgGeom& gp, const PlanLevel& pl, PatchClusterGeom& c) {
  const int NB = gp.NB;
  const std::vector<int>& ap = pl.adj_ptr;
  for (int cs : {2, 4, 8, 16}) {
    auto ranges = [&](int B, std::vector<int>& cut) {
      cut.assign(1, 0);
      int rows = 0, blocks = 0;
      for (int j = 0; j < NB; ++j) {
        const int bj = ap[j + 1] - ap[j];
        if (bj > B) return false;
        if (rows == 32 || blocks + bj > B) {
          cut.push_back(j);
          rows = 0;
          blocks = 0;
        }
        ++rows;
        blocks += bj;
      }
      cut.push_back(NB);
      return (int)cut.size() - 1 <= cs;
    };
    int lo = 1, hi = ap[NB];
    std::vector<int> cut;
    if (!ranges(hi, cut)) continue;  // more than 32 rows per CTA even with all blocks
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (ranges(mid, cut)) hi = mid;
      else lo = mid + 1;
    }
    ranges(hi, cut);
    c = PatchClusterGeom{};
    c.pg = gp;
    c.cs = cs;
    c.max_rows = 0;
    c.max_blocks = 0;
    const int nr = (int)cut.size() - 1;
    for (int r = 0; r <= cs; ++r) c.jsplit[r] = r <= nr ? cut[r] : NB;
    for (int r = 0; r < cs; ++r) {
      c.max_rows = std::max(c.max_rows, c.jsplit[r + 1] - c.jsplit[r]);
      c.max_blocks = std::max(c.max_blocks, ap[c.jsplit[r + 1]] - ap[c.jsplit[r]]);
    }
    if (c.max_rows < 1) c.max_rows = 1;
    if (patch_cluster_smem_bytes<T>(c) <= 227 * 1024) return true;
  }
  return false;
}

// Device geometry of the tensor-core patch solves with windows of G x G
// coarse cells at level k.
PatchMmaGeom mma_geometry(gamblet_ctx* h, int k, int G, const char* dplan, const PlanLevel& pl) {
  const MmaWin& W = pl.mwin[G - 1];
  const LevelDev& L = h->lv[k];
  PatchMmaGeom g{};
  g.NP = W.NP;
  g.nU = W.nU;
  g.n = W.n;
  g.Kp = W.Kp;
  g.Mt = W.Mt;
  g.npair = (int)W.pairs.size();
  g.NB = h->N.size();
  g.jc = h->jc;
  g.diag_o = W.diag_o;
  g.Lpar = 1 << (k - 1);
  g.npatch = L.npar;
  g.w_begin = 0;
  g.w_end = L.npar / W.NP;
  g.U = reinterpret_cast<const int2*>(dplan + W.off[0]);
  g.ubits = reinterpret_cast<const int*>(dplan + W.off[1]);
  g.pairs = reinterpret_cast<const int4*>(dplan + W.off[2]);
  g.rhs_o = reinterpret_cast<const int*>(dplan + W.off[3]);
  g.outmap = reinterpret_cast<const int*>(dplan + W.off[4]);
  return g;
}

// The tensor-core patch solve rounds the scaled patch matrix to float16
// (relative 2^-11 per entry), so it is a candidate only where the requested
// patch tolerance is no tighter than that rounding.
constexpr double kMmaMinPatchTol = 4.8e-4;
// The level CG reads float16 block records on the mixed path when the
// requested level tolerance is this loose (the bench's is 0.05); tighter
// tolerances keep the float32 blocks.
constexpr double kHalfLevelTol = 1e-3;

// Patch solver and launch shape at level k.  Returns 0 for the SIMT patch CG
// (with gp.spp, gp.gather set: lanes per neighbour parent 1, 2, 4 and block
// gather by thread, half-warp or four lanes per block) or G = 1, 2 for the
// tensor-core solves with windows of G x G cells (float32 path only).  The
// candidates are timed on a Morton block of kTuneSample coarse cells in the
// middle of the level (its Rhat rows are overwritten by the full launch that
// follows).
template <typename T>
int tune_patch_shape(gamblet_ctx* h, int k, PatchPcgGeom& gp, T* Rhat, const PatchMmaGeom* mg,
                     const bool* mma_ok) {
  if (!h->opts.autotune || gp.npatch < kTuneMinParents) {
    // fixed rule: the tensor-core windows of 2 x 2 cells where the patch
    // matrices are at least half full of blocks (the coarse levels; the
    // finest level's 9-point operator leaves them sparse)
    const int NB = gp.NB;
    const bool dense = 2.0 * gp.nhalf >= 0.5 * NB * (NB + 1.0);
    if (is_f32<T>() && h->patch_tol >= kMmaMinPatchTol && dense && mma_ok[1]) return 2;
    return 0;
  }
  const std::string key = h->plan->key + "/patch_pcg/" + std::to_string(k) + "/" +
                          std::to_string(sizeof(T)) + "/" + std::to_string(h->patch_tol);
  int code = 0;
  if (!tune_lookup(key, &code)) {
    cudaStream_t s = h->s;
    int* stats = h->pool.zeros<int>(4, s);
    PatchPcgGeom gt = gp;
    gt.i_begin = (gp.npatch / 2 / kTuneSample) * kTuneSample;
    gt.i_end = std::min(gt.i_begin + kTuneSample, gp.npatch);
    float best = 1e30f;
    code = gp.spp * 4 + gp.gather;
    const bool simt_fits = patch_pcg_smem_bytes<T>(gp) <= 227 * 1024;
    for (int spp : {1, 2, 4})
      for (int gather : {0, 1, 2}) {
        if (!simt_fits || gp.NB * spp > 256) continue;
        gt.spp = spp;
        gt.gather = gather;
        const float ms = time_on_stream(s, [&] {
          launch_patch_pcg<T>((const T*)h->lv[k].Ahat, h->lv[k].pmask, gt, Rhat, h->patch_tol,
                              200, stats, h->num_sms, s);
        });
        if (ms < best) {
          best = ms;
          code = spp * 4 + gather;
        }
      }
    if (is_f32<T>() && h->patch_tol >= kMmaMinPatchTol)
      for (int G = 1; G <= 2; ++G) {
        if (!mma_ok[G - 1]) continue;
        PatchMmaGeom mt = mg[G - 1];
        mt.w_begin = gt.i_begin / mt.NP;
        mt.w_end = gt.i_end / mt.NP;
        const float ms = time_on_stream(s, [&] {
          launch_patch_mma((const float*)h->lv[k].Ahat, h->lv[k].pmask, mt, (float*)Rhat,
                           h->patch_tol, 200, stats, h->status, h->num_sms, s);
        });
        if (ms < best) {
          best = ms;
          code = 64 + G;
        }
      }
    tune_store(key, code);
  }
  if (code >= 64) return code - 64;
  gp.spp = code / 4;
  gp.gather = code % 4;
  return 0;
}

// Galerkin kernel of level k (k_galerkin_rows, k_galerkin_warp or
// k_galerkin_warprow), timed on kTuneSampleRows rows in the middle of the
// level (rewritten by the full launch).
template <typename T>
void tune_galerkin_variant(gamblet_ctx* h, int k, GalerkinGeom& gg, const T* Ahat,
                           const T* Rhat, T* Acell) {
  if (!h->opts.autotune || gg.nrow < kTuneMinParents) return;
  const std::string key = h->plan->key + "/galerkin/" + std::to_string(k) + "/" +
                          std::to_string(sizeof(T));
  int v = gg.variant;
  if (!tune_lookup(key, &v)) {
    cudaStream_t s = h->s;
    GalerkinGeom gt = gg;
    gt.i_begin = (gg.nrow / 2 / kTuneSampleRows) * kTuneSampleRows;
    gt.i_end = std::min(gt.i_begin + kTuneSampleRows, gg.nrow);
    float best = 1e30f;
    for (int cand : {0, 1, 2, 3, 4, 5}) {
      if (cand == 2 && 8 * sizeof(T) * 4 * ((size_t)gg.NB + gg.nwin) > 227 * 1024) continue;
      if (cand >= 3 && galerkin_tile_smem_bytes(gg, sizeof(T)) > 227 * 1024) continue;
      gt.variant = cand;
      const float ms = time_on_stream(s, [&] {
        launch_galerkin<T>(Ahat, Rhat, h->lv[k].pmask, gt, Acell, s);
      });
      if (ms < best) {
        best = ms;
        v = cand;
      }
    }
    tune_store(key, v);
  }
  gg.variant = v;
}

// ------------------------------------------------------------ localized setup
template <typename T>
void setup_local(gamblet_ctx* h) {
  cudaStream_t s = h->s;
  Pool& P = h->pool;
  const int q = h->q;
  const int NB = h->N.size();
  if (h->patch_tol < 0 && patch_smem_bytes<T>(NB) > 227 * 1024)
    fail(GAMBLET_ERR_UNSUPPORTED, "patch of " + std::to_string(3 * NB) +
                                      " unknowns exceeds on-chip capacity; lower rho");
  if (NB > 256) fail(GAMBLET_ERR_UNSUPPORTED, "patch neighbourhood too large; lower rho");
  h->patch_stats = P.zeros<int>(4 * (q + 1), s);
  h->patch_flops_iter_k.assign(q + 1, 0.0);
  h->patch_mma_flops_k.assign(q + 1, 0.0);
  h->patch_cluster_k.assign(q + 1, false);
  // level q values in T
  {
    LevelDev& L = h->lv[q];
    const int64_t nv = (int64_t)L.noff * L.npar * 16;
    if (is_f32<T>()) {
      if (!L.Ahat) {  // transformed in float32 by the import already
        float* a32 = P.alloc<float>(nv);
        launch_convert_f64_f32(L.Ahat64, a32, nv, s);
        L.Ahat = a32;
      }
    } else {
      L.Ahat = L.Ahat64;
    }
  }
  OffSet Oq;
  for (const int2& o : h->lv[q].off_h) Oq.add(o.x, o.y);
  std::shared_ptr<const Plan> plan = cached_plan(q, h->opts.rho, h->opts.nbr_rule, Oq, h->N);
  h->plan = plan;
  const char* dplan = P.upload(plan->packed, s);  // every plan table in one copy
  h->dplan = dplan;
  for (int k = q; k >= 2; --k) {
    LevelDev& L = h->lv[k];
    const PlanLevel& pl = plan->lv[k];
    const SymLevel& S = pl.S;
    const int Lpar = 1 << (k - 1);
    L.pair_idx = plan_table<int>(dplan, pl, PlanLevel::kPairIdx);
    // patch solves -> Rhat^(k-1,k)
    T* Rhat = P.alloc<T>((int64_t)NB * 4 * L.npar);
    const double sz = (double)sizeof(T);
    const double pbytes = sz * ((double)L.noff * L.npar * 16 + 4.0 * NB * L.npar);
    if (h->patch_tol < 0) {
      PatchGeom pg{NB, h->jc, h->nbr, L.pair_idx, Lpar, L.npar};
      int tok = h->prof.begin("patch_cholesky", pbytes, h->prof.on ? patch_flops(h, k) : 0.0, s);
      launch_patch_solve<T>((const T*)L.Ahat, L.pmask, pg, Rhat, h->status, h->num_sms, s);
      h->prof.end(tok, s);
    } else {
      PatchPcgGeom gp{NB, h->jc, h->nbr, L.pair_idx, Lpar, L.npar, (int)pl.half.size(),
                      plan_table<int4>(dplan, pl, PlanLevel::kHalf), (int)pl.adj.size(),
                      plan_table<int>(dplan, pl, PlanLevel::kAdjPtr),
                      plan_table<int4>(dplan, pl, PlanLevel::kAdj),
                      plan_table<int>(dplan, pl, PlanLevel::kDiagH), pl.spp, 0, L.npar, 2};
      PatchMmaGeom mg[2];
      bool mma_ok[2];
      for (int G = 1; G <= 2; ++G) {
        mma_ok[G - 1] = is_f32<T>() && pl.mwin[G - 1].ok && L.npar % (G * G) == 0;
        mg[G - 1] = mma_geometry(h, k, G, dplan, pl);
      }
      const bool simt_fits = patch_pcg_smem_bytes<T>(gp) <= 227 * 1024;
      // 0: SIMT patch CG; G = 1, 2: tensor-core windows of G x G cells;
      // 3: SIMT patch CG over a thread-block cluster (patches beyond one CTA)
      int solver = 0;
      const int force = h->opts.patch_gather;
      const bool mma_tol = h->patch_tol >= kMmaMinPatchTol;
      if (force >= 3) {
        solver = force - 2;
        if (!mma_ok[solver - 1])
          fail(GAMBLET_ERR_UNSUPPORTED, "tensor-core patch solves (patch_gather " +
                                            std::to_string(force) +
                                            ") need the mixed path and a window that fits one "
                                            "CTA; lower rho or use patch_gather <= 2");
      } else if (!simt_fits) {
        // the single-CTA kernel cannot hold the patch: the tensor-core window
        // of one cell where its float16 rounding is within the patch
        // tolerance, else the cluster-distributed CG
        solver = (force < 0 && mma_ok[0] && mma_tol) ? 1 : 3;
      } else {
        solver = tune_patch_shape<T>(h, k, gp, Rhat, mg, mma_ok);
        if (force >= 0 && force <= 2) {
          solver = 0;
          gp.gather = force;
        }
      }
      PatchClusterGeom gcl{};
      if (solver == 3 && !cluster_geometry<T>(gp, pl, gcl))
        fail(GAMBLET_ERR_UNSUPPORTED,
             "patch of " + std::to_string(3 * NB) + " unknowns exceeds a 16-CTA cluster; lower rho");
      if (solver == 3) {
        L.shape[0] = gcl.cs;
        L.shape[1] = 5;
        int tok = h->prof.begin("patch_cluster_k" + std::to_string(k), pbytes, 0.0, s);
        CK(launch_patch_pcg_cluster<T>((const T*)L.Ahat, L.pmask, gcl, Rhat, h->patch_tol, 200,
                                       h->patch_stats + 4 * k, s));
        h->prof.end(tok, s);
        h->patch_flops_iter_k[k] = pl.flops_iter;
        h->patch_mma_flops_k[k] = 0.0;
        h->patch_cluster_k[k] = true;
      } else if (solver == 0) {
        L.shape[0] = gp.spp;
        L.shape[1] = gp.gather;
        // flops are added after setup from the measured iteration counts
        int tok = h->prof.begin("patch_pcg_k" + std::to_string(k), pbytes, 0.0, s);
        launch_patch_pcg<T>((const T*)L.Ahat, L.pmask, gp, Rhat, h->patch_tol, 200,
                            h->patch_stats + 4 * k, h->num_sms, s);
        h->prof.end(tok, s);
        h->patch_flops_iter_k[k] = pl.flops_iter;
        h->patch_mma_flops_k[k] = 0.0;
      } else {
        const PatchMmaGeom& g = mg[solver - 1];
        L.shape[0] = 0;
        L.shape[1] = 2 + solver;
        int tok = h->prof.begin("patch_mma_k" + std::to_string(k), pbytes, 0.0, s);
        launch_patch_mma((const float*)L.Ahat, L.pmask, g, (float*)Rhat, h->patch_tol, 200,
                         h->patch_stats + 4 * k, h->status, h->num_sms, s);
        h->prof.end(tok, s);
        h->patch_flops_iter_k[k] = 0.0;
        // executed tensor-core work per product: Mt M-tiles of 128 x 16 x Kp
        h->patch_mma_flops_k[k] = 2.0 * g.Mt * 128.0 * 16.0 * g.Kp;
      }
    }
    CK(cudaGetLastError());
    L.Rhat = Rhat;
    T* RT = P.alloc<T>((int64_t)NB * 4 * L.npar);
    launch_transpose_rhat<T>(Rhat, NB, h->nbr, Lpar, L.npar, RT, s);
    L.RT = RT;
    // Galerkin product -> level k-1 cell stencil (one CTA per coarse row)
    GalerkinGeom gg;
    gg.NB = NB;
    gg.nbr = h->nbr;
    gg.nwin = S.WIN.size();
    gg.win = plan_table<int2>(dplan, pl, PlanLevel::kWin);
    gg.l1_ptr = plan_table<int>(dplan, pl, PlanLevel::kL1Ptr);
    gg.l1_pairs = plan_table<int2>(dplan, pl, PlanLevel::kL1Pairs);
    gg.nout = S.Sp.size();
    gg.out = plan_table<int2>(dplan, pl, PlanLevel::kOut);
    gg.l2_ptr = plan_table<int>(dplan, pl, PlanLevel::kL2Ptr);
    gg.l2_pairs = plan_table<int2>(dplan, pl, PlanLevel::kL2Pairs);
    gg.Lpar = Lpar;
    gg.nrow = L.npar;
    gg.i_begin = 0;
    gg.i_end = L.npar;
    gg.tile_wmin = S.tile_wmin;
    gg.tile_W = S.tile_W;
    gg.t1_ptr = plan_table<int>(dplan, pl, PlanLevel::kT1Ptr);
    gg.t1 = plan_table<int2>(dplan, pl, PlanLevel::kT1);
    gg.nt2 = (int)S.t2.size();
    gg.t2 = plan_table<int4>(dplan, pl, PlanLevel::kT2);
    gg.t2p_ptr = plan_table<int>(dplan, pl, PlanLevel::kT2pPtr);
    gg.t2p = plan_table<int>(dplan, pl, PlanLevel::kT2p);
    // 2 x 2 row tiles while their window boxes stay small enough for
    // several CTAs per SM, else the warp-cooperative kernel; the autotuner
    // decides on large levels
    gg.variant = galerkin_tile_smem_bytes(gg, sizeof(T)) <= 100 * 1024 ? 3 : 1;
    if (sizeof(T) * 4 * ((size_t)NB + (size_t)gg.nwin) > 227 * 1024)
      fail(GAMBLET_ERR_UNSUPPORTED, "Galerkin window exceeds shared memory");
    T* Acell = P.alloc<T>((int64_t)gg.nout * L.npar);
    if (h->opts.galerkin_variant >= 0 && h->opts.galerkin_variant <= 5) {
      gg.variant = h->opts.galerkin_variant;
      if (gg.variant == 2 && 8 * sizeof(T) * 4 * ((size_t)NB + gg.nwin) > 227 * 1024)
        fail(GAMBLET_ERR_UNSUPPORTED, "Galerkin warp-per-row window exceeds shared memory");
      if (gg.variant >= 3 && galerkin_tile_smem_bytes(gg, sizeof(T)) > 227 * 1024)
        fail(GAMBLET_ERR_UNSUPPORTED, "Galerkin tile window exceeds shared memory");
    } else {
      tune_galerkin_variant<T>(h, k, gg, (const T*)L.Ahat, Rhat, Acell);
    }
    L.shape[2] = gg.variant;
    int tok = h->prof.begin(
        "galerkin_k" + std::to_string(k),
        sz * ((double)L.noff * L.npar * 16 + 4.0 * NB * L.npar + (double)gg.nout * L.npar),
        2.0 * (16.0 * S.l1_pairs.size() + 4.0 * S.l2_pairs.size()) * h->lv[k - 1].n_active, s);
    launch_galerkin<T>((const T*)L.Ahat, Rhat, L.pmask, gg, Acell, s);
    h->prof.end(tok, s);
    CK(cudaGetLastError());
    if (k - 1 >= 2) {
      LevelDev& Ln = h->lv[k - 1];
      Ln.off_h = pl.O_next.v;
      Ln.noff = pl.O_next.size();
      Ln.off = plan_table<int2>(dplan, pl, PlanLevel::kOffNext);
      const int* dmap = plan_table<int>(dplan, pl, PlanLevel::kMapNext);
      T* blk = P.alloc<T>((int64_t)Ln.noff * Ln.npar * 16);
      tok = h->prof.begin("cells_to_blocks",
                          sz * ((double)gg.nout * L.npar + (double)Ln.noff * Ln.npar * 16), 0.0, s);
      launch_cells_to_blocks<T>(Acell, L.npar, dmap, Ln.noff, Ln.off, 1 << (k - 2), Ln.npar,
                                Ln.pmask, blk, s);
      h->prof.end(tok, s);
      CK(cudaGetLastError());
      Ln.Ahat = blk;
    } else {
      h->l1map = plan_table<int>(dplan, pl, PlanLevel::kMapNext);
      h->A1L = P.alloc<double>(16);
      launch_level1_factor<T>(Acell, (int)L.npar, h->l1map, h->A1L, h->status, s);
      CK(cudaGetLastError());
      // keep the level-1 cell stencil for the getter
      h->lv[1].Ahat = Acell;
      h->lv[1].noff = S.Sp.size();
      h->lv[1].off_h = S.Sp.v;
    }
  }
  // level-CG operators: coalesced detail blocks and block-Jacobi inverses
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    int o0 = -1, R = 0;
    for (int o = 0; o < L.noff; ++o) {
      if (L.off_h[o].x == 0 && L.off_h[o].y == 0) o0 = o;
      R = std::max(R, std::max(std::abs(L.off_h[o].x), std::abs(L.off_h[o].y)));
    }
    if (o0 < 0) fail(GAMBLET_ERR_INVALID_ARG, "level operator has no diagonal blocks");
    L.o0 = o0;
    L.R = R;
    T* Bd = P.alloc<T>((int64_t)L.noff * 9 * L.npar);
    T* Dinv = P.alloc<T>(9 * L.npar);
    launch_cg_level_setup<T>((const T*)L.Ahat, L.noff, o0, L.npar, L.pmask, Bd, Dinv, s);
    L.Bd = Bd;
    L.Dinv = Dinv;
    L.Bq = nullptr;
    L.bq_scale = nullptr;
    if (is_f32<T>() && h->opts.level_tol >= kHalfLevelTol) {
      // the level CG's product reads each block as one 32-byte float16 record
      // (two 16-byte loads instead of nine scalar ones), with a rounding of
      // 2^-11 relative per entry, far below the level tolerance
      L.Bq = P.alloc<uint4>((int64_t)L.noff * L.npar * 2);
      L.bq_scale = P.alloc<float>(1);
      launch_cg_block_records((const float*)L.Ahat, (const float*)Bd, L.noff, L.npar, L.Bq,
                              L.bq_scale, P.alloc<unsigned>(1), s);
    }
  }
  CK(cudaGetLastError());
}

// ------------------------------------------------------------ exact setup
void setup_exact(gamblet_ctx* h) {
  cudaStream_t s = h->s;
  Pool& P = h->pool;
  const int q = h->q;
  // dense level q
  {
    LevelDev& L = h->lv[q];
    L.D = P.zeros<double>(L.ncell * L.ncell, s);
    launch_dense_from_blocks(L.Ahat64, L.off, L.noff, 1 << (q - 1), L.npar, L.D, s);
  }
  for (int k = q; k >= 2; --k) {
    LevelDev& L = h->lv[k];
    L.det_h.clear();
    L.par_h.clear();
    std::vector<double> scale;
    for (int64_t p = 0; p < L.npar; ++p) {
      const int m = __builtin_popcount(L.pmask_h[p] & 15u);
      for (int t = 0; t < m - 1; ++t) L.det_h.push_back((int32_t)(4 * p + t));
      if (m > 0) {
        L.par_h.push_back((int32_t)(4 * p + 3));
        scale.push_back(-1.0 / std::sqrt((double)m));
      }
    }
    const int nJ = (int)L.det_h.size(), nA = (int)L.par_h.size();
    L.det = P.upload(L.det_h, s);
    L.par = P.upload(L.par_h, s);
    double* dscale = P.upload(scale, s);
    L.Bc = P.alloc<double>((int64_t)nJ * nJ);
    double* Y = P.alloc<double>((int64_t)nJ * nA);
    launch_gather_rows_cols(L.D, (int)L.ncell, L.det, nJ, L.det, nJ, 1.0, nullptr, L.Bc, s);
    launch_gather_rows_cols(L.D, (int)L.ncell, L.det, nJ, L.par, nA, 1.0, dscale, Y, s);
    launch_dpotrf(L.Bc, nJ, h->status, s);
    launch_dpotrs(L.Bc, nJ, Y, nA, s);
    // parent index (not slot) for the Rhat scatter
    std::vector<int32_t> pidx;
    for (int32_t v : L.par_h) pidx.push_back(v >> 2);
    int32_t* dpidx = P.upload(pidx, s);
    L.Rh = P.zeros<double>(L.npar * L.ncell, s);
    launch_dense_rhat(Y, L.det, nJ, dpidx, nA, L.pmask, L.npar, L.Rh, s);
    double* T1 = P.alloc<double>(L.npar * L.ncell);
    launch_dgemm((int)L.npar, (int)L.ncell, (int)L.ncell, 1.0, L.Rh, L.D, 0, 0.0, T1, s);
    double* Ap = P.alloc<double>(L.npar * L.npar);
    launch_dgemm((int)L.npar, (int)L.npar, (int)L.ncell, 1.0, T1, L.Rh, 1, 0.0, Ap, s);
    CK(cudaGetLastError());
    if (k - 1 >= 2) {
      LevelDev& Ln = h->lv[k - 1];
      Ln.D = P.alloc<double>(Ln.ncell * Ln.ncell);
      launch_dense_transform(Ap, Ln.npar, Ln.pmask, Ln.D, s);
    } else {
      h->A1 = Ap;
      h->A1L = P.alloc<double>(16);
      launch_level1_factor_dense(Ap, h->A1L, h->status, s);
    }
    CK(cudaGetLastError());
  }
}

// Threads per parent of the level-CG SpMV at level k: 1 (16 x 16 tiles) or
// 4 (8 x 8 tiles), timed on the whole level with the CG direction vector
// (still zero here; the kernel has no data-dependent branches).
template <typename T>
int tuned_cg_spp(gamblet_ctx* h, int k, const CgLevel& c) {
  if (!h->opts.autotune || c.npar < kTuneMinParents) return c.spp;
  const std::string key = h->plan->key + "/cg_spmv/" + std::to_string(k) + "/" +
                          std::to_string(sizeof(T));
  int best_spp = c.spp;
  if (tune_lookup(key, &best_spp)) return best_spp;
  cudaStream_t s = h->s;
  CgScalars sc{};
  sc.active = 1;
  CgScalars* sc_d = h->pool.upload(std::vector<CgScalars>{sc}, s);
  float best = 1e30f;
  for (int spp : {1, 4, 16}) {
    CgLevel c1 = c;
    c1.spp = spp;
    c1.block_begin = 0;
    c1.spmv_begin = 0;
    const int tmax = cg_tile_side(spp);
    const int ts = std::min(c1.Lpar, tmax) + 2 * c1.R;
    if (cg_spmv_smem_bytes(ts, sizeof(T)) > 227 * 1024) continue;
    prepare_cg_spmv<T>(ts);
    CgLevel* lv_d = h->pool.upload(std::vector<CgLevel>{c1}, s);
    const int blocks = (int)((c1.npar + tmax * tmax - 1) / (tmax * tmax));
    const float ms = time_on_stream(s, [&] {
      launch_cg_spmv<T>(lv_d, 1, blocks, sc_d, ts, s);
    });
    if (ms < best) {
      best = ms;
      best_spp = spp;
    }
  }
  tune_store(key, best_spp);
  return best_spp;
}

// ------------------------------------------------------------ solve buffers
template <typename T>
void alloc_solve(gamblet_ctx* h) {
  Pool& P = h->pool;
  cudaStream_t s = h->s;
  const int q = h->q;
  for (int k = 1; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    L.ghat = P.zeros<T>(L.ncell, s);
    L.v = P.zeros<T>(L.ncell, s);
    if (k >= 2) {
      L.w = P.zeros<T>(L.ncell, s);
      if (!h->exact) {
        L.cr = P.zeros<T>(L.ncell, s);
        L.cz = P.zeros<T>(L.ncell, s);
        L.cp = P.zeros<T>(L.ncell, s);
        L.cAp = P.zeros<T>(L.ncell, s);
      } else {
        L.wc = P.zeros<double>(std::max(L.nJ, 1), s);
      }
    }
  }
  h->g1 = P.zeros<T>(4, s);
  h->U1 = P.zeros<T>(4, s);
  const int64_t nq = h->lv[q].ncell;
  h->u64 = P.zeros<double>(nq, s);
  h->xplain = P.zeros<double>(nq, s);
  h->r64 = P.zeros<double>(nq, s);
  h->z64 = P.zeros<double>(nq, s);
  h->p64 = P.zeros<double>(nq, s);
  h->q64 = P.zeros<double>(nq, s);
  h->g64 = P.zeros<double>(nq, s);
  if (is_f32<T>()) {
    h->rT = P.zeros<T>(nq, s);
    h->zT = P.zeros<T>(nq, s);
  }
  h->dots = P.zeros<double>(8, s);
  if (!h->exact) {
    std::vector<CgLevel> cl;
    int blocks = 0;
    int max_ts = 1, sblocks = 0;
    for (int k = 2; k <= q; ++k) {
      LevelDev& L = h->lv[k];
      CgLevel c;
      c.Bd = L.Bd;
      c.Bq = L.Bq;
      c.bq_inv_scale = L.bq_scale;
      c.Dinv = L.Dinv;
      c.off = L.off;
      c.noff = L.noff;
      c.R = L.R;
      c.Lpar = 1 << (k - 1);
      c.npar = L.npar;
      c.x = L.w;
      c.r = L.cr;
      c.z = L.cz;
      c.p = L.cp;
      c.Ap = L.cAp;
      c.b = L.ghat;
      c.block_begin = blocks;
      blocks += (int)((L.npar + 255) / 256);
      // wide stencils: four threads per parent over 8 x 8 tiles, or sixteen
      // over 4 x 4 tiles for the widest (more CTAs and more loads in flight
      // per byte); the autotuner may overrule the rule on large levels
      c.spp = L.noff > 128 ? 16 : (L.noff > 32 ? 4 : 1);
      c.spp = tuned_cg_spp<T>(h, k, c);
      L.shape[3] = c.spp;
      const int tmax = cg_tile_side(c.spp);
      c.spmv_begin = sblocks;
      sblocks += (int)((L.npar + tmax * tmax - 1) / (tmax * tmax));
      max_ts = std::max(max_ts, std::min(c.Lpar, tmax) + 2 * L.R);
      cl.push_back(c);
    }
    h->cg_spmv_blocks = sblocks;
    h->cg_max_ts = max_ts;
    if (cg_spmv_smem_bytes(max_ts, sizeof(T)) > 227 * 1024)
      fail(GAMBLET_ERR_UNSUPPORTED, "level operator stencil too wide for the CG tile");
    prepare_cg_spmv<T>(max_ts);
    h->cg_nlev = (int)cl.size();
    h->cg_blocks = blocks;
    // from pinned memory: a copy from pageable memory would wait here for
    // every setup kernel queued so far
    h->cg_lv = P.alloc<CgLevel>((int64_t)cl.size());
    if (!cl.empty()) {
      if ((int)cl.size() > h->q) fail(GAMBLET_ERR_INVALID_ARG, "level count exceeds q");
      std::memcpy(h->cg_lv_h, cl.data(), sizeof(CgLevel) * cl.size());
      CK(cudaMemcpyAsync(h->cg_lv, h->cg_lv_h, sizeof(CgLevel) * cl.size(),
                         cudaMemcpyHostToDevice, s));
    }
    h->cg_sc = P.zeros<CgScalars>(std::max(h->cg_nlev, 1), s);
    h->any_active = P.zeros<int>(1, s);
    h->cg_loop_count = P.zeros<int>(1, s);
    h->cg_stats = P.zeros<int>(34, s);
  }
}

// ------------------------------------------------------------ gamblet operator
// The batched level CG as one graph: a device-side while loop (conditional
// node) whose body is one CG iteration of every level; the scalar kernel of
// the body sets the loop condition from the levels' convergence, so the
// whole CG runs without host synchronisation.  Falls back to chunks of
// `chunk` captured iterations with a host check between chunks when the
// driver offers no conditional nodes.
template <typename T>
void build_cg_graph(gamblet_ctx* h, int chunk, double tol2, int maxit) {
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  CK(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond = 0;
  bool while_ok = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault) ==
                  cudaSuccess;
  cudaGraphNode_t node;
  cudaGraphNodeParams cp{};
  if (while_ok) {
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    while_ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp) == cudaSuccess;
  }
  cudaGetLastError();
  if (while_ok) {
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const long long c0 = launches_now();
    CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    launch_cg_spmv<T>(h->cg_lv, h->cg_nlev, h->cg_spmv_blocks, h->cg_sc, h->cg_max_ts, cs);
    launch_cg_rest<T>(h->cg_lv, h->cg_nlev, h->cg_blocks, h->cg_sc, tol2, maxit, h->any_active, cs,
                      cond, 1, h->cg_loop_count, maxit + 2);
    cudaGraph_t captured;
    CK(cudaStreamEndCapture(cs, &captured));
    uncount_launches(launches_now() - c0);  // counted per pass when the loop runs
    h->cg_while = true;
  } else {
    CK(cudaGraphDestroy(g));
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int c = 0; c < chunk; ++c) {
      launch_cg_spmv<T>(h->cg_lv, h->cg_nlev, h->cg_spmv_blocks, h->cg_sc, h->cg_max_ts, cs);
      launch_cg_rest<T>(h->cg_lv, h->cg_nlev, h->cg_blocks, h->cg_sc, tol2, maxit, h->any_active,
                        cs);
    }
    CK(cudaStreamEndCapture(cs, &g));
    h->cg_while = false;
  }
  CK(cudaGraphInstantiate(&h->cg_exec, g, 0));
  CK(cudaGraphDestroy(g));
  CK(cudaStreamDestroy(cs));
}

template <typename T>
void cg_work_per_iteration(gamblet_ctx* h);

// level-CG iterations per captured chunk when the driver offers no
// conditional nodes (the while-loop graph is used otherwise)
constexpr int kCgChunk = 8;

template <typename T>
void run_level_cg(gamblet_ctx* h) {
  cudaStream_t s = h->s;
  if (h->cg_nlev == 0) return;
  const double tol2 = h->opts.level_tol * h->opts.level_tol;
  const int maxit = std::max(h->opts.level_max_iter, 1);
  const int chunk = kCgChunk;
  CK(cudaMemsetAsync(h->cg_sc, 0, sizeof(CgScalars) * h->cg_nlev, s));
  CK(cudaMemsetAsync(h->cg_loop_count, 0, sizeof(int), s));
  launch_cg_init<T>(h->cg_lv, h->cg_nlev, h->cg_blocks, h->cg_sc, s);
  // CG level l solves level k = l + 2; a truncated solve stops at h->kmax
  launch_cg_start(h->cg_sc, h->cg_nlev, std::max(h->kmax - 1, 0), tol2, h->any_active, s);
  if (h->opts.use_graph && !h->cg_exec) build_cg_graph<T>(h, chunk, tol2, maxit);
  if (h->cg_exec && h->cg_while) {
    // the whole CG in one launch (timed as one "level_cg" entry)
    int tok = h->prof.begin("level_cg", 0.0, 0.0, s);
    CK(cudaGraphLaunch(h->cg_exec, s));
    h->prof.end(tok, s);
    CK(cudaGetLastError());
  } else {
    for (int it = 0; it < maxit; it += chunk) {
      if (h->cg_exec) {
        // with graphs the CG kernels are timed together, per chunk
        int tok = h->prof.begin("level_cg", 0.0, 0.0, s);
        CK(cudaGraphLaunch(h->cg_exec, s));
        h->prof.end(tok, s);
      } else {
        for (int c = 0; c < chunk; ++c) {
          int tok = h->prof.begin("level_cg_spmv", 0.0, 0.0, s);
          launch_cg_spmv<T>(h->cg_lv, h->cg_nlev, h->cg_spmv_blocks, h->cg_sc, h->cg_max_ts, s);
          h->prof.end(tok, s);
          tok = h->prof.begin("level_cg_vector", 0.0, 0.0, s);
          launch_cg_rest<T>(h->cg_lv, h->cg_nlev, h->cg_blocks, h->cg_sc, tol2, maxit,
                            h->any_active, s);
          h->prof.end(tok, s);
        }
      }
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h->any_active_h, h->any_active, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*h->any_active_h == 0) break;
    }
  }
  // iteration counts and convergence stay on the device until the solve ends
  // (levels above a truncation are not solved and cannot fail to converge)
  launch_cg_collect(h->cg_sc, h->cg_nlev, h->kmax, tol2, h->cg_while ? h->cg_loop_count : nullptr,
                    h->cg_stats, s);
  CK(cudaGetLastError());
  cg_work_per_iteration<T>(h);
}

// Level-CG counts accumulated on the device since the last call: added to
// the handle's totals and to the kernel profile (synchronises the stream).
void flush_level_stats(gamblet_ctx* h) {
  if (!h->cg_stats || h->cg_nlev == 0) return;
  int st[34];
  CK(cudaMemcpyAsync(st, h->cg_stats, sizeof(st), cudaMemcpyDeviceToHost, h->s));
  CK(cudaMemsetAsync(h->cg_stats, 0, sizeof(st), h->s));
  CK(cudaStreamSynchronize(h->s));
  for (int l = 0; l < h->cg_nlev && l + 2 < 32; ++l) {
    h->level_iters_acc[l + 2] += st[l + 2];
    if (!h->cg_bytes_spmv.empty() && st[l + 2] > 0) {
      const double it = st[l + 2];
      if (h->cg_exec) {
        h->prof.add("level_cg", it * (h->cg_bytes_spmv[l] + h->cg_bytes_vec[l]),
                    it * (h->cg_flops_spmv[l] + h->cg_flops_vec[l]));
      } else {
        h->prof.add("level_cg_spmv", it * h->cg_bytes_spmv[l], it * h->cg_flops_spmv[l]);
        h->prof.add("level_cg_vector", it * h->cg_bytes_vec[l], it * h->cg_flops_vec[l]);
      }
    }
  }
  if (st[32]) h->level_not_conv = true;
  count_launches(4LL * st[33]);  // spmv, update, scalars, direction per pass
}

// in: transformed level-q vector (T); out: transformed (inverse_last = 0) or
// plain (1) level-q vector (T).  in may alias lv[q].ghat.
template <typename T>
void apply_G_up(gamblet_ctx* h, T* out, int inverse_last);

// Restriction, level solves and the coarsest solve of the gamblet operator:
// leaves w^(k) in lv[k].w and U^(1) in h->U1.
template <typename T>
void apply_G_down(gamblet_ctx* h, const T* in) {
  cudaStream_t s = h->s;
  const int q = h->q;
  const int NB = h->N.size();
  LevelDev& Lq = h->lv[q];
  if ((const void*)in != Lq.ghat)
    CK(cudaMemcpyAsync(Lq.ghat, in, sizeof(T) * Lq.ncell, cudaMemcpyDeviceToDevice, s));
  // restriction chain
  for (int k = q; k >= 2; --k) {
    LevelDev& L = h->lv[k];
    T* dst = (T*)(k - 1 >= 2 ? h->lv[k - 1].ghat : h->g1);
    if (h->exact) {
      launch_dgemm((int)L.npar, 1, (int)L.ncell, 1.0, L.Rh, (const double*)L.ghat, 0, 0.0,
                   (double*)dst, s);
      if (k - 1 >= 2) {
        LevelDev& Ln = h->lv[k - 1];
        launch_transform_vec<T>(dst, dst, Ln.npar, Ln.pmask, +1, s);
      }
    } else {
      const double sz = (double)sizeof(T);
      int tok = h->prof.begin("restrict", sz * (4.0 * NB * L.npar + L.ncell + L.npar),
                              8.0 * NB * L.npar, s);
      launch_restrict<T>((const T*)L.Rhat, NB, h->nbr, 1 << (k - 1), L.npar, (const T*)L.ghat, dst,
                         k - 1 >= 2 ? h->lv[k - 1].pmask : nullptr, s);
      h->prof.end(tok, s);
    }
  }
  CK(cudaGetLastError());
  // level solves
  if (h->exact) {
    for (int k = 2; k <= std::min(q, h->kmax); ++k) {
      LevelDev& L = h->lv[k];
      launch_gather_det((const double*)L.ghat, L.det, L.nJ, L.wc, s);
      launch_dpotrs(L.Bc, L.nJ, L.wc, 1, s);
      CK(cudaMemsetAsync(L.w, 0, sizeof(double) * L.ncell, s));
      launch_scatter_det(L.wc, L.det, L.nJ, (double*)L.w, s);
    }
  } else {
    run_level_cg<T>(h);
  }
  launch_level1_solve<T>(h->A1L, (const T*)h->g1, (T*)h->U1, s);
  CK(cudaGetLastError());
}

// Prolongation and summation from U^(1) and the w^(k) in place.
template <typename T>
void apply_G_up(gamblet_ctx* h, T* out, int inverse_last) {
  cudaStream_t s = h->s;
  const int q = h->q;
  const int NB = h->exact ? 0 : h->N.size();
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    const T* vprev = (const T*)(k == 2 ? h->U1 : h->lv[k - 1].v);
    T* dst = (k == q) ? out : (T*)L.v;
    const int inv = (k == q) ? inverse_last : 1;
    const bool detail = k <= h->kmax;  // levels above a truncation only interpolate
    if (h->exact) {
      if (detail) CK(cudaMemcpyAsync(dst, L.w, sizeof(double) * L.ncell, cudaMemcpyDeviceToDevice, s));
      else CK(cudaMemsetAsync(dst, 0, sizeof(double) * L.ncell, s));
      launch_dgemm_t((int)L.ncell, 1, (int)L.npar, 1.0, L.Rh, 1, (const double*)vprev, 0, 1.0,
                     (double*)dst, s);
      if (inv) launch_transform_vec<T>(dst, dst, L.npar, L.pmask, -1, s);
    } else {
      const double sz = (double)sizeof(T);
      int tok = h->prof.begin("prolong", sz * (3.0 * NB * L.npar + 2.0 * L.ncell + L.npar),
                              6.0 * NB * L.npar, s);
      launch_prolong<T>((const T*)L.RT, NB, h->nbr, 1 << (k - 1), L.npar, vprev,
                        detail ? (const T*)L.w : nullptr, L.pmask, inv, dst, s);
      h->prof.end(tok, s);
    }
  }
  CK(cudaGetLastError());
}

// Level-CG traffic and flops per iteration and level (kernel profile).
template <typename T>
void cg_work_per_iteration(gamblet_ctx* h) {
  if (!h->cg_bytes_spmv.empty()) return;
  h->cg_bytes_spmv.assign(h->cg_nlev, 0.0);
  h->cg_flops_spmv.assign(h->cg_nlev, 0.0);
  h->cg_bytes_vec.assign(h->cg_nlev, 0.0);
  h->cg_flops_vec.assign(h->cg_nlev, 0.0);
  for (int l = 0; l < h->cg_nlev; ++l) {
    // the 3x3 detail blocks of B^(k) once per iteration, p read, Ap written
    // (3 active slots); vector kernels: x, r, z, p, Ap, Dinv
    const LevelDev& L = h->lv[l + 2];
    const double sz = (double)sizeof(T);
    h->cg_bytes_spmv[l] = (L.Bq ? 32.0 : 9.0 * sz) * ((double)L.noff * L.npar) + sz * 6.0 * L.npar;
    h->cg_flops_spmv[l] = 2.0 * 9.0 * L.noff * L.npar;
    h->cg_bytes_vec[l] = sz * 3.0 * L.npar * 12;
    h->cg_flops_vec[l] = 3.0 * L.npar * 12;
  }
}

template <typename T>
void apply_G(gamblet_ctx* h, const T* in, T* out, int inverse_last) {
  apply_G_down<T>(h, in);
  apply_G_up<T>(h, out, inverse_last);
}

// Components u^(l) - u^(l-1) in Morton order (plain), level by level.
template <typename T>
void components(gamblet_ctx* h, T* out_q /* ncell_q */, int lev, T* scratch_a, T* scratch_b) {
  cudaStream_t s = h->s;
  const int q = h->q;
  const int NB = h->N.size();
  // v at level `lev`
  T* cur = scratch_a;
  T* nxt = scratch_b;
  if (lev == 1) {
    CK(cudaMemcpyAsync(cur, h->U1, sizeof(T) * 4, cudaMemcpyDeviceToDevice, s));
  } else {
    LevelDev& L = h->lv[lev];
    CK(cudaMemsetAsync(nxt, 0, sizeof(T) * L.npar, s));
    if (h->exact) {
      CK(cudaMemcpyAsync(cur, L.w, sizeof(double) * L.ncell, cudaMemcpyDeviceToDevice, s));
      launch_transform_vec<T>(cur, cur, L.npar, L.pmask, -1, s);
    } else {
      launch_prolong<T>((const T*)L.RT, NB, h->nbr, 1 << (lev - 1), L.npar, nxt, (const T*)L.w,
                        L.pmask, 1, cur, s);
    }
  }
  for (int k = lev + 1; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    if (h->exact) {
      launch_dgemm_t((int)L.ncell, 1, (int)L.npar, 1.0, L.Rh, 1, (const double*)cur, 0, 0.0,
                     (double*)nxt, s);
      launch_transform_vec<T>(nxt, nxt, L.npar, L.pmask, -1, s);
    } else {
      launch_prolong<T>((const T*)L.RT, NB, h->nbr, 1 << (k - 1), L.npar, cur, nullptr, L.pmask,
                        1, nxt, s);
    }
    std::swap(cur, nxt);
  }
  CK(cudaMemcpyAsync(out_q, cur, sizeof(T) * h->lv[q].ncell, cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
}

template <typename T>
T* as_T(gamblet_ctx* h, double* v64, void* vT, int64_t n, bool to) {
  if (!is_f32<T>()) return (T*)v64;
  if (to) launch_convert_f64_f32(v64, (float*)vT, n, h->s);
  return (T*)vT;
}

template <typename T>
gamblet_status solve_impl(gamblet_ctx* h, const double* g_user, double* u_user, double* comps_user,
                          gamblet_info* info) {
  cudaStream_t s = h->s;
  Pool tmp;
  tmp.s = h->s;
  const int q = h->q;
  LevelDev& Lq = h->lv[q];
  const int64_t nq = Lq.ncell;
  flush_level_stats(h);  // counts of earlier calls (compression, diagnostics) are not this solve's
  for (int k = 0; k < 32; ++k) h->level_iters_acc[k] = 0;
  h->level_not_conv = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  double* g_dev = nullptr;
  to_device(tmp, g_dev, g_user, h->n, s);
  // ghat = Q g (float64, Morton order)
  launch_gather_morton(g_dev, h->unknown_of, nq, h->g64, s);
  launch_transform_vec<double>(h->g64, h->g64, Lq.npar, Lq.pmask, +1, s);
  CK(cudaMemsetAsync(h->dots, 0, sizeof(double) * 8, s));
  launch_dots(nq, h->g64, h->g64, nullptr, nullptr, nullptr, nullptr, h->dots, s);
  CK(cudaMemcpyAsync(h->dots_h, h->dots, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double gnorm = std::sqrt(h->dots_h[0]);
  gamblet_status st = GAMBLET_OK;
  int outer = 0;
  double relres = 0;
  // z = G ghat (one pass)
  T* gT = as_T<T>(h, h->g64, h->rT, nq, true);
  T* zT = as_T<T>(h, h->z64, h->zT, nq, false);
  apply_G<T>(h, gT, zT, 0);
  if (is_f32<T>()) launch_convert_f32_f64((const float*)zT, h->z64, nq, s);
  T* comp_scratch = nullptr;
  if (comps_user) {
    // components of the one-pass transform
    T* ca = tmp.alloc<T>(nq);
    T* cb = tmp.alloc<T>(nq);
    T* cq = tmp.alloc<T>(nq);
    double* c64 = tmp.alloc<double>(nq);
    double* cu = tmp.alloc<double>(h->n);
    for (int lev = 1; lev <= q; ++lev) {
      components<T>(h, cq, lev, ca, cb);
      if (is_f32<T>()) launch_convert_f32_f64((const float*)cq, c64, nq, s);
      else CK(cudaMemcpyAsync(c64, cq, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
      launch_scatter_unknown(c64, h->morton_of, h->n, cu, s);
      if (h->mass) {
        double* cm = tmp.alloc<double>(h->n);
        launch_mass_apply(h->n, h->NBq, h->nbrq, h->Minv, cu, h->morton_of, h->unknown_of,
                          1 << q, Lq.ncell, cm, s);
        cu = cm;
      }
      CK(cudaMemcpyAsync(comps_user + (int64_t)(lev - 1) * h->n, cu, sizeof(double) * h->n,
                         cudaMemcpyDefault, s));
    }
    (void)comp_scratch;
  }
  CK(cudaMemcpyAsync(h->u64, h->z64, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
  const int maxit = h->opts.refine_max_iter;
  if (maxit > 0 && gnorm > 0) {
    // flexible CG (one-term orthogonalisation) on Ahat^(q) u = ghat
    double* d = h->dots;
    // r = g - A u
    outer_spmv(h, h->u64, h->q64);
    CK(cudaMemcpyAsync(h->r64, h->g64, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(d, 0, sizeof(double) * 8, s));
    // d[7] = 1 used as unit denominator: r += (-1) * (1/1) q
    double one = 1.0;
    CK(cudaMemcpyAsync(d + 7, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_axpy(nq, d + 7, d + 7, -1.0, h->q64, h->r64, s);
    launch_dots(nq, h->r64, h->r64, nullptr, nullptr, nullptr, nullptr, d, s);
    CK(cudaMemcpyAsync(h->dots_h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    relres = std::sqrt(h->dots_h[0]) / gnorm;
    if (relres > h->opts.refine_tol) {
      T* rT = as_T<T>(h, h->r64, h->rT, nq, true);
      apply_G<T>(h, rT, zT, 0);
      if (is_f32<T>()) launch_convert_f32_f64((const float*)zT, h->z64, nq, s);
      CK(cudaMemcpyAsync(h->p64, h->z64, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
      for (outer = 1; outer <= maxit; ++outer) {
        // stencil read once, xhat read, x written and read, yhat written
        int tok = h->prof.begin("outer_spmv64", 8.0 * ((double)h->qns * Lq.ncell + 4.0 * Lq.ncell),
                                2.0 * h->qns * Lq.ncell + 2.0 * 32.0 * Lq.npar, s);
        outer_spmv(h, h->p64, h->q64);
        h->prof.end(tok, s);
        CK(cudaMemsetAsync(d, 0, sizeof(double) * 4, s));
        // d0 = p.q, d1 = p.r
        launch_dots(nq, h->p64, h->q64, h->p64, h->r64, nullptr, nullptr, d, s);
        launch_axpy(nq, d + 1, d + 0, +1.0, h->p64, h->u64, s);
        launch_axpy(nq, d + 1, d + 0, -1.0, h->q64, h->r64, s);
        launch_dots(nq, nullptr, nullptr, nullptr, nullptr, h->r64, h->r64, d, s);  // d2 = r.r
        CK(cudaMemcpyAsync(h->dots_h, d, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        relres = std::sqrt(h->dots_h[2]) / gnorm;
        if (!(relres == relres)) fail(GAMBLET_ERR_NOT_SPD, "outer iteration produced NaN");
        if (relres <= h->opts.refine_tol) break;
        rT = as_T<T>(h, h->r64, h->rT, nq, true);
        apply_G<T>(h, rT, zT, 0);
        if (is_f32<T>()) launch_convert_f32_f64((const float*)zT, h->z64, nq, s);
        // d3 = z.q ; p = z - (d3 / d0) p
        launch_dots(nq, h->z64, h->q64, nullptr, nullptr, nullptr, nullptr, d + 3, s);
        launch_xpby(nq, h->z64, d + 3, d + 0, -1.0, h->p64, s);
        CK(cudaGetLastError());
      }
      if (outer > maxit) {
        outer = maxit;
        st = GAMBLET_ERR_NOT_CONVERGED;
      }
    }
    // true residual
    outer_spmv(h, h->u64, h->q64);
    CK(cudaMemcpyAsync(h->r64, h->g64, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(d + 7, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_axpy(nq, d + 7, d + 7, -1.0, h->q64, h->r64, s);
    CK(cudaMemsetAsync(d, 0, sizeof(double), s));
    launch_dots(nq, h->r64, h->r64, nullptr, nullptr, nullptr, nullptr, d, s);
    CK(cudaMemcpyAsync(h->dots_h, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    relres = std::sqrt(h->dots_h[0]) / gnorm;
  }
  // u = Q^T uhat, back to unknown order (and, after a mass initialisation,
  // from the coefficients U of psi^(q) to nodal coefficients M^-1,loc U)
  launch_transform_vec<double>(h->u64, h->q64, Lq.npar, Lq.pmask, -1, s);
  double* u_out = is_device_ptr(u_user) ? u_user : tmp.alloc<double>(h->n);
  if (h->mass) {
    double* U = tmp.alloc<double>(h->n);
    launch_scatter_unknown(h->q64, h->morton_of, h->n, U, s);
    launch_mass_apply(h->n, h->NBq, h->nbrq, h->Minv, U, h->morton_of, h->unknown_of, 1 << q,
                      Lq.ncell, u_out, s);
  } else {
    launch_scatter_unknown(h->q64, h->morton_of, h->n, u_out, s);
  }
  if (u_out != u_user)
    CK(cudaMemcpyAsync(u_user, u_out, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  flush_level_stats(h);
  h->prof.resolve();
  check_status(h, "solve");
  if (maxit == 0 && h->level_not_conv) st = GAMBLET_ERR_NOT_CONVERGED;
  if (info) {
    info->status = st;
    info->q = q;
    info->outer_iters = outer;
    for (int k = 0; k < 32; ++k) info->level_iters[k] = h->level_iters_acc[k];
    info->rel_residual = relres;
    info->setup_ms = h->setup_ms;
    info->solve_ms = ms;
    info->patch_iters_max = h->patch_iters_max;
    info->patch_iters_mean = h->patch_iters_mean;
  }
  return st;
}

// ------------------------------------------------- one-pass gradient (reverse)
// Symbolic tables of the reverse pass at level k (all offsets in level-(k-1)
// cell units unless stated):
//  S   plain offsets of A^(k-1): 2 O_(k-1) + (c' - c) over the child slots
//      (the 3 x 3 box when k - 1 = 1);
//  TW  window S + N of T = X Rhat, with the pairs (d, j), S_d + N_j = TW_w;
//  rg  [NB][noff_k] window index of N_j - O_o;
//  yg  [noff_k][NB] (window index of N_j + O_o, index j' of N_j + O_o in N).
struct RevLevel {
  int nS = 0, nTW = 0;
  const int2* S = nullptr;
  const int* tw_ptr = nullptr;
  const int2* tw_pairs = nullptr;
  const int* rg = nullptr;
  const int2* yg = nullptr;
};

// Box lookup (2 obox + 1)^2 -> index in a block-offset list, -1 elsewhere.
std::vector<int> offset_box(const std::vector<int2>& off, int& obox) {
  obox = 0;
  for (const int2& o : off) obox = std::max(obox, std::max(std::abs(o.x), std::abs(o.y)));
  const int side = 2 * obox + 1;
  std::vector<int> box((size_t)side * side, -1);
  for (size_t e = 0; e < off.size(); ++e)
    box[(size_t)(off[e].y + obox) * side + (off[e].x + obox)] = (int)e;
  return box;
}

// Every level's reverse tables and the block-offset boxes, packed into one
// buffer (16-byte aligned pieces) and cached process-wide per plan: they
// depend only on the geometry, and one upload per call replaces a
// synchronising copy per table.
struct RevPack {
  std::vector<char> bytes;
  struct Level {
    int nS = 0, nTW = 0, obox = 0;
    size_t S = 0, tw_ptr = 0, tw_pairs = 0, rg = 0, yg = 0, oidx = 0;
  };
  std::vector<Level> lv;  // index k; lv[1] holds only the box of O_1 (unused)
  int oboxq = 0;
  size_t oidxq = 0;
};

template <typename V>
size_t pack_append(std::vector<char>& buf, const std::vector<V>& v) {
  size_t off = (buf.size() + 15) & ~(size_t)15;
  buf.resize(off + sizeof(V) * v.size());
  if (!v.empty()) std::memcpy(buf.data() + off, v.data(), sizeof(V) * v.size());
  return off;
}

std::shared_ptr<const RevPack> reverse_pack(gamblet_ctx* h) {
  static std::mutex mu;
  static std::map<std::string, std::shared_ptr<const RevPack>> cache;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(h->plan->key);
    if (it != cache.end()) return it->second;
  }
  auto P = std::make_shared<RevPack>();
  const int q = h->q;
  const OffSet& N = h->N;
  P->lv.resize(q + 1);
  for (int k = 2; k <= q; ++k) {
    RevPack::Level& R = P->lv[k];
    OffSet S;
    if (k - 1 == 1) {
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) S.add(dx, dy);
    } else {
      for (const int2& o : h->lv[k - 1].off_h)
        for (int c = 0; c < 4; ++c)
          for (int cp = 0; cp < 4; ++cp)
            S.add(2 * o.x + (cp & 1) - (c & 1), 2 * o.y + (cp >> 1) - (c >> 1));
    }
    OffSet TW;
    for (const int2& d : S.v)
      for (const int2& n : N.v) TW.add(d.x + n.x, d.y + n.y);
    std::vector<std::vector<int2>> lists(TW.size());
    for (int d = 0; d < S.size(); ++d)
      for (int j = 0; j < N.size(); ++j)
        lists[TW.find(S.v[d].x + N.v[j].x, S.v[d].y + N.v[j].y)].push_back(make_int2(d, j));
    std::vector<int> ptr(1, 0);
    std::vector<int2> pairs;
    for (const auto& l : lists) {
      pairs.insert(pairs.end(), l.begin(), l.end());
      ptr.push_back((int)pairs.size());
    }
    const std::vector<int2>& Ok = h->lv[k].off_h;
    const int NB = N.size(), no = (int)Ok.size();
    std::vector<int> rg((size_t)NB * no);
    std::vector<int2> yg((size_t)no * NB);
    for (int j = 0; j < NB; ++j)
      for (int o = 0; o < no; ++o) {
        rg[(size_t)j * no + o] = TW.find(N.v[j].x - Ok[o].x, N.v[j].y - Ok[o].y);
        const int wx = N.v[j].x + Ok[o].x, wy = N.v[j].y + Ok[o].y;
        yg[(size_t)o * NB + j] = make_int2(TW.find(wx, wy), N.find(wx, wy));
      }
    R.nS = S.size();
    R.nTW = TW.size();
    R.S = pack_append(P->bytes, S.v);
    R.tw_ptr = pack_append(P->bytes, ptr);
    R.tw_pairs = pack_append(P->bytes, pairs);
    R.rg = pack_append(P->bytes, rg);
    R.yg = pack_append(P->bytes, yg);
    if (k - 1 >= 2) R.oidx = pack_append(P->bytes, offset_box(h->lv[k - 1].off_h, R.obox));
  }
  P->oidxq = pack_append(P->bytes, offset_box(h->lv[q].off_h, P->oboxq));
  std::lock_guard<std::mutex> lock(mu);
  cache[h->plan->key] = P;
  return P;
}

// The patch-CG geometry of level k as the setup launched it (the plan's
// default shape where the setup used the tensor-core solves).
PatchPcgGeom patch_geometry(gamblet_ctx* h, int k) {
  const PlanLevel& pl = h->plan->lv[k];
  LevelDev& L = h->lv[k];
  const char* dplan = h->dplan;
  const bool simt = L.shape[1] <= 2 && L.shape[0] > 0;
  PatchPcgGeom gp{h->N.size(), h->jc, h->nbr, L.pair_idx, 1 << (k - 1), L.npar,
                  (int)pl.half.size(), plan_table<int4>(dplan, pl, PlanLevel::kHalf),
                  (int)pl.adj.size(), plan_table<int>(dplan, pl, PlanLevel::kAdjPtr),
                  plan_table<int4>(dplan, pl, PlanLevel::kAdj),
                  plan_table<int>(dplan, pl, PlanLevel::kDiagH), simt ? L.shape[0] : pl.spp, 0,
                  L.npar, simt ? L.shape[1] : 2};
  return gp;
}

// Gradient of J = 1/2 |u_loc - u_obs|^2 for the one-pass localized solution
// u_loc = G_loc g (Algorithm 2 with the handle's patch and level solves).
// Forward: the one-pass transform of g and of the misfit (G_loc is
// symmetric, so the second pass is the adjoint of the solve chain and gives
// dJ/dg); reverse: the setup levels from the coarsest to the finest.  T is the
// working precision of the hierarchy (float on the mixed path); J, the
// misfit and the outputs are float64.
template <typename T>
gamblet_status grad_onepass_impl(gamblet_ctx* h, int ncell, const int32_t* cell_nodes,
                                 const double* cell_a, const double* K_ref, const double* g_user,
                                 const double* uobs_user, double* u_user, double* dJ_user,
                                 double* dJdg_user, double* J, gamblet_info* info) {
  cudaStream_t s = h->s;
  const int q = h->q;
  const int NB = h->N.size();
  LevelDev& Lq = h->lv[q];
  const int64_t nq = Lq.ncell;
  Pool tmp;
  tmp.s = s;
  flush_level_stats(h);
  for (int k = 0; k < 32; ++k) h->level_iters_acc[k] = 0;
  h->level_not_conv = false;
  const int kmax_saved = h->kmax;
  h->kmax = q;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // every table of the reverse pass in one copy, and the caller's arrays,
  // before any kernel is queued (copies from pageable host memory wait for
  // the stream)
  std::shared_ptr<const RevPack> pack = reverse_pack(h);
  const char* dpack = tmp.upload(pack->bytes, s);
  double* g_dev = nullptr;
  double* uo_dev = nullptr;
  to_device(tmp, g_dev, g_user, h->n, s);
  to_device(tmp, uo_dev, uobs_user, h->n, s);
  int32_t* cn = nullptr;
  double* ca = nullptr;
  double* kr = nullptr;
  to_device(tmp, cn, cell_nodes, 4 * (int64_t)ncell, s);
  to_device(tmp, ca, cell_a, ncell, s);
  to_device(tmp, kr, K_ref, 16, s);
  double* d = h->dots;
  CK(cudaMemsetAsync(d, 0, sizeof(double) * 8, s));
  const double one = 1.0;
  CK(cudaMemcpyAsync(d + 7, &one, sizeof(double), cudaMemcpyHostToDevice, s));
  // ---- forward: u_hat = G ghat, keeping the intermediates of every level
  launch_gather_morton(g_dev, h->unknown_of, nq, h->g64, s);
  launch_transform_vec<double>(h->g64, h->g64, Lq.npar, Lq.pmask, +1, s);
  T* gT = as_T<T>(h, h->g64, h->rT, nq, true);
  T* zT = as_T<T>(h, h->z64, h->zT, nq, false);
  apply_G<T>(h, gT, zT, 0);
  if (is_f32<T>()) launch_convert_f32_f64((const float*)zT, h->z64, nq, s);
  std::vector<T*> gh(q + 1, nullptr), wg(q + 1, nullptr), vg(q + 1, nullptr);
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    gh[k] = tmp.alloc<T>(L.ncell);
    wg[k] = tmp.alloc<T>(L.ncell);
    CK(cudaMemcpyAsync(gh[k], L.ghat, sizeof(T) * L.ncell, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(wg[k], L.w, sizeof(T) * L.ncell, cudaMemcpyDeviceToDevice, s));
    if (k < q) {
      vg[k] = tmp.alloc<T>(L.ncell);
      CK(cudaMemcpyAsync(vg[k], L.v, sizeof(T) * L.ncell, cudaMemcpyDeviceToDevice, s));
    }
  }
  T* U1g = tmp.alloc<T>(4);
  CK(cudaMemcpyAsync(U1g, h->U1, sizeof(T) * 4, cudaMemcpyDeviceToDevice, s));
  // ---- misfit (transformed) and J
  launch_gather_morton(uo_dev, h->unknown_of, nq, h->r64, s);
  launch_transform_vec<double>(h->r64, h->r64, Lq.npar, Lq.pmask, +1, s);
  CK(cudaMemcpyAsync(h->p64, h->z64, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
  launch_axpy(nq, d + 7, d + 7, -1.0, h->r64, h->p64, s);
  launch_dots(nq, h->p64, h->p64, nullptr, nullptr, nullptr, nullptr, d, s);
  // ---- the misfit through the same chain: lambda^(k), dJ/dg
  T* mT = as_T<T>(h, h->p64, h->rT, nq, true);
  T* dgT = is_f32<T>() ? (T*)h->zT : (T*)h->q64;
  apply_G<T>(h, mT, dgT, 0);
  if (is_f32<T>()) launch_convert_f32_f64((const float*)dgT, h->q64, nq, s);
  // ---- reverse of the setup
  std::vector<T*> Y(q + 1, nullptr);
  int64_t max_rows = 0;
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    Y[k] = tmp.zeros<T>((int64_t)L.noff * L.npar * 16, s);
    launch_ybar_level<T>(Y[k], L.noff, L.off, 1 << (k - 1), L.npar, (const T*)L.w, wg[k], s);
    max_rows = std::max(max_rows, L.npar);
  }
  T* A1bar = tmp.alloc<T>(16);
  launch_abar1<T>(A1bar, (const T*)h->U1, U1g, s);
  T* Rbar = tmp.alloc<T>(max_rows * NB * 4);
  T* M = tmp.alloc<T>(max_rows * NB * 4);
  int* pstats = tmp.zeros<int>(4, s);
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    const int Lpar = 1 << (k - 1);
    const RevPack::Level& pk = pack->lv[k];
    RevLevel R;
    R.nS = pk.nS;
    R.nTW = pk.nTW;
    R.S = reinterpret_cast<const int2*>(dpack + pk.S);
    R.tw_ptr = reinterpret_cast<const int*>(dpack + pk.tw_ptr);
    R.tw_pairs = reinterpret_cast<const int2*>(dpack + pk.tw_pairs);
    R.rg = reinterpret_cast<const int*>(dpack + pk.rg);
    R.yg = reinterpret_cast<const int2*>(dpack + pk.yg);
    const int obox = pk.obox;
    const int* oidx = k - 1 >= 2 ? reinterpret_cast<const int*>(dpack + pk.oidx) : nullptr;
    T* X = tmp.alloc<T>((int64_t)R.nS * L.npar);
    T* Tw = tmp.alloc<T>(L.npar * R.nTW * 4);
    const T* vprev = k == 2 ? U1g : vg[k - 1];
    const T* gbprev = (const T*)(k == 2 ? h->U1 : h->lv[k - 1].v);
    int tok = h->prof.begin("grad_rbar_outer", 0.0, 0.0, s);
    launch_rbar_outer<T>(Rbar, h->nbr, NB, Lpar, L.npar, vprev, gbprev, (const T*)L.ghat, gh[k],
                         s);
    h->prof.end(tok, s);
    tok = h->prof.begin("grad_xbar", 0.0, 0.0, s);
    launch_xbar_cells<T>(X, R.nS, R.S, Lpar, L.npar, k - 1 == 1 ? A1bar : nullptr,
                      k - 1 >= 2 ? Y[k - 1] : nullptr, k - 1 >= 2 ? h->lv[k - 1].npar : 0, oidx,
                      obox, k - 1 >= 2 ? h->lv[k - 1].pmask : nullptr, s);
    h->prof.end(tok, s);
    tok = h->prof.begin("grad_window_product", 0.0, 0.0, s);
    launch_window_product<T>(Tw, R.nTW, R.tw_ptr, R.tw_pairs, X, R.S, (const T*)L.Rhat, NB, Lpar,
                             L.npar, s);
    h->prof.end(tok, s);
    tok = h->prof.begin("grad_rbar_galerkin", 0.0, 0.0, s);
    launch_rbar_galerkin<T>(Rbar, Tw, R.nTW, R.rg, (const T*)L.Ahat, L.noff, L.off, h->nbr, NB,
                            Lpar, L.npar, s);
    h->prof.end(tok, s);
    tok = h->prof.begin("grad_patch_adjoint", 0.0, 0.0, s);
    launch_patch_pcg_adjoint<T>((const T*)L.Ahat, L.pmask, patch_geometry(h, k), Rbar, M,
                                h->patch_tol, 200, pstats, h->num_sms, s);
    h->prof.end(tok, s);
    tok = h->prof.begin("grad_ybar_galerkin", 0.0, 0.0, s);
    launch_ybar_galerkin<T>(Y[k], L.noff, L.off, R.yg, Tw, R.nTW, (const T*)L.Rhat, M, h->nbr, NB,
                            Lpar, L.npar, s);
    h->prof.end(tok, s);
    CK(cudaGetLastError());
  }
  // ---- dJ/dlog a from the finest level's adjoint
  const int oboxq = pack->oboxq;
  const int* oidxq = reinterpret_cast<const int*>(dpack + pack->oidxq);
  const bool dev_dJ = is_device_ptr(dJ_user);
  double* dJ = dev_dJ ? dJ_user : tmp.alloc<double>(ncell);
  int tok = h->prof.begin("grad_cells", 0.0, 0.0, s);
  launch_grad_cells<T>(dJ, ncell, cn, ca, kr, h->morton_of, Y[q], Lq.npar, oidxq, oboxq, Lq.pmask,
                       s);
  h->prof.end(tok, s);
  if (!dev_dJ) CK(cudaMemcpyAsync(dJ_user, dJ, sizeof(double) * ncell, cudaMemcpyDeviceToHost, s));
  // ---- u_loc and dJ/dg back to unknown order
  auto to_user = [&](double* hat, double* user) {
    if (!user) return;
    launch_transform_vec<double>(hat, hat, Lq.npar, Lq.pmask, -1, s);
    double* o = is_device_ptr(user) ? user : tmp.alloc<double>(h->n);
    launch_scatter_unknown(hat, h->morton_of, h->n, o, s);
    if (o != user) CK(cudaMemcpyAsync(user, o, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
  };
  to_user(h->z64, u_user);
  to_user(h->q64, dJdg_user);
  double jh = 0;
  CK(cudaMemcpyAsync(&jh, d, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->kmax = kmax_saved;
  if (J) *J = 0.5 * jh;
  flush_level_stats(h);
  h->prof.resolve();
  check_status(h, "one-pass gradient");
  const gamblet_status st = h->level_not_conv ? GAMBLET_ERR_NOT_CONVERGED : GAMBLET_OK;
  if (info) {
    info->status = st;
    info->q = q;
    info->outer_iters = 0;
    for (int k = 0; k < 32; ++k) info->level_iters[k] = h->level_iters_acc[k];
    info->rel_residual = 0;
    info->setup_ms = h->setup_ms;
    info->solve_ms = ms;
    info->patch_iters_max = h->patch_iters_max;
    info->patch_iters_mean = h->patch_iters_mean;
  }
  return st;
}

gamblet_status set_error(const GbError& e) {
  g_last_error = e.msg;
  return e.st;
}

}  // namespace

namespace {

// gamblet_setup without the status conversion: throws GbError, frees the
// handle on failure.
gamblet_ctx* setup_impl(const gamblet_csr* A, int32_t q, const int32_t* cells,
                        const gamblet_opts* opts) {
  gamblet_ctx* h = nullptr;
  try {
    if (!A || !cells) fail(GAMBLET_ERR_INVALID_ARG, "A and cells must be non-NULL");
    if (A->n < 1 || A->nnz < 1 || !A->rowptr || !A->colind || !A->val)
      fail(GAMBLET_ERR_INVALID_ARG, "empty or incomplete CSR");
    if (q < 2 || q > 15) fail(GAMBLET_ERR_INVALID_ARG, "q must be in [2, 15]");
    if ((int64_t)A->n > ((int64_t)1 << (2 * q)))
      fail(GAMBLET_ERR_INVALID_ARG, "more unknowns than level-q cells");
    h = new gamblet_ctx();
    if (opts) h->opts = *opts;
    else gamblet_default_opts(&h->opts);
    h->s = (cudaStream_t)h->opts.stream;
    h->pool.s = h->s;
    h->prof.on = h->opts.profile != 0;
    h->q = q;
    h->kmax = q;
    h->n = A->n;
    h->exact = !(h->opts.rho > 0);
    h->mixed = h->opts.precision == GAMBLET_MIXED && !h->exact;
    h->patch_tol = h->opts.patch_tol != 0 ? h->opts.patch_tol : (h->mixed ? 1e-3 : 1e-12);
    if (h->opts.precision != GAMBLET_FP64 && h->opts.precision != GAMBLET_MIXED)
      fail(GAMBLET_ERR_INVALID_ARG, "unknown precision");
    if (h->opts.nbr_rule != 0 && h->opts.nbr_rule != 1)
      fail(GAMBLET_ERR_INVALID_ARG, "nbr_rule must be 0 or 1");
    if (h->opts.galerkin_variant < -1 || h->opts.galerkin_variant > 5)
      fail(GAMBLET_ERR_INVALID_ARG, "galerkin_variant must be -1 or 0..5");
    if (h->opts.patch_gather < -1 || h->opts.patch_gather > 4)
      fail(GAMBLET_ERR_INVALID_ARG, "patch_gather must be -1 or 0..4");
    if (h->exact && q > 7)
      fail(GAMBLET_ERR_UNSUPPORTED, "the exact (rho <= 0) transform is limited to q <= 7");
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev));
    for (int k = 0; k < 32; ++k) h->level_iters_acc[k] = 0;
    CK(cudaMallocHost(&h->any_active_h, sizeof(int)));
    CK(cudaMallocHost(&h->dots_h, sizeof(double) * 8));
    CK(cudaMallocHost(&h->status_h, sizeof(int)));
    CK(cudaMallocHost(&h->cg_lv_h, sizeof(CgLevel) * (size_t)std::max(q, 1)));
    h->status = h->pool.zeros<int>(1, h->s);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, h->s));
    if (!h->exact) {
      h->N = neighbour_offsets(h->opts.rho, h->opts.nbr_rule);
      h->jc = h->N.find(0, 0);
      h->nbr = h->pool.upload(h->N.v, h->s);
    }
    build_hierarchy(h, cells);
    import_fine(h, A);
    if (h->exact) {
      setup_exact(h);
      alloc_solve<double>(h);
    } else if (h->mixed) {
      setup_local<float>(h);
      alloc_solve<float>(h);
    } else {
      setup_local<double>(h);
      alloc_solve<double>(h);
    }
    CK(cudaEventRecord(e1, h->s));
    // the level-CG graph is captured while the device still runs the setup
    // (a capture launches nothing), not inside the first solve
    if (!h->exact && h->opts.use_graph && h->cg_nlev > 0 && !h->cg_exec) {
      const double tol2 = h->opts.level_tol * h->opts.level_tol;
      const int maxit = std::max(h->opts.level_max_iter, 1);
      if (h->mixed) build_cg_graph<float>(h, kCgChunk, tol2, maxit);
      else build_cg_graph<double>(h, kCgChunk, tol2, maxit);
    }
    CK(cudaStreamSynchronize(h->s));
    CK(cudaGetLastError());
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->setup_ms = ms;
    if (h->patch_stats && h->patch_tol >= 0) {
      std::vector<int> ps(4 * (q + 1));
      CK(cudaMemcpy(ps.data(), h->patch_stats, sizeof(int) * ps.size(), cudaMemcpyDeviceToHost));
      long long it_sum = 0, n_sum = 0;
      h->patch_iters_max = 0;
      for (int k = 2; k <= q; ++k) {
        h->patch_iters_max = std::max(h->patch_iters_max, ps[4 * k]);
        it_sum += ps[4 * k + 1];
        n_sum += ps[4 * k + 2];
        // algorithmic flops of the patch CG at level k: per iteration the
        // block product (18 flops per used 3x3 block) plus block-Jacobi and
        // vector work, times the iterations actually run
        if (h->patch_mma_flops_k[k] > 0)
          h->prof.add("patch_mma_k" + std::to_string(k), 0.0,
                      (double)ps[4 * k + 3] * h->patch_mma_flops_k[k]);
        else if (h->patch_cluster_k[k])
          h->prof.add("patch_cluster_k" + std::to_string(k), 0.0,
                      (double)ps[4 * k + 1] * h->patch_flops_iter_k[k]);
        else
          h->prof.add("patch_pcg_k" + std::to_string(k), 0.0,
                      (double)ps[4 * k + 1] * h->patch_flops_iter_k[k]);
      }
      h->patch_iters_mean = n_sum > 0 ? (double)it_sum / n_sum : 0.0;
    }
    h->prof.resolve();
    check_status(h, "setup");
    return h;
  } catch (...) {
    if (h) gamblet_destroy(h);
    throw;
  }
}


// Independent problems packed into one hierarchy.  Problem p (q_p levels,
// cells in its own 2^q_p lattice) is given the aligned subtree that starts
// at Morton index base_p of a 2^Q lattice, largest problems first, so the
// subtrees are disjoint and their union is a Morton prefix; the fine
// operator is block diagonal and unknowns are numbered problem by problem.
gamblet_ctx* setup_batched_impl(int32_t nprob, const gamblet_csr* A, const int32_t* q,
                                const int32_t* const* cells, const gamblet_opts* opts,
                                int32_t* offsets) {
  if (nprob < 1 || !A || !q || !cells) fail(GAMBLET_ERR_INVALID_ARG, "nprob >= 1 and non-NULL A, q, cells required");
  int qmax = 0;
  for (int p = 0; p < nprob; ++p) {
    if (q[p] < 1 || q[p] > 15) fail(GAMBLET_ERR_INVALID_ARG, "q[p] must be in [1, 15]");
    if (!cells[p] || A[p].n < 1 || A[p].nnz < 1 || !A[p].rowptr || !A[p].colind || !A[p].val)
      fail(GAMBLET_ERR_INVALID_ARG, "empty or incomplete CSR of problem " + std::to_string(p));
    if ((int64_t)A[p].n > ((int64_t)1 << (2 * q[p])))
      fail(GAMBLET_ERR_INVALID_ARG, "more unknowns than level-q cells in problem " + std::to_string(p));
    qmax = std::max(qmax, (int)q[p]);
  }
  std::vector<int> order(nprob);
  for (int p = 0; p < nprob; ++p) order[p] = p;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return q[a] > q[b]; });
  std::vector<int64_t> base(nprob);
  int64_t total = 0;
  for (int p : order) {
    base[p] = total;  // a multiple of 4^q_p: every earlier subtree is at least as large
    total += (int64_t)1 << (2 * q[p]);
  }
  int Q = std::max(qmax, 2);
  while (((int64_t)1 << (2 * Q)) < total) ++Q;
  if (Q > 15) fail(GAMBLET_ERR_UNSUPPORTED, "the problems do not fit a 2^15 x 2^15 lattice");
  std::vector<BatchSeg> seg(nprob);
  int64_t N = 0, NNZ = 0;
  for (int p = 0; p < nprob; ++p) {
    int x0, y0;
    demorton((uint32_t)base[p], x0, y0);
    seg[p] = BatchSeg{N, NNZ, A[p].n, q[p], x0, y0};
    N += A[p].n;
    NNZ += A[p].nnz;
  }
  if (N >= ((int64_t)1 << 31) || NNZ >= ((int64_t)1 << 31))
    fail(GAMBLET_ERR_UNSUPPORTED, "combined CSR exceeds int32 indexing");
  gamblet_opts o;
  if (opts) o = *opts;
  else gamblet_default_opts(&o);
  cudaStream_t s = (cudaStream_t)o.stream;
  Pool tmp;
  tmp.s = s;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  int32_t* R = tmp.alloc<int32_t>(N + 1);
  int32_t* C = tmp.alloc<int32_t>(NNZ);
  double* V = tmp.alloc<double>(NNZ);
  int32_t* X = tmp.alloc<int32_t>(2 * N);
  std::vector<int32_t> ends(2 * (size_t)nprob);
  for (int p = 0; p < nprob; ++p) {
    const BatchSeg& b = seg[p];
    CK(cudaMemcpyAsync(R + b.row0, A[p].rowptr, sizeof(int32_t) * b.n, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(&ends[2 * p], A[p].rowptr, sizeof(int32_t), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(&ends[2 * p + 1], A[p].rowptr + b.n, sizeof(int32_t), cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(C + b.nnz0, A[p].colind, sizeof(int32_t) * A[p].nnz, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(V + b.nnz0, A[p].val, sizeof(double) * A[p].nnz, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(X + 2 * b.row0, cells[p], sizeof(int32_t) * 2 * b.n, cudaMemcpyDefault, s));
  }
  const int32_t nnz_total = (int32_t)NNZ;
  CK(cudaMemcpyAsync(R + N, &nnz_total, sizeof(int32_t), cudaMemcpyHostToDevice, s));
  BatchSeg* seg_d = tmp.upload(seg, s);
  int* flag = tmp.zeros<int>(1, s);
  launch_batch_fixup(nprob, seg_d, N, NNZ, R, C, X, flag, s);
  CK(cudaGetLastError());
  int flag_h = 0;
  CK(cudaMemcpyAsync(&flag_h, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int p = 0; p < nprob; ++p)
    if (ends[2 * p] != 0 || (int64_t)ends[2 * p + 1] != A[p].nnz)
      fail(GAMBLET_ERR_INVALID_ARG, "problem " + std::to_string(p) +
                                        ": rowptr[0] must be 0 and rowptr[n] must equal nnz");
  if (flag_h == 1) fail(GAMBLET_ERR_INVALID_ARG, "a column index lies outside its problem");
  if (flag_h == 2) fail(GAMBLET_ERR_INVALID_ARG, "a cell lies outside its problem's 2^q lattice");
  const gamblet_csr Ac{(int32_t)N, NNZ, R, C, V};
  gamblet_ctx* h = setup_impl(&Ac, Q, X, &o);
  CK(cudaEventRecord(e1, s));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->setup_ms = ms;  // packing included
  h->nprob = nprob;
  if (offsets) {
    for (int p = 0; p < nprob; ++p) offsets[p] = (int32_t)seg[p].row0;
    offsets[nprob] = (int32_t)N;
  }
  return h;
}

// ------------------------------------------------------------ several right-hand sides
// Buffers of one group of nb <= kMaxRhs right-hand sides: per level the
// transformed right-hand sides, level solutions, CG vectors and prolongated
// vectors, each [nb][ncell_k]; the CG level table and scalars of the group.
template <typename T>
struct RhsGroup {
  int nb = 0;
  std::vector<T*> ghat, w, v, cr, cz, cp, cAp;  // index k
  T* g1 = nullptr;
  T* U1 = nullptr;
  CgLevel* lv = nullptr;
  CgScalars* sc = nullptr;
  int* any = nullptr;
};

template <typename T>
RhsGroup<T> make_group(gamblet_ctx* h, Pool& P, int nb) {
  cudaStream_t s = h->s;
  const int q = h->q;
  RhsGroup<T> G;
  G.nb = nb;
  G.ghat.assign(q + 1, nullptr);
  G.w = G.v = G.cr = G.cz = G.cp = G.cAp = G.ghat;
  for (int k = 2; k <= q; ++k) {
    const int64_t n = h->lv[k].ncell * nb;
    G.ghat[k] = P.zeros<T>(n, s);
    G.w[k] = P.zeros<T>(n, s);
    G.v[k] = P.zeros<T>(n, s);
    G.cr[k] = P.zeros<T>(n, s);
    G.cz[k] = P.zeros<T>(n, s);
    G.cp[k] = P.zeros<T>(n, s);
    G.cAp[k] = P.zeros<T>(n, s);
  }
  G.g1 = P.zeros<T>(4 * nb, s);
  G.U1 = P.zeros<T>(4 * nb, s);
  std::vector<CgLevel> cl(h->cg_nlev);
  CK(cudaMemcpyAsync(cl.data(), h->cg_lv, sizeof(CgLevel) * h->cg_nlev, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int l = 0; l < h->cg_nlev; ++l) {
    const int k = l + 2;
    cl[l].x = G.w[k];
    cl[l].r = G.cr[k];
    cl[l].z = G.cz[k];
    cl[l].p = G.cp[k];
    cl[l].Ap = G.cAp[k];
    cl[l].b = G.ghat[k];
    cl[l].rstride = h->lv[k].ncell;
  }
  G.lv = P.upload(cl, s);
  G.sc = P.zeros<CgScalars>(std::max(h->cg_nlev, 1) * nb, s);
  G.any = P.zeros<int>(1, s);
  return G;
}

// The gamblet operator on nb transformed level-q vectors (in, out: [nb][ncell_q]).
template <typename T>
void apply_G_many(gamblet_ctx* h, RhsGroup<T>& G, const T* in, T* out, int inverse_last) {
  cudaStream_t s = h->s;
  const int q = h->q;
  const int NB = h->N.size();
  const int nb = G.nb;
  const int64_t nq = h->lv[q].ncell;
  CK(cudaMemcpyAsync(G.ghat[q], in, sizeof(T) * nq * nb, cudaMemcpyDeviceToDevice, s));
  for (int k = q; k >= 2; --k) {
    LevelDev& L = h->lv[k];
    const bool lower = k - 1 >= 2;
    int tok = h->prof.begin("restrict", 0.0, 0.0, s);
    launch_restrict_m<T>((const T*)L.Rhat, NB, h->nbr, 1 << (k - 1), L.npar, G.ghat[k], L.ncell,
                         lower ? G.ghat[k - 1] : G.g1, lower ? h->lv[k - 1].ncell : 4,
                         lower ? h->lv[k - 1].pmask : nullptr, nb, s);
    h->prof.end(tok, s);
  }
  if (h->cg_nlev > 0) {
    const double tol2 = h->opts.level_tol * h->opts.level_tol;
    const int maxit = std::max(h->opts.level_max_iter, 1);
    CK(cudaMemsetAsync(G.sc, 0, sizeof(CgScalars) * h->cg_nlev * nb, s));
    launch_cgm_init<T>(G.lv, h->cg_nlev, h->cg_blocks, G.sc, nb, s);
    launch_cgm_start(G.sc, h->cg_nlev * nb, tol2, G.any, s);
    for (int it = 0; it < maxit; it += 8) {
      int tok = h->prof.begin("level_cg", 0.0, 0.0, s);
      for (int c = 0; c < 8; ++c)
        launch_cgm_iteration<T>(G.lv, h->cg_nlev, h->cg_spmv_blocks, h->cg_blocks, G.sc, nb,
                                h->cg_max_ts, tol2, maxit, G.any, s);
      h->prof.end(tok, s);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(h->any_active_h, G.any, sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (*h->any_active_h == 0) break;
    }
  }
  for (int r = 0; r < nb; ++r) launch_level1_solve<T>(h->A1L, G.g1 + 4 * r, G.U1 + 4 * r, s);
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    const T* vprev = k == 2 ? G.U1 : G.v[k - 1];
    const int64_t vstride = k == 2 ? 4 : h->lv[k - 1].ncell;
    T* dst = k == q ? out : G.v[k];
    int tok = h->prof.begin("prolong", 0.0, 0.0, s);
    launch_prolong_m<T>((const T*)L.RT, NB, h->nbr, 1 << (k - 1), L.npar, vprev, vstride, G.w[k],
                        L.ncell, L.pmask, k == q ? inverse_last : 1, dst, L.ncell, nb, s);
    h->prof.end(tok, s);
  }
  CK(cudaGetLastError());
}

// nb right-hand sides (rows of G_user) solved together: the one-pass
// transform preconditions a float64 flexible CG per right-hand side, all
// sharing each pass's matrix reads.
template <typename T>
void solve_group(gamblet_ctx* h, int nb, const double* G_user, double* U_user, double* worst_res,
                 int* max_outer, bool* not_conv) {
  cudaStream_t s = h->s;
  Pool tmp;
  tmp.s = s;
  const int q = h->q;
  LevelDev& Lq = h->lv[q];
  const int64_t nq = Lq.ncell, n = h->n;
  RhsGroup<T> Gp = make_group<T>(h, tmp, nb);
  double* g64 = tmp.zeros<double>(nq * nb, s);
  double* u64 = tmp.zeros<double>(nq * nb, s);
  double* r64 = tmp.zeros<double>(nq * nb, s);
  double* z64 = tmp.zeros<double>(nq * nb, s);
  double* p64 = tmp.zeros<double>(nq * nb, s);
  double* q64 = tmp.zeros<double>(nq * nb, s);
  T* rT = is_f32<T>() ? (T*)tmp.zeros<float>(nq * nb, s) : nullptr;
  T* zT = is_f32<T>() ? (T*)tmp.zeros<float>(nq * nb, s) : nullptr;
  double* d = tmp.zeros<double>(8 * nb, s);
  double* gin = nullptr;
  to_device(tmp, gin, G_user, n * nb, s);
  for (int r = 0; r < nb; ++r) {
    launch_gather_morton(gin + r * n, h->unknown_of, nq, g64 + r * nq, s);
    launch_transform_vec<double>(g64 + r * nq, g64 + r * nq, Lq.npar, Lq.pmask, +1, s);
    launch_dots(nq, g64 + r * nq, g64 + r * nq, nullptr, nullptr, nullptr, nullptr, d + 8 * r, s);
  }
  std::vector<double> dh(8 * nb);
  CK(cudaMemcpyAsync(dh.data(), d, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> gnorm(nb);
  for (int r = 0; r < nb; ++r) gnorm[r] = std::sqrt(dh[8 * r]);
  // z = G r for the whole group (float path through float copies)
  auto precondition = [&](double* src, double* dst) {
    if (is_f32<T>()) {
      launch_convert_f64_f32(src, (float*)rT, nq * nb, s);
      apply_G_many<T>(h, Gp, rT, zT, 0);
      launch_convert_f32_f64((const float*)zT, dst, nq * nb, s);
    } else {
      apply_G_many<T>(h, Gp, (const T*)src, (T*)dst, 0);
    }
  };
  precondition(g64, z64);
  CK(cudaMemcpyAsync(u64, z64, sizeof(double) * nq * nb, cudaMemcpyDeviceToDevice, s));
  const int maxit = h->opts.refine_max_iter;
  std::vector<double> rel(nb, 0.0);
  std::vector<int> active(nb, 0), outer(nb, 0);
  double one = 1.0;
  double* onep = tmp.upload(std::vector<double>(nb, 1.0), s);
  auto residual = [&]() {  // r = g - A u, rel = |r| / |g|
    for (int r = 0; r < nb; ++r) outer_spmv(h, u64 + r * nq, q64 + r * nq);
    CK(cudaMemcpyAsync(r64, g64, sizeof(double) * nq * nb, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(d, 0, sizeof(double) * 8 * nb, s));
    for (int r = 0; r < nb; ++r) {
      launch_axpy(nq, onep + r, onep + r, -1.0, q64 + r * nq, r64 + r * nq, s);
      launch_dots(nq, r64 + r * nq, r64 + r * nq, nullptr, nullptr, nullptr, nullptr, d + 8 * r, s);
    }
    CK(cudaMemcpyAsync(dh.data(), d, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int r = 0; r < nb; ++r) rel[r] = gnorm[r] > 0 ? std::sqrt(dh[8 * r]) / gnorm[r] : 0.0;
  };
  (void)one;
  if (maxit > 0) {
    residual();
    int nact = 0;
    for (int r = 0; r < nb; ++r) nact += active[r] = rel[r] > h->opts.refine_tol;
    if (nact) {
      precondition(r64, z64);
      CK(cudaMemcpyAsync(p64, z64, sizeof(double) * nq * nb, cudaMemcpyDeviceToDevice, s));
      for (int it = 1; it <= maxit && nact; ++it) {
        int tok = h->prof.begin("outer_spmv64", 0.0, 0.0, s);
        for (int r = 0; r < nb; ++r)
          if (active[r]) outer_spmv(h, p64 + r * nq, q64 + r * nq);
        h->prof.end(tok, s);
        CK(cudaMemsetAsync(d, 0, sizeof(double) * 8 * nb, s));
        for (int r = 0; r < nb; ++r) {
          if (!active[r]) continue;
          double* dr = d + 8 * r;
          const int64_t o = r * nq;
          launch_dots(nq, p64 + o, q64 + o, p64 + o, r64 + o, nullptr, nullptr, dr, s);
          launch_axpy(nq, dr + 1, dr + 0, +1.0, p64 + o, u64 + o, s);
          launch_axpy(nq, dr + 1, dr + 0, -1.0, q64 + o, r64 + o, s);
          launch_dots(nq, nullptr, nullptr, nullptr, nullptr, r64 + o, r64 + o, dr, s);
        }
        CK(cudaMemcpyAsync(dh.data(), d, sizeof(double) * 8 * nb, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        nact = 0;
        for (int r = 0; r < nb; ++r) {
          if (!active[r]) continue;
          outer[r] = it;
          rel[r] = gnorm[r] > 0 ? std::sqrt(dh[8 * r + 2]) / gnorm[r] : 0.0;
          if (!(rel[r] == rel[r])) fail(GAMBLET_ERR_NOT_SPD, "outer iteration produced NaN");
          if (rel[r] <= h->opts.refine_tol) active[r] = 0;
          nact += active[r];
        }
        if (!nact) break;
        precondition(r64, z64);
        for (int r = 0; r < nb; ++r) {
          if (!active[r]) continue;
          double* dr = d + 8 * r;
          const int64_t o = r * nq;
          launch_dots(nq, z64 + o, q64 + o, nullptr, nullptr, nullptr, nullptr, dr + 3, s);
          launch_xpby(nq, z64 + o, dr + 3, dr + 0, -1.0, p64 + o, s);
        }
        CK(cudaGetLastError());
      }
      for (int r = 0; r < nb; ++r)
        if (active[r]) *not_conv = true;
    }
    residual();
  }
  for (int r = 0; r < nb; ++r) {
    *worst_res = std::max(*worst_res, rel[r]);
    *max_outer = std::max(*max_outer, outer[r]);
  }
  // back to unknown order (nodal coefficients after a mass initialisation)
  const bool dev_out = is_device_ptr(U_user);
  double* uo = dev_out ? U_user : tmp.alloc<double>(n * nb);
  for (int r = 0; r < nb; ++r) {
    launch_transform_vec<double>(u64 + r * nq, q64 + r * nq, Lq.npar, Lq.pmask, -1, s);
    if (h->mass) {
      double* Ut = tmp.alloc<double>(n);
      launch_scatter_unknown(q64 + r * nq, h->morton_of, n, Ut, s);
      launch_mass_apply(n, h->NBq, h->nbrq, h->Minv, Ut, h->morton_of, h->unknown_of, 1 << q,
                        Lq.ncell, uo + r * n, s);
    } else {
      launch_scatter_unknown(q64 + r * nq, h->morton_of, n, uo + r * n, s);
    }
  }
  if (!dev_out)
    CK(cudaMemcpyAsync(U_user, uo, sizeof(double) * n * nb, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
}

template <typename T>
gamblet_status solve_many_impl(gamblet_ctx* h, int nrhs, const double* G, double* U,
                               gamblet_info* info) {
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, h->s));
  double worst = 0;
  int outer = 0;
  bool not_conv = false;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhs) {
    const int nb = std::min(kMaxRhs, nrhs - r0);
    solve_group<T>(h, nb, G + (int64_t)r0 * h->n, U + (int64_t)r0 * h->n, &worst, &outer,
                   &not_conv);
  }
  CK(cudaEventRecord(e1, h->s));
  CK(cudaEventSynchronize(e1));
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->prof.resolve();
  check_status(h, "solve");
  const gamblet_status st = not_conv ? GAMBLET_ERR_NOT_CONVERGED : GAMBLET_OK;
  if (info) {
    info->status = st;
    info->q = h->q;
    info->outer_iters = outer;
    info->rel_residual = worst;
    info->setup_ms = h->setup_ms;
    info->solve_ms = ms;
    info->patch_iters_max = h->patch_iters_max;
    info->patch_iters_mean = h->patch_iters_mean;
  }
  return st;
}

// Level-q initialisation by the mass matrix (Algorithm 2, lines 2a-5 with
// Definition deflocinvm): M^-1,loc on patches of radius rho_q around every
// node, A^(q),loc = (M^-1,loc)^T A M^-1,loc as a CSR, then the ordinary
// setup on it.  The handle keeps M^-1,loc for the solve's output map.
gamblet_ctx* setup_mass_impl(const gamblet_csr* A, const gamblet_csr* M, int32_t q,
                             const int32_t* cells, double rho_q, const gamblet_opts* opts) {
  if (!A || !M || !cells) fail(GAMBLET_ERR_INVALID_ARG, "A, M and cells must be non-NULL");
  if (A->n < 1 || M->n != A->n || M->nnz < 1 || !M->rowptr || !M->colind || !M->val ||
      A->nnz < 1 || !A->rowptr || !A->colind || !A->val)
    fail(GAMBLET_ERR_INVALID_ARG, "A and M must be complete CSRs of the same size");
  if (q < 2 || q > 15) fail(GAMBLET_ERR_INVALID_ARG, "q must be in [2, 15]");
  if (!(rho_q > 0)) fail(GAMBLET_ERR_INVALID_ARG, "rho_q must be positive");
  if ((int64_t)A->n > ((int64_t)1 << (2 * q)))
    fail(GAMBLET_ERR_INVALID_ARG, "more unknowns than level-q cells");
  gamblet_opts o;
  if (opts) o = *opts;
  else gamblet_default_opts(&o);
  if (o.nbr_rule != 0 && o.nbr_rule != 1) fail(GAMBLET_ERR_INVALID_ARG, "nbr_rule must be 0 or 1");
  cudaStream_t s = (cudaStream_t)o.stream;
  const int n = A->n;
  Pool tmp;
  tmp.s = s;
  int dev = 0, num_sms = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // cells -> Morton codes and the cell -> node map of the level-q lattice
  const int32_t* cells_d = as_device(tmp, cells, 2 * (int64_t)n, s);
  int32_t* morton_of = tmp.alloc<int32_t>(n);
  int* flag = tmp.zeros<int>(4, s);
  launch_cells_to_morton(cells_d, n, q, morton_of, flag, s);
  int flag_h[4];
  CK(cudaMemcpyAsync(flag_h, flag, sizeof(flag_h), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (flag_h[0] == 2) fail(GAMBLET_ERR_INVALID_ARG, "a cell lies outside [0, 2^q)");
  const int64_t ncell = 4 * (((int64_t)flag_h[1] + 1 + 3) / 4);
  int32_t* unknown_of = tmp.alloc<int32_t>(ncell);
  CK(cudaMemsetAsync(unknown_of, 0xff, sizeof(int32_t) * ncell, s));
  uint32_t* pm = tmp.zeros<uint32_t>(ncell / 4, s);
  CK(cudaMemsetAsync(flag, 0, sizeof(int), s));
  launch_scatter_cells(morton_of, n, unknown_of, pm, flag, s);
  // per-node stencils of A and M
  auto stencil = [&](const gamblet_csr* X, int& rx, int& ry) {
    const int32_t* rp = as_device(tmp, X->rowptr, (int64_t)n + 1, s);
    const int32_t* ci = as_device(tmp, X->colind, X->nnz, s);
    const double* va = as_device(tmp, X->val, X->nnz, s);
    int* ext = tmp.zeros<int>(4, s);
    launch_csr_node_extent(n, rp, ci, morton_of, ext, ext + 2, s);
    int ext_h[4];
    CK(cudaMemcpyAsync(ext_h, ext, sizeof(ext_h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ext_h[2]) fail(GAMBLET_ERR_INVALID_ARG, "CSR column index out of range or rowptr decreasing");
    rx = ext_h[0];
    ry = ext_h[1];
    if ((2 * rx + 1) * (2 * ry + 1) > 121)
      fail(GAMBLET_ERR_UNSUPPORTED, "mass initialisation needs a compact fine stencil (|offset| <= 5)");
    double* st = tmp.zeros<double>((int64_t)n * (2 * rx + 1) * (2 * ry + 1), s);
    launch_csr_to_stencil(n, rp, ci, va, morton_of, rx, ry, st, s);
    return st;
  };
  int arx, ary, mrx, mry;
  double* Ast = stencil(A, arx, ary);
  double* Mst = stencil(M, mrx, mry);
  // patch offsets N_q (the same closed-square rule at the fine level)
  const OffSet Nq = neighbour_offsets(rho_q, o.nbr_rule);
  const int NBq = Nq.size(), jcq = Nq.find(0, 0);
  if (mass_patch_smem_bytes(NBq) > 227 * 1024)
    fail(GAMBLET_ERR_UNSUPPORTED, "mass patch exceeds shared memory; lower rho_q");
  int2* nbrq_t = tmp.upload(Nq.v, s);
  double* Minv = tmp.alloc<double>((int64_t)n * NBq);
  int* status = tmp.zeros<int>(1, s);
  launch_mass_patch_inverse(n, NBq, jcq, nbrq_t, Mst, mrx, mry, morton_of, unknown_of, 1 << q,
                            ncell, Minv, status, num_sms, s);
  // symbolic lists of (M^-1,loc)^T A M^-1,loc
  OffSet Aoff, W, D;
  for (int dy = -ary; dy <= ary; ++dy)
    for (int dx = -arx; dx <= arx; ++dx) Aoff.add(dx, dy);
  for (const int2& nj : Nq.v)
    for (const int2& a : Aoff.v) W.add(nj.x - a.x, nj.y - a.y);
  std::vector<int> l1_ptr(W.size() + 1, 0), l2_ptr;
  std::vector<int2> l1, l2;
  for (int w = 0; w < W.size(); ++w) {
    for (int a = 0; a < Aoff.size(); ++a) {
      const int j = Nq.find(W.v[w].x + Aoff.v[a].x, W.v[w].y + Aoff.v[a].y);
      if (j >= 0) l1.push_back(make_int2(a, j));
    }
    l1_ptr[w + 1] = (int)l1.size();
  }
  for (const int2& w : W.v)
    for (const int2& nj : Nq.v) D.add(w.x - nj.x, w.y - nj.y);
  l2_ptr.assign(D.size() + 1, 0);
  for (int d = 0; d < D.size(); ++d) {
    for (int j = 0; j < NBq; ++j) {
      const int w = W.find(D.v[d].x + Nq.v[j].x, D.v[d].y + Nq.v[j].y);
      if (w >= 0) l2.push_back(make_int2(j, w));
    }
    l2_ptr[d + 1] = (int)l2.size();
  }
  std::vector<int> mirror(D.size());
  for (int d = 0; d < D.size(); ++d) mirror[d] = D.find(-D.v[d].x, -D.v[d].y);
  MassTripleGeom tg{NBq, Aoff.size(), W.size(), tmp.upload(W.v, s), tmp.upload(l1_ptr, s),
                    tmp.upload(l1, s), D.size(), tmp.upload(D.v, s), tmp.upload(l2_ptr, s),
                    tmp.upload(l2, s)};
  double* X = tmp.alloc<double>((int64_t)n * D.size());
  launch_mass_triple(n, tg, Ast, Minv, morton_of, unknown_of, 1 << q, ncell, X, s);
  // CSR of A^(q),loc (symmetrised)
  int2* Doff = tmp.upload(D.v, s);
  int32_t* cnt = tmp.alloc<int32_t>(n);
  launch_stencil_counts(n, Doff, D.size(), morton_of, unknown_of, 1 << q, ncell, cnt, s);
  std::vector<int32_t> rowptr_h((size_t)n + 1, 0);
  CK(cudaMemcpyAsync(rowptr_h.data() + 1, cnt, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
  int status_h = 0;
  CK(cudaMemcpyAsync(&status_h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  if (status_h == DEV_NOT_SPD) fail(GAMBLET_ERR_NOT_SPD, "non-positive pivot in a mass patch");
  for (int i = 0; i < n; ++i) {
    if ((int64_t)rowptr_h[i] + rowptr_h[i + 1] >= ((int64_t)1 << 31))
      fail(GAMBLET_ERR_UNSUPPORTED, "initialised operator exceeds int32 CSR indexing");
    rowptr_h[i + 1] += rowptr_h[i];
  }
  const int64_t nnz = rowptr_h[n];
  int32_t* rp = tmp.upload(rowptr_h, s);
  int32_t* ci = tmp.alloc<int32_t>(nnz);
  double* va = tmp.alloc<double>(nnz);
  launch_stencil_to_csr(n, Doff, tmp.upload(mirror, s), D.size(), X, morton_of, unknown_of,
                        1 << q, ncell, rp, ci, va, s);
  CK(cudaGetLastError());
  const gamblet_csr Aq{n, nnz, rp, ci, va};
  gamblet_ctx* h = setup_impl(&Aq, q, cells_d, &o);
  try {
    h->mass = true;
    h->NBq = NBq;
    h->nbrq = h->pool.upload(Nq.v, s);
    h->Minv = h->pool.alloc<double>((int64_t)n * NBq);
    CK(cudaMemcpyAsync(h->Minv, Minv, sizeof(double) * n * NBq, cudaMemcpyDeviceToDevice, s));
    CK(cudaEventRecord(e1, s));
    CK(cudaEventSynchronize(e1));
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    h->setup_ms = ms;  // the mass initialisation included
  } catch (...) {
    gamblet_destroy(h);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return h;
}

// Compression in the normalised basis psi^(1)/||psi^(1)||_a, chi^(k)/||chi^(k)||_a
// (Sec. 5.1): one-pass transform of g, threshold eps * max |c|, rebuild.
template <typename T>
void compress_impl(gamblet_ctx* h, const double* g_user, double eps, double* u_user,
                   int64_t* kept_out, int64_t* total_out) {
  cudaStream_t s = h->s;
  Pool tmp;
  tmp.s = s;
  const int q = h->q;
  LevelDev& Lq = h->lv[q];
  const int64_t nq = Lq.ncell;
  double* g_dev = nullptr;
  to_device(tmp, g_dev, g_user, h->n, s);
  launch_gather_morton(g_dev, h->unknown_of, nq, h->g64, s);
  launch_transform_vec<double>(h->g64, h->g64, Lq.npar, Lq.pmask, +1, s);
  T* gT = as_T<T>(h, h->g64, h->rT, nq, true);
  apply_G_down<T>(h, gT);
  // level 1: c_i = U_i sqrt(A^(1)_ii), A^(1)_ii from the Cholesky factor
  T U1[4];
  double L1[16];
  CK(cudaMemcpyAsync(U1, h->U1, sizeof(T) * 4, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(L1, h->A1L, sizeof(double) * 16, cudaMemcpyDeviceToHost, s));
  unsigned long long* dv = tmp.zeros<unsigned long long>(2, s);  // max bits, kept
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    launch_coef_max<T>((const T*)L.w, (const T*)L.Bd, L.o0, L.npar, L.pmask, dv, s);
  }
  unsigned long long dh[2];
  CK(cudaMemcpyAsync(dh, dv, sizeof(dh), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  const uint32_t m1 = h->lv[1].pmask_h[0] & 15u;
  double c1[4], cmax = 0;
  std::memcpy(&cmax, &dh[0], sizeof(double));
  int64_t total = 0;
  for (int i = 0; i < 4; ++i) {
    double a = 0;
    for (int j = 0; j <= i; ++j) a += L1[i * 4 + j] * L1[i * 4 + j];
    c1[i] = ((m1 >> i) & 1u) ? std::fabs((double)U1[i]) * std::sqrt(a) : 0.0;
    if ((m1 >> i) & 1u) ++total;
    cmax = std::max(cmax, c1[i]);
  }
  for (int k = 2; k <= q; ++k) total += h->lv[k].nJ;
  const double thr = eps * cmax;
  int64_t kept = 0;
  for (int i = 0; i < 4; ++i) {
    if (!((m1 >> i) & 1u)) continue;
    if (c1[i] >= thr) ++kept;
    else U1[i] = T(0);
  }
  CK(cudaMemcpyAsync(h->U1, U1, sizeof(T) * 4, cudaMemcpyHostToDevice, s));
  for (int k = 2; k <= q; ++k) {
    LevelDev& L = h->lv[k];
    launch_coef_threshold<T>((T*)L.w, (const T*)L.Bd, L.o0, L.npar, L.pmask, thr, dv + 1, s);
  }
  T* zT = as_T<T>(h, h->z64, h->zT, nq, false);
  apply_G_up<T>(h, zT, 1);
  if (is_f32<T>()) launch_convert_f32_f64((const float*)zT, h->q64, nq, s);
  else CK(cudaMemcpyAsync(h->q64, zT, sizeof(double) * nq, cudaMemcpyDeviceToDevice, s));
  double* u_out = is_device_ptr(u_user) ? u_user : tmp.alloc<double>(h->n);
  if (h->mass) {
    double* U = tmp.alloc<double>(h->n);
    launch_scatter_unknown(h->q64, h->morton_of, h->n, U, s);
    launch_mass_apply(h->n, h->NBq, h->nbrq, h->Minv, U, h->morton_of, h->unknown_of, 1 << q,
                      Lq.ncell, u_out, s);
  } else {
    launch_scatter_unknown(h->q64, h->morton_of, h->n, u_out, s);
  }
  if (u_out != u_user)
    CK(cudaMemcpyAsync(u_user, u_out, sizeof(double) * h->n, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(dh, dv, sizeof(dh), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  kept += (int64_t)dh[1];
  if (kept_out) *kept_out = kept;
  if (total_out) *total_out = total;
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with
// diagonal d and off-diagonal e (e[i] couples i and i + 1): the negative
// pivots of the LDL^T factorisation of T - x I (Sylvester's law of inertia).
int tridiag_count_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int c = 0;
  double piv = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double off = i > 0 ? e[i - 1] * e[i - 1] : 0.0;
    piv = (d[i] - x) - (i > 0 ? off / piv : 0.0);
    if (piv == 0.0) piv = -1e-300;  // x hits a pivot exactly: treat it as just below
    if (piv < 0) ++c;
  }
  return c;
}

// Extreme eigenvalues of B^(k) by the Lanczos process (steps iterations from
// a fixed pseudo-random start on the detail slots), then bisection on the
// Sturm counts of the Lanczos tridiagonal matrix.
template <typename T>
void level_condition_impl(gamblet_ctx* h, int k, int construction, int steps, double* lmin,
                          double* lmax) {
  cudaStream_t s = h->s;
  LevelDev& L = h->lv[k];
  Pool tmp;
  tmp.s = s;
  const int64_t n = L.ncell;
  double* v = tmp.zeros<double>(n, s);
  double* vp = tmp.zeros<double>(n, s);
  double* w = tmp.zeros<double>(n, s);
  double* d = tmp.zeros<double>(8, s);
  double* t1 = construction == 1 ? tmp.zeros<double>(n, s) : nullptr;
  const int Lpar = 1 << (k - 1);
  // the operator: B^(k) in the stored basis, or M B^(k) M^T for const1
  auto apply = [&](const double* x, double* y) {
    if (construction == 1) {
      launch_detail_basis(L.npar, L.pmask, x, t1, 1, s);
      launch_detail_spmv<T>((const T*)L.Bd, L.off, L.noff, Lpar, L.npar, t1, y, s);
      launch_detail_basis(L.npar, L.pmask, y, y, 0, s);
    } else {
      launch_detail_spmv<T>((const T*)L.Bd, L.off, L.noff, Lpar, L.npar, x, y, s);
    }
  };
  auto dot = [&](const double* a, const double* b) {
    CK(cudaMemsetAsync(d, 0, sizeof(double) * 8, s));
    launch_dots(n, a, b, nullptr, nullptr, nullptr, nullptr, d, s);
    double r = 0;
    CK(cudaMemcpyAsync(&r, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return r;
  };
  launch_detail_start(L.npar, L.pmask, v, s);
  const double nv0 = std::sqrt(dot(v, v));
  if (!(nv0 > 0)) fail(GAMBLET_ERR_INVALID_ARG, "level has no detail unknowns");
  launch_lanczos_step(n, 1.0 / nv0, v, nullptr, 0.0, nullptr, 0.0, v, s);  // normalise
  std::vector<double> al, be;
  double beta = 0;
  const int m = std::max(1, std::min<int>(steps, L.nJ));
  for (int j = 0; j < m; ++j) {
    apply(v, w);
    const double alpha = dot(w, v);
    // w <- w - alpha v - beta v_prev
    launch_lanczos_step(n, 1.0, w, v, -alpha, vp, -beta, w, s);
    al.push_back(alpha);
    const double b = std::sqrt(dot(w, w));
    if (j + 1 == m || !(b > 1e-12 * std::fabs(alpha))) break;
    be.push_back(b);
    // v_prev <- v, v <- w / b
    CK(cudaMemcpyAsync(vp, v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    launch_lanczos_step(n, 1.0 / b, w, nullptr, 0.0, nullptr, 0.0, v, s);
    beta = b;
  }
  CK(cudaGetLastError());
  // Gershgorin interval, then bisection for the smallest and largest
  double lo = 1e300, hi = -1e300;
  for (size_t i = 0; i < al.size(); ++i) {
    const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i < be.size() ? std::fabs(be[i]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  const int mm = (int)al.size();
  auto bisect = [&](int target) {  // smallest x with count_below(x) >= target
    double a = lo, b = hi;
    for (int it = 0; it < 200; ++it) {
      const double c = 0.5 * (a + b);
      if (tridiag_count_below(al, be, c) >= target) b = c;
      else a = c;
    }
    return 0.5 * (a + b);
  };
  *lmin = bisect(1);
  *lmax = bisect(mm);
}

}  // namespace

// ================================================================= C ABI
extern "C" {

void gamblet_default_opts(gamblet_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->rho = 3.0;
  o->nbr_rule = 0;
  o->precision = GAMBLET_FP64;
  o->level_tol = 1e-8;
  o->level_max_iter = 1000;
  o->refine_tol = 1e-13;
  o->refine_max_iter = 50;
  o->patch_tol = 0.0;
  o->use_graph = 1;
  o->profile = 0;
  o->autotune = 1;
  o->galerkin_variant = -1;
  o->patch_gather = -1;
  o->stream = nullptr;
}

gamblet_status gamblet_setup(const gamblet_csr* A, int32_t q, const int32_t* cells,
                             const gamblet_opts* opts, gamblet_handle* out) {
  if (!out) {
    g_last_error = "out is NULL";
    return GAMBLET_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    *out = setup_impl(A, q, cells, opts);
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return GAMBLET_ERR_INVALID_ARG;
  }
}

gamblet_status gamblet_setup_mass(const gamblet_csr* A, const gamblet_csr* M, int32_t q,
                                  const int32_t* cells, double rho_q, const gamblet_opts* opts,
                                  gamblet_handle* out) {
  if (!out) {
    g_last_error = "out is NULL";
    return GAMBLET_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    *out = setup_mass_impl(A, M, q, cells, rho_q, opts);
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return GAMBLET_ERR_INVALID_ARG;
  }
}

gamblet_status gamblet_setup_batched(int32_t nprob, const gamblet_csr* A, const int32_t* q,
                                     const int32_t* const* cells, const gamblet_opts* opts,
                                     gamblet_handle* out, int32_t* offsets) {
  if (!out) {
    g_last_error = "out is NULL";
    return GAMBLET_ERR_INVALID_ARG;
  }
  *out = nullptr;
  try {
    *out = setup_batched_impl(nprob, A, q, cells, opts, offsets);
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return GAMBLET_ERR_INVALID_ARG;
  }
}

gamblet_status gamblet_solve_many(gamblet_handle h, int32_t nrhs, const double* G, double* U,
                                  gamblet_info* info) {
  try {
    if (!h || !G || !U || nrhs < 1)
      fail(GAMBLET_ERR_INVALID_ARG, "handle, G and U must be non-NULL and nrhs >= 1");
    if (h->exact) fail(GAMBLET_ERR_UNSUPPORTED, "several right-hand sides use the localized transform");
    if (h->mixed) return solve_many_impl<float>(h, nrhs, G, U, info);
    return solve_many_impl<double>(h, nrhs, G, U, info);
  } catch (const GbError& e) {
    if (info) info->status = e.st;
    return set_error(e);
  }
}

gamblet_status gamblet_solve_truncated(gamblet_handle h, int32_t k, const double* g, double* u,
                                       gamblet_info* info) {
  try {
    if (!h || !g || !u) fail(GAMBLET_ERR_INVALID_ARG, "handle, g and u must be non-NULL");
    if (k < 1 || k > h->q) fail(GAMBLET_ERR_INVALID_ARG, "k must be in [1, q]");
    struct Restore {  // one-pass, truncated; the handle's options are put back
      gamblet_ctx* h;
      int maxit;
      ~Restore() {
        h->kmax = h->q;
        h->opts.refine_max_iter = maxit;
      }
    } restore{h, h->opts.refine_max_iter};
    h->kmax = k;
    h->opts.refine_max_iter = 0;
    if (h->mixed) return solve_impl<float>(h, g, u, nullptr, info);
    return solve_impl<double>(h, g, u, nullptr, info);
  } catch (const GbError& e) {
    if (info) info->status = e.st;
    return set_error(e);
  }
}

gamblet_status gamblet_level_condition(gamblet_handle h, int32_t k, int32_t construction,
                                       int32_t steps, double* lmin, double* lmax) {
  try {
    if (!h || !lmin || !lmax || k < 2 || k > h->q || steps < 1)
      fail(GAMBLET_ERR_INVALID_ARG, "bad handle, level, steps or output");
    if (construction != 1 && construction != 2)
      fail(GAMBLET_ERR_INVALID_ARG, "construction must be 1 or 2");
    if (h->exact) fail(GAMBLET_ERR_UNSUPPORTED, "diagnostics run on the localized transform");
    if (h->mixed) level_condition_impl<float>(h, k, construction, steps, lmin, lmax);
    else level_condition_impl<double>(h, k, construction, steps, lmin, lmax);
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  }
}

gamblet_status gamblet_compress(gamblet_handle h, const double* g, double eps, double* u,
                                int64_t* kept, int64_t* total) {
  try {
    if (!h || !g || !u) fail(GAMBLET_ERR_INVALID_ARG, "handle, g and u must be non-NULL");
    if (!(eps >= 0)) fail(GAMBLET_ERR_INVALID_ARG, "eps must be >= 0");
    if (h->exact) fail(GAMBLET_ERR_UNSUPPORTED, "compression runs on the localized transform");
    if (h->mixed) compress_impl<float>(h, g, eps, u, kept, total);
    else compress_impl<double>(h, g, eps, u, kept, total);
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  }
}

gamblet_status gamblet_solve(gamblet_handle h, const double* g, double* u, double* components,
                             gamblet_info* info) {
  try {
    if (!h || !g || !u) fail(GAMBLET_ERR_INVALID_ARG, "handle, g and u must be non-NULL");
    if (h->mixed) return solve_impl<float>(h, g, u, components, info);
    return solve_impl<double>(h, g, u, components, info);
  } catch (const GbError& e) {
    if (info) info->status = e.st;
    return set_error(e);
  }
}

gamblet_status gamblet_grad(gamblet_handle h, int32_t ncell, const int32_t* cell_nodes,
                            const double* cell_a, const double* K_ref, const double* u,
                            const double* u_obs, double* dJ, double* J, gamblet_info* info) {
  try {
    if (!h || !cell_nodes || !cell_a || !K_ref || !u || !u_obs || !dJ)
      fail(GAMBLET_ERR_INVALID_ARG, "NULL argument");
    if (ncell < 1) fail(GAMBLET_ERR_INVALID_ARG, "ncell must be positive");
    if (h->mass)
      fail(GAMBLET_ERR_UNSUPPORTED, "the adjoint covers the phi initialisation (A^(q) = A) only");
    cudaStream_t s = h->s;
    Pool tmp;
  tmp.s = h->s;
    const int n = h->n;
    double* ud = nullptr;
    double* uo = nullptr;
    to_device(tmp, ud, u, n, s);
    to_device(tmp, uo, u_obs, n, s);
    // residual u - u_obs and J
    double* res = tmp.alloc<double>(n);
    CK(cudaMemcpyAsync(res, ud, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double* d = tmp.zeros<double>(2, s);
    double one = 1.0;
    CK(cudaMemcpyAsync(d + 1, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    launch_axpy(n, d + 1, d + 1, -1.0, uo, res, s);
    launch_dots(n, res, res, nullptr, nullptr, nullptr, nullptr, d, s);
    double jh = 0;
    CK(cudaMemcpyAsync(&jh, d, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (J) *J = 0.5 * jh;
    // adjoint solve A lam = u - u_obs through the same hierarchy
    double* lam = tmp.alloc<double>(n);
    gamblet_status st = gamblet_solve(h, res, lam, nullptr, info);
    if (st != GAMBLET_OK && st != GAMBLET_ERR_NOT_CONVERGED) return st;
    int32_t* cn = nullptr;
    double* ca = nullptr;
    to_device(tmp, cn, cell_nodes, 4 * (int64_t)ncell, s);
    to_device(tmp, ca, cell_a, ncell, s);
    double kh[16];
    CK(cudaMemcpy(kh, K_ref, sizeof(kh), cudaMemcpyDefault));
    launch_set_kref(kh);
    double* out = nullptr;
    const bool dev_out = is_device_ptr(dJ);
    out = dev_out ? dJ : tmp.alloc<double>(ncell);
    launch_adjoint_contract(ncell, cn, ca, lam, ud, out, s);
    CK(cudaGetLastError());
    if (!dev_out)
      CK(cudaMemcpyAsync(dJ, out, sizeof(double) * ncell, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return st;
  } catch (const GbError& e) {
    if (info) info->status = e.st;
    return set_error(e);
  }
}

gamblet_status gamblet_grad_onepass(gamblet_handle h, int32_t ncell, const int32_t* cell_nodes,
                                    const double* cell_a, const double* K_ref, const double* g,
                                    const double* u_obs, double* u, double* dJ, double* dJ_dg,
                                    double* J, gamblet_info* info) {
  try {
    if (!h || !cell_nodes || !cell_a || !K_ref || !g || !u_obs || !dJ)
      fail(GAMBLET_ERR_INVALID_ARG, "NULL argument");
    if (ncell < 1) fail(GAMBLET_ERR_INVALID_ARG, "ncell must be positive");
    if (h->exact || h->mass || h->nprob != 1 || h->patch_tol < 0 || !h->plan)
      fail(GAMBLET_ERR_UNSUPPORTED,
           "the one-pass gradient needs a localized setup of one problem with A^(q) = A and "
           "iterative patch solves (patch_tol >= 0)");
    for (int k = 2; k <= h->q; ++k)
      if (k < (int)h->patch_cluster_k.size() && h->patch_cluster_k[k])
        fail(GAMBLET_ERR_UNSUPPORTED,
             "the one-pass gradient needs patches that fit one CTA's shared memory (its "
             "adjoint patch solves have no cluster form); lower rho");
    if (h->mixed)
      return grad_onepass_impl<float>(h, ncell, cell_nodes, cell_a, K_ref, g, u_obs, u, dJ, dJ_dg,
                                      J, info);
    return grad_onepass_impl<double>(h, ncell, cell_nodes, cell_a, K_ref, g, u_obs, u, dJ, dJ_dg,
                                     J, info);
  } catch (const GbError& e) {
    if (info) info->status = e.st;
    return set_error(e);
  }
}

gamblet_status gamblet_assemble_cells(int32_t n, const int32_t* rowptr, const int32_t* colind,
                                      int64_t nnz, int32_t ncell, const int32_t* cell_nodes,
                                      const double* log_a, const double* K_ref, double* val,
                                      double* cell_a, void* stream) {
  try {
    if (n < 1 || nnz < 1 || ncell < 1 || !rowptr || !colind || !cell_nodes || !log_a || !K_ref ||
        !val)
      fail(GAMBLET_ERR_INVALID_ARG, "bad sizes or NULL pointer");
    if (!is_device_ptr(rowptr) || !is_device_ptr(colind) || !is_device_ptr(cell_nodes) ||
        !is_device_ptr(log_a) || !is_device_ptr(val))
      fail(GAMBLET_ERR_INVALID_ARG, "pattern, cells, log_a and val must be device pointers");
    cudaStream_t s = (cudaStream_t)stream;
    double kh[16];
    CK(cudaMemcpy(kh, K_ref, sizeof(kh), cudaMemcpyDefault));
    launch_set_kref(kh);
    Pool tmp;
    tmp.s = s;
    int* missing = tmp.zeros<int>(1, s);
    CK(cudaMemsetAsync(val, 0, sizeof(double) * (size_t)nnz, s));
    if (cell_a && !is_device_ptr(cell_a)) fail(GAMBLET_ERR_INVALID_ARG, "cell_a must be device memory");
    launch_assemble_cells(n, rowptr, colind, ncell, cell_nodes, log_a, val, cell_a, missing, s);
    CK(cudaGetLastError());
    int mh = 0;
    CK(cudaMemcpyAsync(&mh, missing, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (mh) fail(GAMBLET_ERR_INVALID_ARG, "a cell's corner pair is missing from the CSR pattern");
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  }
}

gamblet_status gamblet_launch_shapes(gamblet_handle h, int32_t k, int32_t* shapes) {
  if (!h || !shapes || k < 2 || k > h->q || h->exact) {
    g_last_error = "bad handle, level or output (localized transform only)";
    return GAMBLET_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 4; ++i) shapes[i] = h->lv[k].shape[i];
  return GAMBLET_OK;
}

gamblet_status gamblet_level_size(gamblet_handle h, int32_t k, int32_t* n_k, int32_t* nJ_k) {
  if (!h || k < 1 || k > h->q) {
    g_last_error = "bad handle or level";
    return GAMBLET_ERR_INVALID_ARG;
  }
  if (n_k) *n_k = h->lv[k].n_active;
  if (nJ_k) *nJ_k = k >= 2 ? h->lv[k].nJ : 0;
  return GAMBLET_OK;
}

}  // extern "C"

// ----------------------------------------------------------------- getters
namespace {

// canonical index of every Morton cell at level k (-1 if empty)
std::vector<int32_t> canon_map(gamblet_ctx* h, int k) {
  const LevelDev& L = h->lv[k];
  std::vector<int32_t> cm(L.ncell, -1);
  if (k == h->q) {
    if ((int64_t)h->morton_of_h.size() != h->n) {  // fetched on first use
      h->morton_of_h.resize(h->n);
      CK(cudaMemcpyAsync(h->morton_of_h.data(), h->morton_of, sizeof(int32_t) * h->n,
                         cudaMemcpyDeviceToHost, h->s));
      CK(cudaStreamSynchronize(h->s));
    }
    for (int i = 0; i < h->n; ++i) cm[h->morton_of_h[i]] = i;
    return cm;
  }
  int idx = 0;
  for (int y = 0; y < L.L; ++y)
    for (int x = 0; x < L.L; ++x) {
      const uint32_t s = morton((uint32_t)x, (uint32_t)y);
      if ((int64_t)(s >> 2) >= L.npar) continue;  // beyond the stored prefix
      if ((L.pmask_h[s >> 2] >> (s & 3)) & 1u) cm[s] = idx++;
    }
  return cm;
}

// canonical index of each detail slot (4p + t) of level k, -1 otherwise.
std::vector<int32_t> canon_detail(gamblet_ctx* h, int k) {
  const LevelDev& L = h->lv[k];
  std::vector<int32_t> cm_par = canon_map(h, k - 1);
  std::vector<std::pair<int32_t, int32_t>> order;  // (canonical parent, p)
  for (int64_t p = 0; p < L.npar; ++p)
    if (cm_par[p] >= 0) order.push_back({cm_par[p], (int32_t)p});
  std::sort(order.begin(), order.end());
  std::vector<int32_t> cd(L.ncell, -1);
  int idx = 0;
  for (auto& pr : order) {
    const int m = __builtin_popcount(L.pmask_h[pr.second] & 15u);
    for (int t = 0; t < m - 1; ++t) cd[4 * (int64_t)pr.second + t] = idx++;
  }
  return cd;
}

template <typename T>
std::vector<double> download(const void* p, int64_t n, cudaStream_t s) {
  std::vector<T> tmp(n);
  if (n > 0) CK(cudaMemcpyAsync(tmp.data(), p, sizeof(T) * n, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return std::vector<double>(tmp.begin(), tmp.end());
}

struct Coo {
  std::vector<int32_t> r, c;
  std::vector<double> v;
  void add(int32_t i, int32_t j, double x) {
    r.push_back(i);
    c.push_back(j);
    v.push_back(x);
  }
};

// Ahat^(k) (transformed, in blocks) of either path as a callback over blocks.
void level_blocks(gamblet_ctx* h, int k,
                  const std::function<void(int64_t p, int64_t pp, const double* blk)>& f);

}  // namespace

namespace {
void level_blocks(gamblet_ctx* h, int k,
                  const std::function<void(int64_t, int64_t, const double*)>& f) {
  LevelDev& L = h->lv[k];
  cudaStream_t s = h->s;
  if (h->exact) {
    std::vector<double> D = download<double>(L.D, L.ncell * L.ncell, s);
    double blk[16];
    for (int64_t p = 0; p < L.npar; ++p)
      for (int64_t pp = 0; pp < L.npar; ++pp) {
        bool nz = false;
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            blk[a * 4 + b] = D[(4 * p + a) * L.ncell + 4 * pp + b];
            nz = nz || blk[a * 4 + b] != 0.0;
          }
        if (nz) f(p, pp, blk);
      }
    return;
  }
  const int64_t nv = (int64_t)L.noff * L.npar * 16;
  std::vector<double> V = h->mixed ? download<float>(L.Ahat, nv, s) : download<double>(L.Ahat, nv, s);
  const int Lpar = 1 << (k - 1);
  for (int o = 0; o < L.noff; ++o)
    for (int64_t p = 0; p < L.npar; ++p) {
      int x, y;
      demorton((uint32_t)p, x, y);
      const int pp = shift_cell(x, y, L.off_h[o].x, L.off_h[o].y, Lpar, L.npar);
      if (pp < 0) continue;
      f(p, pp, &V[((int64_t)o * L.npar + p) * 16]);
    }
}

Coo get_A(gamblet_ctx* h, int k) {
  Coo out;
  cudaStream_t s = h->s;
  if (k == 1) {
    std::vector<int32_t> cm = canon_map(h, 1);
    std::vector<double> M(16, 0.0);
    if (h->exact) {
      M = download<double>(h->A1, 16, s);
    } else {
      // the level-1 cell stencil has one column per existing level-1 cell
      const LevelDev& L1 = h->lv[1];
      const int64_t nr = h->lv[2].npar;
      std::vector<double> C = h->mixed ? download<float>(L1.Ahat, (int64_t)L1.noff * nr, s)
                                       : download<double>(L1.Ahat, (int64_t)L1.noff * nr, s);
      OffSet Sp;
      for (const int2& d : L1.off_h) Sp.add(d.x, d.y);
      for (int i = 0; i < nr; ++i)
        for (int j = 0; j < nr; ++j) {
          const int code = half_code(Sp, (j & 1) - (i & 1), (j >> 1) - (i >> 1));
          if (code >= 0) M[i * 4 + j] = C[(int64_t)code * nr + i];
          else if (code <= -2) M[i * 4 + j] = C[(int64_t)(-code - 2) * nr + j];
        }
    }
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (cm[i] >= 0 && cm[j] >= 0 && M[i * 4 + j] != 0.0) out.add(cm[i], cm[j], M[i * 4 + j]);
    return out;
  }
  std::vector<int32_t> cm = canon_map(h, k);
  const LevelDev& L = h->lv[k];
  level_blocks(h, k, [&](int64_t p, int64_t pp, const double* blk) {
    double Qr[16], Qc[16];
    qmat<double>((int)(L.pmask_h[p] & 15u), Qr);
    qmat<double>((int)(L.pmask_h[pp] & 15u), Qc);
    for (int c = 0; c < 4; ++c)
      for (int cc = 0; cc < 4; ++cc) {
        const int32_t i = cm[4 * p + c], j = cm[4 * pp + cc];
        if (i < 0 || j < 0) continue;
        double acc = 0;  // (Q^T blk Q)[c][cc]
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) acc += Qr[a * 4 + c] * blk[a * 4 + b] * Qc[b * 4 + cc];
        out.add(i, j, acc);
      }
  });
  return out;
}

Coo get_B(gamblet_ctx* h, int k) {
  Coo out;
  std::vector<int32_t> cd = canon_detail(h, k);
  level_blocks(h, k, [&](int64_t p, int64_t pp, const double* blk) {
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int32_t i = cd[4 * p + a], j = cd[4 * pp + b];
        if (i >= 0 && j >= 0) out.add(i, j, blk[a * 4 + b]);
      }
  });
  return out;
}

Coo get_R(gamblet_ctx* h, int k) {
  Coo out;
  cudaStream_t s = h->s;
  const LevelDev& L = h->lv[k];
  std::vector<int32_t> cmr = canon_map(h, k - 1), cmc = canon_map(h, k);
  if (h->exact) {
    std::vector<double> Rh = download<double>(L.Rh, L.npar * L.ncell, s);
    for (int64_t i = 0; i < L.npar; ++i) {
      if (cmr[i] < 0) continue;
      for (int64_t p = 0; p < L.npar; ++p) {
        double Q[16];
        qmat<double>((int)(L.pmask_h[p] & 15u), Q);
        for (int c = 0; c < 4; ++c) {
          if (cmc[4 * p + c] < 0) continue;
          double acc = 0;
          for (int a = 0; a < 4; ++a) acc += Rh[i * L.ncell + 4 * p + a] * Q[a * 4 + c];
          if (acc != 0.0) out.add(cmr[i], cmc[4 * p + c], acc);
        }
      }
    }
    return out;
  }
  const int NB = h->N.size();
  const int64_t nv = (int64_t)NB * 4 * L.npar;
  std::vector<double> R = h->mixed ? download<float>(L.Rhat, nv, s) : download<double>(L.Rhat, nv, s);
  const int Lpar = 1 << (k - 1);
  for (int64_t i = 0; i < L.npar; ++i) {
    if (cmr[i] < 0) continue;
    int x, y;
    demorton((uint32_t)i, x, y);
    for (int j = 0; j < NB; ++j) {
      const int p = shift_cell(x, y, h->N.v[j].x, h->N.v[j].y, Lpar, L.npar);
      if (p < 0) continue;
      double Q[16];
      qmat<double>((int)(L.pmask_h[p] & 15u), Q);
      for (int c = 0; c < 4; ++c) {
        if (cmc[4 * (int64_t)p + c] < 0) continue;
        double acc = 0;
        for (int a = 0; a < 4; ++a) acc += R[i * 4 * NB + 4 * j + a] * Q[a * 4 + c];
        if (acc != 0.0) out.add(cmr[i], cmc[4 * (int64_t)p + c], acc);
      }
    }
  }
  return out;
}

}  // namespace

extern "C" {

gamblet_status gamblet_get_operator(gamblet_handle h, int32_t which, int32_t k, int64_t capacity,
                                    int64_t* nnz, int32_t* rows, int32_t* cols, double* vals) {
  try {
    if (!h || !nnz) fail(GAMBLET_ERR_INVALID_ARG, "NULL handle or nnz");
    if (k < 1 || k > h->q || (which != 0 && k < 2) || which < 0 || which > 2)
      fail(GAMBLET_ERR_INVALID_ARG, "bad operator or level");
    Coo c = which == 0 ? get_A(h, k) : which == 1 ? get_R(h, k) : get_B(h, k);
    *nnz = (int64_t)c.v.size();
    if (capacity == 0) return GAMBLET_OK;
    if (capacity < *nnz || !rows || !cols || !vals)
      fail(GAMBLET_ERR_INVALID_ARG, "capacity too small or NULL output");
    std::memcpy(rows, c.r.data(), sizeof(int32_t) * c.r.size());
    std::memcpy(cols, c.c.data(), sizeof(int32_t) * c.c.size());
    std::memcpy(vals, c.v.data(), sizeof(double) * c.v.size());
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  }
}

int64_t gamblet_device_bytes(gamblet_handle h) { return h ? h->pool.bytes : 0; }

int32_t gamblet_kernel_stats(gamblet_handle h, gamblet_kernel_stat* out, int32_t capacity) {
  if (!h) return 0;
  const int32_t n = (int32_t)h->prof.stats.size();
  for (int32_t i = 0; i < n && i < capacity && out; ++i) {
    const Prof::Stat& st = h->prof.stats[i];
    std::memset(out[i].name, 0, sizeof(out[i].name));
    std::strncpy(out[i].name, st.name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = st.launches;
    out[i].ms = st.ms;
    out[i].bytes = st.bytes;
    out[i].flops = st.flops;
  }
  return n;
}

void gamblet_reset_kernel_stats(gamblet_handle h) {
  if (h) h->prof.stats.clear();
}

int64_t gamblet_kernel_launches(void) { return (int64_t)gb::g_launches.load(); }

void gamblet_destroy(gamblet_handle h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  else cudaDeviceSynchronize();
  h->pool.release();
  if (h->cg_exec) cudaGraphExecDestroy(h->cg_exec);
  if (h->any_active_h) cudaFreeHost(h->any_active_h);
  if (h->dots_h) cudaFreeHost(h->dots_h);
  if (h->status_h) cudaFreeHost(h->status_h);
  if (h->cg_lv_h) cudaFreeHost(h->cg_lv_h);
  delete h;
}

const char* gamblet_status_string(int32_t status) {
  switch (status) {
    case GAMBLET_OK: return "ok";
    case GAMBLET_ERR_INVALID_ARG: return "invalid argument";
    case GAMBLET_ERR_NOT_SPD: return "matrix not symmetric positive definite (non-positive pivot)";
    case GAMBLET_ERR_NOT_CONVERGED: return "iteration cap reached before the tolerance";
    case GAMBLET_ERR_CUDA: return "CUDA runtime error";
    case GAMBLET_ERR_OUT_OF_MEMORY: return "device out of memory";
    case GAMBLET_ERR_UNSUPPORTED: return "input outside this build's limits";
    default: return "unknown status";
  }
}

const char* gamblet_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

namespace gb {
// error text for the allocation-free entry point (noalloc.cu)
void noalloc_set_error(const char* msg) { g_last_error = msg; }
}  // namespace gb
