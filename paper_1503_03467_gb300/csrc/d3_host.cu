// d3_host.cu - setup, solve and operator getters of the three-dimensional
// gamblet path, and its C ABI (include/gamblet3d.h).
//
// Setup (Algorithm 2, fine to coarse, with psi^(q) = phi): the fine CSR is
// scattered into 8x8 blocks between level-(q-1) cubes and transformed by the
// per-parent Helmert matrices; then for k = q..2 the block-Jacobi factors of
// B^(k), the patch systems of Definition defb (line 11) giving Rhat
// (line 12), and the Galerkin product A^(k-1) = R A^(k) R^T (line 13),
// symmetrised and transformed for the next level.  The symbolic part of
// each level (neighbour offsets N, block offsets O_k, the Minkowski sums
// that drive the Galerkin product) is built here on the host.
//
// Solve (lines 15-18 and the refinement of Sec. 5.4): restriction through
// the levels, all level systems by one batched block-Jacobi CG, the level-1
// Cholesky, prolongation and sum; a float64 flexible CG on the fine CSR
// uses that operator as its preconditioner.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/gamblet3d.h"
#include "d3.cuh"
#include "host.cuh"

using namespace gb::d3;

namespace {

constexpr int kMaxQ3 = 8;
constexpr size_t kSmemLimit = 222 * 1024;  // 227 KB per CTA less the kernels' static reduction buffer
constexpr int kPatchMaxIter = 1000;
constexpr int kCgChunk3 = 8;

int floordiv2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }

struct OffSet3 {
  std::vector<int4> v;
  std::map<std::array<int, 3>, int> idx;
  int add(int x, int y, int z) {
    auto key = std::array<int, 3>{z, y, x};
    auto it = idx.find(key);
    if (it != idx.end()) return it->second;
    const int i = (int)v.size();
    idx[key] = i;
    v.push_back(make_int4(x, y, z, 0));
    return i;
  }
  int find(int x, int y, int z) const {
    auto it = idx.find(std::array<int, 3>{z, y, x});
    return it == idx.end() ? -1 : it->second;
  }
  int size() const { return (int)v.size(); }
  int radius() const {
    int r = 0;
    for (const int4& o : v) r = std::max({r, std::abs(o.x), std::abs(o.y), std::abs(o.z)});
    return r;
  }
  // box lookup table (see OffLookup)
  std::vector<int> table() const {
    const int R = radius(), S = 2 * R + 1;
    std::vector<int> t((size_t)S * S * S, -1);
    for (int i = 0; i < size(); ++i) {
      const int4 o = v[i];
      t[((size_t)(o.z + R) * S + o.y + R) * S + o.x + R] = i;
    }
    return t;
  }
};

// the box [-r, r]^3 clamped to |component| <= cap, row-major (z, y, x)
OffSet3 box3(int r, int cap) {
  r = std::min(r, cap);
  OffSet3 s;
  for (int z = -r; z <= r; ++z)
    for (int y = -r; y <= r; ++y)
      for (int x = -r; x <= r; ++x) s.add(x, y, z);
  return s;
}

// i^rho of Sec. 4.10 in level-(k-1) cell units (rule 0: Euclidean distance
// between closed cubes, sqrt(sum max(|d|-1, 0)^2) <= rho; rule 1: the box
// max |d| <= rho), clamped to the lattice (|d| <= cap).  rho <= 0: all.
OffSet3 neighbours3(double rho, int rule, int cap) {
  OffSet3 s;
  for (int z = -cap; z <= cap; ++z)
    for (int y = -cap; y <= cap; ++y)
      for (int x = -cap; x <= cap; ++x) {
        bool ok = true;
        if (rho > 0) {
          if (rule == 1) {
            ok = std::max({std::abs(x), std::abs(y), std::abs(z)}) <= rho;
          } else {
            const double ex = std::max(std::abs(x) - 1, 0), ey = std::max(std::abs(y) - 1, 0),
                         ez = std::max(std::abs(z) - 1, 0);
            ok = ex * ex + ey * ey + ez * ez <= rho * rho + 1e-12;
          }
        }
        if (ok) s.add(x, y, z);
      }
  return s;
}

struct Lev3 {
  int k = 0;
  int Lpar = 1;            // side of the level-(k-1) lattice (parents)
  int64_t ncell = 0;       // 8^k
  int64_t npar = 0;        // 8^(k-1)
  std::vector<uint32_t> pmask_h;
  uint32_t* pmask = nullptr;
  int n_active = 0, nJ = 0;
  // operator blocks
  OffSet3 O;
  int4* off = nullptr;
  int* lk = nullptr;
  int lkR = 0;
  int* mirror = nullptr;
  int o0 = -1;
  double* Ahat = nullptr;
  double* Dinv = nullptr;
  // patches (k >= 2)
  OffSet3 N;
  int NB = 0, jc = -1;
  int4* nbr = nullptr;
  int* pair = nullptr;
  double* Rhat = nullptr;
  int patch_it_max = 0;
  double patch_it_mean = 0;
  int patch_pairs = 0;     // coupled (a, b) pairs of a patch system
  int nD = 0;
  // solve vectors (8^k entries, Morton order)
  double* gnode = nullptr;
  double* v = nullptr;
  int64_t v0 = 0;          // offset of the level in the CG vectors
  Patch3Geom geom() const {
    Patch3Geom g;
    g.NB = NB;
    g.jc = jc;
    g.noff = O.size();
    g.nbr = nbr;
    g.pair_idx = pair;
    g.Lpar = Lpar;
    g.npatch = npar;
    return g;
  }
};

// A device buffer from the library's pool, released at scope exit.
struct TempBuf {
  void* p = nullptr;
  cudaStream_t s = nullptr;
  TempBuf(size_t bytes, cudaStream_t st) : s(st) {
    if (cudaMallocFromPoolAsync(&p, std::max<size_t>(bytes, 8), library_pool(), s) != cudaSuccess) {
      cudaGetLastError();
      fail(GAMBLET_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(bytes) + " bytes");
    }
  }
  ~TempBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

}  // namespace

struct gamblet3d_ctx {
  Prof prof;
  gamblet_opts opts;
  cudaStream_t s = nullptr;
  int q = 0, n = 0;
  int64_t nnz = 0;
  Pool pool;
  int32_t* rowptr = nullptr;
  int32_t* colind = nullptr;
  double* val = nullptr;
  int32_t* morton_of = nullptr;
  int32_t* unknown_of = nullptr;
  double* qtab = nullptr;
  std::vector<Lev3> lv;  // [0..q], lv[0] unused
  double* U1 = nullptr;
  int* status = nullptr;
  // batched level CG over k = 2..q
  Lcg3Level* cg_lv = nullptr;
  Lcg3Scalars* cg_sc = nullptr;
  double* cg_part = nullptr;
  double *cb = nullptr, *cx = nullptr, *cr = nullptr, *cz = nullptr, *cp = nullptr,
         *cAp = nullptr;
  int cg_nblk = 0, cg_nlev = 0;
  int64_t cg_n = 0;
  std::vector<Lcg3Scalars> sc_h;
  // outer iteration
  double *u = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *qv = nullptr, *rold = nullptr,
         *tmp = nullptr, *dpart = nullptr, *dout = nullptr;
  double setup_ms = 0;
  int setup_status = GAMBLET_OK;
  int patch_it_max = 0;
  double patch_it_mean = 0;
};

namespace {

void check_flags(gamblet3d_ctx* h, const int* flags_d) {
  int f[4];
  CK(cudaMemcpyAsync(f, flags_d, sizeof f, cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  if (f[0] == 2) fail(GAMBLET_ERR_INVALID_ARG, "a cell lies outside [0, 2^q)^3");
  if (f[0] == 1) fail(GAMBLET_ERR_INVALID_ARG, "two unknowns share a cell");
  if (f[2] == 3) fail(GAMBLET_ERR_INVALID_ARG, "a column index lies outside [0, n)");
}

void upload_offsets(gamblet3d_ctx* h, Lev3& L) {
  Pool& P = h->pool;
  L.off = P.upload(L.O.v, h->s);
  L.lkR = L.O.radius();
  L.lk = P.upload(L.O.table(), h->s);
  std::vector<int> mir(L.O.size());
  for (int i = 0; i < L.O.size(); ++i) {
    const int4 o = L.O.v[i];
    mir[i] = L.O.find(-o.x, -o.y, -o.z);
    if (mir[i] < 0) fail(GAMBLET_ERR_INVALID_ARG, "block offset set is not symmetric");
  }
  L.mirror = P.upload(mir, h->s);
  L.o0 = L.O.find(0, 0, 0);
}

// Galerkin lists of level k and the block offsets of level k-1.
struct GalPlan {
  OffSet3 D, E, Onext;
  std::vector<int> l1_ptr, l2_ptr;
  std::vector<int2> l1, l2;
};

GalPlan galerkin_plan(const Lev3& L) {
  GalPlan g;
  const int cap = L.Lpar - 1;
  auto inside = [&](int x, int y, int z) {
    return std::abs(x) <= cap && std::abs(y) <= cap && std::abs(z) <= cap;
  };
  std::vector<std::vector<int2>> l1;
  for (int j = 0; j < L.NB; ++j)
    for (int o = 0; o < L.O.size(); ++o) {
      const int4 a = L.N.v[j], b = L.O.v[o];
      const int x = a.x + b.x, y = a.y + b.y, z = a.z + b.z;
      if (!inside(x, y, z)) continue;
      const int d = g.D.add(x, y, z);
      if ((int)l1.size() <= d) l1.resize(d + 1);
      l1[d].push_back(make_int2(j, o));
    }
  std::vector<std::vector<int2>> l2;
  for (int d = 0; d < g.D.size(); ++d)
    for (int j = 0; j < L.NB; ++j) {
      const int4 a = g.D.v[d], b = L.N.v[j];
      const int x = a.x - b.x, y = a.y - b.y, z = a.z - b.z;
      if (!inside(x, y, z)) continue;
      const int e = g.E.add(x, y, z);
      if ((int)l2.size() <= e) l2.resize(e + 1);
      l2[e].push_back(make_int2(j, d));
    }
  g.l1_ptr.push_back(0);
  for (auto& v : l1) {
    g.l1.insert(g.l1.end(), v.begin(), v.end());
    g.l1_ptr.push_back((int)g.l1.size());
  }
  // outputs in order of decreasing pair count: the eight-lane groups of a
  // warp then take outputs of about the same work
  std::vector<int> order(l2.size());
  for (size_t e = 0; e < order.size(); ++e) order[e] = (int)e;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return l2[a].size() > l2[b].size(); });
  OffSet3 Esorted;
  g.l2_ptr.push_back(0);
  for (int e : order) {
    const int4 o = g.E.v[e];
    Esorted.add(o.x, o.y, o.z);
    g.l2.insert(g.l2.end(), l2[e].begin(), l2[e].end());
    g.l2_ptr.push_back((int)g.l2.size());
  }
  g.E = Esorted;
  // parent offsets of level k-1 (level k-2 cell units) reached by the
  // outputs: floor((x + e) / 2) over the child slot bits x
  const int capn = std::max(L.Lpar / 2 - 1, 0);
  std::vector<std::array<int, 3>> cand;
  for (const int4& e : g.E.v)
    for (int bits = 0; bits < 8; ++bits) {
      const int ox = floordiv2((bits & 1) + e.x), oy = floordiv2(((bits >> 1) & 1) + e.y),
                oz = floordiv2(((bits >> 2) & 1) + e.z);
      if (std::abs(ox) <= capn && std::abs(oy) <= capn && std::abs(oz) <= capn)
        cand.push_back({oz, oy, ox});
    }
  std::sort(cand.begin(), cand.end());
  cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
  for (auto& c : cand) g.Onext.add(c[2], c[1], c[0]);
  return g;
}

std::vector<double> qtable() {
  std::vector<double> t(256 * 64);
  for (int m = 0; m < 256; ++m)
    for (int a = 0; a < 8; ++a)
      for (int c = 0; c < 8; ++c) t[m * 64 + a * 8 + c] = q8(m, a, c);
  return t;
}

double ms_between(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0;
  CK(cudaEventElapsedTime(&ms, a, b));
  return ms;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  EventPair() {
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
  }
  ~EventPair() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

gamblet3d_ctx* setup3(const gamblet_csr* A, int q, const int32_t* cells, const gamblet_opts* o) {
  if (!A || !cells) fail(GAMBLET_ERR_INVALID_ARG, "A or cells is NULL");
  if (A->n < 1 || A->nnz < 0 || !A->rowptr || (A->nnz > 0 && (!A->colind || !A->val)))
    fail(GAMBLET_ERR_INVALID_ARG, "malformed CSR");
  if (q < 2 || q > kMaxQ3) fail(GAMBLET_ERR_INVALID_ARG, "q must satisfy 2 <= q <= 8");
  if (A->nnz > INT32_MAX) fail(GAMBLET_ERR_UNSUPPORTED, "more than 2^31 - 1 stored entries");
  auto h = std::make_unique<gamblet3d_ctx>();
  if (o) h->opts = *o;
  else gamblet_default_opts(&h->opts);
  if (h->opts.precision != GAMBLET_FP64)
    fail(GAMBLET_ERR_UNSUPPORTED, "the three-dimensional path computes in float64 only");
  if (!(h->opts.level_tol > 0) || !(h->opts.refine_tol >= 0) || h->opts.level_max_iter < 1 ||
      h->opts.refine_max_iter < 0 || h->opts.patch_tol < 0)
    fail(GAMBLET_ERR_INVALID_ARG, "bad tolerance or iteration cap");
  h->s = (cudaStream_t)h->opts.stream;
  h->pool.s = h->s;
  h->prof.on = h->opts.profile != 0;
  Prof& prof = h->prof;
  cudaStream_t s = h->s;
  Pool& P = h->pool;
  h->q = q;
  h->n = A->n;
  h->nnz = A->nnz;
  const int n = h->n;
  EventPair ev;
  CK(cudaEventRecord(ev.a, s));

  // fine CSR and cells on the device
  std::vector<int32_t> rp((size_t)n + 1);
  to_host(rp.data(), A->rowptr, (int64_t)n + 1);
  if (rp[0] != 0 || rp[n] != A->nnz) fail(GAMBLET_ERR_INVALID_ARG, "rowptr[0] != 0 or rowptr[n] != nnz");
  for (int i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) fail(GAMBLET_ERR_INVALID_ARG, "rowptr is not non-decreasing");
  h->rowptr = P.upload(rp, s);
  to_device(P, h->colind, A->colind, A->nnz, s);
  to_device(P, h->val, A->val, A->nnz, s);
  const int32_t* cells_d = as_device(P, cells, (int64_t)3 * n, s);

  // hierarchy
  h->lv.resize(q + 1);
  for (int k = 1; k <= q; ++k) {
    Lev3& L = h->lv[k];
    L.k = k;
    L.Lpar = 1 << (k - 1);
    L.ncell = (int64_t)1 << (3 * k);
    L.npar = (int64_t)1 << (3 * (k - 1));
    L.pmask = P.zeros<uint32_t>(L.npar, s);
  }
  int* flags = P.zeros<int>(4, s);
  h->morton_of = P.alloc<int32_t>(n);
  h->unknown_of = P.alloc<int32_t>(h->lv[q].ncell);
  CK(cudaMemsetAsync(h->unknown_of, 0xff, sizeof(int32_t) * h->lv[q].ncell, s));
  launch_cells_to_morton3(cells_d, n, q, h->morton_of, flags, s);
  launch_scatter3(h->morton_of, n, h->unknown_of, h->lv[q].pmask, flags, s);
  for (int k = q; k >= 2; --k) launch_coarsen3(h->lv[k].pmask, h->lv[k - 1].npar, h->lv[k - 1].pmask, s);
  launch_csr_extent3(n, h->rowptr, h->colind, h->morton_of, flags + 1, flags + 2, s);
  CK(cudaGetLastError());
  check_flags(h.get(), flags);
  int ext = 0;
  CK(cudaMemcpy(&ext, flags + 1, sizeof(int), cudaMemcpyDeviceToHost));
  for (int k = 1; k <= q; ++k) {
    Lev3& L = h->lv[k];
    L.pmask_h.resize(L.npar);
    CK(cudaMemcpyAsync(L.pmask_h.data(), L.pmask, sizeof(uint32_t) * L.npar, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  for (int k = 1; k <= q; ++k) {
    Lev3& L = h->lv[k];
    for (uint32_t m : L.pmask_h) {
      const int c = __builtin_popcount(m & 255u);
      L.n_active += c;
      if (c > 0) L.nJ += c - 1;
    }
  }
  h->qtab = P.upload(qtable(), s);
  h->status = P.zeros<int>(1, s);

  // level q blocks
  {
    Lev3& L = h->lv[q];
    L.O = box3(ext, L.Lpar - 1);
    upload_offsets(h.get(), L);
    L.Ahat = P.zeros<double>((int64_t)L.O.size() * L.npar * 64, s);
    OffLookup lk{L.lk, L.lkR};
    const double blk_bytes = (double)L.O.size() * L.npar * 64 * sizeof(double);
    const int tk = prof.begin("import3", (double)h->nnz * 16 + blk_bytes * 2, 0.0, s);
    launch_csr_to_blocks3(n, h->rowptr, h->colind, h->val, h->morton_of, lk, q, L.npar, L.Ahat, s);
    launch_transform_blocks3(L.Ahat, L.Ahat, L.off, L.mirror, L.O.size(), L.npar, L.Lpar, L.pmask,
                             0, h->qtab, s);
    prof.end(tk, s);
  }
  const double ptol = h->opts.patch_tol > 0 ? h->opts.patch_tol : 1e-12;
  int* it_stats = P.zeros<int>(3 * (q + 1), s);
  for (int k = q; k >= 2; --k) {
    Lev3& L = h->lv[k];
    if (L.o0 < 0) fail(GAMBLET_ERR_INVALID_ARG, "the diagonal block offset is missing");
    L.Dinv = P.alloc<double>(L.npar * 64);
    const int td = prof.begin("dinv3", (double)L.npar * 128 * sizeof(double), 0.0, s);
    launch_detail_inverse3(L.Ahat, L.o0, L.npar, L.pmask, L.Dinv, h->status, s);
    prof.end(td, s);
    // patches
    L.N = neighbours3(h->opts.rho, h->opts.nbr_rule, L.Lpar - 1);
    L.NB = L.N.size();
    L.jc = L.N.find(0, 0, 0);
    if (patch_cg3_smem(L.NB) > kSmemLimit)
      fail(GAMBLET_ERR_UNSUPPORTED, "patch of " + std::to_string(L.NB) +
                                        " cubes exceeds one CTA's shared memory (level " +
                                        std::to_string(k) + ")");
    std::vector<int> pair((size_t)L.NB * L.NB);
    for (int a = 0; a < L.NB; ++a)
      for (int b = 0; b < L.NB; ++b) {
        const int4 na = L.N.v[a], nb = L.N.v[b];
        pair[(size_t)a * L.NB + b] = L.O.find(nb.x - na.x, nb.y - na.y, nb.z - na.z);
      }
    L.nbr = P.upload(L.N.v, s);
    L.pair = P.upload(pair, s);
    L.Rhat = P.alloc<double>(L.npar * L.NB * 8);
    int npairs = 0;
    for (int v : pair) npairs += v >= 0;
    L.patch_pairs = npairs;
    const int tp = prof.begin("patch_cg3_k" + std::to_string(k), 0.0, 0.0, s);
    launch_patch_cg3(L.Ahat, L.Dinv, L.pmask, L.geom(), ptol, kPatchMaxIter, L.Rhat,
                     it_stats + 3 * k, s);
    prof.end(tp, s);
    CK(cudaGetLastError());
    // Galerkin product into level k-1
    GalPlan g = galerkin_plan(L);
    L.nD = g.D.size();
    if (galerkin3_smem(L.NB, L.nD) > kSmemLimit)
      fail(GAMBLET_ERR_UNSUPPORTED, "Galerkin row of level " + std::to_string(k) +
                                        " exceeds one CTA's shared memory");
    Lev3& C = h->lv[k - 1];
    C.O = g.Onext;
    upload_offsets(h.get(), C);
    const int64_t nblk = (int64_t)C.O.size() * C.npar * 64;
    TempBuf raw(sizeof(double) * (size_t)nblk, s);
    CK(cudaMemsetAsync(raw.p, 0, sizeof(double) * (size_t)nblk, s));
    Galerkin3Geom gg;
    gg.NB = L.NB;
    gg.nbr = L.nbr;
    gg.Lpar = L.Lpar;
    gg.npatch = L.npar;
    gg.nD = L.nD;
    gg.l1_ptr = P.upload(g.l1_ptr, s);
    gg.l1 = P.upload(g.l1, s);
    gg.nE = g.E.size();
    gg.E = P.upload(g.E.v, s);
    gg.l2_ptr = P.upload(g.l2_ptr, s);
    gg.l2 = P.upload(g.l2, s);
    gg.out_lk = OffLookup{C.lk, C.lkR};
    gg.noff = L.O.size();
    gg.noff_out = C.O.size();
    gg.npar_out = C.npar;
    {
      // per active coarse row: phase 1 reads 64 block entries per (j, o) pair,
      // phase 2 an 8-vector per (j', d) pair
      const double rows = (double)C.n_active;
      const double fl = rows * (128.0 * g.l1.size() + 16.0 * g.l2.size());
      const double by = (double)L.O.size() * L.npar * 512 + (double)L.npar * L.NB * 64 +
                        (double)nblk * sizeof(double);
      const int tg = prof.begin("galerkin3_k" + std::to_string(k), by, fl, s);
      launch_galerkin3(L.Ahat, L.Rhat, L.pmask, gg, raw.as<double>(), s);
      prof.end(tg, s);
    }
    C.Ahat = P.alloc<double>(nblk);
    const int tt = prof.begin("transform3", (double)nblk * 3 * sizeof(double), 0.0, s);
    launch_transform_blocks3(raw.as<double>(), C.Ahat, C.off, C.mirror, C.O.size(), C.npar,
                             C.Lpar, C.pmask, 1, h->qtab, s);
    prof.end(tt, s);
    CK(cudaGetLastError());
  }
  // solve buffers
  for (int k = 1; k <= q; ++k) {
    Lev3& L = h->lv[k];
    L.gnode = P.zeros<double>(L.ncell, s);
    L.v = P.zeros<double>(L.ncell, s);
  }
  h->U1 = P.zeros<double>(8, s);
  std::vector<Lcg3Level> cg;
  int64_t v0 = 0;
  int blk = 0;
  for (int k = 2; k <= q; ++k) {
    Lev3& L = h->lv[k];
    L.v0 = v0;
    Lcg3Level c;
    c.A = L.Ahat;
    c.Dinv = L.Dinv;
    c.off = L.off;
    c.noff = L.O.size();
    c.Lpar = L.Lpar;
    c.npar = L.npar;
    c.v0 = v0;
    c.blk0 = blk;
    c.nblk = (int)((L.npar + 31) / 32);
    cg.push_back(c);
    v0 += L.npar * 8;
    blk += c.nblk;
  }
  h->cg_n = v0;
  h->cg_nblk = blk;
  h->cg_nlev = (int)cg.size();
  h->cg_lv = P.upload(cg, s);
  h->cg_sc = P.zeros<Lcg3Scalars>(h->cg_nlev, s);
  h->cg_part = P.zeros<double>((int64_t)blk * 3, s);
  h->cb = P.zeros<double>(v0, s);
  h->cx = P.zeros<double>(v0, s);
  h->cr = P.zeros<double>(v0, s);
  h->cz = P.zeros<double>(v0, s);
  h->cp = P.zeros<double>(v0, s);
  h->cAp = P.zeros<double>(v0, s);
  h->sc_h.resize(h->cg_nlev);
  h->u = P.zeros<double>(n, s);
  h->r = P.zeros<double>(n, s);
  h->z = P.zeros<double>(n, s);
  h->p = P.zeros<double>(n, s);
  h->qv = P.zeros<double>(n, s);
  h->rold = P.zeros<double>(n, s);
  h->tmp = P.zeros<double>(n, s);
  h->dpart = P.zeros<double>(2 * 1024, s);
  h->dout = P.zeros<double>(2, s);
  CK(cudaEventRecord(ev.b, s));
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  h->setup_ms = ms_between(ev.a, ev.b);
  prof.resolve();
  if (const int gv = guard_take())
    fail(GAMBLET_ERR_CUDA, "internal index guard " + std::to_string(gv) + " failed in the setup");
  int st = 0;
  CK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st == DEV_NOT_SPD) fail(GAMBLET_ERR_NOT_SPD, "non-positive pivot in a block-Jacobi factor");
  std::vector<int> its(3 * (q + 1));
  CK(cudaMemcpy(its.data(), it_stats, sizeof(int) * its.size(), cudaMemcpyDeviceToHost));
  int64_t sum = 0, cnt = 0;
  for (int k = 2; k <= q; ++k) {
    Lev3& L = h->lv[k];
    // CG work of the patch systems: per iteration the product with the
    // patch's detail blocks (49 multiply-adds per coupled pair), the
    // block-Jacobi step (49 per parent) and about ten vector operations per
    // unknown; the blocks are read from memory on every iteration
    const double per_it_fl = 2.0 * 49 * L.patch_pairs + 2.0 * 49 * L.NB + 10.0 * 7 * L.NB;
    const double per_it_by = (double)L.patch_pairs * 7 * 56 + (double)L.NB * 7 * 64;
    prof.add("patch_cg3_k" + std::to_string(k), per_it_by * its[3 * k + 1], per_it_fl * its[3 * k + 1]);
    L.patch_it_max = its[3 * k];
    L.patch_it_mean = its[3 * k + 2] ? (double)its[3 * k + 1] / its[3 * k + 2] : 0.0;
    h->patch_it_max = std::max(h->patch_it_max, L.patch_it_max);
    sum += its[3 * k + 1];
    cnt += its[3 * k + 2];
  }
  h->patch_it_mean = cnt ? (double)sum / cnt : 0.0;
  if (h->patch_it_max >= kPatchMaxIter) h->setup_status = GAMBLET_ERR_NOT_CONVERGED;
  return h.release();
}

// dot products x . y (and x . w) in float64, deterministic
void dots(gamblet3d_ctx* h, int64_t n, const double* x, const double* y, const double* w,
          double* out) {
  const int nb = dot3_blocks(n);
  launch_dot3(n, x, y, w, h->dpart, h->s);
  launch_dot3_finish(h->dpart, nb, w ? 2 : 1, h->dout, h->s);
  CK(cudaMemcpyAsync(out, h->dout, sizeof(double) * (w ? 2 : 1), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
}

// All level systems B^(k) w^(k) = W g^(k) at once (right-hand sides in cb,
// solutions in cx); returns false if a level hit its iteration cap.
bool level_cg(gamblet3d_ctx* h, int* iters) {
  cudaStream_t s = h->s;
  if (h->cg_nlev == 0) return true;
  Prof& prof = h->prof;
  const double tol = h->opts.level_tol;
  const int maxit = h->opts.level_max_iter;
  launch_lcg3_start(h->cg_lv, h->cg_nlev, h->cg_nblk, h->cb, h->cx, h->cr, h->cz, h->cp,
                    h->cg_part, s);
  launch_lcg3_init_scalars(h->cg_lv, h->cg_nlev, h->cg_part, h->cg_sc, tol, s);
  for (int done = 0; done < maxit; done += kCgChunk3) {
    CK(cudaMemcpyAsync(h->sc_h.data(), h->cg_sc, sizeof(Lcg3Scalars) * h->cg_nlev,
                       cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    bool any = false;
    for (auto& c : h->sc_h) any |= c.active == 1;
    if (!any) break;
    const int tc = prof.begin("level_cg3", 0.0, 0.0, s);
    for (int it = 0; it < kCgChunk3; ++it) {
      launch_lcg3_spmv(h->cg_lv, h->cg_nlev, h->cg_nblk, h->cg_sc, h->cp, h->cAp, h->cg_part, s);
      launch_lcg3_alpha(h->cg_lv, h->cg_nlev, h->cg_part, h->cg_sc, s);
      launch_lcg3_update(h->cg_lv, h->cg_nlev, h->cg_nblk, h->cg_sc, h->cp, h->cAp, h->cx, h->cr,
                         h->cz, h->cg_part, s);
      launch_lcg3_beta(h->cg_lv, h->cg_nlev, h->cg_part, h->cg_sc, tol, maxit, s);
      launch_lcg3_direction(h->cg_lv, h->cg_nlev, h->cg_nblk, h->cg_sc, h->cz, h->cp, s);
    }
    prof.end(tc, s);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(h->sc_h.data(), h->cg_sc, sizeof(Lcg3Scalars) * h->cg_nlev,
                     cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool ok = true;
  for (int l = 0; l < h->cg_nlev; ++l) {
    const int k = l + 2;
    if (iters && k < 32) iters[k] += h->sc_h[l].iters;
    if (h->sc_h[l].active != 0) ok = false;
    // the iterations this level ran: its detail blocks (49 values of 8
    // bytes each) once per iteration, and about twelve passes over the
    // level's vectors (8 doubles per parent)
    const Lev3& L = h->lv[k];
    const double it = h->sc_h[l].iters;
    prof.add("level_cg3", it * ((double)L.O.size() * L.npar * 392 + 12.0 * 64 * L.npar),
             it * (2.0 * 49 * L.O.size() * L.npar + 2.0 * 49 * L.npar + 12.0 * 8 * L.npar));
  }
  return ok;
}

// out = G in: the one-pass gamblet operator (restriction, level solves,
// prolongation and sum); comps (device, q x n) receives the components.
bool apply_G3(gamblet3d_ctx* h, const double* in, double* out, double* comps, int* iters) {
  cudaStream_t s = h->s;
  const int q = h->q;
  Prof& prof = h->prof;
  double rb = 0, rf = 0;
  for (int k = 2; k <= q; ++k) {
    const Lev3& L = h->lv[k];
    rb += (double)L.npar * L.NB * 64 + (double)L.npar * 8 * 8 * 3;
    rf += 2.0 * L.npar * L.NB * 8 + 2.0 * 64 * L.npar;
  }
  const int tr = prof.begin("restrict3", rb, rf, s);
  launch_gather3(in, h->unknown_of, h->lv[q].ncell, h->lv[q].gnode, s);
  for (int k = q; k >= 2; --k) {
    Lev3& L = h->lv[k];
    double* ghat = h->cb + L.v0;
    launch_transform_vec3(L.gnode, ghat, L.npar, L.pmask, +1, h->qtab, s);
    launch_restrict3(L.Rhat, ghat, L.pmask, L.geom(), h->lv[k - 1].gnode, s);
  }
  prof.end(tr, s);
  const bool ok = level_cg(h, iters);
  launch_coarsest3(h->lv[1].Ahat, h->lv[1].pmask_h[0], h->lv[1].gnode, h->qtab, h->U1, h->status,
                   s);
  const double* vprev = h->U1;
  const int tq = prof.begin("prolong3", rb, rf, s);
  for (int k = 2; k <= q; ++k) {
    Lev3& L = h->lv[k];
    launch_prolong3(L.Rhat, vprev, h->cx + L.v0, L.pmask, L.geom(), h->qtab, L.v, s);
    vprev = L.v;
  }
  launch_scatter_unknown3(h->lv[q].v, h->morton_of, h->n, out, s);
  prof.end(tq, s);
  if (comps) {
    for (int k0 = 1; k0 <= q; ++k0) {
      const double* vp = k0 == 1 ? h->U1 : nullptr;
      for (int k = std::max(k0, 2); k <= q; ++k) {
        Lev3& L = h->lv[k];
        launch_prolong3(L.Rhat, vp, k == k0 ? h->cx + L.v0 : nullptr, L.pmask, L.geom(), h->qtab,
                        L.v, s);
        vp = L.v;
      }
      launch_scatter_unknown3(vp, h->morton_of, h->n, comps + (int64_t)(k0 - 1) * h->n, s);
    }
  }
  CK(cudaGetLastError());
  return ok;
}

gamblet_status solve3(gamblet3d_ctx* h, const double* g, double* u, double* comps,
                      gamblet_info* info) {
  cudaStream_t s = h->s;
  const int n = h->n, q = h->q;
  Pool tmp;
  tmp.s = s;
  EventPair ev;
  CK(cudaEventRecord(ev.a, s));
  const double* gd = as_device(tmp, g, n, s);
  const bool u_dev = is_device_ptr(u);
  double* ud = u_dev ? u : h->u;
  double* cd = nullptr;
  const bool c_dev = comps && is_device_ptr(comps);
  if (comps) cd = c_dev ? comps : tmp.alloc<double>((int64_t)q * n);
  int iters[32] = {0};
  bool ok = true;
  int outer = 0;
  double gg = 0;
  dots(h, n, gd, gd, nullptr, &gg);
  const double gnorm = std::sqrt(gg);
  if (h->opts.refine_max_iter == 0) {
    ok &= apply_G3(h, gd, ud, cd, iters);
  } else {
    // flexible CG (Polak-Ribiere beta), u_0 = 0
    CK(cudaMemsetAsync(ud, 0, sizeof(double) * n, s));
    CK(cudaMemcpyAsync(h->r, gd, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    ok &= apply_G3(h, h->r, h->z, cd, iters);
    CK(cudaMemcpyAsync(h->p, h->z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    double rz = 0;
    dots(h, n, h->r, h->z, nullptr, &rz);
    const double stop = h->opts.refine_tol * gnorm;
    bool conv = gnorm == 0.0;
    while (!conv && outer < h->opts.refine_max_iter) {
      const int to = h->prof.begin("outer_spmv3", (double)h->nnz * 12 + (double)n * 24,
                                   2.0 * h->nnz, s);
      launch_csr_spmv3(n, h->rowptr, h->colind, h->val, h->p, h->qv, s);
      h->prof.end(to, s);
      double pq = 0;
      dots(h, n, h->p, h->qv, nullptr, &pq);
      if (!(pq > 0)) break;
      const double alpha = rz / pq;
      launch_axpby3(n, alpha, h->p, 1.0, ud, s);
      CK(cudaMemcpyAsync(h->rold, h->r, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      launch_axpby3(n, -alpha, h->qv, 1.0, h->r, s);
      ++outer;
      double rr = 0;
      dots(h, n, h->r, h->r, nullptr, &rr);
      if (std::sqrt(rr) <= stop) {
        conv = true;
        break;
      }
      ok &= apply_G3(h, h->r, h->z, nullptr, iters);
      double zz[2];
      dots(h, n, h->z, h->r, h->rold, zz);
      const double beta = (zz[0] - zz[1]) / rz;
      rz = zz[0];
      launch_axpby3(n, 1.0, h->z, beta, h->p, s);
    }
    if (!conv) ok = false;
  }
  // final residual |g - A u| / |g| in float64
  launch_csr_spmv3(n, h->rowptr, h->colind, h->val, ud, h->tmp, s);
  launch_axpby3(n, 1.0, gd, -1.0, h->tmp, s);
  double res2 = 0;
  dots(h, n, h->tmp, h->tmp, nullptr, &res2);
  if (!u_dev) CK(cudaMemcpyAsync(u, ud, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (comps && !c_dev)
    CK(cudaMemcpyAsync(comps, cd, sizeof(double) * (size_t)q * n, cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(ev.b, s));
  CK(cudaStreamSynchronize(s));
  h->prof.resolve();
  int st = 0;
  CK(cudaMemcpy(&st, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st == DEV_NOT_SPD) fail(GAMBLET_ERR_NOT_SPD, "non-positive pivot in the level-1 Cholesky");
  if (info) {
    info->status = ok ? GAMBLET_OK : GAMBLET_ERR_NOT_CONVERGED;
    info->q = q;
    info->outer_iters = outer;
    for (int k = 0; k < 32; ++k) info->level_iters[k] = iters[k];
    info->rel_residual = gnorm > 0 ? std::sqrt(res2) / gnorm : 0.0;
    info->setup_ms = h->setup_ms;
    info->solve_ms = ms_between(ev.a, ev.b);
    info->patch_iters_max = h->patch_it_max;
    info->patch_iters_mean = h->patch_it_mean;
  }
  return ok ? GAMBLET_OK : GAMBLET_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------- getters
bool active_cell(const gamblet3d_ctx* h, int k, int64_t m) {
  return (h->lv[k].pmask_h[m >> 3] >> (m & 7)) & 1u;
}

// level-k Morton index -> oracle index (-1 inactive)
std::vector<int32_t> oracle_index(const gamblet3d_ctx* h, int k) {
  const int64_t nc = h->lv[k].ncell;
  std::vector<int32_t> map(nc, -1);
  if (k == h->q) {
    CK(cudaMemcpy(map.data(), h->unknown_of, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost));
    return map;
  }
  const int64_t L = (int64_t)1 << k;
  std::vector<std::pair<int64_t, int64_t>> keys;
  for (int64_t m = 0; m < nc; ++m) {
    if (!active_cell(h, k, m)) continue;
    int x, y, z;
    demorton3((uint32_t)m, x, y, z);
    keys.push_back({((int64_t)z * L + y) * L + x, m});
  }
  std::sort(keys.begin(), keys.end());
  for (size_t r = 0; r < keys.size(); ++r) map[keys[r].second] = (int32_t)r;
  return map;
}

// parent -> first row of its details in the oracle's W^(k) order
std::vector<int32_t> detail_base(const gamblet3d_ctx* h, int k) {
  const Lev3& L = h->lv[k];
  std::vector<int32_t> pm = oracle_index(h, k - 1);
  std::vector<std::pair<int32_t, int64_t>> order;
  for (int64_t P = 0; P < L.npar; ++P)
    if (pm[P] >= 0) order.push_back({pm[P], P});
  std::sort(order.begin(), order.end());
  std::vector<int32_t> base(L.npar, -1);
  int32_t row = 0;
  for (auto& e : order) {
    base[e.second] = row;
    row += std::max(__builtin_popcount(L.pmask_h[e.second] & 255u) - 1, 0);
  }
  return base;
}

struct Coo {
  std::vector<int32_t> r, c;
  std::vector<double> v;
};

void get_operator3(const gamblet3d_ctx* h, int which, int k, Coo& out) {
  const int q = h->q;
  if (k < 1 || k > q || (which != 0 && k < 2) || which < 0 || which > 2)
    fail(GAMBLET_ERR_INVALID_ARG, "bad operator or level");
  std::vector<double> Q = qtable();
  const Lev3& L = h->lv[k];
  if (which == 0 || which == 2) {
    const int noff = L.O.size();
    std::vector<double> A((size_t)noff * L.npar * 64);
    CK(cudaMemcpy(A.data(), L.Ahat, sizeof(double) * A.size(), cudaMemcpyDeviceToHost));
    std::vector<int32_t> map = which == 0 ? oracle_index(h, k) : std::vector<int32_t>();
    std::vector<int32_t> base = which == 2 ? detail_base(h, k) : std::vector<int32_t>();
    for (int o = 0; o < noff; ++o)
      for (int64_t p = 0; p < L.npar; ++p) {
        const uint32_t mp = L.pmask_h[p];
        if (!mp) continue;
        int x, y, z;
        demorton3((uint32_t)p, x, y, z);
        const int4 d = L.O.v[o];
        const int pn = shift3(x, y, z, d.x, d.y, d.z, L.Lpar);
        if (pn < 0 || !L.pmask_h[pn]) continue;
        const uint32_t mn = L.pmask_h[pn];
        const double* B = &A[((size_t)o * L.npar + p) * 64];
        if (which == 2) {
          const int na = __builtin_popcount(mp) - 1, nb = __builtin_popcount(mn) - 1;
          for (int a = 0; a < na; ++a)
            for (int b = 0; b < nb; ++b) {
              out.r.push_back(base[p] + a);
              out.c.push_back(base[pn] + b);
              out.v.push_back(B[a * 8 + b]);
            }
          continue;
        }
        // A(p, pn) = Q_p^T Ahat Q_pn
        const double* Qp = &Q[(size_t)mp * 64];
        const double* Qn = &Q[(size_t)mn * 64];
        for (int sa = 0; sa < 8; ++sa) {
          if (!((mp >> sa) & 1)) continue;
          for (int sb = 0; sb < 8; ++sb) {
            if (!((mn >> sb) & 1)) continue;
            double v = 0;
            for (int a = 0; a < 8; ++a)
              for (int b = 0; b < 8; ++b) v += Qp[a * 8 + sa] * B[a * 8 + b] * Qn[b * 8 + sb];
            out.r.push_back(map[p * 8 + sa]);
            out.c.push_back(map[(int64_t)pn * 8 + sb]);
            out.v.push_back(v);
          }
        }
      }
    return;
  }
  // R^(k-1,k): row i (level k-1), columns the children of the patch parents
  std::vector<double> R((size_t)L.npar * L.NB * 8);
  CK(cudaMemcpy(R.data(), L.Rhat, sizeof(double) * R.size(), cudaMemcpyDeviceToHost));
  std::vector<int32_t> rmap = oracle_index(h, k - 1), cmap = oracle_index(h, k);
  for (int64_t i = 0; i < L.npar; ++i) {
    if (!L.pmask_h[i]) continue;
    int x, y, z;
    demorton3((uint32_t)i, x, y, z);
    for (int j = 0; j < L.NB; ++j) {
      const int4 d = L.N.v[j];
      const int P = shift3(x, y, z, d.x, d.y, d.z, L.Lpar);
      if (P < 0 || !L.pmask_h[P]) continue;
      const uint32_t m = L.pmask_h[P];
      const double* Qm = &Q[(size_t)m * 64];
      const double* rh = &R[((size_t)i * L.NB + j) * 8];
      for (int sc = 0; sc < 8; ++sc) {
        if (!((m >> sc) & 1)) continue;
        double v = 0;
        for (int c = 0; c < 8; ++c) v += Qm[c * 8 + sc] * rh[c];
        out.r.push_back(rmap[i]);
        out.c.push_back(cmap[(int64_t)P * 8 + sc]);
        out.v.push_back(v);
      }
    }
  }
}

}  // namespace

extern "C" {

gamblet_status gamblet3d_setup(const gamblet_csr* A, int32_t q, const int32_t* cells,
                               const gamblet_opts* opts, gamblet3d_handle* out) {
  if (!out) return set_error(GbError{GAMBLET_ERR_INVALID_ARG, "out is NULL"});
  *out = nullptr;
  try {
    gamblet3d_ctx* h = setup3(A, q, cells, opts);
    *out = h;
    if (h->setup_status != GAMBLET_OK)
      return set_error(GbError{(gamblet_status)h->setup_status,
                               "a patch CG reached its iteration cap"});
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  } catch (const std::exception& e) {
    return set_error(GbError{GAMBLET_ERR_INVALID_ARG, e.what()});
  }
}

gamblet_status gamblet3d_solve(gamblet3d_handle h, const double* g, double* u, double* components,
                               gamblet_info* info) {
  if (!h || !g || !u) return set_error(GbError{GAMBLET_ERR_INVALID_ARG, "NULL handle, g or u"});
  try {
    const gamblet_status st = solve3(h, g, u, components, info);
    if (st != GAMBLET_OK) return set_error(GbError{st, "an iteration cap was hit"});
    return st;
  } catch (const GbError& e) {
    return set_error(e);
  } catch (const std::exception& e) {
    return set_error(GbError{GAMBLET_ERR_INVALID_ARG, e.what()});
  }
}

gamblet_status gamblet3d_level_size(gamblet3d_handle h, int32_t k, int32_t* n_k, int32_t* nJ_k) {
  if (!h || k < 1 || k > h->q)
    return set_error(GbError{GAMBLET_ERR_INVALID_ARG, "bad handle or level"});
  if (n_k) *n_k = h->lv[k].n_active;
  if (nJ_k) *nJ_k = k >= 2 ? h->lv[k].nJ : 0;
  return GAMBLET_OK;
}

gamblet_status gamblet3d_get_operator(gamblet3d_handle h, int32_t which, int32_t k,
                                      int64_t capacity, int64_t* nnz, int32_t* rows, int32_t* cols,
                                      double* vals) {
  if (!h || !nnz) return set_error(GbError{GAMBLET_ERR_INVALID_ARG, "NULL handle or nnz"});
  try {
    Coo c;
    get_operator3(h, which, k, c);
    *nnz = (int64_t)c.v.size();
    if (capacity > 0) {
      if (!rows || !cols || !vals)
        return set_error(GbError{GAMBLET_ERR_INVALID_ARG, "NULL output array"});
      const int64_t m = std::min<int64_t>(capacity, (int64_t)c.v.size());
      std::copy(c.r.begin(), c.r.begin() + m, rows);
      std::copy(c.c.begin(), c.c.begin() + m, cols);
      std::copy(c.v.begin(), c.v.begin() + m, vals);
    }
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  }
}

gamblet_status gamblet3d_level_geometry(gamblet3d_handle h, int32_t k, int32_t* geom) {
  if (!h || !geom || k < 2 || k > h->q)
    return set_error(GbError{GAMBLET_ERR_INVALID_ARG, "bad handle, level or output"});
  const Lev3& L = h->lv[k];
  geom[0] = L.NB;
  geom[1] = L.O.size();
  geom[2] = L.patch_it_max;
  geom[3] = L.nD;
  return GAMBLET_OK;
}

int32_t gamblet3d_kernel_stats(gamblet3d_handle h, gamblet_kernel_stat* out, int32_t capacity) {
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

void gamblet3d_reset_kernel_stats(gamblet3d_handle h) {
  if (h) h->prof.stats.clear();
}

int64_t gamblet3d_device_bytes(gamblet3d_handle h) { return h ? h->pool.bytes : 0; }

void gamblet3d_destroy(gamblet3d_handle h) {
  if (!h) return;
  cudaStreamSynchronize(h->s);
  delete h;
}

}  // extern "C"
