// tune.cu - the launch-shape autotuner of the setup and the level CG: the
// SIMT patch CG's lanes and gather, the tensor-core patch windows, the
// cluster split of patches beyond one CTA, the Galerkin kernel variant and
// the level-CG SpMV tile, chosen by timing candidates on a sample of each
// large level once per geometry and precision in a process.  Every
// candidate computes the same rows; only the summation order (and, for the
// tensor-core windows, the float16 rounding of the scaled patch matrix)
// differs.
#include "host.cuh"

namespace gb {
namespace hs {

// ------------------------------------------------------------ autotuner
// Launch shapes chosen by timing the candidates on the device, once per
// geometry key, level and working precision in a process, then reused by
// every later setup of that geometry (the results depend on the shape only
// through summation order).  Levels smaller than kTuneMinParents keep the
// fixed rule: their kernels are too short for the choice to matter.
// Patch solves: a 256 x 128 Morton block of coarse cells, about fifteen
// patches per CTA of the persistent SIMT kernels, so that the timing sees
// their steady state (with two per CTA the launch and the tail dominated,
// and the tuner's choice on the finest level changed from run to run)
constexpr int64_t kTuneSample = 32768;
// Galerkin rows are cheap and one variant packs eight rows per CTA: a larger
// sample keeps every candidate's grid larger than the GPU
constexpr int64_t kTuneSampleRows = 16384;
// Galerkin levels from 4096 rows are tuned (a whole level up to the sample
// size): below that the fixed rule (pairs of targets, 128 threads) holds
constexpr int64_t kTuneMinRows = 4096;

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
    // lanes per neighbour parent; the block gather by four lanes per block
    // row (gathers 0 and 1 lose to it at every level size measured, and each
    // candidate costs cold-start time; both stay available as forced shapes)
    for (int spp : {1, 2, 4})
      for (int gather : {2}) {
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

// Galerkin kernel of level k (the tile kernel over pairs of targets with 4, 8
// or 16 lanes per pair at 256 or 128 threads per CTA, or, where a tile's
// window does not fit shared memory, k_galerkin_rows, k_galerkin_warp or
// k_galerkin_warprow), timed on kTuneSampleRows rows in the middle of the
// level (rewritten by the full launch).
template <typename T>
void tune_galerkin_variant(gamblet_ctx* h, int k, GalerkinGeom& gg, const T* Ahat,
                           const T* Rhat, T* Acell) {
  if (!h->opts.autotune || gg.nrow < kTuneMinRows) return;
  const std::string key = h->plan->key + "/galerkin/" + std::to_string(k) + "/" +
                          std::to_string(sizeof(T));
  // code: variant + 16 * (tile kernels launched with 128 threads per CTA)
  int v = gg.variant;
  if (!tune_lookup(key, &v)) {
    cudaStream_t s = h->s;
    GalerkinGeom gt = gg;
    gt.i_begin = (gg.nrow / 2 / kTuneSampleRows) * kTuneSampleRows;
    gt.i_end = std::min(gt.i_begin + kTuneSampleRows, gg.nrow);
    float best = 1e30f;
    // where the tile fits: the pair-of-targets tile kernels (6, 7, 8), which
    // beat the single-target ones (3, 4, 5) and the row kernels (0, 1, 2) on
    // every level measured, at 256 and 128 threads; else the row kernels
    const bool tile = galerkin_tile_smem_bytes(gg, sizeof(T)) <= 227 * 1024;
    for (int cand : {0, 1, 2, 6, 7, 8})
      for (int half : {0, 1}) {
        if (tile != (cand >= 3)) continue;
        if (cand == 2 && 8 * sizeof(T) * 4 * ((size_t)gg.NB + gg.nwin) > 227 * 1024) continue;
        if (half && cand < 3) continue;
        gt.variant = cand;
        gt.tile_threads = half ? 128 : 256;
        const float ms = time_on_stream(s, [&] {
          launch_galerkin<T>(Ahat, Rhat, h->lv[k].pmask, gt, Acell, s);
        });
        if (ms < best) {
          best = ms;
          v = cand + 16 * half;
        }
      }
    tune_store(key, v);
  }
  gg.variant = v % 16;
  gg.tile_threads = v >= 16 ? 128 : 256;
}

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

template bool cluster_geometry<float>(const PatchPcgGeom&, const PlanLevel&, PatchClusterGeom&);
template bool cluster_geometry<double>(const PatchPcgGeom&, const PlanLevel&, PatchClusterGeom&);
template int tune_patch_shape<float>(gamblet_ctx*, int, PatchPcgGeom&, float*, const PatchMmaGeom*,
                                     const bool*);
template int tune_patch_shape<double>(gamblet_ctx*, int, PatchPcgGeom&, double*,
                                      const PatchMmaGeom*, const bool*);
template void tune_galerkin_variant<float>(gamblet_ctx*, int, GalerkinGeom&, const float*,
                                           const float*, float*);
template void tune_galerkin_variant<double>(gamblet_ctx*, int, GalerkinGeom&, const double*,
                                            const double*, double*);
template int tuned_cg_spp<float>(gamblet_ctx*, int, const CgLevel&);
template int tuned_cg_spp<double>(gamblet_ctx*, int, const CgLevel&);

}  // namespace hs
}  // namespace gb
