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
// The symbolic plan is built in plan.cu, launch shapes are tuned in tune.cu,
// the gradient through the one-pass transform is grad.cu, the operator
// getters getters.cu; host.cuh holds the handle and the shared helpers.
#include "host.cuh"

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

namespace {

thread_local std::string g_last_error;

}  // namespace


namespace gb {
namespace hs {
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
  const char* dplan = P.upload_owned(plan, plan->packed, s);  // every plan table in one copy
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
    gg.t1 = plan_table<int2>(dplan, pl, PlanLevel::kT1);
    gg.nt1u = S.n_read;
    gg.nitems = (int)S.t1_items.size();
    gg.t1_items = plan_table<int4>(dplan, pl, PlanLevel::kT1Items);
    gg.nt2 = (int)S.t2.size();
    gg.t2 = plan_table<int4>(dplan, pl, PlanLevel::kT2);
    gg.t2p_ptr = plan_table<int>(dplan, pl, PlanLevel::kT2pPtr);
    gg.t2p = plan_table<int>(dplan, pl, PlanLevel::kT2p);
    gg.nt3 = (int)S.t3p_ptr.size() - 1;
    gg.t3 = plan_table<int4>(dplan, pl, PlanLevel::kT3);
    gg.t3p_ptr = plan_table<int>(dplan, pl, PlanLevel::kT3pPtr);
    gg.t3p = plan_table<uint32_t>(dplan, pl, PlanLevel::kT3p);
    // 2 x 2 row tiles while their window boxes stay small enough for
    // several CTAs per SM, else the warp-cooperative kernel; the autotuner
    // decides on large levels
    gg.variant = galerkin_tile_smem_bytes(gg, sizeof(T)) <= 100 * 1024 ? 7 : 1;
    gg.tile_threads = gg.variant == 7 ? 128 : 256;  // small levels: more CTAs to fill the GPU
    if (sizeof(T) * 4 * ((size_t)NB + (size_t)gg.nwin) > 227 * 1024)
      fail(GAMBLET_ERR_UNSUPPORTED, "Galerkin window exceeds shared memory");
    T* Acell = P.alloc<T>((int64_t)gg.nout * L.npar);
    if (h->opts.galerkin_variant >= 0 && h->opts.galerkin_variant <= 8) {
      gg.variant = h->opts.galerkin_variant;
      gg.tile_threads = 256;
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
    T* Dinv = P.alloc<T>(9 * L.npar);
    const PlanLevel& pl = h->plan->lv[k];
    const bool records = is_f32<T>() && h->opts.level_tol >= kHalfLevelTol && !pl.hidx.empty();
    // with the records the CG never reads the coalesced copy Bd; the
    // diagnostics that do (compression, condition estimates) build it on
    // first use (level_detail_blocks)
    T* Bd = records ? nullptr : P.alloc<T>((int64_t)L.noff * 9 * L.npar);
    unsigned* amax = records ? P.alloc<unsigned>(1) : nullptr;
    launch_cg_level_setup<T>((const T*)L.Ahat, L.noff, o0, L.npar, L.pmask, Bd, Dinv, amax, s);
    L.Bd = Bd;
    L.Dinv = Dinv;
    L.Bq = nullptr;
    L.bq_scale = nullptr;
    L.nhoff = 0;
    L.hoff = nullptr;
    if (records) {
      // the level CG's product reads each block as one 32-byte float16 record
      // (two 16-byte loads instead of nine scalar ones), with a rounding of
      // 2^-11 relative per entry, far below the level tolerance; B^(k) is
      // symmetric, so only the blocks of the half-plane offsets are stored
      L.nhoff = (int)pl.hidx.size();
      L.hoff = plan_table<int2>(h->dplan, pl, PlanLevel::kHOff);
      L.Bq = P.alloc<uint4>((int64_t)L.nhoff * L.npar * 2);
      L.bq_scale = P.alloc<float>(1);
      launch_cg_block_records((const float*)L.Ahat, plan_table<int>(h->dplan, pl, PlanLevel::kHIdx),
                              L.nhoff, L.npar, amax, L.Bq, L.bq_scale, s);
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
      c.hoff = L.hoff;
      c.nhoff = L.nhoff;
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

gamblet_status set_error(const GbError& e) {
  g_last_error = e.msg;
  return e.st;
}

}  // namespace hs
}  // namespace gb

namespace gb {
namespace hs {

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
    if (h->opts.galerkin_variant < -1 || h->opts.galerkin_variant > 8)
      fail(GAMBLET_ERR_INVALID_ARG, "galerkin_variant must be -1 or 0..8");
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
    to_host(&ends[2 * p], A[p].rowptr, 1);
    to_host(&ends[2 * p + 1], A[p].rowptr + b.n, 1);
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

}  // namespace hs
}  // namespace gb

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
    to_host(kh, K_ref, 16);
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
    to_host(kh, K_ref, 16);
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
