// grad.cu - the gradient of J = 1/2 |u_loc - u_obs|^2 through the one-pass
// localized transform (the reverse mode of Algorithm 2's solve and localized
// setup; the paper differentiates nothing, the reading is stated where the
// reverse pass is designed) and its C ABI entry point gamblet_grad_onepass.
#include "host.cuh"

namespace gb {
namespace hs {

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
  const char* dpack = tmp.upload_owned(pack, pack->bytes, s);
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

}  // namespace hs
}  // namespace gb

extern "C" {

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

}  // extern "C"
