// solve_host.cu - the solve phase behind the C ABI: the gamblet operator
// G (restriction chain, Eq. eqyguugy6t; all level CGs batched, Eq.
// eqsdjoejddi1; coarsest solve; prolongation and summation, Theorem
// thddwedmgugyug), its use as the preconditioner of a float64 flexible CG on
// A^(q) (Sec. 5.4), several right-hand sides per pass, truncated solves,
// compression in the normalised basis (Sec. 5.1) and the extreme eigenvalues
// of B^(k) (Theorem thmodhehiudhehd).
#include "host.cuh"

namespace gb {
namespace hs {

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
    h->cg_bytes_spmv[l] = (L.Bq ? 32.0 * L.nhoff : 9.0 * sz * L.noff) * (double)L.npar +
                          sz * 6.0 * L.npar;
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
// the gradient through the one-pass transform (grad.cu) uses both precisions
template float* as_T<float>(gamblet_ctx*, double*, void*, int64_t, bool);
template double* as_T<double>(gamblet_ctx*, double*, void*, int64_t, bool);
template void apply_G<float>(gamblet_ctx*, const float*, float*, int);
template void apply_G<double>(gamblet_ctx*, const double*, double*, int);

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
        // u += (d1 / d0) p, r -= (d1 / d0) q, d2 = r.r
        launch_update_ur(nq, d + 1, d + 0, h->p64, h->q64, h->u64, h->r64, d + 2, s);
        CK(cudaMemcpyAsync(h->dots_h, d, sizeof(double) * 4, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        relres = std::sqrt(h->dots_h[2]) / gnorm;
        if (!(relres == relres)) fail(GAMBLET_ERR_NOT_SPD, "outer iteration produced NaN");
        if (relres <= h->opts.refine_tol) break;
        rT = as_T<T>(h, h->r64, h->rT, nq, true);
        apply_G<T>(h, rT, zT, 0);
        // d3 = z.q ; p = z - (d3 / d0) p
        if (is_f32<T>())
          launch_widen_dot(nq, (const float*)zT, h->z64, h->q64, d + 3, s);
        else
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

// The coalesced detail blocks Bd of level k, built on first use where the
// setup skipped them (the level CG of the mixed path reads its block records
// instead); they live in the handle's pool until gamblet_destroy.
template <typename T>
const T* level_detail_blocks(gamblet_ctx* h, int k) {
  LevelDev& L = h->lv[k];
  if (!L.Bd) {
    T* Bd = h->pool.alloc<T>((int64_t)L.noff * 9 * L.npar);
    launch_extract_detail<T>((const T*)L.Ahat, L.noff, L.npar, Bd, h->s);
    L.Bd = Bd;
  }
  return (const T*)L.Bd;
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
    launch_coef_max<T>((const T*)L.w, level_detail_blocks<T>(h, k), L.o0, L.npar, L.pmask, dv, s);
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
    launch_coef_threshold<T>((T*)L.w, level_detail_blocks<T>(h, k), L.o0, L.npar, L.pmask, thr,
                             dv + 1, s);
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
  const T* Bd = level_detail_blocks<T>(h, k);
  auto apply = [&](const double* x, double* y) {
    if (construction == 1) {
      launch_detail_basis(L.npar, L.pmask, x, t1, 1, s);
      launch_detail_spmv<T>(Bd, L.off, L.noff, Lpar, L.npar, t1, y, s);
      launch_detail_basis(L.npar, L.pmask, y, y, 0, s);
    } else {
      launch_detail_spmv<T>(Bd, L.off, L.noff, Lpar, L.npar, x, y, s);
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

template void build_cg_graph<float>(gamblet_ctx*, int, double, int);
template void build_cg_graph<double>(gamblet_ctx*, int, double, int);

}  // namespace hs
}  // namespace gb

extern "C" {

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

}  // extern "C"
