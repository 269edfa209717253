// getters.cu - the level operators of a handle as COO triplets in the
// caller's numbering (gamblet_get_operator): A^(k), R^(k-1,k) and B^(k) of
// Sec. 4 read back from the device blocks and transformed back from the
// per-parent Helmert basis.
#include "host.cuh"

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

}  // extern "C"
