// plan.cu - the symbolic plan of a geometry: everything the localized setup
// (Algorithm 2 with Definition defb) derives from the geometry alone - the
// patch neighbourhoods i^rho (Sec. 4.10), the block offset sets of every
// level A^(k) (exact Minkowski sums of the interpolation and operator
// supports), the patch block lists, the Galerkin pair lists (Eq. eqhuhiuv)
// and the tables of the tensor-core patch windows - built once per geometry
// and cached process-wide; and a host-only check of those tables against
// their definitions (gamblet_plan_check).
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "host.cuh"

namespace gb {
namespace hs {

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
  // phase 2: the output targets of the tile and, per target, the window
  // positions its patch reaches
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
  std::vector<char> read(W * W, 0);  // window positions phase 2 reads
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
      read[u] = 1;
    }
    tl.push_back(std::move(t));
  }
  // the window products t_r(u) are kept only at the positions phase 2 reads,
  // numbered in box order (cid), so that a tile's shared memory holds
  // |read| instead of W^2 positions; the pair lists below carry cid
  std::vector<int> cid(W * W, -1);
  int ncid = 0;
  for (int u = 0; u < W * W; ++u)
    if (read[u]) cid[u] = ncid++;
  if (W * W > 65536) fail(GAMBLET_ERR_UNSUPPORTED, "window too large for tiled Galerkin");
  // the same targets in horizontal pairs (c, c + (1, 0)) where both exist
  // (tl is in (y, x) order here): one list of window positions u per pair,
  // the union of the two targets' lists, with both targets' j at u
  {
    struct Group {
      int4 a, b;
      std::vector<uint32_t> ent;
    };
    std::vector<Group> gl;
    const int4 none = make_int4(0, 0, -1, -1);
    for (size_t e = 0; e < tl.size(); ++e) {
      Group gr;
      gr.a = tl[e].t;
      gr.b = none;
      std::map<int, std::pair<int, int>> at;  // u -> (j of a, j of b)
      for (int pu : tl[e].pairs) at[pu >> 8] = {pu & 0xff, 0xff};
      if (e + 1 < tl.size() && tl[e + 1].t.y == tl[e].t.y && tl[e + 1].t.x == tl[e].t.x + 1) {
        gr.b = tl[e + 1].t;
        for (int pu : tl[e + 1].pairs) {
          auto it = at.find(pu >> 8);
          if (it == at.end()) at[pu >> 8] = {0xff, pu & 0xff};
          else it->second.second = pu & 0xff;
        }
        ++e;
      }
      for (const auto& kv : at) {
        if (kv.first > 0xffff) fail(GAMBLET_ERR_UNSUPPORTED, "window too large for tiled Galerkin");
        gr.ent.push_back((uint32_t)cid[kv.first] | ((uint32_t)kv.second.first << 16) |
                         ((uint32_t)kv.second.second << 24));
      }
      gl.push_back(std::move(gr));
    }
    std::stable_sort(gl.begin(), gl.end(), [](const Group& a, const Group& b) {
      return a.ent.size() > b.ent.size();
    });
    S.t3p_ptr.assign(1, 0);
    for (const Group& gr : gl) {
      S.t3.push_back(gr.a);
      S.t3.push_back(gr.b);
      S.t3p.insert(S.t3p.end(), gr.ent.begin(), gr.ent.end());
      S.t3p_ptr.push_back((int)S.t3p.size());
    }
  }
  std::stable_sort(tl.begin(), tl.end(), [](const Target& a, const Target& b) {
    return a.pairs.size() > b.pairs.size();
  });
  S.t2p_ptr.assign(1, 0);
  for (const Target& t : tl) {
    S.t2.push_back(t.t);
    for (int pu : t.pairs) S.t2p.push_back((pu & 0xff) | (cid[pu >> 8] << 8));
    S.t2p_ptr.push_back((int)S.t2p.size());
  }
  // phase 1: the block list of every window position that phase 2 reads (the
  // others - the part of the window below the half-plane targets' patches -
  // are left out: their products would never be used)
  S.t1_ptr.assign((size_t)W * W + 1, 0);
  for (int uy = 0; uy < W; ++uy)
    for (int ux = 0; ux < W; ++ux) {
      const int u = uy * W + ux;
      for (int o = 0; o < O_k.size() && read[u]; ++o) {
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
  // the positions phase 2 reads, by decreasing block count: the threads of a
  // CTA take them round-robin, so the lanes of a warp walk lists of about
  // the same length and the threads' totals differ by at most one list
  // phase-1 work items: the read positions with their block lists, sorted by
  // decreasing length; the kernel deals them to its threads in alternating
  // direction, so that the threads' totals even out
  for (int u = 0; u < W * W; ++u)
    if (read[u])
      S.t1_items.push_back(make_int4(u | (cid[u] << 16), S.t1_ptr[u], S.t1_ptr[u + 1], 0));
  std::stable_sort(S.t1_items.begin(), S.t1_items.end(), [](const int4& a, const int4& b) {
    return a.z - a.y > b.z - b.y;
  });
  S.n_read = ncid;
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
    // half-plane of the symmetric block stencil (the level CG stores one
    // block per pair of opposite offsets)
    bool sym = true;
    for (const int2& d : pl.S.O.v) sym = sym && pl.S.O.find(-d.x, -d.y) >= 0;
    for (int o = 0; o < pl.S.O.size() && sym; ++o) {
      const int2 d = pl.S.O.v[o];
      if (d.y > 0 || (d.y == 0 && d.x >= 0)) {
        pl.hidx.push_back(o);
        pl.hoff.push_back(d);
      }
    }
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
    pl.table_off[PlanLevel::kT1] = put_v(S.t1);
    pl.table_off[PlanLevel::kT2] = put_v(S.t2);
    pl.table_off[PlanLevel::kT2pPtr] = put_v(S.t2p_ptr);
    pl.table_off[PlanLevel::kT2p] = put_v(S.t2p);
    pl.table_off[PlanLevel::kT1Items] = put_v(S.t1_items);
    pl.table_off[PlanLevel::kT3] = put_v(S.t3);
    pl.table_off[PlanLevel::kT3pPtr] = put_v(S.t3p_ptr);
    pl.table_off[PlanLevel::kT3p] = put_v(S.t3p);
    pl.table_off[PlanLevel::kOffNext] = put_v(pl.O_next.v);
    pl.table_off[PlanLevel::kMapNext] = put_v(pl.map_next);
    pl.table_off[PlanLevel::kHIdx] = put_v(pl.hidx);
    pl.table_off[PlanLevel::kHOff] = put_v(pl.hoff);
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

}  // namespace hs
}  // namespace gb

namespace gb {
namespace hs {

// Consistency of a plan's tables with their definitions, derived a second way
// (from the contributions each table must carry rather than the way the
// builder enumerates them).  counts: levels, t1 entries, phase-1 items,
// phase-2 target incidences, half-plane offsets.
void check_plan(const Plan& P, int q, const OffSet& N, int64_t* counts) {
  auto need = [](bool ok, int k, const std::string& what) {
    if (!ok) fail(GAMBLET_ERR_INVALID_ARG, "plan level " + std::to_string(k) + ": " + what);
  };
  const int NB = N.size();
  int64_t n_t1 = 0, n_items = 0, n_inc = 0, n_half = 0;
  for (int k = q; k >= 2; --k) {
    const PlanLevel& pl = P.lv[k];
    const SymLevel& S = pl.S;
    const int Lpar = 1 << (k - 1);
    // half-plane of the level stencil: one of d, -d for every d != 0, and 0
    std::vector<int> want_h;
    for (int o = 0; o < S.O.size(); ++o) {
      const int2 d = S.O.v[o];
      need(S.O.find(-d.x, -d.y) >= 0, k, "block stencil not symmetric");
      if (d.y > 0 || (d.y == 0 && d.x >= 0)) want_h.push_back(o);
    }
    need(pl.hidx == want_h && pl.hoff.size() == want_h.size(), k, "half-plane offsets");
    for (size_t h = 0; h < want_h.size(); ++h)
      need(pl.hoff[h].x == S.O.v[want_h[h]].x && pl.hoff[h].y == S.O.v[want_h[h]].y, k,
           "half-plane offset values");
    n_half += (int64_t)want_h.size();
    // tile geometry: row r of the 2 x 2 tile sits at rv[r] from the origin
    const int W = S.tile_W, wmin = S.tile_wmin;
    const int2 rv[4] = {make_int2(0, 0), make_int2(1, 0), make_int2(0, 1), make_int2(1, 1)};
    auto box = [&](int x, int y) {
      const int ux = x - wmin, uy = y - wmin;
      return (ux >= 0 && ux < W && uy >= 0 && uy < W) ? uy * W + ux : -1;
    };
    // positions read by phase 2: c + N_j for every output target c of a row,
    // where some row's window holds it
    std::set<int> win4;
    for (int r = 0; r < 4; ++r)
      for (const int2& w : S.WIN.v) {
        const int u = box(rv[r].x + w.x, rv[r].y + w.y);
        need(u >= 0, k, "window outside the tile box");
        win4.insert(u);
      }
    std::set<int> read;
    std::map<std::pair<int, int>, std::set<std::pair<int, int>>> inc;  // target -> (j, u)
    for (int r = 0; r < 4; ++r)
      for (const int2& d : S.Sp.v) {
        const int cx = rv[r].x + d.x, cy = rv[r].y + d.y;
        for (int j = 0; j < NB; ++j) {
          const int u = box(cx + N.v[j].x, cy + N.v[j].y);
          if (u >= 0 && win4.count(u)) {
            inc[{cx, cy}].insert({j, u});
            read.insert(u);
          }
        }
        inc[{cx, cy}];  // targets without positions still carry outputs
      }
    // phase-1 items: the read positions, once each, with their box-order index
    std::vector<int> cid_of(W * W, -1);
    {
      int c = 0;
      for (int u : read) cid_of[u] = c++;
    }
    need((int)S.t1_items.size() == (int)read.size() && S.n_read == (int)read.size(), k,
         "phase-1 items do not match the read positions");
    std::set<int> seen;
    for (size_t e = 0; e < S.t1_items.size(); ++e) {
      const int4 it = S.t1_items[e];
      const int u = it.x & 0xffff, c = it.x >> 16;
      need(read.count(u) && !seen.count(u), k, "phase-1 item position");
      seen.insert(u);
      need(c == cid_of[u], k, "phase-1 item index");
      need(it.y == S.t1_ptr[u] && it.z == S.t1_ptr[u + 1], k, "phase-1 item range");
      if (e > 0) need(it.z - it.y <= S.t1_items[e - 1].z - S.t1_items[e - 1].y, k, "item order");
    }
    n_items += (int64_t)S.t1_items.size();
    // phase 1: every contribution A_hat[o][u] R_hat_r(j) with u = r + N_j - O_o
    // at a read position, exactly once, and nothing else
    std::set<std::tuple<int, int, int, int>> want1, have1;  // (u, o, r, j)
    for (int r = 0; r < 4; ++r)
      for (int j = 0; j < NB; ++j)
        for (int o = 0; o < S.O.size(); ++o) {
          const int wx = N.v[j].x - S.O.v[o].x, wy = N.v[j].y - S.O.v[o].y;
          if (std::abs(wx) > Lpar - 1 || std::abs(wy) > Lpar - 1) continue;
          const int u = box(rv[r].x + wx, rv[r].y + wy);
          if (u >= 0 && read.count(u)) want1.insert({u, o, r, j});
        }
    for (int u = 0; u < W * W; ++u)
      for (int e = S.t1_ptr[u]; e < S.t1_ptr[u + 1]; ++e) {
        for (int r = 0; r < 4; ++r) {
          const int j = ((unsigned)S.t1[e].y >> (8 * r)) & 0xffu;
          if (j != 0xff) {
            need(read.count(u) > 0, k, "phase-1 entry at an unread position");
            const bool fresh = have1.insert({u, S.t1[e].x, r, j}).second;
            need(fresh, k, "phase-1 contribution listed twice");
          }
        }
        ++n_t1;
      }
    need(have1 == want1, k, "phase-1 contributions");
    // phase 2, single targets: row offsets and the pair lists
    std::map<std::pair<int, int>, std::set<std::pair<int, int>>> got2, got3;
    for (size_t e = 0; e < S.t2.size(); ++e) {
      const int4 t = S.t2[e];
      const int d[4] = {(int)(short)(t.z & 0xffff), t.z >> 16, (int)(short)(t.w & 0xffff),
                        t.w >> 16};
      for (int r = 0; r < 4; ++r)
        need(d[r] == S.Sp.find(t.x - rv[r].x, t.y - rv[r].y), k, "phase-2 output offsets");
      auto& g = got2[{t.x, t.y}];
      for (int q2 = S.t2p_ptr[e]; q2 < S.t2p_ptr[e + 1]; ++q2) {
        const int j = S.t2p[q2] & 0xff, c = S.t2p[q2] >> 8;
        need(c >= 0 && c < (int)read.size(), k, "phase-2 position index");
        g.insert({j, c});
      }
    }
    // phase 2, pairs of targets (c, c + (1, 0))
    need((int)S.t3.size() == 2 * ((int)S.t3p_ptr.size() - 1), k, "pair records");
    for (size_t e = 0; 2 * e < S.t3.size(); ++e) {
      const int4 a = S.t3[2 * e], b = S.t3[2 * e + 1];
      const bool has_b = (b.z != -1 || b.w != -1);
      if (has_b) need(b.x == a.x + 1 && b.y == a.y, k, "pair partner");
      auto& ga = got3[{a.x, a.y}];
      for (int q3 = S.t3p_ptr[e]; q3 < S.t3p_ptr[e + 1]; ++q3) {
        const uint32_t pu = S.t3p[q3];
        const int c = (int)(pu & 0xffffu), ja = (int)((pu >> 16) & 0xffu), jb = (int)(pu >> 24);
        need(c < (int)read.size() && (ja != 0xff || jb != 0xff), k, "pair entry");
        if (ja != 0xff) ga.insert({ja, c});
        if (jb != 0xff) {
          need(has_b, k, "pair entry for a missing partner");
          got3[{b.x, b.y}].insert({jb, c});
        }
      }
      if (has_b) got3[{b.x, b.y}];
    }
    // both lists carry exactly the incidences of the definition
    std::map<std::pair<int, int>, std::set<std::pair<int, int>>> want2;
    for (const auto& kv : inc) {
      auto& w = want2[kv.first];
      for (const auto& ju : kv.second) w.insert({ju.first, cid_of[ju.second]});
      n_inc += (int64_t)kv.second.size();
    }
    need(got2 == want2, k, "phase-2 pair lists (single targets)");
    need(got3 == want2, k, "phase-2 pair lists (pairs of targets)");
    // patch matrices (Definition defb): one stored block per neighbour pair
    // ja >= jb coupled through O_k, in bank-coloured slots; each row's
    // adjacency walks every block touching it (the other side transposed)
    std::set<std::tuple<int, int, int>> wantb, haveb;  // (ja, jb, o)
    for (int a = 0; a < NB; ++a)
      for (int b = 0; b < NB; ++b) {
        const int o = S.O.find(N.v[b].x - N.v[a].x, N.v[b].y - N.v[a].y);
        need(S.pair_idx[(size_t)a * NB + b] == o, k, "patch pair index");
        if (a >= b && o >= 0) wantb.insert({a, b, o});
      }
    for (const int4& hb : pl.half)
      if (hb.x >= 0) need(haveb.insert({hb.x, hb.y, hb.z}).second, k, "patch block stored twice");
    need(haveb == wantb, k, "patch blocks");
    for (int j = 0; j < NB; ++j) {
      std::set<std::pair<int, int>> wanta, havea;  // (other, transposed) of each touching block
      for (const auto& t : wantb) {
        if (std::get<0>(t) == j) wanta.insert({std::get<1>(t), 0});
        else if (std::get<1>(t) == j) wanta.insert({std::get<0>(t), 1});
      }
      for (int e = pl.adj_ptr[j]; e < pl.adj_ptr[j + 1]; ++e) {
        const int4 ad = pl.adj[e];
        const int4 hb = pl.half[ad.x];
        need(ad.z == 0 ? (hb.x == j && hb.y == ad.y) : (hb.y == j && hb.x == ad.y), k,
             "patch adjacency entry");
        havea.insert({ad.y, ad.z});
      }
      need(havea == wanta && pl.adj_ptr[j + 1] - pl.adj_ptr[j] == (int)wanta.size(), k,
           "patch adjacency of a row");
      need(pl.half[pl.diag_h[j]].x == j && pl.half[pl.diag_h[j]].y == j, k, "patch diagonal");
    }
    // tensor-core windows of G x G cells: the union of the patches, the
    // membership bits, the union's blocks, right-hand-side offsets and the
    // output map
    for (int G = 1; G <= 2; ++G) {
      const MmaWin& Wn = pl.mwin[G - 1];
      std::set<std::pair<int, int>> U;
      for (int c = 0; c < G * G; ++c)
        for (const int2& o : N.v) U.insert({(c & 1) + o.x, (c >> 1) + o.y});
      need((int)Wn.U.size() == (int)U.size() && Wn.nU == (int)U.size() && Wn.NP == G * G, k,
           "window union size");
      std::map<std::pair<int, int>, int> uidx;
      for (int u = 0; u < Wn.nU; ++u) {
        need(U.count({Wn.U[u].x, Wn.U[u].y}) && !uidx.count({Wn.U[u].x, Wn.U[u].y}), k,
             "window union member");
        uidx[{Wn.U[u].x, Wn.U[u].y}] = u;
        int bits = 0;
        for (int c = 0; c < G * G; ++c)
          if (N.find(Wn.U[u].x - (c & 1), Wn.U[u].y - (c >> 1)) >= 0) bits |= 1 << c;
        need(Wn.ubits[u] == bits, k, "window membership bits");
        for (int c = 0; c < G * G; ++c)
          need(Wn.rhs_o[(size_t)c * Wn.nU + u] ==
                   S.O.find((c & 1) - Wn.U[u].x, (c >> 1) - Wn.U[u].y),
               k, "window right-hand-side offset");
      }
      std::set<std::tuple<int, int, int>> wantw, havew;
      for (int a = 0; a < Wn.nU; ++a)
        for (int b = 0; b < a; ++b) {
          const int o = S.O.find(Wn.U[b].x - Wn.U[a].x, Wn.U[b].y - Wn.U[a].y);
          if (o >= 0) wantw.insert({a, b, o});
        }
      for (const int4& pr : Wn.pairs) havew.insert({pr.x, pr.y, pr.z});
      need(havew == wantw && Wn.pairs.size() == wantw.size(), k, "window blocks");
      for (int c = 0; c < G * G; ++c)
        for (int j = 0; j < NB; ++j)
          need(Wn.outmap[(size_t)c * NB + j] ==
                   uidx.at({(c & 1) + N.v[j].x, (c >> 1) + N.v[j].y}),
               k, "window output map");
      need(Wn.diag_o == S.O.find(0, 0), k, "window diagonal offset");
    }
    // the level-(k-1) block stencil: every coupling d of the cell stencil S
    // between child c of a parent and some child of another lies in O_(k-1),
    // and the conversion map points at d in the computed half-plane (or at
    // -d, read transposed)
    if (k - 1 >= 2) {
      const OffSet& On = pl.O_next;
      const int Lp = 1 << (k - 2);
      auto decodes_to = [&](int m, int dx, int dy) {
        if (m >= 0) return S.Sp.v[m].x == dx && S.Sp.v[m].y == dy;
        if (m <= -2) return S.Sp.v[-m - 2].x == -dx && S.Sp.v[-m - 2].y == -dy;
        return false;
      };
      for (const int2& d : S.S.v)
        for (int c = 0; c < 4; ++c)
          for (int cc = 0; cc < 4; ++cc) {
            const int ex = d.x - ((cc & 1) - (c & 1)), ey = d.y - ((cc >> 1) - (c >> 1));
            if ((ex & 1) || (ey & 1)) continue;
            const int Dx = ex / 2, Dy = ey / 2;
            if (std::abs(Dx) > Lp - 1 || std::abs(Dy) > Lp - 1) continue;
            const int o = On.find(Dx, Dy);
            need(o >= 0, k, "cell coupling missing from the next block stencil");
            need(decodes_to(pl.map_next[(size_t)o * 16 + c * 4 + cc], d.x, d.y), k,
                 "block conversion map");
          }
    }
  }
  if (counts) {
    counts[0] = q - 1;
    counts[1] = n_t1;
    counts[2] = n_items;
    counts[3] = n_inc;
    counts[4] = n_half;
  }
}

}  // namespace hs
}  // namespace gb

extern "C" gamblet_status gamblet_plan_check(int32_t q, double rho, int32_t nbr_rule,
                                             int64_t* counts) {
  using namespace gb::hs;
  try {
    if (q < 2 || q > 12) fail(GAMBLET_ERR_INVALID_ARG, "q must be in [2, 12]");
    if (!(rho > 0) || rho > 8) fail(GAMBLET_ERR_INVALID_ARG, "rho must be in (0, 8]");
    if (nbr_rule != 0 && nbr_rule != 1) fail(GAMBLET_ERR_INVALID_ARG, "nbr_rule must be 0 or 1");
    OffSet Oq;  // the Q1 operator's 3 x 3 block stencil on a full square
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) Oq.add(dx, dy);
    const OffSet N = neighbour_offsets(rho, nbr_rule);
    const auto plan = build_plan(q, Oq, N, "check");
    check_plan(*plan, q, N, counts);
    return GAMBLET_OK;
  } catch (const GbError& e) {
    return set_error(e);
  } catch (const std::exception& e) {
    return set_error(GbError{GAMBLET_ERR_INVALID_ARG, e.what()});
  }
}
