// Step 1 on the host (Sec. 3, Sec. 6 step 1, Sec. 7.1): overlapping subdomains,
// r-hop extensions, index sets I and B, the batched row spaces, sparsity patterns,
// assembly incidence and the interface pairs used by the projection of step 3.
#include "mor_plan.h"

#include <algorithm>
#include <cmath>
#include <atomic>
#include <thread>

#include "../../include/mor.h"

namespace mor {
namespace {

template <class F>
void parallel_for(int n, int n_threads, F f) {
  if (n <= 0) return;
  int nt = std::max(1, std::min(n_threads, n));
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      int i;
      while ((i = next.fetch_add(1)) < n) f(i, t);
    });
  for (auto& x : th) x.join();
}

// per-thread scratch, stamped with subdomain id + 1 so it never needs clearing
struct Scratch {
  std::vector<int32_t> ball, vert, loc_mark, loc, wmark, wloc;
  std::vector<uint8_t> tplus, tomega;
  void init(int64_t n_nodes, int64_t n_tets) {
    ball.assign(n_nodes, 0);
    vert.assign(n_nodes, 0);
    loc_mark.assign(n_nodes, 0);
    loc.assign(n_nodes, 0);
    wmark.assign(n_nodes, 0);
    wloc.assign(n_nodes, 0);
    tplus.assign(n_tets, 0);
    tomega.assign(n_tets, 0);
  }
};

// variable-length rows of one subdomain before packing
struct LocalRows {
  std::vector<int64_t> ptr{0};
  std::vector<int32_t> cols;  // local column indices
  std::vector<int64_t> inc_ptr{0};
  std::vector<int32_t> inc_tet;
  std::vector<uint32_t> inc_code;
};

struct SubOut {
  LocalRows P, W;
  std::vector<int32_t> w2p_local;  // omega dof -> plus-local index
  std::vector<int32_t> o2w_local;  // owned dof -> omega-local index
  std::string err;
};

void build_rows(const std::vector<int32_t>& row_nodes, const int32_t* tets,
                const std::vector<int64_t>& n2t_ptr, const std::vector<int32_t>& n2t,
                const std::vector<uint8_t>& tflag, const std::vector<int32_t>& mark,
                const std::vector<int32_t>& loc, int32_t stamp, LocalRows& R) {
  std::vector<int32_t> cand;
  for (int32_t g : row_nodes) {
    cand.clear();
    for (int64_t q = n2t_ptr[g]; q < n2t_ptr[g + 1]; ++q) {
      int32_t e = n2t[q];
      if (!tflag[e]) continue;
      for (int b = 0; b < 4; ++b) {
        int32_t vb = tets[4 * (int64_t)e + b];
        if (mark[vb] == stamp) cand.push_back(loc[vb]);
      }
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    R.cols.insert(R.cols.end(), cand.begin(), cand.end());
    R.ptr.push_back((int64_t)R.cols.size());
    for (int64_t q = n2t_ptr[g]; q < n2t_ptr[g + 1]; ++q) {
      int32_t e = n2t[q];
      if (!tflag[e]) continue;
      uint32_t code = 0;
      for (int b = 0; b < 4; ++b) {
        int32_t vb = tets[4 * (int64_t)e + b];
        if (vb == g) code |= (uint32_t)b;
        uint32_t slot = kNoSlot;
        if (mark[vb] == stamp) {
          auto it = std::lower_bound(cand.begin(), cand.end(), loc[vb]);
          slot = (uint32_t)(it - cand.begin());
        }
        code |= slot << (2 + 7 * b);
      }
      R.inc_tet.push_back(e);
      R.inc_code.push_back(code);
    }
    R.inc_ptr.push_back((int64_t)R.inc_tet.size());
  }
}

void make_tiles(const std::vector<int64_t>& begin, const std::vector<int64_t>& end,
                HostTiles& t) {
  int n_sd = (int)begin.size();
  t.lo.resize(n_sd);
  t.hi.resize(n_sd);
  for (int i = 0; i < n_sd; ++i) {
    t.lo[i] = (int32_t)t.sd.size();
    for (int64_t r = begin[i]; r < end[i]; r += kTileRows) {
      t.sd.push_back(i);
      t.r0.push_back((int32_t)r);
      t.r1.push_back((int32_t)std::min<int64_t>(end[i], r + kTileRows));
    }
    t.hi[i] = (int32_t)t.sd.size();
  }
}

void pack_ell(const std::vector<SubOut>& outs, bool plus, const std::vector<int64_t>& off,
              int64_t n_rows, HostEll& E, std::vector<int64_t>& inc_ptr,
              std::vector<int32_t>& inc_tet, std::vector<uint32_t>& inc_code) {
  int32_t W = 0;
  for (auto& o : outs) {
    const LocalRows& R = plus ? o.P : o.W;
    for (size_t r = 0; r + 1 < R.ptr.size(); ++r)
      W = std::max<int32_t>(W, (int32_t)(R.ptr[r + 1] - R.ptr[r]));
  }
  int64_t n_slices = (n_rows + kSlice - 1) / kSlice;
  E.n_rows = n_rows;
  E.W = W;
  E.width.assign(n_slices, 0);
  E.col.assign(n_slices * kSlice * (int64_t)W, -1);
  inc_ptr.assign(n_rows + 1, 0);
  inc_tet.clear();
  inc_code.clear();
  for (size_t i = 0; i < outs.size(); ++i) {
    const LocalRows& R = plus ? outs[i].P : outs[i].W;
    int64_t nr = (int64_t)R.ptr.size() - 1;
    for (int64_t r = 0; r < nr; ++r) {
      int64_t row = off[i] + r;
      int64_t len = R.ptr[r + 1] - R.ptr[r];
      int64_t s = row / kSlice;
      E.width[s] = std::max<int32_t>(E.width[s], (int32_t)len);
      for (int64_t j = 0; j < len; ++j)
        E.col[s * kSlice * W + j * kSlice + (row % kSlice)] =
            (int32_t)(off[i] + R.cols[R.ptr[r] + j]);
      for (int64_t q = R.inc_ptr[r]; q < R.inc_ptr[r + 1]; ++q) {
        inc_tet.push_back(R.inc_tet[q]);
        inc_code.push_back(R.inc_code[q]);
      }
      inc_ptr[row + 1] = (int64_t)inc_tet.size();
    }
  }
}

}  // namespace

int build_host_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                    const uint8_t* dirichlet, const int32_t* owner, int32_t r_hops,
                    HostPlan& hp, std::string& err) {
  if (n_nodes <= 0 || n_tets <= 0 || !tets || !dirichlet || !owner) {
    err = "mor_build_subdomains: empty mesh or null array";
    return MOR_ERR_ARG;
  }
  if (n_nodes > INT32_MAX || n_tets > INT32_MAX / 4) {
    err = "mor_build_subdomains: mesh too large for int32 indices";
    return MOR_ERR_ARG;
  }
  if (r_hops == 0 || r_hops < -1) {
    err = "mor_build_subdomains: r_hops must be >= 1, or -1 for the per-subdomain rule";
    return MOR_ERR_ARG;
  }
  for (int64_t q = 0; q < 4 * n_tets; ++q)
    if (tets[q] < 0 || tets[q] >= n_nodes) {
      err = "mor_build_subdomains: element vertex index out of range";
      return MOR_ERR_BAD_MESH;
    }
  int32_t n_sd = 0;
  for (int64_t v = 0; v < n_nodes; ++v) {
    if (owner[v] < 0) {
      err = "mor_build_subdomains: negative owner label";
      return MOR_ERR_ARG;
    }
    n_sd = std::max(n_sd, owner[v] + 1);
  }
  hp = HostPlan();
  hp.n_nodes = n_nodes;
  hp.n_tets = n_tets;
  hp.n_sd = n_sd;
  hp.r_hops = r_hops;

  // global node -> element incidence (ascending element ids)
  hp.n2t_ptr.assign(n_nodes + 1, 0);
  for (int64_t q = 0; q < 4 * n_tets; ++q) hp.n2t_ptr[tets[q] + 1]++;
  for (int64_t v = 0; v < n_nodes; ++v) hp.n2t_ptr[v + 1] += hp.n2t_ptr[v];
  hp.n2t.assign(4 * n_tets, 0);
  {
    std::vector<int64_t> fill(hp.n2t_ptr.begin(), hp.n2t_ptr.end() - 1);
    for (int64_t e = 0; e < n_tets; ++e)
      for (int a = 0; a < 4; ++a) hp.n2t[fill[tets[4 * e + a]]++] = (int32_t)e;
  }

  // owned nodes per subdomain (ascending)
  std::vector<std::vector<int32_t>> P(n_sd);
  for (int64_t v = 0; v < n_nodes; ++v) P[owner[v]].push_back((int32_t)v);
  for (int i = 0; i < n_sd; ++i)
    if (P[i].empty()) {
      err = "mor_build_subdomains: owner label " + std::to_string(i) + " is unused";
      return MOR_ERR_ARG;
    }

  int n_threads = (int)std::max(1u, std::thread::hardware_concurrency());
  n_threads = std::min(n_threads, 32);
  // hops per subdomain: fixed, or about half the width of the owned set
  // (max(1, round(cbrt(|P_i|) / 2)): the extension roughly doubles the diameter)
  hp.r_sd.resize(n_sd);
  for (int i = 0; i < n_sd; ++i)
    hp.r_sd[i] = r_hops > 0 ? r_hops
                            : std::max(1, (int32_t)std::lround(std::cbrt((double)P[i].size()) / 2.0));
  std::vector<Scratch> scratch(std::min(n_threads, n_sd));
  for (auto& s : scratch) s.init(n_nodes, n_tets);
  hp.sets.resize(n_sd);
  std::vector<SubOut> outs(n_sd);
  const auto& n2t_ptr = hp.n2t_ptr;
  const auto& n2t = hp.n2t;

  parallel_for(n_sd, (int)scratch.size(), [&](int i, int t) {
    Scratch& S = scratch[t];
    const int32_t st = i + 1;
    SubSets& ss = hp.sets[i];
    SubOut& so = outs[i];
    // r-hop ball of P_i over element edges
    std::vector<int32_t> ball_list = P[i], frontier = P[i], next;
    for (int32_t v : P[i]) S.ball[v] = st;
    for (int h = 0; h < hp.r_sd[i]; ++h) {
      next.clear();
      for (int32_t v : frontier)
        for (int64_t q = n2t_ptr[v]; q < n2t_ptr[v + 1]; ++q)
          for (int b = 0; b < 4; ++b) {
            int32_t w = tets[4 * (int64_t)n2t[q] + b];
            if (S.ball[w] != st) {
              S.ball[w] = st;
              next.push_back(w);
              ball_list.push_back(w);
            }
          }
      frontier.swap(next);
    }
    // T_i^+ = elements touching the ball
    for (int32_t v : ball_list)
      for (int64_t q = n2t_ptr[v]; q < n2t_ptr[v + 1]; ++q) {
        int32_t e = n2t[q];
        if (!S.tplus[e]) {
          S.tplus[e] = 1;
          ss.plus_tets.push_back(e);
        }
      }
    std::sort(ss.plus_tets.begin(), ss.plus_tets.end());
    // nodes of T_i^+: interior (all elements in T_i^+) -> I, others -> B
    for (int32_t e : ss.plus_tets)
      for (int b = 0; b < 4; ++b) {
        int32_t v = tets[4 * (int64_t)e + b];
        if (S.vert[v] == st) continue;
        S.vert[v] = st;
        if (dirichlet[v]) continue;
        bool interior = true;
        for (int64_t q = n2t_ptr[v]; q < n2t_ptr[v + 1] && interior; ++q)
          interior = S.tplus[n2t[q]] != 0;
        (interior ? ss.I : ss.B).push_back(v);
      }
    std::sort(ss.I.begin(), ss.I.end());
    std::sort(ss.B.begin(), ss.B.end());
    // omega_i = elements touching P_i
    for (int32_t v : P[i])
      for (int64_t q = n2t_ptr[v]; q < n2t_ptr[v + 1]; ++q) {
        int32_t e = n2t[q];
        if (!S.tomega[e]) {
          S.tomega[e] = 1;
          ss.omega_tets.push_back(e);
        }
      }
    std::sort(ss.omega_tets.begin(), ss.omega_tets.end());
    for (int32_t e : ss.omega_tets)
      for (int b = 0; b < 4; ++b) {
        int32_t v = tets[4 * (int64_t)e + b];
        if (S.wmark[v] == st || dirichlet[v]) continue;
        S.wmark[v] = st;
        ss.omega.push_back(v);
      }
    std::sort(ss.omega.begin(), ss.omega.end());
    for (size_t w = 0; w < ss.omega.size(); ++w) S.wloc[ss.omega[w]] = (int32_t)w;
    for (int32_t v : P[i])
      if (!dirichlet[v]) ss.owned.push_back(v);
    // plus-local numbering: I then B
    for (size_t l = 0; l < ss.I.size(); ++l) {
      S.loc_mark[ss.I[l]] = st;
      S.loc[ss.I[l]] = (int32_t)l;
    }
    for (size_t l = 0; l < ss.B.size(); ++l) {
      S.loc_mark[ss.B[l]] = st;
      S.loc[ss.B[l]] = (int32_t)(ss.I.size() + l);
    }
    so.w2p_local.resize(ss.omega.size());
    for (size_t w = 0; w < ss.omega.size(); ++w) {
      int32_t v = ss.omega[w];
      if (S.loc_mark[v] != st || S.loc[v] >= (int32_t)ss.I.size()) {
        so.err = "omega_i is not interior to its extension (r_hops too small)";
        break;
      }
      so.w2p_local[w] = S.loc[v];
    }
    so.o2w_local.resize(ss.owned.size());
    for (size_t o = 0; o < ss.owned.size(); ++o) so.o2w_local[o] = S.wloc[ss.owned[o]];
    if (so.err.empty()) {
      std::vector<int32_t> prow(ss.I);
      prow.insert(prow.end(), ss.B.begin(), ss.B.end());
      build_rows(prow, tets, n2t_ptr, n2t, S.tplus, S.loc_mark, S.loc, st, so.P);
      build_rows(ss.omega, tets, n2t_ptr, n2t, S.tomega, S.wmark, S.wloc, st, so.W);
    }
    // clear the element flags for the next subdomain on this thread
    for (int32_t e : ss.plus_tets) S.tplus[e] = 0;
    for (int32_t e : ss.omega_tets) S.tomega[e] = 0;
  });
  for (auto& o : outs)
    if (!o.err.empty()) {
      err = "mor_build_subdomains: " + o.err;
      return MOR_ERR_ARG;
    }

  // batched layouts
  hp.Poff.assign(n_sd + 1, 0);
  hp.Woff.assign(n_sd + 1, 0);
  hp.Ooff.assign(n_sd + 1, 0);
  hp.nI.resize(n_sd);
  hp.nB.resize(n_sd);
  for (int i = 0; i < n_sd; ++i) {
    const SubSets& ss = hp.sets[i];
    hp.nI[i] = (int32_t)ss.I.size();
    hp.nB[i] = (int32_t)ss.B.size();
    hp.Poff[i + 1] = hp.Poff[i] + ss.I.size() + ss.B.size();
    hp.Woff[i + 1] = hp.Woff[i] + ss.omega.size();
    hp.Ooff[i + 1] = hp.Ooff[i] + ss.owned.size();
  }
  hp.nP = hp.Poff[n_sd];
  hp.nW = hp.Woff[n_sd];
  hp.nO = hp.Ooff[n_sd];
  if (hp.nP > INT32_MAX / 2 || hp.nW > INT32_MAX / 2) {
    err = "mor_build_subdomains: batched rows exceed int32 range";
    return MOR_ERR_ARG;
  }
  hp.p_node.resize(hp.nP);
  hp.p_sd.resize(hp.nP);
  hp.p_isB.resize(hp.nP);
  hp.w_node.resize(hp.nW);
  hp.w_sd.resize(hp.nW);
  hp.w2p.resize(hp.nW);
  hp.w2o.assign(hp.nW, -1);
  hp.o2w.resize(hp.nO);
  hp.o_node.resize(hp.nO);
  hp.o_sd.resize(hp.nO);
  std::vector<int32_t> node2orow(n_nodes, -1);
  for (int i = 0; i < n_sd; ++i) {
    const SubSets& ss = hp.sets[i];
    int64_t p0 = hp.Poff[i], w0 = hp.Woff[i], o0 = hp.Ooff[i];
    for (size_t l = 0; l < ss.I.size(); ++l) {
      hp.p_node[p0 + l] = ss.I[l];
      hp.p_sd[p0 + l] = i;
      hp.p_isB[p0 + l] = 0;
    }
    for (size_t l = 0; l < ss.B.size(); ++l) {
      hp.p_node[p0 + ss.I.size() + l] = ss.B[l];
      hp.p_sd[p0 + ss.I.size() + l] = i;
      hp.p_isB[p0 + ss.I.size() + l] = 1;
    }
    for (size_t w = 0; w < ss.omega.size(); ++w) {
      hp.w_node[w0 + w] = ss.omega[w];
      hp.w_sd[w0 + w] = i;
      hp.w2p[w0 + w] = (int32_t)(p0 + outs[i].w2p_local[w]);
    }
    for (size_t o = 0; o < ss.owned.size(); ++o) {
      int32_t wr = (int32_t)(w0 + outs[i].o2w_local[o]);
      hp.o2w[o0 + o] = wr;
      hp.w2o[wr] = (int32_t)(o0 + o);
      hp.o_node[o0 + o] = ss.owned[o];
      hp.o_sd[o0 + o] = i;
      node2orow[ss.owned[o]] = (int32_t)(o0 + o);
    }
  }
  pack_ell(outs, true, hp.Poff, hp.nP, hp.pat_P, hp.incP_ptr, hp.incP_tet, hp.incP_code);
  pack_ell(outs, false, hp.Woff, hp.nW, hp.pat_W, hp.incW_ptr, hp.incW_tet, hp.incW_code);
  if (hp.pat_P.W >= (int32_t)kNoSlot || hp.pat_W.W >= (int32_t)kNoSlot) {
    err = "mor_build_subdomains: node degree too large for the incidence code";
    return MOR_ERR_BAD_MESH;
  }

  // row tiles
  {
    std::vector<int64_t> b(n_sd), e(n_sd);
    for (int i = 0; i < n_sd; ++i) {
      b[i] = hp.Poff[i];
      e[i] = hp.Poff[i + 1];
    }
    make_tiles(b, e, hp.tP_all);
    for (int i = 0; i < n_sd; ++i) e[i] = hp.Poff[i] + hp.nI[i];
    make_tiles(b, e, hp.tP_I);
    for (int i = 0; i < n_sd; ++i) {
      b[i] = hp.Poff[i] + hp.nI[i];
      e[i] = hp.Poff[i + 1];
    }
    make_tiles(b, e, hp.tP_B);
    for (int i = 0; i < n_sd; ++i) {
      b[i] = hp.Woff[i];
      e[i] = hp.Woff[i + 1];
    }
    make_tiles(b, e, hp.tW);
    for (int i = 0; i < n_sd; ++i) {
      b[i] = hp.Ooff[i];
      e[i] = hp.Ooff[i + 1];
    }
    make_tiles(b, e, hp.tO);
  }

  // interface entries: free u, v sharing an element, owner(u) < owner(v)
  struct Entry {
    int32_t i, j, u, v;
    bool operator<(const Entry& o) const {
      if (i != o.i) return i < o.i;
      if (j != o.j) return j < o.j;
      if (u != o.u) return u < o.u;
      return v < o.v;
    }
    bool operator==(const Entry& o) const {
      return i == o.i && j == o.j && u == o.u && v == o.v;
    }
  };
  std::vector<Entry> ents;
  for (int64_t u = 0; u < n_nodes; ++u) {
    if (dirichlet[u]) continue;
    for (int64_t q = hp.n2t_ptr[u]; q < hp.n2t_ptr[u + 1]; ++q)
      for (int b = 0; b < 4; ++b) {
        int32_t v = tets[4 * (int64_t)hp.n2t[q] + b];
        if (dirichlet[v] || owner[v] <= owner[u]) continue;
        ents.push_back(Entry{owner[u], owner[v], (int32_t)u, v});
      }
  }
  std::sort(ents.begin(), ents.end());
  ents.erase(std::unique(ents.begin(), ents.end()), ents.end());
  hp.pair_ptr.assign(1, 0);
  for (size_t q = 0; q < ents.size(); ++q) {
    if (q == 0 || ents[q].i != ents[q - 1].i || ents[q].j != ents[q - 1].j) {
      if (q > 0) hp.pair_ptr.push_back((int64_t)q);
      hp.pair_i.push_back(ents[q].i);
      hp.pair_j.push_back(ents[q].j);
    }
    hp.e_urow.push_back(node2orow[ents[q].u]);
    hp.e_vrow.push_back(node2orow[ents[q].v]);
    hp.e_unode.push_back(ents[q].u);
    hp.e_vnode.push_back(ents[q].v);
  }
  if (!ents.empty()) hp.pair_ptr.push_back((int64_t)ents.size());
  return MOR_OK;
}

}  // namespace mor
