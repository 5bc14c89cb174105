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

// Rows of one local space (rows numbered by their local index): the sorted local
// columns of every row (nodes sharing an element of `elems` with it) and its incidence
// entries (the elements of `elems` holding the row's node, ascending).  Element-driven:
// every element's four local vertex indices are looked up once into W.evl, the
// (element, vertex) pairs are bucketed by row in element order, and each row then
// reads only the small table.  W holds the work arrays (reused across calls).
struct RowWork {
  std::vector<int32_t> evl;    // 4 per element: local index of each vertex, or -1
  std::vector<int64_t> start;  // per row: first (element, vertex) pair
  std::vector<int64_t> fill;
  std::vector<int32_t> pairs;  // 4 * element position + vertex slot, bucketed by row
  std::vector<int32_t> seen, slot_of, cand;
};

// per-thread scratch, stamped with subdomain id + 1 so it never needs clearing
struct Scratch {
  std::vector<int32_t> ball, vert, loc_mark, loc, wmark, wloc;
  std::vector<uint8_t> tplus, tomega;
  RowWork rows;  // build_rows work arrays
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

// Sort ids whose flags are set: a scan of the flag array over their range when that range
// is short (a few times the count, as for compact subdomains), else a comparison sort.
void sort_flagged(std::vector<int32_t>& ids, const std::vector<uint8_t>& flag) {
  if (ids.empty()) return;
  int32_t lo = INT32_MAX, hi = -1;
  for (int32_t e : ids) {
    lo = std::min(lo, e);
    hi = std::max(hi, e);
  }
  if ((int64_t)hi - lo + 1 <= 16 * (int64_t)ids.size()) {
    ids.clear();
    for (int32_t e = lo; e <= hi; ++e)
      if (flag[e]) ids.push_back(e);
  } else {
    std::sort(ids.begin(), ids.end());
  }
}

void build_rows(int64_t n_rows, const std::vector<int32_t>& elems, const int32_t* tets,
                const std::vector<int32_t>& mark, const std::vector<int32_t>& loc,
                int32_t stamp, LocalRows& R, RowWork& W) {
  const int64_t ne = (int64_t)elems.size();
  W.evl.resize(4 * ne);
  W.start.assign(n_rows + 1, 0);
  for (int64_t p = 0; p < ne; ++p) {
    const int32_t* t = tets + 4 * (int64_t)elems[p];
    for (int b = 0; b < 4; ++b) {
      const int32_t vb = t[b];
      const int32_t l = mark[vb] == stamp ? loc[vb] : -1;
      W.evl[4 * p + b] = l;
      if (l >= 0) ++W.start[l + 1];
    }
  }
  for (int64_t r = 0; r < n_rows; ++r) W.start[r + 1] += W.start[r];
  W.fill.assign(W.start.begin(), W.start.end() - 1);
  W.pairs.resize(W.start[n_rows]);
  for (int64_t p = 0; p < ne; ++p)
    for (int b = 0; b < 4; ++b) {
      const int32_t l = W.evl[4 * p + b];
      if (l >= 0) W.pairs[W.fill[l]++] = (int32_t)(4 * p + b);
    }
  W.seen.assign(n_rows, -1);
  if ((int64_t)W.slot_of.size() < n_rows) W.slot_of.resize(n_rows);
  R.cols.reserve(R.cols.size() + 16 * n_rows);
  R.ptr.reserve(R.ptr.size() + n_rows);
  R.inc_tet.reserve(R.inc_tet.size() + W.start[n_rows]);
  R.inc_code.reserve(R.inc_code.size() + W.start[n_rows]);
  R.inc_ptr.reserve(R.inc_ptr.size() + n_rows);
  for (int64_t row = 0; row < n_rows; ++row) {
    auto& cand = W.cand;
    cand.clear();
    for (int64_t k = W.start[row]; k < W.start[row + 1]; ++k) {
      const int32_t* ev = W.evl.data() + (W.pairs[k] & ~3);
      for (int b = 0; b < 4; ++b) {
        const int32_t l = ev[b];
        if (l >= 0 && W.seen[l] != row) {
          W.seen[l] = (int32_t)row;
          cand.push_back(l);
        }
      }
    }
    std::sort(cand.begin(), cand.end());
    for (size_t k = 0; k < cand.size(); ++k) W.slot_of[cand[k]] = (int32_t)k;
    R.cols.insert(R.cols.end(), cand.begin(), cand.end());
    R.ptr.push_back((int64_t)R.cols.size());
    for (int64_t k = W.start[row]; k < W.start[row + 1]; ++k) {
      const int32_t pb = W.pairs[k];
      const int32_t* ev = W.evl.data() + (pb & ~3);
      uint32_t code = (uint32_t)(pb & 3);
      for (int b = 0; b < 4; ++b) {
        const uint32_t slot = ev[b] >= 0 ? (uint32_t)W.slot_of[ev[b]] : kNoSlot;
        code |= slot << (2 + 7 * b);
      }
      R.inc_tet.push_back(elems[pb >> 2]);
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

// Pack the rows of all subdomains into one sliced-ELL pattern and incidence CSR.  Row
// lengths and incidence offsets come first (prefix sums), then every subdomain writes
// its own contiguous rows in parallel; a slice may straddle two subdomains, so slice
// widths are a separate pass over the row lengths.
void pack_ell(const std::vector<SubOut>& outs, bool plus, const std::vector<int64_t>& off,
              int64_t n_rows, HostEll& E, std::vector<int64_t>& inc_ptr,
              BigVec<int32_t>& inc_tet, BigVec<uint32_t>& inc_code, int n_threads) {
  const int n_sd = (int)outs.size();
  std::vector<int32_t> len(n_rows, 0);
  inc_ptr.assign(n_rows + 1, 0);
  std::vector<int32_t> wmax(n_sd, 0);
  parallel_for(n_sd, n_threads, [&](int i, int) {
    const LocalRows& R = plus ? outs[i].P : outs[i].W;
    int32_t m = 0;
    for (size_t r = 0; r + 1 < R.ptr.size(); ++r) {
      len[off[i] + r] = (int32_t)(R.ptr[r + 1] - R.ptr[r]);
      m = std::max(m, len[off[i] + r]);
      inc_ptr[off[i] + r + 1] = R.inc_ptr[r + 1] - R.inc_ptr[r];
    }
    wmax[i] = m;
  });
  for (int64_t r = 0; r < n_rows; ++r) inc_ptr[r + 1] += inc_ptr[r];
  int32_t W = 0;
  for (int i = 0; i < n_sd; ++i) W = std::max(W, wmax[i]);
  const int64_t n_slices = (n_rows + kSlice - 1) / kSlice;
  E.n_rows = n_rows;
  E.W = W;
  E.width.assign(n_slices, 0);
  for (int64_t r = 0; r < n_rows; ++r)
    E.width[r / kSlice] = std::max(E.width[r / kSlice], len[r]);
  // every entry is written exactly once below: the slots of each row by the thread of
  // its subdomain (padding slots -1), the rows past n_rows in the last slice here
  E.col.resize(n_slices * kSlice * (int64_t)W);
  inc_tet.resize(inc_ptr[n_rows]);
  inc_code.resize(inc_ptr[n_rows]);
  for (int64_t row = n_rows; row < n_slices * kSlice; ++row)
    for (int64_t j = 0; j < W; ++j)
      E.col[(row / kSlice) * kSlice * W + j * kSlice + (row % kSlice)] = -1;
  parallel_for(n_sd, n_threads, [&](int i, int) {
    const LocalRows& R = plus ? outs[i].P : outs[i].W;
    const int64_t nr = (int64_t)R.ptr.size() - 1;
    for (int64_t r = 0; r < nr; ++r) {
      const int64_t row = off[i] + r, s = row / kSlice;
      const int64_t l = R.ptr[r + 1] - R.ptr[r];
      for (int64_t j = 0; j < W; ++j)
        E.col[s * kSlice * W + j * kSlice + (row % kSlice)] =
            j < l ? (int32_t)(off[i] + R.cols[R.ptr[r] + j]) : -1;
      int64_t q = inc_ptr[row];
      for (int64_t k = R.inc_ptr[r]; k < R.inc_ptr[r + 1]; ++k, ++q) {
        inc_tet[q] = R.inc_tet[k];
        inc_code[q] = R.inc_code[k];
      }
    }
  });
}

// spread the low 10 bits of v to every third bit
uint32_t spread3(uint32_t v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// I and B in Morton order of the node positions quantised to 1024 cells per axis of
// the bounding box of I u B (ties by node id); codes in the same order
void morton_order(const double* xyz, const std::vector<int32_t>& I,
                  const std::vector<int32_t>& B, std::vector<int32_t>& Ip,
                  std::vector<int32_t>& Bp, std::vector<uint32_t>& code) {
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  bool first = true;
  if (xyz)
    for (const auto* seg : {&I, &B})
      for (int32_t v : *seg)
        for (int a = 0; a < 3; ++a) {
          double x = xyz[3 * (int64_t)v + a];
          if (first || x < lo[a]) lo[a] = x;
          if (first || x > hi[a]) hi[a] = x;
          if (a == 2) first = false;
        }
  auto key = [&](int32_t v) -> uint32_t {
    if (!xyz) return 0u;
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
      double w = hi[a] - lo[a];
      double t = w > 0.0 ? (xyz[3 * (int64_t)v + a] - lo[a]) / w * 1024.0 : 0.0;
      q[a] = (uint32_t)std::min(1023.0, std::max(0.0, std::floor(t)));
    }
    return (spread3(q[2]) << 2) | (spread3(q[1]) << 1) | spread3(q[0]);
  };
  code.clear();
  for (int s = 0; s < 2; ++s) {
    const std::vector<int32_t>& src = s == 0 ? I : B;
    std::vector<std::pair<uint32_t, int32_t>> kv(src.size());
    for (size_t l = 0; l < src.size(); ++l) kv[l] = {key(src[l]), src[l]};
    std::sort(kv.begin(), kv.end());
    std::vector<int32_t>& dst = s == 0 ? Ip : Bp;
    dst.resize(src.size());
    for (size_t l = 0; l < kv.size(); ++l) {
      dst[l] = kv[l].second;
      code.push_back(kv[l].first);
    }
  }
}

}  // namespace

int build_global_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                      const uint8_t* dirichlet, const int32_t* owner, int32_t r_hops,
                      HostPlan& g, std::string& err) {
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
  g = HostPlan();
  g.n_nodes = n_nodes;
  g.n_tets = n_tets;
  g.n_sd = n_sd;
  g.r_hops = r_hops;

  // global node -> element incidence (ascending element ids): counts and slots taken
  // with atomics on all cores, then every node's list sorted
  const int nthr_g = (int)std::min(32u, std::max(1u, std::thread::hardware_concurrency()));
  g.n2t_ptr.assign(n_nodes + 1, 0);
  g.n2t.resize(4 * n_tets);
  {
    std::vector<std::atomic<int64_t>> cnt(n_nodes);
    const int64_t ech = 1 << 16;
    const int n_ech = (int)((n_tets + ech - 1) / ech);
    parallel_for((int)((n_nodes + ech - 1) / ech), nthr_g, [&](int c, int) {
      const int64_t v1 = std::min(n_nodes, (int64_t)(c + 1) * ech);
      for (int64_t v = (int64_t)c * ech; v < v1; ++v) cnt[v].store(0, std::memory_order_relaxed);
    });
    parallel_for(n_ech, nthr_g, [&](int c, int) {
      const int64_t e1 = std::min(n_tets, (int64_t)(c + 1) * ech);
      for (int64_t q = 4 * (int64_t)c * ech; q < 4 * e1; ++q)
        cnt[tets[q]].fetch_add(1, std::memory_order_relaxed);
    });
    for (int64_t v = 0; v < n_nodes; ++v)
      g.n2t_ptr[v + 1] = g.n2t_ptr[v] + cnt[v].load(std::memory_order_relaxed);
    parallel_for((int)((n_nodes + ech - 1) / ech), nthr_g, [&](int c, int) {
      const int64_t v1 = std::min(n_nodes, (int64_t)(c + 1) * ech);
      for (int64_t v = (int64_t)c * ech; v < v1; ++v)
        cnt[v].store(g.n2t_ptr[v], std::memory_order_relaxed);
    });
    parallel_for(n_ech, nthr_g, [&](int c, int) {
      const int64_t e1 = std::min(n_tets, (int64_t)(c + 1) * ech);
      for (int64_t e = (int64_t)c * ech; e < e1; ++e)
        for (int a = 0; a < 4; ++a)
          g.n2t[cnt[tets[4 * e + a]].fetch_add(1, std::memory_order_relaxed)] = (int32_t)e;
    });
    parallel_for((int)((n_nodes + ech - 1) / ech), nthr_g, [&](int c, int) {
      const int64_t v1 = std::min(n_nodes, (int64_t)(c + 1) * ech);
      for (int64_t v = (int64_t)c * ech; v < v1; ++v)
        std::sort(g.n2t.begin() + g.n2t_ptr[v], g.n2t.begin() + g.n2t_ptr[v + 1]);
    });
  }

  // node adjacency (nodes sharing an element), for the r-hop balls: two passes over
  // chunks of nodes, each node deduplicating its element neighbours locally
  {
    const int64_t ach = 1 << 13;
    const int n_ach = (int)((n_nodes + ach - 1) / ach);
    g.adj_ptr.assign(n_nodes + 1, 0);
    auto neighbours = [&](int64_t v, std::vector<int32_t>& nb) {
      nb.clear();
      for (int64_t q = g.n2t_ptr[v]; q < g.n2t_ptr[v + 1]; ++q)
        for (int b = 0; b < 4; ++b) {
          const int32_t w = tets[4 * (int64_t)g.n2t[q] + b];
          if (w != v) nb.push_back(w);
        }
      std::sort(nb.begin(), nb.end());
      nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
    };
    parallel_for(n_ach, nthr_g, [&](int c, int) {
      std::vector<int32_t> nb;
      const int64_t v1 = std::min(n_nodes, (int64_t)(c + 1) * ach);
      for (int64_t v = (int64_t)c * ach; v < v1; ++v) {
        neighbours(v, nb);
        g.adj_ptr[v + 1] = (int64_t)nb.size();
      }
    });
    for (int64_t v = 0; v < n_nodes; ++v) g.adj_ptr[v + 1] += g.adj_ptr[v];
    g.adj.resize(g.adj_ptr[n_nodes]);
    parallel_for(n_ach, nthr_g, [&](int c, int) {
      std::vector<int32_t> nb;
      const int64_t v1 = std::min(n_nodes, (int64_t)(c + 1) * ach);
      for (int64_t v = (int64_t)c * ach; v < v1; ++v) {
        neighbours(v, nb);
        std::copy(nb.begin(), nb.end(), g.adj.begin() + g.adj_ptr[v]);
      }
    });
  }

  // owned nodes per subdomain (ascending)
  g.Pown.assign(n_sd, {});
  for (int64_t v = 0; v < n_nodes; ++v) g.Pown[owner[v]].push_back((int32_t)v);
  for (int i = 0; i < n_sd; ++i)
    if (g.Pown[i].empty()) {
      err = "mor_build_subdomains: owner label " + std::to_string(i) + " is unused";
      return MOR_ERR_ARG;
    }
  // hops per subdomain: fixed, or about half the width of the owned set
  // (max(1, round(cbrt(|P_i|) / 2)): the extension roughly doubles the diameter)
  g.r_sd.resize(n_sd);
  for (int i = 0; i < n_sd; ++i)
    g.r_sd[i] = r_hops > 0 ? r_hops
                           : std::max(1, (int32_t)std::lround(std::cbrt((double)g.Pown[i].size()) / 2.0));

  // owned free nodes (O space, by subdomain, ascending node ids)
  g.Ooff.assign(n_sd + 1, 0);
  for (int i = 0; i < n_sd; ++i) {
    int64_t c = 0;
    for (int32_t v : g.Pown[i]) c += dirichlet[v] == 0;
    g.Ooff[i + 1] = g.Ooff[i] + c;
  }
  g.nO = g.Ooff[n_sd];
  g.o_node.resize(g.nO);
  g.o_sd.resize(g.nO);
  std::vector<int32_t> g_node2orow(n_nodes, -1);
  for (int i = 0; i < n_sd; ++i) {
    int64_t o = g.Ooff[i];
    for (int32_t v : g.Pown[i])
      if (!dirichlet[v]) {
        g.o_node[o] = v;
        g.o_sd[o] = i;
        g_node2orow[v] = (int32_t)o;
        ++o;
      }
  }

  // interface entries: free u, v sharing an element, owner(u) < owner(v)
  struct Entry {
    int32_t i, j, u, v;
  };
  // Each free node u lists its free neighbours v with owner(v) > owner(u) once, in
  // ascending order (from the adjacency), in chunks of nodes on all cores; the chunks
  // are concatenated in node order and a stable sort by subdomain pair then yields the
  // entries ordered by (i, j, u, v).
  const int64_t chunk = 1 << 13;
  const int n_chunks = (int)((n_nodes + chunk - 1) / chunk);
  std::vector<std::vector<Entry>> parts(n_chunks);
  parallel_for(n_chunks, nthr_g, [&](int c, int) {
    auto& out = parts[c];
    const int64_t u1 = std::min(n_nodes, (int64_t)(c + 1) * chunk);
    for (int64_t u = (int64_t)c * chunk; u < u1; ++u) {
      if (dirichlet[u]) continue;
      for (int64_t q = g.adj_ptr[u]; q < g.adj_ptr[u + 1]; ++q) {
        const int32_t v = g.adj[q];
        if (!dirichlet[v] && owner[v] > owner[u])
          out.push_back(Entry{owner[u], owner[v], (int32_t)u, v});
      }
    }
  });
  std::vector<Entry> ents;
  {
    size_t n_ent = 0;
    for (const auto& pt : parts) n_ent += pt.size();
    ents.reserve(n_ent);
    for (auto& pt : parts) {
      ents.insert(ents.end(), pt.begin(), pt.end());
      std::vector<Entry>().swap(pt);
    }
  }
  std::stable_sort(ents.begin(), ents.end(), [](const Entry& a, const Entry& b) {
    return a.i != b.i ? a.i < b.i : a.j < b.j;
  });
  g.pair_ptr.assign(1, 0);
  for (size_t q = 0; q < ents.size(); ++q) {
    if (q == 0 || ents[q].i != ents[q - 1].i || ents[q].j != ents[q - 1].j) {
      if (q > 0) g.pair_ptr.push_back((int64_t)q);
      g.pair_i.push_back(ents[q].i);
      g.pair_j.push_back(ents[q].j);
    }
    g.e_urow.push_back(g_node2orow[ents[q].u]);
    g.e_vrow.push_back(g_node2orow[ents[q].v]);
    g.e_unode.push_back(ents[q].u);
    g.e_vnode.push_back(ents[q].v);
  }
  if (!ents.empty()) g.pair_ptr.push_back((int64_t)ents.size());
  return MOR_OK;
}

// per-thread work arrays of the wave builder, stamped with subdomain id + 1
struct PlanScratch::Impl {
  std::vector<Scratch> s;
};
PlanScratch::PlanScratch() : impl(new Impl) {}
PlanScratch::~PlanScratch() { delete impl; }

int build_wave_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                    const uint8_t* dirichlet, const double* xyz, const HostPlan& g, int s0,
                    int s1, HostPlan& w, PlanScratch& ps, std::string& err) {
  const int nw = s1 - s0;
  w = HostPlan();
  w.n_nodes = n_nodes;
  w.n_tets = n_tets;
  w.n_sd = nw;
  w.r_hops = g.r_hops;
  w.r_sd.assign(g.r_sd.begin() + s0, g.r_sd.begin() + s1);
  // per-thread scratch: 6 node arrays + 2 element flag arrays; at most 32 threads and
  // about 24 GB of scratch in total
  const double per_thread = 24.0 * (double)n_nodes + 2.0 * (double)n_tets;
  int nthr = (int)std::max(1u, std::thread::hardware_concurrency());
  nthr = std::min({nthr, 32, std::max(1, (int)(24e9 / per_thread)), std::max(nw, 1)});
  auto& scratch = ps.impl->s;
  const int have = (int)scratch.size();
  if (have < nthr) {
    // zero the new scratch on the threads themselves (parallel first touch)
    scratch.resize(nthr);
    parallel_for(nthr - have, nthr - have,
                 [&](int q, int) { scratch[have + q].init(n_nodes, n_tets); });
  }
  w.sets.resize(nw);
  std::vector<SubOut> outs(nw);
  const auto& n2t_ptr = g.n2t_ptr;
  const auto& n2t = g.n2t;

  parallel_for(nw, nthr, [&](int li, int t) {
    Scratch& S = scratch[t];
    const int i = s0 + li;
    const int32_t st = i + 1;
    SubSets& ss = w.sets[li];
    SubOut& so = outs[li];
    // r-hop ball of P_i over element edges
    std::vector<int32_t> ball_list = g.Pown[i], frontier = g.Pown[i], next;
    for (int32_t v : g.Pown[i]) S.ball[v] = st;
    for (int h = 0; h < g.r_sd[i]; ++h) {
      next.clear();
      for (int32_t v : frontier)
        for (int64_t q = g.adj_ptr[v]; q < g.adj_ptr[v + 1]; ++q) {
          const int32_t w = g.adj[q];
          if (S.ball[w] != st) {
            S.ball[w] = st;
            next.push_back(w);
            ball_list.push_back(w);
          }
        }
      frontier.swap(next);
    }
    // T_i^+ = elements touching the ball, ascending
    for (int32_t v : ball_list)
      for (int64_t q = n2t_ptr[v]; q < n2t_ptr[v + 1]; ++q) {
        int32_t e = n2t[q];
        if (!S.tplus[e]) {
          S.tplus[e] = 1;
          ss.plus_tets.push_back(e);
        }
      }
    sort_flagged(ss.plus_tets, S.tplus);
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
    // a subdomain whose extension covers the whole domain has no lifting problem
    // (Eq. (8) has no boundary data) and no interface; the batched kernels assume
    // every subdomain has rows in I and in B
    if (ss.B.empty() || ss.I.empty())
      so.err = "subdomain " + std::to_string(i) +
               (ss.B.empty() ? " has an empty boundary set B (its extension covers the "
                               "domain: use more subdomains or fewer hops)"
                             : " has an empty interior set I");
    // clear the element flags for the next subdomain on this thread
    for (int32_t e : ss.plus_tets) S.tplus[e] = 0;
  });
  // the rest per subdomain, largest T_i^+ first (the tasks differ in size by 2-3x on
  // box partitions; dynamic scheduling then ends the pass evenly across the threads)
  std::vector<int> order(nw);
  for (int li = 0; li < nw; ++li) order[li] = li;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return w.sets[a].plus_tets.size() > w.sets[b].plus_tets.size();
  });
  parallel_for(nw, nthr, [&](int oi, int t) {
    Scratch& S = scratch[t];
    const int li = order[oi];
    const int i = s0 + li;
    const int32_t st = i + 1;
    SubSets& ss = w.sets[li];
    SubOut& so = outs[li];
    // omega_i = elements touching P_i, ascending
    for (int32_t v : g.Pown[i])
      for (int64_t q = n2t_ptr[v]; q < n2t_ptr[v + 1]; ++q) {
        int32_t e = n2t[q];
        if (!S.tomega[e]) {
          S.tomega[e] = 1;
          ss.omega_tets.push_back(e);
        }
      }
    sort_flagged(ss.omega_tets, S.tomega);
    for (int32_t e : ss.omega_tets)
      for (int b = 0; b < 4; ++b) {
        int32_t v = tets[4 * (int64_t)e + b];
        if (S.wmark[v] == st || dirichlet[v]) continue;
        S.wmark[v] = st;
        ss.omega.push_back(v);
      }
    std::sort(ss.omega.begin(), ss.omega.end());
    for (size_t w = 0; w < ss.omega.size(); ++w) S.wloc[ss.omega[w]] = (int32_t)w;
    for (int32_t v : g.Pown[i])
      if (!dirichlet[v]) ss.owned.push_back(v);
    // plus-local numbering: I then B, each in Morton order
    morton_order(xyz, ss.I, ss.B, ss.Ip, ss.Bp, ss.pcode);
    for (size_t l = 0; l < ss.Ip.size(); ++l) {
      S.loc_mark[ss.Ip[l]] = st;
      S.loc[ss.Ip[l]] = (int32_t)l;
    }
    for (size_t l = 0; l < ss.Bp.size(); ++l) {
      S.loc_mark[ss.Bp[l]] = st;
      S.loc[ss.Bp[l]] = (int32_t)(ss.Ip.size() + l);
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
      build_rows((int64_t)(ss.Ip.size() + ss.Bp.size()), ss.plus_tets, tets, S.loc_mark,
                 S.loc, st, so.P, S.rows);
      build_rows((int64_t)ss.omega.size(), ss.omega_tets, tets, S.wmark, S.wloc, st, so.W,
                 S.rows);
    }
    // clear the element flags for the next subdomain on this thread
    for (int32_t e : ss.omega_tets) S.tomega[e] = 0;
  });
  for (auto& o : outs)
    if (!o.err.empty()) {
      err = "mor_build_subdomains: " + o.err;
      return MOR_ERR_ARG;
    }
  HostPlan& hp = w;
  const int n_sd = nw;
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
  hp.p_code.resize(hp.nP);
  hp.w_node.resize(hp.nW);
  hp.w_sd.resize(hp.nW);
  hp.w2p.resize(hp.nW);
  hp.w2o.assign(hp.nW, -1);
  hp.o2w.resize(hp.nO);
  hp.o_node.resize(hp.nO);
  hp.o_sd.resize(hp.nO);
  parallel_for(n_sd, nthr, [&](int i, int) {
    const SubSets& ss = hp.sets[i];
    int64_t p0 = hp.Poff[i], w0 = hp.Woff[i], o0 = hp.Ooff[i];
    for (size_t l = 0; l < ss.Ip.size(); ++l) {
      hp.p_node[p0 + l] = ss.Ip[l];
      hp.p_sd[p0 + l] = i;
      hp.p_isB[p0 + l] = 0;
    }
    for (size_t l = 0; l < ss.Bp.size(); ++l) {
      hp.p_node[p0 + ss.Ip.size() + l] = ss.Bp[l];
      hp.p_sd[p0 + ss.Ip.size() + l] = i;
      hp.p_isB[p0 + ss.Ip.size() + l] = 1;
    }
    for (size_t l = 0; l < ss.pcode.size(); ++l) hp.p_code[p0 + l] = ss.pcode[l];
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
    }
  });
  pack_ell(outs, true, hp.Poff, hp.nP, hp.pat_P, hp.incP_ptr, hp.incP_tet, hp.incP_code,
           nthr);
  pack_ell(outs, false, hp.Woff, hp.nW, hp.pat_W, hp.incW_ptr, hp.incW_tet, hp.incW_code,
           nthr);
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

  return MOR_OK;
}

int build_host_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                    const uint8_t* dirichlet, const int32_t* owner, int32_t r_hops,
                    const double* xyz, HostPlan& hp, std::string& err) {
  HostPlan g;
  int rc = build_global_plan(n_nodes, n_tets, tets, dirichlet, owner, r_hops, g, err);
  if (rc != MOR_OK) return rc;
  PlanScratch ps;
  rc = build_wave_plan(n_nodes, n_tets, tets, dirichlet, xyz, g, 0, g.n_sd, hp, ps, err);
  if (rc != MOR_OK) return rc;
  // the global parts: incidence, owned sets, interface entries
  hp.n2t_ptr.swap(g.n2t_ptr);
  hp.n2t.swap(g.n2t);
  hp.Pown.swap(g.Pown);
  hp.pair_i.swap(g.pair_i);
  hp.pair_j.swap(g.pair_j);
  hp.pair_ptr.swap(g.pair_ptr);
  hp.e_urow.swap(g.e_urow);
  hp.e_vrow.swap(g.e_vrow);
  hp.e_unode.swap(g.e_unode);
  hp.e_vnode.swap(g.e_vnode);
  return MOR_OK;
}

namespace {

constexpr int kMinAggRows = 8;

// leading equal bits (of 30) of two Morton codes
int lead_equal(uint32_t a, uint32_t b) {
  uint32_t x = (a ^ b) & 0x3FFFFFFFu;
  int n = 30;
  while (x) {
    x >>= 1;
    --n;
  }
  return n;
}

// prefix length b whose run count is closest (in ratio) to want, from the histogram of
// leading equal bits between consecutive codes (a boundary at level b where lead < b)
int pick_bits(const uint32_t* code, int n, double want) {
  if (n <= 1 || want <= 1.0) return 0;
  int hist[31] = {0};
  for (int l = 1; l < n; ++l) ++hist[lead_equal(code[l - 1], code[l])];
  int best = 0;
  double best_err = 1e300, runs = 1.0;
  for (int b = 0; b <= 30; ++b) {
    if (b > 0) runs += hist[b - 1];
    double err = std::fabs(std::log(runs / want));
    if (err < best_err) {
      best_err = err;
      best = b;
    }
  }
  return best;
}

// run starts of equal (code >> (30 - b)), short runs joined to the previous run (a short
// first run to the next one)
void cut_runs(const uint32_t* code, int n, int b, std::vector<int>& starts) {
  starts.clear();
  if (n <= 0) return;
  const int sh = 30 - b;
  std::vector<int> raw{0};
  for (int l = 1; l < n; ++l)
    if (b > 0 && (code[l] >> sh) != (code[l - 1] >> sh)) raw.push_back(l);
  for (size_t r = 0; r < raw.size(); ++r) {
    int e = r + 1 < raw.size() ? raw[r + 1] : n;
    if (starts.empty() || e - raw[r] >= kMinAggRows) starts.push_back(raw[r]);
  }
  if (starts.size() >= 2 && starts[1] - starts[0] < kMinAggRows) starts.erase(starts.begin() + 1);
}

}  // namespace

void build_aggregates(const HostPlan& hp, int target_rows, int max_agg, AggPlan& ap) {
  const int n_sd = hp.n_sd;
  ap = AggPlan();
  ap.aloc.assign(hp.nP, 0);
  ap.aoff.assign(n_sd + 1, 0);
  ap.nca[0].assign(n_sd, 0);
  ap.nca[1].assign(n_sd, 0);
  std::vector<int> sI, sB;
  for (int i = 0; i < n_sd; ++i) {
    const int nI = hp.nI[i], nB = hp.nB[i];
    const uint32_t* cI = hp.p_code.data() + hp.Poff[i];
    const uint32_t* cB = cI + nI;
    double t = std::max(1, target_rows);
    for (int attempt = 0; attempt < 64; ++attempt) {
      cut_runs(cI, nI, pick_bits(cI, nI, nI / t), sI);
      cut_runs(cB, nB, pick_bits(cB, nB, nB / t), sB);
      if ((int)(sI.size() + sB.size()) <= max_agg) break;
      t *= 1.25;
    }
    int32_t* al = ap.aloc.data() + hp.Poff[i];
    for (size_t r = 0; r < sI.size(); ++r) {
      int e = r + 1 < sI.size() ? sI[r + 1] : nI;
      for (int l = sI[r]; l < e; ++l) al[l] = (int32_t)r;
    }
    for (size_t r = 0; r < sB.size(); ++r) {
      int e = r + 1 < sB.size() ? sB[r + 1] : nB;
      for (int l = sB[r]; l < e; ++l) al[nI + l] = (int32_t)(sI.size() + r);
    }
    ap.nca[0][i] = (int32_t)sI.size();
    ap.nca[1][i] = (int32_t)(sI.size() + sB.size());
    ap.aoff[i + 1] = ap.aoff[i] + ap.nca[1][i];
  }
  const int64_t n_agg = ap.aoff[n_sd];
  for (int set = 0; set < 2; ++set) {
    const HostTiles& T = set == 0 ? hp.tP_I : hp.tP_all;
    const size_t nt = T.sd.size();
    ap.toff[set].assign(nt + 1, 0);
    ap.tfirst[set].assign(n_agg, 0);
    ap.tcount[set].assign(n_agg, 0);
    for (size_t t = 0; t < nt; ++t) {
      const int sd = T.sd[t];
      const int a0 = ap.aloc[T.r0[t]], a1 = ap.aloc[T.r1[t] - 1];
      const int ns = a1 - a0 + 1;
      ap.max_slots = std::max(ap.max_slots, ns);
      ap.toff[set][t + 1] = ap.toff[set][t] + ns;
      for (int a = a0; a <= a1; ++a) {
        int64_t ga = ap.aoff[sd] + a;
        if (ap.tcount[set][ga]++ == 0) ap.tfirst[set][ga] = (int32_t)t;
      }
    }
    ap.eoff[set].assign(n_sd + 1, 0);
    for (int i = 0; i < n_sd; ++i)
      ap.eoff[set][i + 1] = ap.eoff[set][i] + (int64_t)ap.nca[set][i] * ap.nca[set][i];
  }
}

}  // namespace mor
