// Host-side plan of step 1 (Sec. 3, Sec. 6 step 1, Sec. 7.1): subdomain index sets,
// the batched row spaces, sparsity patterns, assembly incidence and interface pairs.
// Pure C++; no CUDA types.
#pragma once
#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

namespace mor {

// Allocator whose resize() leaves new elements default-initialised (uninitialised for
// integers): the large plan arrays are written in full by the threads that build them,
// so no serial zero fill touches their pages first.
template <class T>
struct UninitAlloc : std::allocator<T> {
  template <class U>
  struct rebind {
    using other = UninitAlloc<U>;
  };
  UninitAlloc() = default;
  template <class U>
  UninitAlloc(const UninitAlloc<U>&) noexcept {}
  template <class U>
  void construct(U* p) noexcept {
    ::new (static_cast<void*>(p)) U;
  }
  template <class U, class... A>
  void construct(U* p, A&&... a) {
    ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};
template <class T>
using BigVec = std::vector<T, UninitAlloc<T>>;

constexpr int kSlice = 32;      // sliced-ELL slice height (rows)
constexpr int kTileRows = 128;  // rows per CUDA block tile in row-tiled kernels
constexpr uint32_t kNoSlot = 127;

// Fixed-stride sliced ELL pattern: slice s holds rows [32 s, 32 s + 32); entry (row r,
// slot j) lives at (r >> 5) * 32 * W + j * 32 + (r & 31); col = -1 marks padding.
struct HostEll {
  int64_t n_rows = 0;
  int32_t W = 0;
  std::vector<int32_t> width;  // per slice
  BigVec<int32_t> col;
};

// Row tiles of one row set; a tile never straddles two subdomains.
struct HostTiles {
  std::vector<int32_t> sd, r0, r1;   // per tile
  std::vector<int32_t> lo, hi;       // per subdomain: tile range
};

struct SubSets {
  std::vector<int32_t> I, B, omega, owned, plus_tets, omega_tets;  // ascending node ids
  // the rows of I and B in P-space order: each sorted by the Morton code of the node
  // position in the bounding box of T_i^+ (codes in pcode, I rows then B rows), so a
  // box of any dyadic size holds a contiguous run of rows
  std::vector<int32_t> Ip, Bp;
  std::vector<uint32_t> pcode;
};

struct HostPlan {
  int64_t n_nodes = 0, n_tets = 0;
  int32_t n_sd = 0;
  int32_t r_hops = 0;           // < 0: per-subdomain rule, see r_sd
  std::vector<int32_t> r_sd;    // hops used for each subdomain
  std::vector<SubSets> sets;
  // batched row spaces: P (I then B rows of every omega_i^+), W (free nodes of every
  // omega_i), O (owned free nodes)
  std::vector<int64_t> Poff, Woff, Ooff;
  std::vector<int32_t> nI, nB;
  int64_t nP = 0, nW = 0, nO = 0;
  std::vector<int32_t> p_node, p_sd, w_node, w_sd, w2p, w2o, o2w, o_node, o_sd;
  std::vector<uint8_t> p_isB;
  std::vector<uint32_t> p_code;  // 30-bit Morton code of each P row (see SubSets)
  std::vector<std::vector<int32_t>> Pown;  // owned nodes of each subdomain (global plan)
  // patterns on T_i^+ (P space) and omega_i (W space); columns are space indices
  HostEll pat_P, pat_W;
  // assembly incidence, CSR over rows: element id and code
  // code bits 0..1 = local vertex a of the row, bits 2+7b..8+7b = slot of vertex b
  // in the row's pattern (kNoSlot = not a DOF)
  std::vector<int64_t> incP_ptr, incW_ptr;
  BigVec<int32_t> incP_tet, incW_tet;
  BigVec<uint32_t> incP_code, incW_code;
  HostTiles tP_all, tP_I, tP_B, tW, tO;
  // interface entries (u in sd i, v in sd j, i < j, u ~ v through an element)
  std::vector<int32_t> pair_i, pair_j;
  std::vector<int64_t> pair_ptr;
  std::vector<int32_t> e_urow, e_vrow, e_unode, e_vnode;  // O rows and global nodes
  // global node -> element incidence
  std::vector<int64_t> n2t_ptr;
  std::vector<int32_t> n2t;
  // global plan only: node adjacency over element edges (ascending, without the node)
  std::vector<int64_t> adj_ptr;
  std::vector<int32_t> adj;
};

// Aggregates of the coarse level of the local preconditioner: the I rows and the B rows
// of each subdomain (Morton order) are cut into runs of equal Morton prefix, the prefix
// length per segment chosen for about target_rows rows a run; runs shorter than 8 rows
// join a neighbouring run of their segment; at most max_agg runs per subdomain (coarser
// prefixes otherwise).  I aggregates are numbered first.  Set 0 = the I tiles (A_II
// solves, I aggregates), set 1 = all P tiles (H^+ solves, all aggregates).
struct AggPlan {
  std::vector<int32_t> aloc;        // per P row: aggregate within its subdomain
  std::vector<int32_t> aoff;        // n_sd + 1: global id of the first aggregate
  std::vector<int32_t> nca[2];      // per subdomain: aggregates of set 0 / 1
  std::vector<int64_t> toff[2];     // per tile + 1: partial rows of the tile
  std::vector<int32_t> tfirst[2], tcount[2];  // per global aggregate
  std::vector<int64_t> eoff[2];     // n_sd + 1: offsets of the nca x nca blocks
  int max_slots = 0;                // most aggregates meeting one tile
};
void build_aggregates(const HostPlan& hp, int target_rows, int max_agg, AggPlan& ap);

// Returns 0 or a MOR_ERR_* code (err receives a message).
// xyz (host, n_nodes x 3) orders the rows of each subdomain; with xyz = nullptr they
// stay in ascending node order (all codes 0).
int build_host_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                    const uint8_t* dirichlet, const int32_t* owner, int32_t r_hops,
                    const double* xyz, HostPlan& hp, std::string& err);

// The two halves of build_host_plan, for meshes whose per-subdomain structures do not fit
// at once.  build_global_plan: n_sd, r_sd, node -> element incidence, owned sets (Pown),
// the global O space (Ooff, o_node, o_sd) and the interface entries.  build_wave_plan:
// the per-subdomain sets, row spaces, patterns, incidences and tiles of subdomains
// [s0, s1), numbered 0 .. s1 - s0 - 1, using the incidence and owned sets of g; its O
// rows are the global O rows [g.Ooff[s0], g.Ooff[s1]) in the same order.
struct PlanScratch {
  struct Impl;
  Impl* impl;
  PlanScratch();
  ~PlanScratch();
  PlanScratch(const PlanScratch&) = delete;
  PlanScratch& operator=(const PlanScratch&) = delete;
};
int build_global_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                      const uint8_t* dirichlet, const int32_t* owner, int32_t r_hops,
                      HostPlan& g, std::string& err);
int build_wave_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                    const uint8_t* dirichlet, const double* xyz, const HostPlan& g, int s0,
                    int s1, HostPlan& w, PlanScratch& ps, std::string& err);

}  // namespace mor
