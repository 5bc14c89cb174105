// Host-side plan of step 1 (Sec. 3, Sec. 6 step 1, Sec. 7.1): subdomain index sets,
// the batched row spaces, sparsity patterns, assembly incidence and interface pairs.
// Pure C++; no CUDA types.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace mor {

constexpr int kSlice = 32;      // sliced-ELL slice height (rows)
constexpr int kTileRows = 128;  // rows per CUDA block tile in row-tiled kernels
constexpr uint32_t kNoSlot = 127;

// Fixed-stride sliced ELL pattern: slice s holds rows [32 s, 32 s + 32); entry (row r,
// slot j) lives at (r >> 5) * 32 * W + j * 32 + (r & 31); col = -1 marks padding.
struct HostEll {
  int64_t n_rows = 0;
  int32_t W = 0;
  std::vector<int32_t> width;  // per slice
  std::vector<int32_t> col;
};

// Row tiles of one row set; a tile never straddles two subdomains.
struct HostTiles {
  std::vector<int32_t> sd, r0, r1;   // per tile
  std::vector<int32_t> lo, hi;       // per subdomain: tile range
};

struct SubSets {
  std::vector<int32_t> I, B, omega, owned, plus_tets, omega_tets;
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
  // patterns on T_i^+ (P space) and omega_i (W space); columns are space indices
  HostEll pat_P, pat_W;
  // assembly incidence, CSR over rows: element id and code
  // code bits 0..1 = local vertex a of the row, bits 2+7b..8+7b = slot of vertex b
  // in the row's pattern (kNoSlot = not a DOF)
  std::vector<int64_t> incP_ptr, incW_ptr;
  std::vector<int32_t> incP_tet, incW_tet;
  std::vector<uint32_t> incP_code, incW_code;
  HostTiles tP_all, tP_I, tP_B, tW, tO;
  // interface entries (u in sd i, v in sd j, i < j, u ~ v through an element)
  std::vector<int32_t> pair_i, pair_j;
  std::vector<int64_t> pair_ptr;
  std::vector<int32_t> e_urow, e_vrow, e_unode, e_vnode;  // O rows and global nodes
  // global node -> element incidence
  std::vector<int64_t> n2t_ptr;
  std::vector<int32_t> n2t;
};

// Returns 0 or a MOR_ERR_* code (err receives a message).
int build_host_plan(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                    const uint8_t* dirichlet, const int32_t* owner, int32_t r_hops,
                    HostPlan& hp, std::string& err);

}  // namespace mor
