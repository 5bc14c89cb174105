// C ABI of libmor (include/mor.h): handles, device memory, and the launch sequence of
// the three steps of the paper's framework (Sec. 6) on one GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <future>
#include <mutex>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mor.h"
#include "mor_kernels.h"
#include "mor_plan.h"

using namespace mor;

std::atomic<long long> mor::g_kernel_launches{0};

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(expr)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (expr);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return fail(e_ == cudaErrorMemoryAllocation ? MOR_ERR_OOM : MOR_ERR_CUDA,      \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));               \
  } while (0)

#define TRY(expr)              \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != MOR_OK) return rc_; \
  } while (0)

// Device allocations owned by one object.  Handle memory uses cudaMalloc.  A call's
// workspace is "pooled": stream-ordered allocations from the device's default memory
// pool on the call's stream, freed on that stream when the workspace goes out of
// scope, so repeated calls reuse memory without cudaMalloc/cudaFree synchronisation.
void keep_default_pool_warm() {
  static std::mutex mu;
  static std::vector<int> done;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lock(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;  // freed blocks stay in the pool (this process only)
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  done.push_back(dev);
}

struct Allocs {
  std::vector<void*> ptrs;
  bool pooled = false;
  cudaStream_t pool_st = nullptr;
  Allocs() = default;
  Allocs(const Allocs&) = delete;
  Allocs& operator=(const Allocs&) = delete;
  void use_pool(cudaStream_t st) {
    keep_default_pool_warm();
    pooled = true;
    pool_st = st;
  }
  ~Allocs() {
    for (void* p : ptrs) {
      if (pooled)
        cudaFreeAsync(p, pool_st);
      else
        cudaFree(p);
    }
  }
  template <class T>
  int alloc(T** p, size_t n, bool zero = true, cudaStream_t st = nullptr) {
    if (n == 0) n = 1;
    cudaError_t e = pooled ? cudaMallocAsync((void**)p, n * sizeof(T), pool_st)
                           : cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
      *p = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? MOR_ERR_OOM : MOR_ERR_CUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ptrs.push_back(*p);
    if (zero) {
      e = cudaMemsetAsync(*p, 0, n * sizeof(T), st);
      if (e != cudaSuccess) return fail(MOR_ERR_CUDA, cudaGetErrorString(e));
    }
    return MOR_OK;
  }
  template <class T, class Al>
  int upload(T** p, const std::vector<T, Al>& h, cudaStream_t st) {
    TRY(alloc(p, h.size(), false));
    if (!h.empty()) {
      cudaError_t e = cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T),
                                      cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return fail(MOR_ERR_CUDA, cudaGetErrorString(e));
    }
    return MOR_OK;
  }
};

int upload_tiles(Allocs& A, const HostTiles& h, DTiles& d, cudaStream_t st) {
  int32_t *sd, *r0, *r1, *lo, *hi;
  TRY(A.upload(&sd, h.sd, st));
  TRY(A.upload(&r0, h.r0, st));
  TRY(A.upload(&r1, h.r1, st));
  TRY(A.upload(&lo, h.lo, st));
  TRY(A.upload(&hi, h.hi, st));
  d.n = (int)h.sd.size();
  d.n_sd = (int)h.lo.size();
  d.sd = sd;
  d.r0 = r0;
  d.r1 = r1;
  d.lo = lo;
  d.hi = hi;
  return MOR_OK;
}

// ---- kernel timing (roofline) ------------------------------------------------------
// family = 2 * kind + wide (kind 0 sparse product, 1 x/r update, 2 p update, 3 coarse
// solve).  The events of one step: before the product, after the product, after the
// x/r update, after the coarse kernel, after the p update.
constexpr int kFamilies = 8;
struct Prof {
  bool on = false;
  double launches[kFamilies] = {}, ms[kFamilies] = {}, bytes[kFamilies] = {};
  std::vector<std::array<cudaEvent_t, 5>> pool;
  struct Pending {
    int wide;
    double bytes[4];
    size_t ev;
  };
  std::vector<Pending> pending;
  size_t used = 0;
  const cudaEvent_t* take() {
    if (used == pool.size()) {
      std::array<cudaEvent_t, 5> e;
      for (auto& x : e) cudaEventCreate(&x);
      pool.push_back(e);
    }
    return pool[used++].data();
  }
  void collect() {
    // event interval of each kind: product [0,1], x/r [1,2], p update [3,4], coarse [2,3]
    static const int from[4] = {0, 1, 3, 2};
    for (auto& p : pending)
      for (int kind = 0; kind < 4; ++kind) {
        float t = 0.f;
        int e0 = from[kind];
        if (cudaEventElapsedTime(&t, pool[p.ev][e0], pool[p.ev][e0 + 1]) == cudaSuccess) {
          int f = 2 * kind + p.wide;
          launches[f] += 1;
          ms[f] += t;
          bytes[f] += p.bytes[kind];
        }
      }
    pending.clear();
    used = 0;
  }
};
Prof g_prof;

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// budget of the bounded device-side waits, seconds of SM clock
double g_wait_budget_s = 1.0;
long long wait_budget_cycles() {
  int dev = 0, khz = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
  if (khz <= 0) khz = 2000000;
  return (long long)(g_wait_budget_s * 1e3 * (double)khz);
}
int round_up4(int x) { return (x + 3) & ~3; }

}  // namespace

// error reporting for the other translation units (same thread-local message)
int mor::set_error(int code, const std::string& msg) { return fail(code, msg); }

// ======================================================================================
struct mor_subdomains_s {
  HostPlan hp;
  Allocs mem;
  const double* xyz = nullptr;
  const int32_t* tets = nullptr;
  const double* kappa = nullptr;
  int32_t *p_node, *p_sd, *w_node, *w_sd, *w2p, *w2o, *o2w, *o_node, *o_sd;
  uint8_t* p_isB;
  int32_t *patP_col, *patP_w, *patW_col, *patW_w;
  int64_t *incP_ptr, *incW_ptr;
  int32_t *incP_tet, *incW_tet;
  uint32_t *incP_code, *incW_code;
  DTiles tP_all, tP_I, tP_B, tW, tO;
  int64_t* pair_ptr;
  int32_t *e_urow, *e_vrow, *e_unode, *e_vnode;
  int64_t* n2t_ptr;
  int32_t* n2t;
  std::vector<int32_t> nbr_ptr, nbr_sd, nbr_blk;
  int64_t n_iface = 0;
  int max_tiles = 0;
  // streamed plans (mor_build_subdomains_streamed): hp holds the global part only and
  // mor_build_bases builds the per-subdomain part wave by wave from these host copies
  bool streamed = false;
  int wave_sd = 0;
  int sd_base = 0;  // batch id of this plan's first subdomain (waves of a streamed plan)
  std::vector<int32_t> h_tets;
  std::vector<uint8_t> h_dir;
  std::vector<double> h_xyz;
};

struct mor_bases_s {
  int n_sd = 0, k = 0, kp = 0, kq = 0, m = 0;
  Allocs mem;
  // R_BB per subdomain (paper sketch or explicit SVD only)
  double* Rbb = nullptr;
  std::vector<int64_t> rbb_off;
  std::vector<int32_t> rbb_m;
  bool tc = false;  // tc_gram 2: the interface blocks of step 3 on the tensor cores too
  double *Q = nullptr, *bt = nullptr, *sigma = nullptr;
  int* kept = nullptr;
  std::vector<int32_t> h_kept;
  std::vector<double> h_sigma;
  std::vector<int64_t> Ooff;
  int64_t stats[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

struct mor_reduced_s {
  int n_sd = 0, kq = 0, n_pairs = 0;
  int64_t dim = 0;
  Allocs mem;
  double* blocks = nullptr;
  double* bt = nullptr;
  int32_t *nbr_ptr, *nbr_sd, *nbr_blk;
  std::vector<int32_t> h_nbr_ptr, h_nbr_sd, h_nbr_blk;
};

// ======================================================================================
extern "C" {

const char* mor_last_error(void) { return g_err.c_str(); }

}  // extern "C"

namespace {

// device copies of the per-subdomain part of a plan (sets, row spaces, patterns,
// incidences, tiles)
int upload_heavy(mor_subdomains_s* h, cudaStream_t st) {
  const HostPlan& hp = h->hp;
  Allocs& A = h->mem;
  TRY(A.upload(&h->p_node, hp.p_node, st));
  TRY(A.upload(&h->p_sd, hp.p_sd, st));
  TRY(A.upload(&h->p_isB, hp.p_isB, st));
  TRY(A.upload(&h->w_node, hp.w_node, st));
  TRY(A.upload(&h->w_sd, hp.w_sd, st));
  TRY(A.upload(&h->w2p, hp.w2p, st));
  TRY(A.upload(&h->w2o, hp.w2o, st));
  TRY(A.upload(&h->o2w, hp.o2w, st));
  TRY(A.upload(&h->patP_col, hp.pat_P.col, st));
  TRY(A.upload(&h->patP_w, hp.pat_P.width, st));
  TRY(A.upload(&h->patW_col, hp.pat_W.col, st));
  TRY(A.upload(&h->patW_w, hp.pat_W.width, st));
  TRY(A.upload(&h->incP_ptr, hp.incP_ptr, st));
  TRY(A.upload(&h->incW_ptr, hp.incW_ptr, st));
  TRY(A.upload(&h->incP_tet, hp.incP_tet, st));
  TRY(A.upload(&h->incW_tet, hp.incW_tet, st));
  TRY(A.upload(&h->incP_code, hp.incP_code, st));
  TRY(A.upload(&h->incW_code, hp.incW_code, st));
  TRY(upload_tiles(A, hp.tP_all, h->tP_all, st));
  TRY(upload_tiles(A, hp.tP_I, h->tP_I, st));
  TRY(upload_tiles(A, hp.tP_B, h->tP_B, st));
  TRY(upload_tiles(A, hp.tW, h->tW, st));
  TRY(upload_tiles(A, hp.tO, h->tO, st));
  h->max_tiles = std::max({h->tP_all.n, h->tW.n, h->tO.n, h->tP_B.n, 1});
  return MOR_OK;
}

// device copies of the global part (O space, interface entries, incidence) and the
// block-sparse neighbour structure of the reduced matrix
int upload_light(mor_subdomains_s* h, cudaStream_t st) {
  const HostPlan& hp = h->hp;
  Allocs& A = h->mem;
  TRY(A.upload(&h->o_node, hp.o_node, st));
  TRY(A.upload(&h->o_sd, hp.o_sd, st));
  TRY(A.upload(&h->pair_ptr, hp.pair_ptr, st));
  TRY(A.upload(&h->e_urow, hp.e_urow, st));
  TRY(A.upload(&h->e_vrow, hp.e_vrow, st));
  TRY(A.upload(&h->e_unode, hp.e_unode, st));
  TRY(A.upload(&h->e_vnode, hp.e_vnode, st));
  TRY(A.upload(&h->n2t_ptr, hp.n2t_ptr, st));
  TRY(A.upload(&h->n2t, hp.n2t, st));
  h->n_iface = (int64_t)hp.e_urow.size();
  // pair p gives blocks 2p = (i, j) and 2p + 1 = (j, i)
  std::vector<std::vector<std::pair<int32_t, int32_t>>> rows(hp.n_sd);
  for (size_t p = 0; p < hp.pair_i.size(); ++p) {
    rows[hp.pair_i[p]].emplace_back(hp.pair_j[p], (int32_t)(2 * p));
    rows[hp.pair_j[p]].emplace_back(hp.pair_i[p], (int32_t)(2 * p + 1));
  }
  h->nbr_ptr.assign(1, 0);
  for (auto& r : rows) {
    std::sort(r.begin(), r.end());
    for (auto& e : r) {
      h->nbr_sd.push_back(e.first);
      h->nbr_blk.push_back(e.second);
    }
    h->nbr_ptr.push_back((int32_t)h->nbr_sd.size());
  }
  return MOR_OK;
}

int mesh_xyz_host(const mor_mesh* mesh, std::vector<double>& xyz, cudaStream_t st) {
  xyz.resize((size_t)mesh->n_nodes * 3);
  if (!xyz.empty()) {
    CK(cudaMemcpyAsync(xyz.data(), mesh->xyz_dev, xyz.size() * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
  }
  return MOR_OK;
}

}  // namespace

extern "C" {

int mor_build_subdomains(const mor_mesh* mesh, const int32_t* owner, int32_t r_hops,
                         void* stream, mor_subdomains** out) {
  if (!mesh || !owner || !out) return fail(MOR_ERR_ARG, "mor_build_subdomains: null argument");
  if (!mesh->xyz_dev || !mesh->tets_dev || !mesh->kappa_dev)
    return fail(MOR_ERR_ARG, "mor_build_subdomains: null device mesh array");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  auto h = std::make_unique<mor_subdomains_s>();
  std::string err;
  // node positions order the rows of each subdomain (Morton order within I and B)
  std::vector<double> xyz_host;
  TRY(mesh_xyz_host(mesh, xyz_host, st));
  int rc = build_host_plan(mesh->n_nodes, mesh->n_tets, mesh->tets, mesh->dirichlet, owner,
                           r_hops, xyz_host.empty() ? nullptr : xyz_host.data(), h->hp, err);
  if (rc != MOR_OK) return fail(rc, err);
  h->xyz = mesh->xyz_dev;
  h->tets = mesh->tets_dev;
  h->kappa = mesh->kappa_dev;
  TRY(upload_heavy(h.get(), st));
  TRY(upload_light(h.get(), st));
  CK(cudaStreamSynchronize(st));
  *out = h.release();
  return MOR_OK;
}

int mor_build_subdomains_streamed(const mor_mesh* mesh, const int32_t* owner, int32_t r_hops,
                                  int32_t wave_subdomains, void* stream,
                                  mor_subdomains** out) {
  if (!mesh || !owner || !out || wave_subdomains < 1)
    return fail(MOR_ERR_ARG, "mor_build_subdomains_streamed: bad argument");
  if (!mesh->xyz_dev || !mesh->tets_dev || !mesh->kappa_dev)
    return fail(MOR_ERR_ARG, "mor_build_subdomains_streamed: null device mesh array");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  auto h = std::make_unique<mor_subdomains_s>();
  std::string err;
  int rc = build_global_plan(mesh->n_nodes, mesh->n_tets, mesh->tets, mesh->dirichlet, owner,
                             r_hops, h->hp, err);
  if (rc != MOR_OK) return fail(rc, err);
  h->streamed = true;
  h->wave_sd = wave_subdomains;
  h->h_tets.assign(mesh->tets, mesh->tets + 4 * mesh->n_tets);
  h->h_dir.assign(mesh->dirichlet, mesh->dirichlet + mesh->n_nodes);
  TRY(mesh_xyz_host(mesh, h->h_xyz, st));
  h->xyz = mesh->xyz_dev;
  h->tets = mesh->tets_dev;
  h->kappa = mesh->kappa_dev;
  TRY(upload_light(h.get(), st));
  CK(cudaStreamSynchronize(st));
  *out = h.release();
  return MOR_OK;
}

int mor_build_subdomains_host(const mor_mesh_host* mesh, const int32_t* owner,
                              int32_t r_hops, int32_t wave_subdomains, void* stream,
                              mor_subdomains** out) {
  if (!mesh || !owner || !out || !mesh->tets || !mesh->dirichlet || !mesh->xyz ||
      !mesh->kappa || mesh->n_nodes < 1 || mesh->n_tets < 1 || wave_subdomains < 0)
    return fail(MOR_ERR_ARG, "mor_build_subdomains_host: bad argument");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  auto h = std::make_unique<mor_subdomains_s>();
  // device copies owned by the handle; the host -> device copies overlap step 1 on the
  // host, which reads the host arrays directly
  double *xyz_d, *kappa_d;
  int32_t* tets_d;
  Allocs& A = h->mem;
  TRY(A.alloc(&xyz_d, (size_t)mesh->n_nodes * 3, false, st));
  TRY(A.alloc(&tets_d, (size_t)mesh->n_tets * 4, false, st));
  TRY(A.alloc(&kappa_d, (size_t)mesh->n_tets, false, st));
  CK(cudaMemcpyAsync(xyz_d, mesh->xyz, (size_t)mesh->n_nodes * 3 * sizeof(double),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(tets_d, mesh->tets, (size_t)mesh->n_tets * 4 * sizeof(int32_t),
                     cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(kappa_d, mesh->kappa, (size_t)mesh->n_tets * sizeof(double),
                     cudaMemcpyHostToDevice, st));
  std::string err;
  int rc;
  if (wave_subdomains > 0) {
    rc = build_global_plan(mesh->n_nodes, mesh->n_tets, mesh->tets, mesh->dirichlet, owner,
                           r_hops, h->hp, err);
    if (rc != MOR_OK) {
      cudaStreamSynchronize(st);  // the copies read the caller's arrays
      return fail(rc, err);
    }
    h->streamed = true;
    h->wave_sd = wave_subdomains;
    h->h_tets.assign(mesh->tets, mesh->tets + 4 * mesh->n_tets);
    h->h_dir.assign(mesh->dirichlet, mesh->dirichlet + mesh->n_nodes);
    h->h_xyz.assign(mesh->xyz, mesh->xyz + 3 * mesh->n_nodes);
  } else {
    rc = build_host_plan(mesh->n_nodes, mesh->n_tets, mesh->tets, mesh->dirichlet, owner,
                         r_hops, mesh->xyz, h->hp, err);
    if (rc != MOR_OK) {
      cudaStreamSynchronize(st);
      return fail(rc, err);
    }
  }
  h->xyz = xyz_d;
  h->tets = tets_d;
  h->kappa = kappa_d;
  if (!h->streamed) TRY(upload_heavy(h.get(), st));
  TRY(upload_light(h.get(), st));
  CK(cudaStreamSynchronize(st));
  *out = h.release();
  return MOR_OK;
}

int mor_subdomains_counts(const mor_subdomains* h, int32_t* n_sub_out, int64_t* counts) {
  if (!h) return fail(MOR_ERR_ARG, "mor_subdomains_counts: null handle");
  if (n_sub_out) *n_sub_out = h->hp.n_sd;
  if (counts && h->streamed) {
    // only the global part is kept: owned DOFs and hops; the rest is -1
    for (int i = 0; i < h->hp.n_sd; ++i) {
      int64_t* c = counts + 7 * (int64_t)i;
      for (int q = 0; q < 7; ++q) c[q] = -1;
      c[3] = h->hp.Ooff[i + 1] - h->hp.Ooff[i];
      c[6] = (int64_t)h->hp.r_sd[i];
    }
    return MOR_OK;
  }
  if (counts)
    for (int i = 0; i < h->hp.n_sd; ++i) {
      const SubSets& s = h->hp.sets[i];
      int64_t* c = counts + 7 * (int64_t)i;
      c[0] = (int64_t)s.I.size();
      c[1] = (int64_t)s.B.size();
      c[2] = (int64_t)s.omega.size();
      c[3] = (int64_t)s.owned.size();
      c[4] = (int64_t)s.plus_tets.size();
      c[5] = (int64_t)s.omega_tets.size();
      c[6] = (int64_t)h->hp.r_sd[i];
    }
  return MOR_OK;
}

int mor_subdomains_indices(const mor_subdomains* h, int32_t sub, int32_t which, int32_t* out) {
  if (!h || !out || sub < 0 || sub >= h->hp.n_sd || which < 0 || which > 5)
    return fail(MOR_ERR_ARG, "mor_subdomains_indices: bad argument");
  if (h->streamed)
    return fail(MOR_ERR_STATE, "mor_subdomains_indices: streamed plans keep no index sets");
  const SubSets& s = h->hp.sets[sub];
  const std::vector<int32_t>* v[6] = {&s.I, &s.B, &s.omega, &s.owned, &s.plus_tets,
                                      &s.omega_tets};
  std::memcpy(out, v[which]->data(), v[which]->size() * sizeof(int32_t));
  return MOR_OK;
}

int mor_basis_opts_default(mor_basis_opts* o) {
  if (!o) return fail(MOR_ERR_ARG, "mor_basis_opts_default: null");
  o->rank = 8;
  o->oversample = 5;
  o->ranks = nullptr;
  o->eps = 0.0;
  o->seed = 0;
  o->precision = MOR_MIXED;
  o->sketch = MOR_SKETCH_FIELD;
  o->cg_rtol = 1e-9;
  o->max_iter = 20000;
  o->replace_every = 40;
  o->normwise = 1;
  o->drift_restart = 1.5;
  o->sketch_rtol = 0.0;
  o->tau = 1e-12;
  o->orth_tol = 1e-14;
  o->coarse_rows = -1;
  o->h1_weighted = 0;
  o->sketch_div = 0;
  o->tc_gram = 1;
  o->explicit_svd = 0;
  o->sub_begin = 0;
  o->sub_end = 0;
  return MOR_OK;
}

}  // extern "C"

// ======================================================================================
namespace {

// device matrices of one build
struct Mat {
  int32_t *width = nullptr, *col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  int W = 0;
  EllView<double> e64() const { return EllView<double>{width, col, v64, W}; }
  EllView<float> e32() const { return EllView<float>{width, col, v32, W}; }
};

struct Build {
  const mor_subdomains_s* S;
  const mor_basis_opts* o;
  cudaStream_t st;
  Allocs mem;
  int n_sd, k, kp, kq, m;
  bool mixed;
  // pinned poll word
  int* h_poll = nullptr;
  int* d_poll = nullptr;
  // workspace
  double *vR64 = nullptr;
  void *xT = nullptr, *rT = nullptr, *pT = nullptr, *qT = nullptr, *bT = nullptr;
  CgState cs{};
  RefineState rs{};
  int64_t iters[4] = {0, 0, 0, 0};
  int64_t sweeps = 0, not_conv = 0, floor_cols = 0;
  bool debug = getenv("MOR_DEBUG") != nullptr;
  ~Build() {
    if (h_poll) cudaFreeHost(h_poll);
  }

  // sum of active[] over the subdomains (and of second[] into h_poll[1])
  int poll(const int* active, const int* second = nullptr) {
    launch_count_active(n_sd, active, d_poll, st, second);
    CK(cudaMemcpyAsync(h_poll, d_poll, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return h_poll[0];
  }
  // per matrix set: max row sum of |A| per subdomain (rounding-level bound)
  double* anorm[2] = {nullptr, nullptr};
  // per matrix set (profiling only): rows and stored entries of each subdomain
  int32_t* sd_rows[2] = {nullptr, nullptr};
  int64_t* sd_nnz[2] = {nullptr, nullptr};

  // coarse levels of the two-level preconditioner: [0] A_II (I tiles), [1] H^+ (all P
  // tiles)
  Coarse<float> co32[2];
  Coarse<double> co64[2];
  template <typename T>
  const Coarse<T>& coarse_of(int set) const {
    if constexpr (sizeof(T) == 4)
      return co32[set];
    else
      return co64[set];
  }

  template <typename T>
  int solve(const DTiles& tl, const Mat& A, const T* dinvT, const double* b64, double* x64,
            int nc, int which, double rtol, int set) {
    const Coarse<T>& co = coarse_of<T>(set);
    cs.sd_rows = sd_rows[set];
    cs.sd_nnz = sd_nnz[set];
    // columns [0, ncn) share the block-normwise reference; the load column (forward
    // solve, column k) keeps its own
    const int ncn = o->normwise ? std::min(nc, k) : 0;
    EllView<T> AT;
    if constexpr (sizeof(T) == 4)
      AT = A.e32();
    else
      AT = A.e64();
    T* x = (T*)xT;
    T* r = (T*)rT;
    T* p = (T*)pT;
    T* q = (T*)qT;
    T* b = (T*)bT;
    double rtol2 = rtol * rtol;
    double pb[4] = {0, 0, 0, 0};
    // bytes come from the device work counters (cs.work), attributed when the build
    // finishes; the events time every launch
    // one CG per (subdomain, column) in precision T on the full system, with the
    // recursively updated residual replaced by the binary64 residual b - A x64 every
    // replace_every iterations and whenever the recursion reports convergence
    // (residual replacement keeps the search directions, so no Krylov restart)
    launch_zero_rows(tl, x64, kp, st);
    launch_residual64(tl, A.e64(), b64, x64, vR64, kp, nc, ncn, rtol2, 1, false, anorm[set],
                      rs, st);
    if (poll(rs.active) == 0) return MOR_OK;
    launch_cast<T>(tl, vR64, b, kp, st);
    launch_cg_init<T>(tl, b, x, r, p, dinvT, kp, nc, ncn, cs, co, st);
    const int check = 8;
    const int every = std::max(check, o->replace_every / check * check);
    int it = 0;
    while (true) {
      int chunk = std::min(check, o->max_iter - it);
      for (int c = 0; c < chunk; ++c) {
        const cudaEvent_t* ev = nullptr;
        if (g_prof.on) {
          ev = g_prof.take();
          g_prof.pending.push_back(
              Prof::Pending{sizeof(T) == 4 ? 0 : 1, {pb[0], pb[1], pb[2], pb[3]},
                            g_prof.used - 1});
        }
        launch_cg_step<T>(tl, AT, x, r, p, q, dinvT, kp, rtol2, cs, co, st, ev);
      }
      it += chunk;
      int act = poll(cs.active);
      if (act == 0 || it % every == 0 || it >= o->max_iter) {
        launch_accum_reset<T>(tl, x, x64, kp, st);
        launch_residual64(tl, A.e64(), b64, x64, vR64, kp, nc, ncn, rtol2, 0, false,
                          anorm[set], rs, st);
        ++sweeps;
        int ract = poll(rs.active, rs.nnear);
        if (ract > 0 && h_poll[1] > 0) {
          // some open column is within reach of the rounding level: measure the exact
          // reference || |A| |x| + |b| || and test again
          launch_residual64(tl, A.e64(), b64, x64, vR64, kp, nc, ncn, rtol2, 0, true,
                            anorm[set], rs, st);
          ++sweeps;
          ract = poll(rs.active);
        }
        if (debug) {
          std::vector<double> orr((size_t)n_sd * kp), obb((size_t)n_sd * kp);
          cudaMemcpy(orr.data(), rs.orr, orr.size() * sizeof(double), cudaMemcpyDeviceToHost);
          cudaMemcpy(obb.data(), rs.obb, obb.size() * sizeof(double), cudaMemcpyDeviceToHost);
          double worst = 0.0;
          int wi = -1;
          for (size_t i = 0; i < orr.size(); ++i)
            if ((int)(i % kp) < nc && obb[i] > 0 && orr[i] / obb[i] > worst) {
              worst = orr[i] / obb[i];
              wi = (int)i;
            }
          fprintf(stderr, "[mor] solve %d it %d active %d recursive-active %d worst %.3e (sd %d col %d)\n",
                  which, it, ract, act, std::sqrt(worst), wi / kp, wi % kp);
        }
        if (debug && (ract == 0 || it >= o->max_iter)) {
          std::vector<int> its(n_sd);
          cudaMemcpy(its.data(), cs.iters, n_sd * sizeof(int), cudaMemcpyDeviceToHost);
          std::sort(its.begin(), its.end());
          long tot = 0;
          for (int v : its) tot += v;
          fprintf(stderr, "[mor] solve %d recursion iterations per subdomain: min %d median %d max %d "
                  "(busy fraction %.2f)\n", which, its.front(), its[n_sd / 2], its.back(),
                  (double)tot / ((double)n_sd * std::max(1, it)));
        }
        if (ract == 0 || it >= o->max_iter) {
          // columns that ended on the attainable-accuracy test instead of rtol
          std::vector<int> nfl(n_sd);
          CK(cudaMemcpyAsync(nfl.data(), rs.nfloor, n_sd * sizeof(int), cudaMemcpyDeviceToHost,
                             st));
          CK(cudaStreamSynchronize(st));
          for (int v : nfl) floor_cols += v;
          if (ract > 0) not_conv += ract;
          break;
        }
        launch_cg_replace<T>(tl, vR64, r, p, dinvT, kp, o->drift_restart, cs, rs, co, st);
      }
    }
    iters[which] += it;
    CK(cudaGetLastError());
    return MOR_OK;
  }

};

// ---- paper-literal weights (Lemma 4.1, Eq. (14)) with dense per-subdomain factors ----
// Dense H^+ in [I; B] order (I rows in the plan's order, B rows in ascending node order,
// the order of the oracle), its Cholesky factor, and the factor's trailing block L_BB
// with R_BB = L_BB^T (Lemma 4.1: R_BB^T R_BB = S_B).
struct DenseWeights {
  int n_sd = 0, n_max = 0, m_max = 0, i_max = 0;
  std::vector<int32_t> h_nI, h_M, h_nH;
  std::vector<int64_t> h_boff, h_bboff;
  int32_t *p_loc = nullptr, *nI = nullptr, *M = nullptr, *nH = nullptr, *zero = nullptr;
  int32_t *bnode = nullptr, *bprow = nullptr;
  int64_t *hoff = nullptr, *boff = nullptr, *bboff = nullptr;
  double *H = nullptr, *Lbb = nullptr, *Rbb = nullptr;
};

// dense problems above this order are refused (the dense path serves small subdomains,
// as the paper's explicit SVD does)
constexpr int kDenseMaxOrder = 6144;

int dense_weights(const HostPlan& hp, const int32_t* p_sd_dev, Allocs& Mem,
                  const EllView<double>& Hp, DenseWeights& D, cudaStream_t st) {
  const int n_sd = hp.n_sd;
  D.n_sd = n_sd;
  D.h_nI.resize(n_sd);
  D.h_M.resize(n_sd);
  D.h_nH.resize(n_sd);
  std::vector<int32_t> p_loc(hp.nP), bnode, bprow;
  std::vector<int64_t> hoff(n_sd + 1, 0), boff(n_sd + 1, 0), bboff(n_sd + 1, 0);
  for (int i = 0; i < n_sd; ++i) {
    const int nI = hp.nI[i], nB = hp.nB[i];
    const int64_t P0 = hp.Poff[i];
    D.h_nI[i] = nI;
    D.h_M[i] = nB;
    D.h_nH[i] = nI + nB;
    if (nI + nB > kDenseMaxOrder)
      return fail(MOR_ERR_ARG, "mor_build_bases: paper-literal weights need |I| + |B| <= " +
                                   std::to_string(kDenseMaxOrder) + " (dense factors)");
    D.n_max = std::max(D.n_max, nI + nB);
    D.m_max = std::max(D.m_max, nB);
    D.i_max = std::max(D.i_max, nI);
    for (int l = 0; l < nI; ++l) p_loc[P0 + l] = l;
    std::vector<std::pair<int32_t, int64_t>> b(nB);
    for (int l = 0; l < nB; ++l) b[l] = {hp.p_node[P0 + nI + l], P0 + nI + l};
    std::sort(b.begin(), b.end());
    for (int l = 0; l < nB; ++l) {
      p_loc[b[l].second] = nI + l;
      bnode.push_back(b[l].first);
      bprow.push_back((int32_t)b[l].second);
    }
    hoff[i + 1] = hoff[i] + (int64_t)(nI + nB) * (nI + nB);
    boff[i + 1] = boff[i] + nB;
    bboff[i + 1] = bboff[i] + (int64_t)nB * nB;
  }
  D.h_boff = boff;
  D.h_bboff = bboff;
  std::vector<int32_t> zero(n_sd, 0);
  TRY(Mem.upload(&D.p_loc, p_loc, st));
  TRY(Mem.upload(&D.nI, D.h_nI, st));
  TRY(Mem.upload(&D.M, D.h_M, st));
  TRY(Mem.upload(&D.nH, D.h_nH, st));
  TRY(Mem.upload(&D.zero, zero, st));
  TRY(Mem.upload(&D.bnode, bnode, st));
  TRY(Mem.upload(&D.bprow, bprow, st));
  TRY(Mem.upload(&D.hoff, hoff, st));
  TRY(Mem.upload(&D.boff, boff, st));
  TRY(Mem.upload(&D.bboff, bboff, st));
  TRY(Mem.alloc(&D.H, (size_t)hoff[n_sd], true, st));
  TRY(Mem.alloc(&D.Lbb, (size_t)std::max<int64_t>(bboff[n_sd], 1), true, st));
  TRY(Mem.alloc(&D.Rbb, (size_t)std::max<int64_t>(bboff[n_sd], 1), true, st));
  // dense H^+ of every subdomain (order nH = nI + nB), its Cholesky factor in place
  launch_ell_to_dense(hp.nP, p_sd_dev, D.p_loc, D.p_loc, Hp, D.zero, D.nH, D.zero, D.nH, D.nH,
                      D.hoff, D.H, st);
  int* bad;
  TRY(Mem.alloc(&bad, 1, true, st));
  launch_potrf(n_sd, D.n_max, D.H, D.hoff, D.nH, bad, st);
  // L_BB = the trailing nB x nB block of the factor, R_BB = L_BB^T
  launch_transpose_block(n_sd, D.m_max, D.H, D.hoff, D.nH, D.nI, D.M, D.Lbb, D.bboff, 0, st);
  launch_transpose_block(n_sd, D.m_max, D.H, D.hoff, D.nH, D.nI, D.M, D.Rbb, D.bboff, 1, st);
  int h_bad = 0;
  CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h_bad) return fail(MOR_ERR_CUDA, "mor_build_bases: H^+ is not positive definite");
  return MOR_OK;
}

}  // namespace

// step 2 for every subdomain of a plan whose per-subdomain part is on the device;
// m_force > 0 fixes the widest rank (so that waves of a streamed plan share k and kq)
static int build_bases_core(const mor_subdomains* sd, const mor_basis_opts* opts,
                            int m_force, void* stream, mor_bases** out) {
  if (!sd || !opts || !out) return fail(MOR_ERR_ARG, "mor_build_bases: null argument");
  *out = nullptr;
  const mor_basis_opts& o = *opts;
  const int n_sd_h = sd->hp.n_sd;
  const bool tol_mode = o.eps > 0.0;
  if (o.sketch_div < 0) return fail(MOR_ERR_ARG, "mor_build_bases: sketch_div must be >= 0");
  if (o.tc_gram < 0 || o.tc_gram > 2)
    return fail(MOR_ERR_ARG, "mor_build_bases: tc_gram must be 0, 1 or 2");
  if (o.sketch_div > 0 && (!tol_mode || m_force > 0))
    return fail(MOR_ERR_ARG, "mor_build_bases: sketch_div needs eps > 0 and a one-shot plan");
  std::vector<int32_t> h_rank(n_sd_h), h_k(n_sd_h);
  for (int i = 0; i < n_sd_h; ++i) h_rank[i] = o.ranks ? o.ranks[i] : o.rank;
  int m_max = 0;
  for (int i = 0; i < n_sd_h; ++i) {
    if (o.sketch_div > 0) {
      // the paper's sketch size k_i = floor(M_i / 8) (Sec. 7.1): sigma_j > eps among
      // them are kept, so the rank entry is not used
      h_k[i] = std::max(1, sd->hp.nB[i] / o.sketch_div);
      h_rank[i] = h_k[i];
    } else {
      if (h_rank[i] < 1 || o.oversample < 0)
        return fail(MOR_ERR_ARG, "mor_build_bases: ranks >= 1 and oversample >= 0 required");
      h_k[i] = h_rank[i] + o.oversample;
    }
    m_max = std::max(m_max, o.sketch_div > 0 ? h_k[i] : h_rank[i]);
  }
  if (m_force > 0) m_max = std::max(m_max, m_force);
  // widest sketch; the load column sits at k
  const int k = o.sketch_div > 0 ? m_max : m_max + o.oversample;
  const int kp = round_up4(k + 1);
  // columns per subdomain kept for the reduced system: fixed rank m_max + 1; in
  // tolerance mode the widest kept count + 1, known after the weighted SVD (at most k)
  int kq = round_up4((tol_mode ? k : m_max) + 1);
  int mcols = tol_mode ? k : m_max;
  const bool wide = kp > 80;
  if (kp > 512)
    return fail(MOR_ERR_ARG, "mor_build_bases: sketch width must be <= 511 columns");
  if (!tol_mode && kq > 128)
    return fail(MOR_ERR_ARG, "mor_build_bases: rank + 1 must be <= 128 basis columns");
  if (!(o.eps >= 0.0)) return fail(MOR_ERR_ARG, "mor_build_bases: eps must be >= 0");
  if (o.precision != MOR_FP64 && o.precision != MOR_MIXED)
    return fail(MOR_ERR_ARG, "mor_build_bases: unknown precision");
  if (o.sketch != MOR_SKETCH_FIELD && o.sketch != MOR_SKETCH_PAPER)
    return fail(MOR_ERR_ARG, "mor_build_bases: unknown sketch");
  const bool dense = o.sketch == MOR_SKETCH_PAPER || o.explicit_svd != 0;
  if (dense && m_force > 0)
    return fail(MOR_ERR_ARG, "mor_build_bases: paper-literal weights need a one-shot plan");
  if (o.explicit_svd && o.sketch_div > 0)
    return fail(MOR_ERR_ARG, "mor_build_bases: explicit_svd has no sketch (sketch_div)");
  if (!(o.cg_rtol > 0.0) || o.max_iter < 1 || o.replace_every < 1 || !(o.drift_restart >= 1.0))
    return fail(MOR_ERR_ARG, "mor_build_bases: bad solver tolerances");

  cudaStream_t st = (cudaStream_t)stream;
  const mor_subdomains_s& S = *sd;
  const HostPlan& hp = S.hp;
  Build B;
  B.S = &S;
  B.o = opts;
  B.st = st;
  B.n_sd = hp.n_sd;
  B.k = k;
  B.kp = kp;
  B.kq = kq;
  B.m = mcols;
  B.mixed = o.precision == MOR_MIXED;
  Allocs& M = B.mem;
  M.use_pool(st);
  const int n_sd = hp.n_sd;
  const int64_t nP = hp.nP, nW = hp.nW, nO = hp.nO;
  const int WP = hp.pat_P.W, WW = hp.pat_W.W;
  const int64_t nEllP = ceil_div(nP, 32) * 32 * WP;
  const int64_t nEllW = ceil_div(nW, 32) * 32 * WW;
  const int64_t nEllO = ceil_div(nO, 32) * 32 * WW;

  CK(cudaMallocHost((void**)&B.h_poll, 2 * sizeof(int)));
  TRY(M.alloc(&B.d_poll, 2, true, st));
  int* d_err;
  TRY(M.alloc(&d_err, 1, true, st));

  // ---- assembly (Sec. 2, Sec. 4): A^+, H^+ on T_i^+; A, H_i on omega_i ----
  double *valA_P, *valH_P, *loadP, *valA_W, *valH_W, *loadW;
  TRY(M.alloc(&valA_P, nEllP, true, st));
  TRY(M.alloc(&valH_P, nEllP, true, st));
  TRY(M.alloc(&loadP, nP, true, st));
  TRY(M.alloc(&valA_W, nEllW, true, st));
  TRY(M.alloc(&valH_W, nEllW, true, st));
  TRY(M.alloc(&loadW, nW, true, st));
  launch_assemble(nP, S.incP_ptr, S.incP_tet, S.incP_code, WP, S.xyz, S.tets, S.kappa,
                  o.h1_weighted, valA_P,
                  valH_P, loadP, d_err, st);
  launch_assemble(nW, S.incW_ptr, S.incW_tet, S.incW_code, WW, S.xyz, S.tets, S.kappa,
                  o.h1_weighted, valA_W,
                  valH_W, loadW, d_err, st);

  // ---- extraction of the blocks used by the solves ----
  auto make_mat = [&](Mat& mt, int64_t n_rows, int W, bool f32) -> int {
    int64_t n = ceil_div(n_rows, 32) * 32 * W;
    mt.W = W;
    TRY(M.alloc(&mt.width, ceil_div(n_rows, 32), true, st));
    TRY(M.alloc(&mt.col, n, false, st));
    CK(cudaMemsetAsync(mt.col, 0xFF, n * sizeof(int32_t), st));
    TRY(M.alloc(&mt.v64, n, true, st));
    if (f32) TRY(M.alloc(&mt.v32, n, true, st));
    return MOR_OK;
  };
  Mat A_II, A_IB, A_BI, Hp, Hi, App;
  double *dA64, *dH64;
  float *dA32, *dH32;
  TRY(make_mat(A_II, nP, WP, true));
  TRY(make_mat(A_IB, nP, WP, false));
  TRY(make_mat(A_BI, nP, WP, false));
  TRY(make_mat(Hp, nP, WP, true));
  TRY(make_mat(Hi, nW, WW, false));
  TRY(make_mat(App, nO, WW, false));
  TRY(M.alloc(&dA64, nP, true, st));
  TRY(M.alloc(&dH64, nP, true, st));
  TRY(M.alloc(&dA32, nP, true, st));
  TRY(M.alloc(&dH32, nP, true, st));
  const double drop = 1e-12;  // structural zeros of the element stiffness (Kuhn split)
  launch_extract(nP, nullptr, S.p_isB, 0, S.patP_col, S.patP_w, WP, valA_P, nullptr, S.p_isB, 0,
                 drop, WP, A_II.width, A_II.col, A_II.v64, A_II.v32, dA64, dA32, st);
  launch_extract(nP, nullptr, S.p_isB, 0, S.patP_col, S.patP_w, WP, valA_P, nullptr, S.p_isB, 1,
                 drop, WP, A_IB.width, A_IB.col, A_IB.v64, nullptr, nullptr, nullptr, st);
  launch_extract(nP, nullptr, S.p_isB, 1, S.patP_col, S.patP_w, WP, valA_P, nullptr, S.p_isB, 0,
                 drop, WP, A_BI.width, A_BI.col, A_BI.v64, nullptr, nullptr, nullptr, st);
  launch_extract(nP, nullptr, nullptr, 0, S.patP_col, S.patP_w, WP, valH_P, nullptr, nullptr, 0,
                 -1.0, WP, Hp.width, Hp.col, Hp.v64, Hp.v32, dH64, dH32, st);
  launch_extract(nW, nullptr, nullptr, 0, S.patW_col, S.patW_w, WW, valH_W, nullptr, nullptr, 0,
                 -1.0, WW, Hi.width, Hi.col, Hi.v64, nullptr, nullptr, nullptr, st);
  launch_extract(nO, S.o2w, nullptr, 0, S.patW_col, S.patW_w, WW, valA_W, S.w2o, nullptr, 0,
                 drop, WW, App.width, App.col, App.v64, nullptr, nullptr, nullptr, st);
  int h_err = 0;
  CK(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h_err) return fail(MOR_ERR_BAD_MESH, "mor_build_bases: element with non-positive volume");

  // ---- coarse level of the local preconditioner (set 0: A_II, set 1: H^+) ----
  // automatic size: small aggregates where the coarse product runs in binary32 (fewer
  // iterations for a cheap product), larger ones at GB300's low binary64 rate
  const int coarse_rows = o.coarse_rows < 0 ? (B.mixed ? 35 : 300) : o.coarse_rows;
  if (coarse_rows > 0) {
    AggPlan ap;
    build_aggregates(hp, coarse_rows, kMaxAgg, ap);
    if (ap.max_slots > kMaxSlots)
      return fail(MOR_ERR_ARG, "mor_build_bases: too many aggregates meet one row tile");
    const int64_t n_agg = ap.aoff[n_sd];
    int32_t *aloc, *aoff;
    TRY(M.upload(&aloc, ap.aloc, st));
    TRY(M.upload(&aoff, ap.aoff, st));
    const size_t tsz_c = B.mixed ? sizeof(float) : sizeof(double);
    void* yc;
    TRY(M.alloc((unsigned char**)&yc, (size_t)n_agg * kp * tsz_c, true, st));
    int* d_bad;
    TRY(M.alloc(&d_bad, 1, true, st));
    // the binary32 path forms the coarse product on the tensor cores (tc_gram >= 1)
    // for up to 128 columns
    const bool coarse_tc = B.mixed && o.tc_gram != 0 && kp <= 128;
    int* d_tc_err = nullptr;
    if (coarse_tc) TRY(M.alloc(&d_tc_err, 1, true, st));
    // E (binary64, assembled) and the inversion workspace, shared by both matrices
    int n_max[2] = {1, 1};
    int64_t ne_max = 1;
    for (int set = 0; set < 2; ++set) {
      for (int i = 0; i < n_sd; ++i) n_max[set] = std::max(n_max[set], ap.nca[set][i]);
      ne_max = std::max<int64_t>(ne_max, ap.eoff[set][n_sd]);
    }
    const int nm = std::max(n_max[0], n_max[1]);
    double *E, *sc;
    float *W, *P;
    {
      Allocs Wk;  // released after the inversions
      Wk.use_pool(st);
      TRY(Wk.alloc(&E, ne_max, false, st));
      TRY(Wk.alloc(&W, ne_max, false, st));
      TRY(Wk.alloc(&P, (size_t)n_sd * kCoarsePivots * kCoarsePivots, false, st));
      TRY(Wk.alloc(&sc, (size_t)n_sd * nm, false, st));
      for (int set = 0; set < 2; ++set) {
        const DTiles& tl = set == 0 ? S.tP_I : S.tP_all;
        const Mat& Am = set == 0 ? A_II : Hp;
        int32_t *nca, *tfirst, *tcount;
        int64_t *toff, *eoff;
        TRY(M.upload(&nca, ap.nca[set], st));
        TRY(M.upload(&tfirst, ap.tfirst[set], st));
        TRY(M.upload(&tcount, ap.tcount[set], st));
        TRY(M.upload(&toff, ap.toff[set], st));
        TRY(M.upload(&eoff, ap.eoff[set], st));
        const int64_t ne = ap.eoff[set][n_sd];
        // partial r_c.y_c per row block: blocks of at least kCoarseRowsMin (SIMT) or
        // kCoarseTcM rows
        const int nrb = std::max((n_max[set] + kCoarseRowsMin - 1) / kCoarseRowsMin,
                                 (n_max[set] + kCoarseTcM - 1) / kCoarseTcM);
        void *einv, *cpart;
        double* dpart;
        TRY(M.alloc((unsigned char**)&einv, (size_t)std::max<int64_t>(ne, 1) * tsz_c, true, st));
        TRY(M.alloc((unsigned char**)&cpart, (size_t)std::max<int64_t>(ap.toff[set].back(), 1) *
                                                 kp * tsz_c, true, st));
        TRY(M.alloc(&dpart, (size_t)n_sd * nrb * kp, true, st));
        CK(cudaMemsetAsync(E, 0, sizeof(double) * std::max<int64_t>(ne, 1), st));
        launch_coarse_matrix(tl, Am.e64(), aloc, nca, eoff, E, st);
        if (B.mixed)
          launch_coarse_invert<float>(n_sd, n_max[set], nca, eoff, E, W, P, sc, (float*)einv,
                                      d_bad, st);
        else
          launch_coarse_invert<double>(n_sd, n_max[set], nca, eoff, E, W, P, sc,
                                       (double*)einv, d_bad, st);
        auto fill = [&](auto& c, auto* ei, auto* cp, auto* y) {
          c.aloc = aloc;
          c.aoff = aoff;
          c.nca = nca;
          c.tfirst = tfirst;
          c.tcount = tcount;
          c.toff = toff;
          c.eoff = eoff;
          c.einv = ei;
          c.cpart = cp;
          c.yc = y;
          c.dpart = dpart;
          c.n_max = n_max[set];
        };
        if (B.mixed)
          fill(B.co32[set], (const float*)einv, (float*)cpart, (float*)yc);
        else
          fill(B.co64[set], (const double*)einv, (double*)cpart, (double*)yc);
        if (coarse_tc) {
          // E^{-1} as tensor-core operand blocks: ceil(n / 128) x ceil(n / 32) per
          // subdomain, 16 KB each
          std::vector<int64_t> h_off(n_sd + 1, 0);
          int blocks_max = 0;
          for (int i = 0; i < n_sd; ++i) {
            const int nc = ap.nca[set][i];
            const int nb = ((nc + kCoarseTcM - 1) / kCoarseTcM) * ((nc + 31) / 32);
            blocks_max = std::max(blocks_max, nb);
            h_off[i + 1] = h_off[i] + nb;
          }
          int64_t* etc_off;
          uint4* etc;
          TRY(M.upload(&etc_off, h_off, st));
          TRY(M.alloc(&etc, (size_t)std::max<int64_t>(h_off[n_sd], 1) * 1024, false, st));
          launch_coarse_tc_pack(n_sd, blocks_max, nca, eoff, (const float*)einv, etc_off, etc,
                                st);
          // r_c planes: ceil(n / 32) blocks of 2 x NP x 32 bf16 per subdomain
          const int NP = (kp + 15) & ~15;
          std::vector<int64_t> h_rc(n_sd + 1, 0);
          for (int i = 0; i < n_sd; ++i) h_rc[i + 1] = h_rc[i] + (ap.nca[set][i] + 31) / 32;
          int64_t* rcb_off;
          __nv_bfloat16* rcb;
          TRY(M.upload(&rcb_off, h_rc, st));
          TRY(M.alloc(&rcb, (size_t)std::max<int64_t>(h_rc[n_sd], 1) * 2 * NP * 32, true, st));
          B.co32[set].rcb = rcb;
          B.co32[set].rcb_off = rcb_off;
          B.co32[set].etc = etc;
          B.co32[set].etc_off = etc_off;
          B.co32[set].tc_err = d_tc_err;
          B.co32[set].tc_budget = wait_budget_cycles();
        }
      }
      CK(cudaStreamSynchronize(st));
    }
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_bad)  // an aggregate matrix that is not SPD: keep the Jacobi preconditioner
      for (int set = 0; set < 2; ++set) {
        B.co32[set] = Coarse<float>();
        B.co64[set] = Coarse<double>();
      }
  }

  // ---- paper-literal weights: dense H^+ factor, R_BB (Lemma 4.1) ----
  DenseWeights DW;
  if (dense) TRY(dense_weights(hp, S.p_sd, M, Hp.e64(), DW, st));

  // ---- solver workspace ----
  size_t tsz = B.mixed ? sizeof(float) : sizeof(double);
  double *vS, *vG, *vF, *vX;
  TRY(M.alloc(&vS, nP * kp, true, st));
  TRY(M.alloc(&vG, nP * kp, true, st));
  TRY(M.alloc(&vF, nP * kp, true, st));
  TRY(M.alloc(&vX, nP * kp, true, st));
  TRY(M.alloc(&B.vR64, nP * kp, true, st));
  {
    unsigned char *a, *b, *c, *d, *e;
    TRY(M.alloc(&a, nP * kp * tsz, true, st));
    TRY(M.alloc(&b, nP * kp * tsz, true, st));
    TRY(M.alloc(&c, nP * kp * tsz, true, st));
    TRY(M.alloc(&d, nP * kp * tsz, true, st));
    TRY(M.alloc(&e, nP * kp * tsz, true, st));
    B.xT = a;
    B.rT = b;
    B.pT = c;
    B.qT = d;
    B.bT = e;
  }
  int mt = S.max_tiles;
  TRY(M.alloc(&B.cs.rz, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.bb, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.alpha, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.beta, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.rr, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.rzf, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.gam, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.pr, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.alpha32, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.beta32, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.gam32, (size_t)n_sd * kp, true, st));
  if (g_prof.on) {
    // work counters and, per matrix set, rows and stored entries of every subdomain
    TRY(M.alloc(&B.cs.work, (size_t)4 * n_sd, true, st));
    for (int set = 0; set < 2; ++set) {
      const HostTiles& ht = set == 0 ? hp.tP_I : hp.tP_all;
      std::vector<int32_t> rows(n_sd, 0);
      for (size_t t = 0; t < ht.sd.size(); ++t) rows[ht.sd[t]] += ht.r1[t] - ht.r0[t];
      TRY(M.upload(&B.sd_rows[set], rows, st));
      TRY(M.alloc(&B.sd_nnz[set], n_sd, true, st));
      launch_count_sd_nnz(set == 0 ? S.tP_I : S.tP_all, set == 0 ? A_II.e64() : Hp.e64(),
                          B.sd_nnz[set], st);
    }
  }
  TRY(M.alloc(&B.cs.done, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.cs.part1, (size_t)mt * kp, true, st));
  TRY(M.alloc(&B.cs.part2, (size_t)mt * kp, true, st));
  TRY(M.alloc(&B.cs.counter, n_sd, true, st));
  TRY(M.alloc(&B.cs.iters, n_sd, true, st));
  TRY(M.alloc(&B.cs.active, n_sd, true, st));
  TRY(M.alloc(&B.rs.obb, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.rs.orr, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.rs.scale, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.rs.part, (size_t)mt * kp, true, st));
  TRY(M.alloc(&B.rs.part2, (size_t)mt * kp, true, st));
  TRY(M.alloc(&B.rs.part3, (size_t)mt * kp, true, st));
  TRY(M.alloc(&B.rs.oaa, (size_t)n_sd * kp, true, st));
  TRY(M.alloc(&B.rs.nfloor, n_sd, true, st));
  TRY(M.alloc(&B.rs.nnear, n_sd, true, st));
  TRY(M.alloc(&B.rs.xx, (size_t)n_sd * kp, true, st));
  for (int set = 0; set < 2; ++set) {
    TRY(M.alloc(&B.anorm[set], n_sd, true, st));
    launch_row_abs_max(set == 0 ? S.tP_I : S.tP_all, set == 0 ? A_II.e64() : Hp.e64(),
                       B.anorm[set], st);
  }
  TRY(M.alloc(&B.rs.counter, n_sd, true, st));
  TRY(M.alloc(&B.rs.active, n_sd, true, st));
  double *Xw, *Yw, *Zw, *u0w, *V = nullptr, *AV = nullptr, *bP;
  TRY(M.alloc(&Xw, nW * kp, true, st));
  TRY(M.alloc(&Yw, nW * kp, true, st));
  TRY(M.alloc(&Zw, nW * kp, true, st));
  TRY(M.alloc(&u0w, nW, true, st));
  TRY(M.alloc(&bP, nO, true, st));
  double *G, *evals, *evecs, *Mm, *gpart, *eigw = nullptr;
  int *gcnt, *kcnt;
  // the k x k work of the sketch and the diagonal-block update on kq <= 128 columns;
  // the explicit SVD can keep more columns than its (unused) sketch width
  const int kb = o.explicit_svd ? std::max(kp, 128) : kp;
  TRY(M.alloc(&G, (size_t)n_sd * kb * kb, true, st));
  TRY(M.alloc(&evals, (size_t)n_sd * kb, true, st));
  TRY(M.alloc(&evecs, (size_t)n_sd * kb * kb, true, st));
  TRY(M.alloc(&Mm, (size_t)n_sd * kb * kb, true, st));
  {
    // Gram partials: per row tile for the small Grams (at most 80 x 80), per row chunk
    // of a subdomain for the wide ones
    const size_t nk = (size_t)std::min(kb, 80);
    size_t gsz = (size_t)mt * nk * nk;
    if (wide || kb > 80) {
      // the sketch Grams (k x k) and the diagonal-block Gram (at most 128 x 128)
      gsz = std::max(gsz, (size_t)n_sd * gram_wide_chunks(n_sd, k, k) * k * k);
      gsz = std::max(gsz, (size_t)n_sd * 16 * 128 * 128);
      TRY(M.alloc(&eigw, (size_t)n_sd * 2 * kb * kb, false, st));
    }
    TRY(M.alloc(&gpart, gsz, true, st));
  }
  TRY(M.alloc(&gcnt, n_sd, true, st));
  TRY(M.alloc(&kcnt, n_sd, true, st));
  // the small kernels serve widths up to 80 columns, the wide ones the rest
  // tensor-core Grams (mixed precision): partials per (subdomain, row chunk)
  const bool use_tc = B.mixed && o.tc_gram != 0;
  double* tcpart = nullptr;
  int64_t* tcrange = nullptr;
  int* tcerr = nullptr;
  if (use_tc) {
    const size_t n = (size_t)std::min(std::max(kb, 4), 128);
    TRY(M.alloc(&tcpart, (size_t)n_sd * tc_gram_chunks(n_sd) * n * n, false, st));
    TRY(M.alloc(&tcrange, (size_t)2 * n_sd, true, st));
    TRY(M.alloc(&tcerr, 1, true, st));
  }
  const long long tc_budget = wait_budget_cycles();
  auto gram = [&](const DTiles& tl, const double* X, int ldx, int nx, const double* Y,
                  int ldy, int ny, int ldg) {
    if (use_tc && nx <= 128 && ny <= 128)
      launch_tc_gram(tl, n_sd, X, ldx, nx, Y, ldy, ny, tcpart, tcrange, G, ldg,
                     (int64_t)ldg * ldg, tc_budget, tcerr, st);
    else if (nx > 80 || ny > 80)
      launch_gram_wide(tl, n_sd, X, ldx, nx, Y, ldy, ny, gpart, G, ldg, (int64_t)ldg * ldg,
                       st);
    else
      launch_gram(tl, n_sd, X, ldx, nx, Y, ldy, ny, gpart, gcnt, G, ldg, st);
  };
  auto sym_eig = [&](int ld, int n, double* ev, double* V_) {
    if (n > 80)
      launch_sym_eig_wide(n_sd, G, ld, n, ev, V_, eigw, st);
    else
      launch_sym_eig(n_sd, G, ld, n, ev, V_, st);
  };
  auto rowmul = [&](const DTiles& tl, const double* X, int ldx, int nin, int ldm, double* Y,
                    int ldy, int nout) {
    if (nin > 80 || nout > 80 || ldy > 80)
      launch_rowmul_wide(tl, X, ldx, nin, Mm, ldm, Y, ldy, nout, st);
    else
      launch_rowmul(tl, X, ldx, nin, Mm, ldm, Y, ldy, nout, st);
  };

  auto bases = std::make_unique<mor_bases_s>();
  mor_bases_s& Bo = *bases;
  Bo.n_sd = n_sd;
  Bo.k = k;
  Bo.kp = kp;
  Bo.Ooff = hp.Ooff;
  TRY(Bo.mem.alloc(&Bo.sigma, (size_t)n_sd * kp, true, st));
  TRY(Bo.mem.alloc(&Bo.kept, n_sd, true, st));

  auto solve = [&](const DTiles& tl, const Mat& A, bool isA, const double* b64, double* x64,
                   int nc, int which, double rtol) -> int {
    const int set = isA ? 0 : 1;
    if (B.mixed)
      return B.solve<float>(tl, A, isA ? dA32 : dH32, b64, x64, nc, which, rtol, set);
    return B.solve<double>(tl, A, isA ? dA64 : dH64, b64, x64, nc, which, rtol, set);
  };
  const double rt = o.cg_rtol;
  const double rt_sketch = o.sketch_rtol > 0.0 ? o.sketch_rtol : o.cg_rtol;

  // ---- sketch: W = ((H^+)^{-1} L xi)_B ----
  float2* lsplit;
  TRY(M.alloc(&lsplit, (size_t)hp.n_tets * 10, false, st));
  launch_elem_chol(hp.n_tets, S.xyz, S.tets, S.kappa, o.h1_weighted, lsplit, st);
  int32_t *d_ksd, *d_msd, *d_msel;
  TRY(M.upload(&d_ksd, h_k, st));
  TRY(M.upload(&d_msd, h_rank, st));
  TRY(M.alloc(&d_msel, n_sd, true, st));
  // the reduced system stores the widest kept count + 1 columns per subdomain (tolerance
  // mode), and the output buffers are sized once that count is known
  auto finish_kq = [&]() -> int {
    if (tol_mode && m_force == 0) {
      // the reduced system stores the widest kept count + 1 columns per subdomain
      std::vector<int> msel(n_sd);
      CK(cudaMemcpyAsync(msel.data(), d_msel, n_sd * sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      mcols = 0;
      for (int v : msel) mcols = std::max(mcols, v);
      kq = round_up4(mcols + 1);
    }
    if (kq > 128)
      return fail(MOR_ERR_ARG, "mor_build_bases: more than 127 singular values above eps in a "
                               "subdomain (at most 128 basis columns per subdomain)");
    B.kq = kq;
    B.m = mcols;
    Bo.kq = kq;
    Bo.m = mcols;
    TRY(M.alloc(&V, nO * kq, true, st));
    TRY(M.alloc(&AV, nO * kq, true, st));
    TRY(Bo.mem.alloc(&Bo.Q, nO * kq, true, st));
    TRY(Bo.mem.alloc(&Bo.bt, (size_t)n_sd * kq, true, st));
    return MOR_OK;
  };
  const double* colsW = Zw;  // X^ U_m (or R_i^{-1} U_m), W rows
  int colsLd = kp;
  // Eq. (14) explicitly, with dense factors: Z_I = A_II^{-1} [A_IB | b_I] (the last
  // column is u_0 of Prob. "aux1"), Z = C_i Z_I, Y = R_i Z with R_i = chol(H_i)^T,
  // X = Y R_BB^{-1}, and the SVD X = U Sigma V^T through eig(X^T X) = V Sigma^2 V^T;
  // the basis columns are R_i^{-1} U_m with U_m = X V_m Sigma_m^{-1}
  auto explicit_svd_bases = [&]() -> int {
    const int mB = DW.m_max, iM = DW.i_max;
    if (mB > 1024)
      return fail(MOR_ERR_ARG, "mor_build_bases: explicit_svd needs |B| <= 1024");
    const int ldz = mB + 1, ldm = round_up4(std::max(mB, 1));
    std::vector<int64_t> aoff(n_sd + 1, 0), zoff(n_sd), woff(n_sd), hioff(n_sd + 1, 0);
    std::vector<int32_t> nWsd(n_sd), ldz_v(n_sd, ldz), ncz(n_sd, ldz);
    int w_max = 0;
    for (int i = 0; i < n_sd; ++i) {
      aoff[i + 1] = aoff[i] + (int64_t)DW.h_nI[i] * DW.h_nI[i];
      zoff[i] = hp.Poff[i] * ldz;
      woff[i] = hp.Woff[i];
      nWsd[i] = (int32_t)(hp.Woff[i + 1] - hp.Woff[i]);
      w_max = std::max(w_max, nWsd[i]);
      hioff[i + 1] = hioff[i] + (int64_t)nWsd[i] * nWsd[i];
    }
    if (w_max > kDenseMaxOrder)
      return fail(MOR_ERR_ARG, "mor_build_bases: explicit_svd needs |omega_i| <= 6144");
    std::vector<int32_t> w_loc(nW), w_sdv(nW), w_row(nW);
    for (int i = 0; i < n_sd; ++i)
      for (int64_t r = hp.Woff[i]; r < hp.Woff[i + 1]; ++r) {
        w_loc[r] = (int32_t)(r - hp.Woff[i]);
        w_sdv[r] = i;
        w_row[r] = (int32_t)(r - hp.Woff[i]);
      }
    std::vector<int64_t> poff(hp.Poff.begin(), hp.Poff.begin() + n_sd);
    int64_t *d_aoff, *d_zoff, *d_woff, *d_hioff, *d_poff;
    int32_t *d_nW, *d_ldz, *d_ncz, *d_wloc, *d_wsd, *d_wrow;
    TRY(M.upload(&d_aoff, aoff, st));
    TRY(M.upload(&d_zoff, zoff, st));
    TRY(M.upload(&d_woff, woff, st));
    TRY(M.upload(&d_hioff, hioff, st));
    TRY(M.upload(&d_poff, poff, st));
    TRY(M.upload(&d_nW, nWsd, st));
    TRY(M.upload(&d_ldz, ldz_v, st));
    TRY(M.upload(&d_ncz, ncz, st));
    TRY(M.upload(&d_wloc, w_loc, st));
    TRY(M.upload(&d_wsd, w_sdv, st));
    TRY(M.upload(&d_wrow, w_row, st));
    int* bad;
    TRY(M.alloc(&bad, 1, true, st));
    // A_II = L_A L_A^T (dense), U_A = L_A^T
    double *Ad, *UA, *Zi, *Zw2, *Yw2, *Hd, *Ui, *Um;
    TRY(M.alloc(&Ad, (size_t)std::max<int64_t>(aoff[n_sd], 1), true, st));
    TRY(M.alloc(&UA, (size_t)std::max<int64_t>(aoff[n_sd], 1), true, st));
    launch_ell_to_dense(nP, S.p_sd, DW.p_loc, DW.p_loc, A_II.e64(), DW.zero, DW.nI, DW.zero,
                        DW.nI, DW.nI, d_aoff, Ad, st);
    launch_potrf(n_sd, iM, Ad, d_aoff, DW.nI, bad, st);
    launch_transpose_block(n_sd, iM, Ad, d_aoff, DW.nI, DW.zero, DW.nI, UA, d_aoff, 1, st);
    // [A_IB | b_I] on the I rows of the P space (columns: B in ascending node order)
    TRY(M.alloc(&Zi, (size_t)nP * ldz, true, st));
    launch_ell_to_dense(nP, S.p_sd, DW.p_loc, DW.p_loc, A_IB.e64(), DW.zero, DW.nI, DW.nI,
                        DW.M, d_ldz, d_zoff, Zi, st);
    launch_set_col(S.tP_I, loadP, Zi, ldz, mB, st);
    // A_II Z_I = [A_IB | b_I]: forward with L_A (column j = row j of U_A), backward
    // with U_A (column j = row j of L_A)
    launch_trsv_cols(n_sd, iM, ldz, UA, d_aoff, DW.nI, DW.nI, DW.zero, Zi, d_poff, ldz, d_ncz,
                     1, st);
    launch_trsv_cols(n_sd, iM, ldz, Ad, d_aoff, DW.nI, DW.nI, DW.zero, Zi, d_poff, ldz, d_ncz,
                     0, st);
    launch_gather_rows(nW, S.w2p, Zi, ldz, mB, u0w, 1, 0, 1, st);
    TRY(M.alloc(&Zw2, (size_t)nW * ldm, true, st));
    TRY(M.alloc(&Yw2, (size_t)nW * ldm, true, st));
    launch_gather_rows(nW, S.w2p, Zi, ldz, 0, Zw2, ldm, 0, mB, st);
    // H_i = L_i L_i^T (dense, W order), R_i = U_i = L_i^T; Y = R_i Z
    TRY(M.alloc(&Hd, (size_t)std::max<int64_t>(hioff[n_sd], 1), true, st));
    TRY(M.alloc(&Ui, (size_t)std::max<int64_t>(hioff[n_sd], 1), true, st));
    launch_ell_to_dense(nW, d_wsd, d_wloc, d_wloc, Hi.e64(), DW.zero, d_nW, DW.zero, d_nW, d_nW,
                        d_hioff, Hd, st);
    launch_potrf(n_sd, w_max, Hd, d_hioff, d_nW, bad, st);
    launch_transpose_block(n_sd, w_max, Hd, d_hioff, d_nW, DW.zero, d_nW, Ui, d_hioff, 1, st);
    launch_trmv_upper(n_sd, w_max, mB, Ui, d_hioff, d_nW, Zw2, Yw2, d_woff, ldm, DW.M, st);
    // X = Y R_BB^{-1}, one W row per warp
    launch_trsv_rows(DW.Rbb, DW.bboff, DW.M, Yw2, d_woff, ldm, d_wsd, d_wrow, (int)nW, st);
    int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_bad)
      return fail(MOR_ERR_CUDA, "mor_build_bases: A_II or H_i is not positive definite");
    // X^T X = V Sigma^2 V^T (binary64 Jacobi); sigma_j^2 stored like the randomized path's
    double *Gx, *evx, *Vx, *Mx, *gp, *ew = nullptr;
    TRY(M.alloc(&Gx, (size_t)n_sd * ldm * ldm, true, st));
    TRY(M.alloc(&evx, (size_t)n_sd * ldm, true, st));
    TRY(M.alloc(&Vx, (size_t)n_sd * ldm * ldm, true, st));
    TRY(M.alloc(&Mx, (size_t)n_sd * ldm * ldm, true, st));
    TRY(M.alloc(&gp, (size_t)std::max<int64_t>(
                         (int64_t)n_sd * gram_wide_chunks(n_sd, mB, mB) * mB * mB,
                         (int64_t)mt * std::min(ldm, 80) * std::min(ldm, 80)), true, st));
    if (mB > 80) {
      launch_gram_wide(S.tW, n_sd, Yw2, ldm, mB, Yw2, ldm, mB, gp, Gx, ldm, (int64_t)ldm * ldm,
                       st);
      TRY(M.alloc(&ew, (size_t)n_sd * 2 * ldm * ldm, false, st));
      launch_sym_eig_wide(n_sd, Gx, ldm, mB, evx, Vx, ew, st);
    } else {
      launch_gram(S.tW, n_sd, Yw2, ldm, mB, Yw2, ldm, mB, gp, gcnt, Gx, ldm, st);
      launch_sym_eig(n_sd, Gx, ldm, mB, evx, Vx, st);
    }
    // kept directions: the first m_i, or sigma_j > eps (Eq. (15)); U_m = X V_m Sigma_m^-1
    std::vector<int32_t> keep(n_sd);
    for (int i = 0; i < n_sd; ++i) keep[i] = tol_mode ? DW.h_M[i] : h_rank[i];
    int32_t* d_keep;
    TRY(M.upload(&d_keep, keep, st));
    if (tol_mode)
      launch_make_M(n_sd, 4, evx, Vx, ldm, mB, o.eps * o.eps, mB, Mx, d_msel, st, d_keep);
    else
      launch_make_M(n_sd, 3, evx, Vx, ldm, mB, 0.0, mB, Mx, d_msel, st, d_keep);
    if (!tol_mode) mcols = std::min(m_max, mB);
    TRY(finish_kq());
    TRY(M.alloc(&Um, (size_t)nW * ldm, true, st));
    launch_rowmul_wide(S.tW, Yw2, ldm, mB, Mx, ldm, Um, ldm, mcols, st);
    // basis columns R_i^{-1} U_m: backward substitution with U_i (column j = row j of L_i)
    launch_trsv_cols(n_sd, w_max, mcols, Hd, d_hioff, d_nW, d_nW, DW.zero, Um, d_woff, ldm,
                     d_msel, 0, st);
    colsW = Um;
    colsLd = ldm;
    // singular values: the explicit path reports all |B_i| of them
    Bo.k = mB;
    Bo.kp = ldm;
    TRY(Bo.mem.alloc(&Bo.sigma, (size_t)n_sd * ldm, true, st));
    CK(cudaMemcpyAsync(Bo.sigma, evx, (size_t)n_sd * ldm * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
    return MOR_OK;
  };
  if (o.explicit_svd) {
    TRY(explicit_svd_bases());
  } else {
    if (o.sketch == MOR_SKETCH_PAPER) {
      // W = R_BB^{-1} S (Sec. 6): S Gaussian on B (rows in ascending node order), a
      // backward substitution with R_BB (its column j is row j of L_BB), then W goes to
      // the B rows of the P space
      double* Sb;
      TRY(M.alloc(&Sb, (size_t)std::max<int64_t>(DW.h_boff[n_sd], 1) * k, true, st));
      launch_node_normals(n_sd, DW.m_max, DW.bnode, DW.boff, DW.M, d_ksd, k, o.seed,
                          (uint32_t)S.sd_base, Sb, k, st);
      launch_trsv_cols(n_sd, DW.m_max, k, DW.Lbb, DW.bboff, DW.M, DW.M, DW.zero, Sb, DW.boff,
                       k, d_ksd, 0, st);
      CK(cudaMemsetAsync(vG, 0, nP * kp * sizeof(double), st));
      launch_scatter_rows(DW.h_boff[n_sd], DW.bprow, Sb, k, vG, kp, k, st);
    } else {
      launch_sketch_rhs(0, nP, S.p_sd, S.incP_ptr, S.incP_tet, S.incP_code, lsplit, k, o.seed,
                        (uint32_t)S.sd_base, vS, kp, st, d_ksd);
      TRY(solve(S.tP_all, Hp, false, vS, vG, k, 0, rt_sketch));
    }

    // ---- forward solve A_II [X | u_0] = [A_IB W | b_I] (Prob. "aux1", Eq. (7), and the lifting of Eq. (8)) ----
    launch_spmm<double>(S.tP_I, A_IB.e64(), vG, vF, kp, st);
    launch_set_col(S.tP_I, loadP, vF, kp, k, st);
    TRY(solve(S.tP_I, A_II, true, vF, vX, k + 1, 1, rt));

    // ---- X = C_i X_full, orthonormalise in the H_i inner product (twice) ----
    launch_gather_rows(nW, S.w2p, vX, kp, 0, Xw, kp, 0, kp, st);
    launch_gather_rows(nW, S.w2p, vX, kp, k, u0w, 1, 0, 1, st);
    for (int pass = 0; pass < 2; ++pass) {
      launch_spmm<double>(S.tW, Hi.e64(), Xw, Yw, kp, st);
      gram(S.tW, Xw, kp, k, Yw, kp, k, kp);
      sym_eig(kp, k, evals, evecs);
      launch_make_M(n_sd, 0, evals, evecs, kp, k, o.orth_tol, 0, Mm, kcnt, st);
      rowmul(S.tW, Xw, kp, k, kp, Zw, kp, k);
      std::swap(Xw, Zw);
    }

    // ---- adjoint: T = A_BI A_II^{-1} C_i^T H_i X^ (two left solves, the transposed form of Eq. (24)) ----
    launch_spmm<double>(S.tW, Hi.e64(), Xw, Yw, kp, st);
    CK(cudaMemsetAsync(vF, 0, nP * kp * sizeof(double), st));
    launch_scatter_rows(nW, S.w2p, Yw, kp, vF, kp, kp, st);
    TRY(solve(S.tP_I, A_II, true, vF, vX, k, 2, rt));
    CK(cudaMemsetAsync(vS, 0, nP * kp * sizeof(double), st));
    launch_spmm<double>(S.tP_B, A_BI.e64(), vX, vS, kp, st);
    // S_B^{-1} T = ((H^+)^{-1} [0; T])_B  (Lemma 4.1 / block inverse of H^+)
    TRY(solve(S.tP_all, Hp, false, vS, vG, k, 3, rt));
    gram(S.tP_B, vS, kp, k, vG, kp, k, kp);
    // eig(G_B) = sigma_j^2 (kept on the device as squares); the rotation of the top
    // `rank` directions gives the basis X^ U_m = R_i^{-1} Qh U_m
    sym_eig(kp, k, Bo.sigma, evecs);
    // fixed rank: the first m_i directions; tolerance mode: sigma_j > eps (Eq. (15))
    if (tol_mode)
      launch_make_M(n_sd, 2, Bo.sigma, evecs, kp, k, o.eps * o.eps, k, Mm, d_msel, st, d_ksd);
    else
      launch_make_M(n_sd, 1, Bo.sigma, evecs, kp, k, 0.0, mcols, Mm, d_msel, st, d_msd);
    TRY(finish_kq());
    rowmul(S.tW, Xw, kp, k, kp, Zw, kp, mcols);
    colsW = Zw;
  }

  // ---- V = D_i [u_0, X^ U_m], diagonal-block update Q_i = V W Lambda^{-1/2} ----
  launch_gather_rows(nO, S.o2w, u0w, 1, 0, V, kq, 0, 1, st);
  launch_gather_rows(nO, S.o2w, colsW, colsLd, 0, V, kq, 1, mcols, st);
  launch_spmm<double>(S.tO, App.e64(), V, AV, kq, st);
  // V^T A V stays binary64 in every precision: the reduced system takes the diagonal
  // blocks Q_i^T A_ii Q_i as the identity, and Q_i = V W Lambda^{-1/2} amplifies the
  // Gram's error on directions of small energy
  if (mcols + 1 > 80)
    launch_gram_wide(S.tO, n_sd, V, kq, mcols + 1, AV, kq, mcols + 1, gpart, G, kq,
                     (int64_t)kq * kq, st);
  else
    launch_gram(S.tO, n_sd, V, kq, mcols + 1, AV, kq, mcols + 1, gpart, gcnt, G, kq, st);
  sym_eig(kq, mcols + 1, evals, evecs);
  launch_make_M(n_sd, 0, evals, evecs, kq, mcols + 1, o.tau, 0, Mm, Bo.kept, st);
  rowmul(S.tO, V, kq, mcols + 1, kq, Bo.Q, kq, mcols + 1);
  // b~_i = Q_i^T b[P_i]
  launch_gather_rows(nO, S.o2w, loadW, 1, 0, bP, 1, 0, 1, st);
  launch_gram_vec(S.tO, n_sd, Bo.Q, kq, kq, bP, 1, gpart, gcnt, Bo.bt, kq, st);
  CK(cudaGetLastError());

  if (dense) {
    // R_BB per subdomain for mor_bases_get_rbb
    TRY(Bo.mem.alloc(&Bo.Rbb, (size_t)std::max<int64_t>(DW.h_bboff[n_sd], 1), false, st));
    CK(cudaMemcpyAsync(Bo.Rbb, DW.Rbb, (size_t)DW.h_bboff[n_sd] * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
    Bo.rbb_off = DW.h_bboff;
    Bo.rbb_m = DW.h_M;
  }
  if (B.co32[0].tc_err) {
    int h_err = 0;
    CK(cudaMemcpyAsync(&h_err, B.co32[0].tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_err)
      return fail(MOR_ERR_TIMEOUT, "mor_build_bases: a wait of the tensor-core coarse product "
                                   "ran out of its budget (mor_set_wait_budget)");
  }
  if (use_tc) {
    int h_tcerr = 0;
    CK(cudaMemcpyAsync(&h_tcerr, tcerr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h_tcerr)
      return fail(MOR_ERR_TIMEOUT, "mor_build_bases: a tensor-core Gram's wait ran out of its "
                                   "budget (mor_set_wait_budget)");
    Bo.tc = o.tc_gram >= 2;
  }
  Bo.h_kept.resize(n_sd);
  Bo.h_sigma.resize((size_t)n_sd * Bo.kp);
  CK(cudaMemcpyAsync(Bo.h_kept.data(), Bo.kept, n_sd * sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(Bo.h_sigma.data(), Bo.sigma, (size_t)n_sd * Bo.kp * sizeof(double),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (auto& s : Bo.h_sigma) s = std::sqrt(std::max(s, 0.0));
  if (g_prof.on) {
    g_prof.collect();
    // algorithmic bytes of the work the CG kernels actually did (converged subdomains
    // and column packs are skipped): sparse product = stored entries (value + index)
    // of the active subdomains + read p and write q per open (row, 16-byte pack); x/r
    // update = read x, r, p, q and write x, r per open (row, pack); p update = read r,
    // p and write p per open (row, pack); coarse = E^{-1} entries read.  Diagonal,
    // aggregate-index and y_c reads are not counted.
    std::vector<unsigned long long> wt((size_t)4 * n_sd);
    CK(cudaMemcpy(wt.data(), B.cs.work, wt.size() * sizeof(unsigned long long),
                  cudaMemcpyDeviceToHost));
    double w[4] = {0, 0, 0, 0};
    for (int k2 = 0; k2 < 4; ++k2)
      for (int i = 0; i < n_sd; ++i) w[k2] += (double)wt[(size_t)k2 * n_sd + i];
    const double tsz = B.mixed ? 4.0 : 8.0;
    const int wide = B.mixed ? 0 : 1;
    g_prof.bytes[0 + wide] += w[0] * (tsz + 4.0) + w[1] * 16.0 * 2.0;
    g_prof.bytes[2 + wide] += w[1] * 16.0 * 6.0;
    g_prof.bytes[4 + wide] += w[2] * 16.0 * 3.0;
    g_prof.bytes[6 + wide] += w[3] * tsz;
  }
  Bo.stats[0] = B.iters[0];
  Bo.stats[1] = B.iters[1];
  Bo.stats[2] = B.iters[2];
  Bo.stats[3] = B.iters[3];
  Bo.stats[4] = B.sweeps;
  Bo.stats[5] = B.not_conv;
  Bo.stats[6] = B.floor_cols;
  *out = bases.release();
  if (B.not_conv > 0)
    return fail(MOR_ERR_NOT_CONVERGED, "mor_build_bases: " + std::to_string(B.not_conv) +
                                           " local solve columns did not converge");
  return MOR_OK;
}

// streamed plans: the per-subdomain part of waves of sd->wave_sd subdomains is built on
// the host, uploaded, and run through build_bases_core; Q, b~, sigma and the kept
// counts of each wave go to their rows of the global handle
static int build_bases_streamed(const mor_subdomains* sd, const mor_basis_opts* opts,
                                void* stream, mor_bases** out) {
  const HostPlan& g = sd->hp;
  const mor_basis_opts& o = *opts;
  cudaStream_t st = (cudaStream_t)stream;
  const int sb = o.sub_begin, se = o.sub_end > 0 ? o.sub_end : g.n_sd;
  if (sb < 0 || se > g.n_sd || sb >= se)
    return fail(MOR_ERR_ARG, "mor_build_bases: bad subdomain range");
  int m_max = 0;
  for (int i = 0; i < g.n_sd; ++i) m_max = std::max(m_max, o.ranks ? o.ranks[i] : o.rank);
  auto bases = std::make_unique<mor_bases_s>();
  mor_bases_s& Bo = *bases;
  PlanScratch ps;
  int64_t not_conv = 0;
  // the host plan of the next wave is built while the device works on the current one
  auto plan_async = [&](int s0, HostPlan* out, std::string* err) {
    const int s1 = std::min(se, s0 + sd->wave_sd);
    return std::async(std::launch::async, [=, &g, &ps] {
      return build_wave_plan(g.n_nodes, g.n_tets, sd->h_tets.data(), sd->h_dir.data(),
                             sd->h_xyz.data(), g, s0, s1, *out, ps, *err);
    });
  };
  auto next_plan = std::make_unique<HostPlan>();
  std::string next_err;
  std::future<int> next = plan_async(sb, next_plan.get(), &next_err);
  bool first = true;
  for (int s0 = sb; s0 < se; s0 += sd->wave_sd) {
    const int s1 = std::min(se, s0 + sd->wave_sd), nw = s1 - s0;
    auto W = std::make_unique<mor_subdomains_s>();
    int rc = next.get();
    if (rc != MOR_OK) return fail(rc, next_err);
    W->hp = std::move(*next_plan);
    if (s1 < se) next = plan_async(s1, next_plan.get(), &next_err);
    // a return below leaves the pending plan to be joined by the future's destructor
    W->xyz = sd->xyz;
    W->tets = sd->tets;
    W->kappa = sd->kappa;
    W->sd_base = s0;
    TRY(upload_heavy(W.get(), st));
    mor_basis_opts ow = o;
    if (o.ranks) ow.ranks = o.ranks + s0;
    mor_bases* bw = nullptr;
    rc = build_bases_core(W.get(), &ow, m_max, stream, &bw);
    std::unique_ptr<mor_bases_s> wb(bw);
    if (rc == MOR_ERR_NOT_CONVERGED)
      not_conv += wb->stats[5];
    else if (rc != MOR_OK)
      return rc;
    if (first) {
      first = false;
      Bo.n_sd = g.n_sd;
      Bo.tc = wb->tc;
      Bo.k = wb->k;
      Bo.kp = wb->kp;
      Bo.kq = wb->kq;
      Bo.m = wb->m;
      Bo.Ooff = g.Ooff;
      TRY(Bo.mem.alloc(&Bo.Q, (size_t)g.nO * Bo.kq, true, st));
      TRY(Bo.mem.alloc(&Bo.bt, (size_t)g.n_sd * Bo.kq, true, st));
      TRY(Bo.mem.alloc(&Bo.sigma, (size_t)g.n_sd * Bo.kp, true, st));
      TRY(Bo.mem.alloc(&Bo.kept, g.n_sd, true, st));
      Bo.h_kept.assign(g.n_sd, 0);
      Bo.h_sigma.assign((size_t)g.n_sd * Bo.kp, 0.0);
    }
    const int64_t o0 = g.Ooff[s0], no = g.Ooff[s1] - o0;
    CK(cudaMemcpyAsync(Bo.Q + o0 * Bo.kq, wb->Q, (size_t)no * Bo.kq * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Bo.bt + (int64_t)s0 * Bo.kq, wb->bt, (size_t)nw * Bo.kq * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Bo.sigma + (int64_t)s0 * Bo.kp, wb->sigma,
                       (size_t)nw * Bo.kp * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Bo.kept + s0, wb->kept, nw * sizeof(int), cudaMemcpyDeviceToDevice, st));
    std::copy(wb->h_kept.begin(), wb->h_kept.end(), Bo.h_kept.begin() + s0);
    std::copy(wb->h_sigma.begin(), wb->h_sigma.end(), Bo.h_sigma.begin() + (int64_t)s0 * Bo.kp);
    for (int q = 0; q < 8; ++q) Bo.stats[q] += wb->stats[q];
    CK(cudaStreamSynchronize(st));  // the wave's memory is released after its copies
  }
  *out = bases.release();
  if (not_conv > 0)
    return fail(MOR_ERR_NOT_CONVERGED, "mor_build_bases: " + std::to_string(not_conv) +
                                           " local solve columns did not converge");
  return MOR_OK;
}

extern "C" {

int mor_build_bases(const mor_subdomains* sd, const mor_basis_opts* opts, void* stream,
                    mor_bases** out) {
  if (!sd || !opts || !out) return fail(MOR_ERR_ARG, "mor_build_bases: null argument");
  if (sd->streamed) return build_bases_streamed(sd, opts, stream, out);
  if (opts->sub_begin != 0 || (opts->sub_end > 0 && opts->sub_end != sd->hp.n_sd))
    return fail(MOR_ERR_ARG, "mor_build_bases: a subdomain range needs a streamed plan");
  return build_bases_core(sd, opts, 0, stream, out);
}

int mor_bases_info(const mor_bases* h, int32_t* kq, int32_t* k, int32_t* kept,
                   int64_t* total_kept) {
  if (!h) return fail(MOR_ERR_ARG, "mor_bases_info: null handle");
  if (kq) *kq = h->kq;
  if (k) *k = h->k;
  int64_t tot = 0;
  for (int i = 0; i < h->n_sd; ++i) {
    if (kept) kept[i] = h->h_kept[i];
    tot += h->h_kept[i];
  }
  if (total_kept) *total_kept = tot;
  return MOR_OK;
}

int mor_bases_sigma(const mor_bases* h, double* sigma) {
  if (!h || !sigma) return fail(MOR_ERR_ARG, "mor_bases_sigma: null argument");
  for (int i = 0; i < h->n_sd; ++i)
    for (int j = 0; j < h->k; ++j) sigma[(int64_t)i * h->k + j] = h->h_sigma[(int64_t)i * h->kp + j];
  return MOR_OK;
}

int mor_bases_get_Q(const mor_bases* h, int32_t sub, double* out) {
  if (!h || !out || sub < 0 || sub >= h->n_sd) return fail(MOR_ERR_ARG, "mor_bases_get_Q: bad argument");
  int64_t r0 = h->Ooff[sub], r1 = h->Ooff[sub + 1];
  CK(cudaMemcpy(out, h->Q + r0 * h->kq, (r1 - r0) * h->kq * sizeof(double),
                cudaMemcpyDeviceToHost));
  return MOR_OK;
}

int mor_bases_get_rbb(const mor_bases* h, int32_t sub, double* out) {
  if (!h || !out || sub < 0 || sub >= h->n_sd)
    return fail(MOR_ERR_ARG, "mor_bases_get_rbb: bad argument");
  if (!h->Rbb)
    return fail(MOR_ERR_STATE, "mor_bases_get_rbb: bases built without dense weights");
  const int64_t m = h->rbb_m[sub];
  CK(cudaMemcpy(out, h->Rbb + h->rbb_off[sub], (size_t)(m * m) * sizeof(double),
                cudaMemcpyDeviceToHost));
  return MOR_OK;
}

int mor_bases_get_bt(const mor_bases* h, double* out) {
  if (!h || !out) return fail(MOR_ERR_ARG, "mor_bases_get_bt: null argument");
  CK(cudaMemcpy(out, h->bt, (size_t)h->n_sd * h->kq * sizeof(double), cudaMemcpyDeviceToHost));
  return MOR_OK;
}

int mor_bases_stats(const mor_bases* h, int64_t* stats) {
  if (!h || !stats) return fail(MOR_ERR_ARG, "mor_bases_stats: null argument");
  for (int i = 0; i < 8; ++i) stats[i] = h->stats[i];
  return MOR_OK;
}

int mor_project(const mor_subdomains* sd, const mor_bases* b, void* stream, mor_reduced** out) {
  if (!sd || !b || !out) return fail(MOR_ERR_ARG, "mor_project: null argument");
  *out = nullptr;
  if (b->n_sd != sd->hp.n_sd) return fail(MOR_ERR_STATE, "mor_project: bases of another plan");
  cudaStream_t st = (cudaStream_t)stream;
  auto r = std::make_unique<mor_reduced_s>();
  const HostPlan& hp = sd->hp;
  r->n_sd = hp.n_sd;
  r->kq = b->kq;
  r->n_pairs = (int)hp.pair_i.size();
  r->dim = (int64_t)hp.n_sd * b->kq;
  Allocs& A = r->mem;
  double* aval;
  TRY(A.alloc(&aval, sd->n_iface, false, st));
  launch_iface_vals(sd->n_iface, sd->e_unode, sd->e_vnode, sd->n2t_ptr, sd->n2t, sd->xyz,
                    sd->tets, sd->kappa, aval, st);
  TRY(A.alloc(&r->blocks, (size_t)2 * std::max(r->n_pairs, 1) * b->kq * b->kq, true, st));
  if (b->tc && b->kq <= 128) {
    // K~_ij = sum over interface entries of a_e Q[u_e]^T Q[v_e] on the tensor cores
    Allocs W;
    W.use_pool(st);
    double *part, *Gp;
    int* err;
    const size_t nb = (size_t)std::max(r->n_pairs, 1) * b->kq * b->kq;
    TRY(W.alloc(&part, nb, false, st));
    TRY(W.alloc(&Gp, nb, false, st));
    TRY(W.alloc(&err, 1, true, st));
    launch_tc_pair_blocks(r->n_pairs, sd->pair_ptr, sd->e_urow, sd->e_vrow, aval, b->Q, b->kq,
                          part, Gp, r->blocks, wait_budget_cycles(), err, st);
    int h = 0;
    CK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h)
      return fail(MOR_ERR_TIMEOUT, "mor_project: a tensor-core wait ran out of its budget");
  } else {
    launch_pair_blocks(r->n_pairs, sd->pair_ptr, sd->e_urow, sd->e_vrow, aval, b->Q, b->kq,
                       r->blocks, st);
  }
  TRY(A.alloc(&r->bt, r->dim, false, st));
  CK(cudaMemcpyAsync(r->bt, b->bt, r->dim * sizeof(double), cudaMemcpyDeviceToDevice, st));
  r->h_nbr_ptr = sd->nbr_ptr;
  r->h_nbr_sd = sd->nbr_sd;
  r->h_nbr_blk = sd->nbr_blk;
  TRY(A.upload(&r->nbr_ptr, r->h_nbr_ptr, st));
  TRY(A.upload(&r->nbr_sd, r->h_nbr_sd, st));
  TRY(A.upload(&r->nbr_blk, r->h_nbr_blk, st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  *out = r.release();
  return MOR_OK;
}

int mor_reduced_info(const mor_reduced* h, int64_t* dim, int64_t* n_blocks) {
  if (!h) return fail(MOR_ERR_ARG, "mor_reduced_info: null handle");
  if (dim) *dim = h->dim;
  if (n_blocks) *n_blocks = 2 * (int64_t)h->n_pairs;
  return MOR_OK;
}

int mor_reduced_dense(const mor_reduced* h, double* out) {
  if (!h || !out) return fail(MOR_ERR_ARG, "mor_reduced_dense: null argument");
  if (h->dim > 20000) return fail(MOR_ERR_ARG, "mor_reduced_dense: system too large");
  int kq = h->kq;
  std::vector<double> blk((size_t)2 * h->n_pairs * kq * kq);
  if (!blk.empty())
    CK(cudaMemcpy(blk.data(), h->blocks, blk.size() * sizeof(double), cudaMemcpyDeviceToHost));
  std::memset(out, 0, (size_t)h->dim * h->dim * sizeof(double));
  for (int64_t i = 0; i < h->dim; ++i) out[i * h->dim + i] = 1.0;
  for (int i = 0; i < h->n_sd; ++i)
    for (int q = h->h_nbr_ptr[i]; q < h->h_nbr_ptr[i + 1]; ++q) {
      int j = h->h_nbr_sd[q];
      const double* B = blk.data() + (size_t)h->h_nbr_blk[q] * kq * kq;
      for (int a = 0; a < kq; ++a)
        for (int c = 0; c < kq; ++c)
          out[((int64_t)i * kq + a) * h->dim + (int64_t)j * kq + c] = B[a * kq + c];
    }
  return MOR_OK;
}

int mor_solve_reduced(const mor_reduced* h, double rtol, int32_t max_iter, void* stream,
                      double* x_dev, mor_solve_info* info) {
  if (!h || !x_dev || !(rtol > 0.0) || max_iter < 1)
    return fail(MOR_ERR_ARG, "mor_solve_reduced: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Allocs A;
  A.use_pool(st);
  RcgState s{};
  s.x = x_dev;
  TRY(A.alloc(&s.r, h->dim, false, st));
  TRY(A.alloc(&s.p, h->dim, false, st));
  TRY(A.alloc(&s.q, h->dim, false, st));
  TRY(A.alloc(&s.part, (size_t)2 * h->n_sd, true, st));
  TRY(A.alloc(&s.counter, 1, true, st));
  TRY(A.alloc(&s.scal, 8, true, st));
  TRY(A.alloc(&s.flag, 2, true, st));
  int hf[2] = {0, 0};
  unsigned* sync;
  TRY(A.alloc(&sync, 4, true, st));
  const int grid = launch_rcg_persistent(h->n_sd, h->kq, h->nbr_ptr, h->nbr_sd, h->nbr_blk,
                                         h->blocks, h->bt, rtol * rtol, max_iter, s, sync,
                                         wait_budget_cycles(), st);
  if (grid > 0) {
    unsigned hs[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(hs, sync, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hf, s.flag, sizeof(hf), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hs[2] != 0)
      return fail(MOR_ERR_TIMEOUT, "mor_solve_reduced: a grid-barrier wait ran out of its "
                                   "budget (mor_set_wait_budget)");
  } else {
    cudaGetLastError();  // no cooperative launch: three launches per step
    launch_rcg_init(h->n_sd, h->kq, h->bt, s, st);
    int it = 0;
    while (it < max_iter) {
      int chunk = std::min(16, max_iter - it);
      for (int c = 0; c < chunk; ++c)
        launch_rcg_step(h->n_sd, h->kq, h->nbr_ptr, h->nbr_sd, h->nbr_blk, h->blocks,
                        rtol * rtol, s, st);
      it += chunk;
      CK(cudaMemcpyAsync(hf, s.flag, sizeof(hf), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (hf[0]) break;
    }
  }
  CK(cudaGetLastError());
  double sc[8];
  CK(cudaMemcpy(sc, s.scal, sizeof(sc), cudaMemcpyDeviceToHost));
  // energy b~^T x
  std::vector<double> hx(h->dim), hb(h->dim);
  CK(cudaMemcpy(hx.data(), x_dev, h->dim * sizeof(double), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(hb.data(), h->bt, h->dim * sizeof(double), cudaMemcpyDeviceToHost));
  double E = 0.0;
  for (int64_t i = 0; i < h->dim; ++i) E += hb[i] * hx[i];
  if (info) {
    info->iterations = hf[1];
    info->converged = hf[0] && sc[4] <= rtol * rtol * sc[1];
    info->rel_residual = sc[1] > 0 ? std::sqrt(sc[4] / sc[1]) : 0.0;
    info->energy = E;
  }
  if (!(hf[0] && sc[4] <= rtol * rtol * sc[1]))
    return fail(MOR_ERR_NOT_CONVERGED, "mor_solve_reduced: max_iter reached");
  return MOR_OK;
}

int mor_set_wait_budget(double seconds) {
  // at least 1 ms: after a wait runs out, the tensor-core kernels wait once more, with
  // the same budget, for their MMAs in flight (microseconds) before releasing TMEM
  if (!(seconds >= 1e-3) || seconds > 3600.0)
    return fail(MOR_ERR_ARG, "mor_set_wait_budget: seconds must lie in [0.001, 3600]");
  g_wait_budget_s = seconds;
  return MOR_OK;
}

int mor_debug_wait_timeout(double seconds, int32_t* timed_out) {
  if (!timed_out || !(seconds >= 0.0) || seconds > 10.0)
    return fail(MOR_ERR_ARG, "mor_debug_wait_timeout: bad argument");
  Allocs A;
  unsigned* sync;
  int* status;
  TRY(A.alloc(&sync, 4, true));
  TRY(A.alloc(&status, 1, true));
  const double keep = g_wait_budget_s;
  g_wait_budget_s = seconds;
  const long long cycles = wait_budget_cycles();
  g_wait_budget_s = keep;
  launch_wait_unset_flag(sync, cycles, status, nullptr);
  int h = -1;
  CK(cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost));
  *timed_out = h == 1 ? 1 : 0;
  if (h == 1) return fail(MOR_ERR_TIMEOUT, "mor_debug_wait_timeout: the wait ran out");
  return MOR_OK;
}

int mor_lift(const mor_subdomains* sd, const mor_bases* b, const double* x_dev, double* u_dev,
             void* stream) {
  if (!sd || !b || !x_dev || !u_dev) return fail(MOR_ERR_ARG, "mor_lift: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(u_dev, 0, sd->hp.n_nodes * sizeof(double), st));
  launch_lift(sd->hp.nO, sd->o_node, sd->o_sd, b->Q, b->kq, x_dev, u_dev, st);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(st));
  return MOR_OK;
}

int mor_energy_norm(const mor_subdomains* sd, const double* u1_dev, const double* u2_dev,
                    double* out, void* stream) {
  if (!sd || !u1_dev || !out) return fail(MOR_ERR_ARG, "mor_energy_norm: null argument");
  cudaStream_t st = (cudaStream_t)stream;
  Allocs A;
  double* part;
  double* res;
  int64_t nb = ceil_div(sd->hp.n_tets, 256);
  TRY(A.alloc(&part, nb, false, st));
  TRY(A.alloc(&res, 1, false, st));
  launch_energy(sd->hp.n_tets, sd->xyz, sd->tets, sd->kappa, u1_dev, u2_dev, part, res, st);
  double h = 0;
  CK(cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *out = std::sqrt(std::max(h, 0.0));
  return MOR_OK;
}

int mor_debug_plan_check(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                         const uint8_t* dirichlet, const int32_t* owner, const double* xyz,
                         int32_t r_hops, int32_t wave_subdomains, int32_t coarse_rows,
                         int64_t* out) {
  if (!tets || !dirichlet || !owner || !out || wave_subdomains < 1 || coarse_rows < 1)
    return fail(MOR_ERR_ARG, "mor_debug_plan_check: bad argument");
  std::string err;
  HostPlan full, g;
  int rc = build_host_plan(n_nodes, n_tets, tets, dirichlet, owner, r_hops, xyz, full, err);
  if (rc != MOR_OK) return fail(rc, err);
  rc = build_global_plan(n_nodes, n_tets, tets, dirichlet, owner, r_hops, g, err);
  if (rc != MOR_OK) return fail(rc, err);
  int64_t bad = 0, waves = 0;
  if (g.nO != full.nO || g.o_node != full.o_node || g.o_sd != full.o_sd ||
      g.pair_ptr != full.pair_ptr || g.e_urow != full.e_urow || g.e_vrow != full.e_vrow)
    ++bad;
  PlanScratch ps;
  for (int s0 = 0; s0 < g.n_sd; s0 += wave_subdomains, ++waves) {
    const int s1 = std::min(g.n_sd, s0 + wave_subdomains);
    HostPlan w;
    rc = build_wave_plan(n_nodes, n_tets, tets, dirichlet, xyz, g, s0, s1, w, ps, err);
    if (rc != MOR_OK) return fail(rc, err);
    const int64_t P0 = full.Poff[s0], W0 = full.Woff[s0], O0 = full.Ooff[s0];
    if (w.nP != full.Poff[s1] - P0 || w.nW != full.Woff[s1] - W0 ||
        w.nO != full.Ooff[s1] - O0) {
      ++bad;
      continue;
    }
    for (int64_t r = 0; r < w.nP; ++r) {
      if (w.p_node[r] != full.p_node[P0 + r] || w.p_code[r] != full.p_code[P0 + r]) ++bad;
      const int64_t sw = r / kSlice, sf = (P0 + r) / kSlice;
      for (int j = 0; j < std::max(w.pat_P.W, full.pat_P.W); ++j) {
        int32_t cw = j < w.pat_P.width[sw] ? w.pat_P.col[(sw * kSlice + 0) * w.pat_P.W +
                                                         j * kSlice + r % kSlice] : -1;
        int32_t cf = j < full.pat_P.width[sf]
                         ? full.pat_P.col[sf * kSlice * full.pat_P.W + j * kSlice +
                                          (P0 + r) % kSlice]
                         : -1;
        if ((cw < 0) != (cf < 0) || (cf >= 0 && cf != cw + P0)) ++bad;
      }
      for (int64_t q = w.incP_ptr[r], qf = full.incP_ptr[P0 + r]; q < w.incP_ptr[r + 1];
           ++q, ++qf)
        if (w.incP_tet[q] != full.incP_tet[qf] || w.incP_code[q] != full.incP_code[qf]) ++bad;
    }
    for (int64_t x = 0; x < w.nW; ++x)
      if (w.w2p[x] + P0 != full.w2p[W0 + x]) ++bad;
    for (int64_t o = 0; o < w.nO; ++o)
      if (w.o_node[o] != full.o_node[O0 + o] || w.o2w[o] + W0 != full.o2w[O0 + o]) ++bad;
  }
  // aggregates of the coarse level: contiguous, ordered I then B, within the caps
  AggPlan ap;
  build_aggregates(full, coarse_rows, kMaxAgg, ap);
  int64_t agg_bad = 0, max_nc = 0;
  for (int i = 0; i < full.n_sd; ++i) {
    const int n0 = ap.nca[0][i], n1 = ap.nca[1][i];
    max_nc = std::max<int64_t>(max_nc, n1);
    if (n1 > kMaxAgg || n0 > n1) ++agg_bad;
    const int32_t* al = ap.aloc.data() + full.Poff[i];
    const int nrow = full.nI[i] + full.nB[i];
    for (int l = 0; l < nrow; ++l) {
      if (al[l] < 0 || al[l] >= n1) ++agg_bad;
      if (l > 0 && (al[l] < al[l - 1] || al[l] > al[l - 1] + 1)) ++agg_bad;
      if ((l < full.nI[i]) != (al[l] < n0)) ++agg_bad;
    }
  }
  out[0] = full.n_sd;
  out[1] = full.nP;
  out[2] = waves;
  out[3] = bad;
  out[4] = agg_bad;
  out[5] = ap.max_slots;
  out[6] = max_nc;
  out[7] = full.nO;
  return MOR_OK;
}

int mor_debug_sketch_rhs(const mor_subdomains* sd, const mor_basis_opts* opts, int32_t sub,
                         double* out, void* stream) {
  if (!sd || !opts || !out || sub < 0 || sub >= sd->hp.n_sd)
    return fail(MOR_ERR_ARG, "mor_debug_sketch_rhs: bad argument");
  if (sd->streamed)
    return fail(MOR_ERR_STATE, "mor_debug_sketch_rhs: not available for streamed plans");
  const HostPlan& hp = sd->hp;
  cudaStream_t st = (cudaStream_t)stream;
  int k = opts->rank + opts->oversample;
  int64_t row0 = hp.Poff[sub], n_rows = hp.Poff[sub + 1] - row0;
  Allocs A;
  float2* lsplit;
  double* res;
  TRY(A.alloc(&lsplit, (size_t)hp.n_tets * 10, false, st));
  TRY(A.alloc(&res, (hp.nP) * (size_t)k, true, st));
  launch_elem_chol(hp.n_tets, sd->xyz, sd->tets, sd->kappa, opts->h1_weighted, lsplit, st);
  launch_sketch_rhs(row0, n_rows, sd->p_sd, sd->incP_ptr, sd->incP_tet, sd->incP_code, lsplit,
                    k, opts->seed, 0u, res, k, st, nullptr);
  CK(cudaGetLastError());
  std::vector<double> tmp((size_t)n_rows * k);
  CK(cudaMemcpyAsync(tmp.data(), res + row0 * k, tmp.size() * sizeof(double),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  // P rows are in Morton order within I and B; report I then B in ascending node order
  const SubSets& ss = hp.sets[sub];
  const int64_t nI = (int64_t)ss.I.size();
  for (int64_t l = 0; l < n_rows; ++l) {
    int32_t v = hp.p_node[row0 + l];
    int64_t dst = l < nI ? std::lower_bound(ss.I.begin(), ss.I.end(), v) - ss.I.begin()
                         : nI + (std::lower_bound(ss.B.begin(), ss.B.end(), v) - ss.B.begin());
    std::copy(tmp.begin() + l * k, tmp.begin() + (l + 1) * k, out + dst * k);
  }
  return MOR_OK;
}

int mor_debug_tc_gram(int64_t rows, int32_t nx, int32_t ny, const double* X_dev,
                      const double* Y_dev, double* G_dev, void* stream) {
  if (rows < 0 || nx < 1 || ny < 1 || nx > 128 || ny > 128 || !G_dev ||
      (rows > 0 && (!X_dev || !Y_dev)))
    return fail(MOR_ERR_ARG, "mor_debug_tc_gram: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Allocs A;
  A.use_pool(st);
  double* part;
  int64_t* range;
  int* err;
  TRY(A.alloc(&part, (size_t)nx * ny, false, st));
  TRY(A.alloc(&range, 2, true, st));
  TRY(A.alloc(&err, 1, true, st));
  launch_tc_gram_rows(rows, X_dev, nx, nx, Y_dev, ny, ny, part, range, G_dev,
                      wait_budget_cycles(), err, st);
  int h = 0;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) return fail(MOR_ERR_TIMEOUT, "mor_debug_tc_gram: a wait ran out of its budget");
  return MOR_OK;
}

int mor_debug_coarse_inverse(int32_t n, const double* E_dev, double* Einv_dev, void* stream) {
  if (n < 1 || n > kMaxAgg || !E_dev || !Einv_dev)
    return fail(MOR_ERR_ARG, "mor_debug_coarse_inverse: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  Allocs A;
  A.use_pool(st);
  int32_t* nca;
  int64_t* eoff;
  float *W, *P;
  double* sc;
  int* bad;
  const int32_t h_n = n;
  const int64_t h_off = 0;
  TRY(A.alloc(&nca, 1, false, st));
  TRY(A.alloc(&eoff, 1, false, st));
  TRY(A.alloc(&W, (size_t)n * n, false, st));
  TRY(A.alloc(&P, (size_t)kCoarsePivots * kCoarsePivots, false, st));
  TRY(A.alloc(&sc, (size_t)n, false, st));
  TRY(A.alloc(&bad, 1, true, st));
  CK(cudaMemcpyAsync(nca, &h_n, sizeof h_n, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(eoff, &h_off, sizeof h_off, cudaMemcpyHostToDevice, st));
  launch_coarse_invert<double>(1, n, nca, eoff, E_dev, W, P, sc, Einv_dev, bad, st);
  int h = 0;
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (h) return fail(MOR_ERR_ARG, "mor_debug_coarse_inverse: a pivot is not positive");
  return MOR_OK;
}

int mor_profile_enable(int32_t on) {
  g_prof.on = on != 0;
  return MOR_OK;
}
int mor_profile_reset(void) {
  for (int f = 0; f < kFamilies; ++f) g_prof.launches[f] = g_prof.ms[f] = g_prof.bytes[f] = 0;
  return MOR_OK;
}
int mor_profile_query(int32_t family, double* out) {
  if (family < 0 || family >= kFamilies || !out)
    return fail(MOR_ERR_ARG, "mor_profile_query: bad argument");
  out[0] = g_prof.launches[family];
  out[1] = g_prof.ms[family];
  out[2] = g_prof.bytes[family];
  out[3] = 0;
  return MOR_OK;
}
int mor_autotune(int32_t on) {
  if (on < 0)
    autotune_reset();
  else
    autotune_enable(on != 0);
  return MOR_OK;
}

int mor_autotune_report(int64_t* out, int32_t max_entries, int32_t* n) {
  if (!n || max_entries < 0 || (max_entries > 0 && !out))
    return fail(MOR_ERR_ARG, "mor_autotune_report: bad argument");
  *n = autotune_entries(out, max_entries);
  return MOR_OK;
}

int mor_kernel_launches(int64_t* out) {
  if (!out) return fail(MOR_ERR_ARG, "mor_kernel_launches: null");
  *out = (int64_t)g_kernel_launches.load();
  return MOR_OK;
}

void mor_free_subdomains(mor_subdomains* h) { delete h; }
void mor_free_bases(mor_bases* h) { delete h; }
void mor_free_reduced(mor_reduced* h) { delete h; }

}  // extern "C"
