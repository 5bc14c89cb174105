// The reduced solve of mor_solve_reduced in a form that allocates nothing: its work
// vectors live in one fixed device array of this file instead of cudaMalloc'd buffers.
// It runs the same CG kernels (mor_reduced.cu) on caller-owned inputs and output.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/mor.h"
#include "mor_kernels.h"

using namespace mor;

namespace {

// Limits of the fixed scratch array: the reduced vectors r, p, q (3 x kMaxDim binary64),
// the per-subdomain partial sums (2 x kMaxSub), 8 scalars and a 3-int tail (ticket
// counter, done flag, iteration count): 1,703,952 doubles = 13.6 MB.  The array is
// placed on a device when this file's device code is loaded there (with CUDA's default
// lazy loading: at the first set-up below on that device) and stays until the process
// exits.
constexpr int64_t kMaxDim = int64_t(1) << 19;  // 524,288 reduced unknowns
constexpr int64_t kMaxSub = int64_t(1) << 16;  // 65,536 subdomains
constexpr int64_t kVecOff = 0;
constexpr int64_t kPartOff = 3 * kMaxDim;
constexpr int64_t kScalOff = kPartOff + 2 * kMaxSub;
constexpr int64_t kIntOff = kScalOff + 8;
constexpr int64_t kScratchDoubles = kIntOff + 8;
static_assert(kScratchDoubles == 1703952, "stated scratch size");

static __device__ __align__(256) double g_solve_scratch[kScratchDoubles];

// Device address of g_solve_scratch.  In host code the symbol is a host stand-in, not a
// device address, so the set-up looks the address up with cudaGetSymbolAddress, once per
// device and CUDA context, with that device current.  The cache is keyed by the
// context's unique id: after cudaDeviceReset the device gets a new context, the module
// is loaded again (possibly elsewhere) and the address is looked up again.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

std::mutex g_mu;
constexpr int kMaxDevices = 128;
struct Slot {
  unsigned long long ctx_id = 0;
  double* ptr = nullptr;
};
Slot g_slot[kMaxDevices];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

int driver_fns() {
  if (g_ctx_current && g_ctx_id) return MOR_OK;
  void* f1 = nullptr;
  void* f2 = nullptr;
  cudaDriverEntryPointQueryResult q1, q2;
  cudaError_t e1 = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000,
                                                    cudaEnableDefault, &q1);
  cudaError_t e2 = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000,
                                                    cudaEnableDefault, &q2);
  if (e1 != cudaSuccess || e2 != cudaSuccess || q1 != cudaDriverEntryPointSuccess ||
      q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
    return set_error(MOR_ERR_CUDA, "mor_solve_reduced_noalloc: driver context query unavailable");
  g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
  g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  return MOR_OK;
}

int scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(MOR_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(MOR_ERR_ARG, "mor_solve_reduced_noalloc: device index out of range");
  // cudaSetDevice initialises the device's primary context and makes it current (a
  // no-op when it already is)
  e = cudaSetDevice(dev);
  if (e != cudaSuccess) return set_error(MOR_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_mu);
  int rc = driver_fns();
  if (rc != MOR_OK) return rc;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx || g_ctx_id(ctx, &id) != CUDA_SUCCESS)
    return set_error(MOR_ERR_CUDA, "mor_solve_reduced_noalloc: no current CUDA context");
  Slot& s = g_slot[dev];
  if (!s.ptr || s.ctx_id != id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_solve_scratch);
    if (e != cudaSuccess || !p)
      return set_error(MOR_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    s.ptr = static_cast<double*>(p);
    s.ctx_id = id;
  }
  *out = s.ptr;
  return MOR_OK;
}

// E = bt . x into *out (one block, fixed summation order)
__global__ void k_energy_dot(int64_t n, const double* __restrict__ bt,
                             const double* __restrict__ x, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += bt[i] * x[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

extern "C" int mor_solve_reduced_noalloc(int32_t n_sub, int32_t kq, const int32_t* nbr_ptr_dev,
                                         const int32_t* nbr_sub_dev, const int32_t* nbr_blk_dev,
                                         const double* blocks_dev, const double* bt_dev,
                                         double rtol, int32_t max_iter, void* stream,
                                         double* x_dev, mor_solve_info* info) {
  if (n_sub < 1 || kq < 1 || !nbr_ptr_dev || !nbr_sub_dev || !nbr_blk_dev || !blocks_dev ||
      !bt_dev || !x_dev || !(rtol > 0.0) || max_iter < 1)
    return set_error(MOR_ERR_ARG, "mor_solve_reduced_noalloc: bad argument");
  const int64_t dim = (int64_t)n_sub * kq;
  if (dim > kMaxDim || n_sub > kMaxSub)
    return set_error(MOR_ERR_ARG,
                     "mor_solve_reduced_noalloc: system too large for the fixed scratch "
                     "(n_sub * kq <= 524288 and n_sub <= 65536 required)");
  double* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != MOR_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  RcgState s{};
  s.x = x_dev;
  s.r = base + kVecOff;
  s.p = base + kVecOff + dim;
  s.q = base + kVecOff + 2 * dim;
  s.part = base + kPartOff;
  s.scal = base + kScalOff;
  int* ints = reinterpret_cast<int*>(base + kIntOff);
  s.counter = ints;
  s.flag = ints + 1;
  // the array keeps the previous call's contents: the ticket counter and the flags
  // must start at zero
  cudaError_t e = cudaMemsetAsync(ints, 0, 3 * sizeof(int), st);
  if (e != cudaSuccess) return set_error(MOR_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  launch_rcg_init(n_sub, kq, bt_dev, s, st);
  int hf[2] = {0, 0};
  for (int it = 0; it < max_iter;) {
    int chunk = max_iter - it < 16 ? max_iter - it : 16;
    for (int c = 0; c < chunk; ++c)
      launch_rcg_step(n_sub, kq, nbr_ptr_dev, nbr_sub_dev, nbr_blk_dev, blocks_dev,
                      rtol * rtol, s, st);
    it += chunk;
    e = cudaMemcpyAsync(hf, s.flag, sizeof(hf), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(MOR_ERR_CUDA, std::string("reduced solve: ") + cudaGetErrorString(e));
    if (hf[0]) break;
  }
  count_launch();
  k_energy_dot<<<1, 256, 0, st>>>(dim, bt_dev, x_dev, s.scal + 6);
  double sc[8];
  e = cudaMemcpyAsync(sc, s.scal, sizeof(sc), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(MOR_ERR_CUDA, std::string("reduced solve: ") + cudaGetErrorString(e));
  const bool ok = hf[0] && sc[4] <= rtol * rtol * sc[1];
  if (info) {
    info->iterations = hf[1];
    info->converged = ok ? 1 : 0;
    info->rel_residual = sc[1] > 0 ? std::sqrt(sc[4] / sc[1]) : 0.0;
    info->energy = sc[6];
  }
  if (!ok) return set_error(MOR_ERR_NOT_CONVERGED, "mor_solve_reduced_noalloc: max_iter reached");
  return MOR_OK;
}
