// Step 3 (Eq. (23), Sec. 6 step 3): the off-diagonal blocks of Q^T A Q from the
// interface couplings of neighbouring subdomains, the reduced CG solve (diagonal
// preconditioner = identity because every diagonal block is I after the step-2
// update), and the lift u~ = sum_i S_i Q_i x_i.
#include "mor_dev.cuh"
#include "mor_kernels.h"

#include <algorithm>

namespace mor {
namespace {

constexpr int kPairThreads = 512;
constexpr int kPairPerThread = 32;  // 512 * 32 >= 128 * 128
constexpr int kPairChunk = 32;

__global__ void __launch_bounds__(kPairThreads)
    k_pair_blocks(const int64_t* __restrict__ pair_ptr, const int32_t* __restrict__ urow,
                  const int32_t* __restrict__ vrow, const double* __restrict__ aval,
                  const double* __restrict__ Q, int kq, double* blocks) {
  extern __shared__ double sh[];
  double* Qu = sh;
  double* Qv = Qu + kPairChunk * kq;
  double* av = Qv + kPairChunk * kq;
  int p = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  int64_t e0 = pair_ptr[p], e1 = pair_ptr[p + 1];
  int nout = kq * kq;
  double acc[kPairPerThread];
#pragma unroll
  for (int m = 0; m < kPairPerThread; ++m) acc[m] = 0.0;
  for (int64_t base = e0; base < e1; base += kPairChunk) {
    int ne = (int)min((int64_t)kPairChunk, e1 - base);
    for (int idx = tid; idx < ne * kq; idx += nth) {
      int ee = idx / kq, c = idx % kq;
      Qu[ee * kq + c] = Q[(int64_t)urow[base + ee] * kq + c];
      Qv[ee * kq + c] = Q[(int64_t)vrow[base + ee] * kq + c];
    }
    for (int ee = tid; ee < ne; ee += nth) av[ee] = aval[base + ee];
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kPairPerThread; ++m) {
      int o = tid + m * nth;
      if (o < nout) {
        int i = o / kq, j = o % kq;
        double s = 0.0;
        for (int ee = 0; ee < ne; ++ee) s += av[ee] * Qu[ee * kq + i] * Qv[ee * kq + j];
        acc[m] += s;
      }
    }
    __syncthreads();
  }
  double* Bij = blocks + (int64_t)(2 * p) * nout;
  double* Bji = blocks + (int64_t)(2 * p + 1) * nout;
#pragma unroll
  for (int m = 0; m < kPairPerThread; ++m) {
    int o = tid + m * nth;
    if (o < nout) {
      int i = o / kq, j = o % kq;
      Bij[i * kq + j] = acc[m];
      Bji[j * kq + i] = acc[m];
    }
  }
}

// ---- reduced CG: one block per block row (subdomain), global last-block reductions
__device__ __forceinline__ double block_sum128(double x, double* red) {
  red[threadIdx.x] = x;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool last_global(int* counter, int nblk) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    int prev = atomicAdd(counter, 1);
    is_last = (prev == nblk - 1);
    if (is_last) *counter = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

__device__ double sum_parts(const double* part, int n, int stride, int off, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(part + (int64_t)i * stride + off);
  return block_sum128(s, red);
}

__global__ void k_rcg_init(int n_sd, int kq, const double* __restrict__ bt, RcgState s) {
  __shared__ double red[128];
  int sd = blockIdx.x;
  double loc = 0.0;
  for (int i = threadIdx.x; i < kq; i += blockDim.x) {
    int64_t g = (int64_t)sd * kq + i;
    double b = bt[g];
    s.x[g] = 0.0;
    s.r[g] = b;
    s.p[g] = b;
    loc += b * b;
  }
  double t = block_sum128(loc, red);
  if (threadIdx.x == 0) s.part[2 * sd] = t;
  if (!last_global(s.counter, n_sd)) return;
  double bb = sum_parts(s.part, n_sd, 2, 0, red);
  if (threadIdx.x == 0) {
    s.scal[0] = bb;
    s.scal[1] = bb;
    s.scal[2] = 0.0;
    s.scal[3] = 0.0;
    s.scal[4] = bb;
    s.flag[0] = (bb > 0.0) ? 0 : 1;
    s.flag[1] = 0;
  }
}

__global__ void k_rcg_spmv(int n_sd, int kq, const int32_t* __restrict__ nbr_ptr,
                           const int32_t* __restrict__ nbr_sd, const int32_t* __restrict__ nbr_blk,
                           const double* __restrict__ blocks, RcgState s) {
  __shared__ double red[128];
  int sd = blockIdx.x;
  double loc = 0.0;
  for (int i = threadIdx.x; i < kq; i += blockDim.x) {
    int64_t g = (int64_t)sd * kq + i;
    double acc = s.p[g];
    for (int q = nbr_ptr[sd]; q < nbr_ptr[sd + 1]; ++q) {
      const double* B = blocks + (int64_t)nbr_blk[q] * kq * kq + (int64_t)i * kq;
      const double* pj = s.p + (int64_t)nbr_sd[q] * kq;
      for (int l = 0; l < kq; ++l) acc += B[l] * pj[l];
    }
    s.q[g] = acc;
    loc += s.p[g] * acc;
  }
  double t = block_sum128(loc, red);
  if (threadIdx.x == 0) s.part[2 * sd] = t;
  if (!last_global(s.counter, n_sd)) return;
  double pq = sum_parts(s.part, n_sd, 2, 0, red);
  if (threadIdx.x == 0) s.scal[2] = (s.flag[0] || !(pq > 0.0)) ? 0.0 : s.scal[0] / pq;
}

__global__ void k_rcg_update_xr(int n_sd, int kq, double tol2, RcgState s) {
  __shared__ double red[128];
  int sd = blockIdx.x;
  double al = s.scal[2];
  double loc = 0.0;
  for (int i = threadIdx.x; i < kq; i += blockDim.x) {
    int64_t g = (int64_t)sd * kq + i;
    s.x[g] += al * s.p[g];
    double r = s.r[g] - al * s.q[g];
    s.r[g] = r;
    loc += r * r;
  }
  double t = block_sum128(loc, red);
  if (threadIdx.x == 0) s.part[2 * sd + 1] = t;
  if (!last_global(s.counter, n_sd)) return;
  double rr = sum_parts(s.part, n_sd, 2, 1, red);
  if (threadIdx.x == 0) {
    double be = 0.0;
    if (!s.flag[0]) {
      s.flag[1] += 1;
      s.scal[4] = rr;
      if (rr <= tol2 * s.scal[1] || !(s.scal[0] > 0.0)) {
        s.flag[0] = 1;
      } else {
        be = rr / s.scal[0];
        s.scal[0] = rr;
      }
    }
    s.scal[3] = be;
  }
}

__global__ void k_rcg_update_p(int kq, RcgState s) {
  int sd = blockIdx.x;
  double be = s.scal[3];
  for (int i = threadIdx.x; i < kq; i += blockDim.x) {
    int64_t g = (int64_t)sd * kq + i;
    s.p[g] = s.r[g] + be * s.p[g];
  }
}

// The whole reduced CG in one cooperative launch: blocks take block rows sd =
// blockIdx.x, blockIdx.x + gridDim.x, ...; the three phases of an iteration (q = K~ p
// with p.q; x and r update with r.r; p update) are separated by grid barriers with
// bounded waits.  Every block forms the scalars itself from the same partial sums in
// the same order (sum_parts), so all blocks take the same decisions; the arithmetic is
// that of the three-kernel iteration.  sync[0] barrier count, sync[1] generation,
// sync[2] error (a wait ran out).
__global__ void __launch_bounds__(128)
    k_rcg_persistent(int n_sd, int kq, const int32_t* __restrict__ nbr_ptr,
                     const int32_t* __restrict__ nbr_sd, const int32_t* __restrict__ nbr_blk,
                     const double* __restrict__ blocks, const double* __restrict__ bt,
                     double tol2, int max_iter, RcgState s, unsigned* sync,
                     long long budget) {
  __shared__ double red[128];
  unsigned* count = sync;
  volatile unsigned* gen = sync + 1;
  volatile int* err = reinterpret_cast<volatile int*>(sync + 2);
  // x = 0, r = p = b~, ||b~||^2
  for (int sd = blockIdx.x; sd < n_sd; sd += gridDim.x) {
    double loc = 0.0;
    for (int i = threadIdx.x; i < kq; i += blockDim.x) {
      const int64_t g = (int64_t)sd * kq + i;
      const double b = bt[g];
      s.x[g] = 0.0;
      s.r[g] = b;
      s.p[g] = b;
      loc += b * b;
    }
    const double t = block_sum128(loc, red);
    if (threadIdx.x == 0) s.part[2 * sd] = t;
  }
  if (!grid_barrier(count, gen, err, budget)) return;
  const double bb = sum_parts(s.part, n_sd, 2, 0, red);
  double rz = bb, rr = bb;
  int done = bb > 0.0 ? 0 : 1, it = 0;
  while (!done && it < max_iter) {
    // q = K~ p (identity diagonal blocks) and p.q
    for (int sd = blockIdx.x; sd < n_sd; sd += gridDim.x) {
      double loc = 0.0;
      for (int i = threadIdx.x; i < kq; i += blockDim.x) {
        const int64_t g = (int64_t)sd * kq + i;
        double acc = s.p[g];
        for (int q = nbr_ptr[sd]; q < nbr_ptr[sd + 1]; ++q) {
          const double* B = blocks + (int64_t)nbr_blk[q] * kq * kq + (int64_t)i * kq;
          const double* pj = s.p + (int64_t)nbr_sd[q] * kq;
          for (int l = 0; l < kq; ++l) acc += B[l] * pj[l];
        }
        s.q[g] = acc;
        loc += s.p[g] * acc;
      }
      const double t = block_sum128(loc, red);
      if (threadIdx.x == 0) s.part[2 * sd] = t;
    }
    if (!grid_barrier(count, gen, err, budget)) return;
    const double pq = sum_parts(s.part, n_sd, 2, 0, red);
    const double al = pq > 0.0 ? rz / pq : 0.0;
    for (int sd = blockIdx.x; sd < n_sd; sd += gridDim.x) {
      double loc = 0.0;
      for (int i = threadIdx.x; i < kq; i += blockDim.x) {
        const int64_t g = (int64_t)sd * kq + i;
        s.x[g] += al * s.p[g];
        const double r = s.r[g] - al * s.q[g];
        s.r[g] = r;
        loc += r * r;
      }
      const double t = block_sum128(loc, red);
      if (threadIdx.x == 0) s.part[2 * sd + 1] = t;
    }
    if (!grid_barrier(count, gen, err, budget)) return;
    rr = sum_parts(s.part, n_sd, 2, 1, red);
    ++it;
    double be = 0.0;
    if (rr <= tol2 * bb || !(rz > 0.0)) {
      done = 1;
    } else {
      be = rr / rz;
      rz = rr;
    }
    if (!done) {
      for (int sd = blockIdx.x; sd < n_sd; sd += gridDim.x)
        for (int i = threadIdx.x; i < kq; i += blockDim.x) {
          const int64_t g = (int64_t)sd * kq + i;
          s.p[g] = s.r[g] + be * s.p[g];
        }
      if (!grid_barrier(count, gen, err, budget)) return;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    s.scal[0] = rz;
    s.scal[1] = bb;
    s.scal[4] = rr;
    s.flag[0] = done;
    s.flag[1] = it;
  }
}

// a bounded wait on a flag that nothing sets (the timeout path of the grid barrier)
__global__ void k_wait_unset_flag(unsigned* sync, long long budget, int* status) {
  volatile unsigned* gen = sync + 1;
  volatile int* err = reinterpret_cast<volatile int*>(sync + 2);
  if (threadIdx.x == 0) *status = bounded_wait(gen, *gen, err, budget) ? 0 : 1;
}

__global__ void k_lift(int64_t n_o, const int32_t* __restrict__ o_node,
                       const int32_t* __restrict__ o_sd, const double* __restrict__ Q, int kq,
                       const double* __restrict__ x, double* u) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n_o) return;
  const double* xs = x + (int64_t)o_sd[r] * kq;
  double s = 0.0;
  for (int c = 0; c < kq; ++c) s += Q[r * kq + c] * xs[c];
  u[o_node[r]] = s;
}

}  // namespace

void launch_pair_blocks(int n_pairs, const int64_t* pair_ptr, const int32_t* urow,
                        const int32_t* vrow, const double* aval, const double* Q, int kq,
                        double* blocks, cudaStream_t st) {
  if (n_pairs <= 0) return;
  size_t sm = sizeof(double) * (2 * (size_t)kPairChunk * kq + kPairChunk);
  static bool attr = false;
  if (!attr) {  // kq up to 128: 66 KB
    cudaFuncSetAttribute(k_pair_blocks, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         100 * 1024);
    attr = true;
  }
  count_launch();
  k_pair_blocks<<<n_pairs, kPairThreads, sm, st>>>(pair_ptr, urow, vrow, aval, Q, kq, blocks);
}

void launch_rcg_init(int n_sd, int kq, const double* bt, const RcgState& s,
                     cudaStream_t st) {
  count_launch();
  k_rcg_init<<<n_sd, 128, 0, st>>>(n_sd, kq, bt, s);
}

void launch_rcg_step(int n_sd, int kq, const int32_t* nbr_ptr, const int32_t* nbr_sd,
                     const int32_t* nbr_blk, const double* blocks, double tol2,
                     const RcgState& s, cudaStream_t st) {
  count_launch();
  k_rcg_spmv<<<n_sd, 128, 0, st>>>(n_sd, kq, nbr_ptr, nbr_sd, nbr_blk, blocks, s);
  count_launch();
  k_rcg_update_xr<<<n_sd, 128, 0, st>>>(n_sd, kq, tol2, s);
  count_launch();
  k_rcg_update_p<<<n_sd, 128, 0, st>>>(kq, s);
}

int launch_rcg_persistent(int n_sd, int kq, const int32_t* nbr_ptr, const int32_t* nbr_sd,
                          const int32_t* nbr_blk, const double* blocks, const double* bt,
                          double tol2, int max_iter, const RcgState& s, unsigned* sync,
                          long long budget, cudaStream_t st) {
  int dev = 0, nsm = 0, per_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rcg_persistent, 128, 0) !=
          cudaSuccess ||
      per_sm < 1)
    return -1;
  int grid = std::min(n_sd, nsm * per_sm);
  RcgState sc = s;
  void* args[] = {&n_sd, &kq, (void*)&nbr_ptr, (void*)&nbr_sd, (void*)&nbr_blk,
                  (void*)&blocks, (void*)&bt, &tol2, &max_iter, &sc, &sync, &budget};
  count_launch();
  if (cudaLaunchCooperativeKernel((const void*)k_rcg_persistent, grid, 128, args, 0, st) !=
      cudaSuccess)
    return -1;
  return grid;
}

void launch_wait_unset_flag(unsigned* sync, long long budget, int* status, cudaStream_t st) {
  count_launch();
  k_wait_unset_flag<<<1, 32, 0, st>>>(sync, budget, status);
}

void launch_lift(int64_t n_o, const int32_t* o_node, const int32_t* o_sd, const double* Q,
                 int kq, const double* x, double* u, cudaStream_t st) {
  if (n_o <= 0) return;
  count_launch();
  k_lift<<<(unsigned)((n_o + 255) / 256), 256, 0, st>>>(n_o, o_node, o_sd, Q, kq, x, u);
}

}  // namespace mor
