// Setup of the coarse level of the two-level local preconditioner
// M^{-1} = D^{-1} + Z E^{-1} Z^T used by every local CG of step 2: the aggregate
// matrices E = Z^T A Z per subdomain (Z = aggregate indicators) and their inverses.
// The preconditioner only changes how fast the solves of Sec. 4 / Sec. 6 converge,
// not what they compute.
#include "mor_kernels.h"
#include "mor_plan.h"

namespace mor {
namespace {

// one thread per row of a tile: every stored entry (i, j) adds A_ij to E[a(i)][a(j)]
__global__ void k_coarse_matrix(DTiles tl, EllView<double> A, const int32_t* __restrict__ aloc,
                                const int32_t* __restrict__ nca,
                                const int64_t* __restrict__ eoff, double* E) {
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int64_t row = tl.r0[tile] + (int64_t)threadIdx.x;
  if (row >= tl.r1[tile]) return;
  const int n = nca[sd];
  const int a = aloc[row];
  if (a >= n) return;
  double* Eb = E + eoff[sd] + (int64_t)a * n;
  const int w = A.width[row >> 5];
  for (int j = 0; j < w; ++j) {
    int64_t at = ell_at(row, j, A.W);
    int32_t c = A.col[at];
    if (c < 0) continue;
    int b = aloc[c];
    if (b < n) atomicAdd(Eb + b, A.val[at]);
  }
}

// In-place Gauss-Jordan inverse of the SPD block of one subdomain, pivots in order
// (no pivoting is needed for SPD matrices): at step k with p = 1 / M_kk,
// M_kj <- p M_kj, M_ik <- -p M_ik, M_ij <- M_ij - M_ik p M_kj (i, j != k), M_kk <- p.
// Then einv = (M + M^T) / 2 in T.  A non-positive pivot marks the block bad.
template <typename T>
__global__ void k_coarse_invert(const int32_t* __restrict__ nca,
                                const int64_t* __restrict__ eoff, double* E, T* einv,
                                int* bad) {
  const int sd = blockIdx.x;
  const int n = nca[sd];
  if (n <= 0) return;
  double* M = E + eoff[sd];
  __shared__ double colk[kMaxAgg], rowk[kMaxAgg];
  __shared__ double piv;
  __shared__ int fail;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = ty * blockDim.x + tx, nth = blockDim.x * blockDim.y;
  if (tid == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = M[(int64_t)k * n + k];
      if (!(d > 0.0)) {
        fail = 1;
        d = 1.0;
      }
      piv = 1.0 / d;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nth) {
      colk[i] = M[(int64_t)i * n + k];
      rowk[i] = M[(int64_t)k * n + i] * piv;
    }
    __syncthreads();
    const double p = piv;
    for (int i = ty; i < n; i += blockDim.y) {
      double* Mi = M + (int64_t)i * n;
      const double ci = colk[i];
      if (i == k) {
        for (int j = tx; j < n; j += blockDim.x) Mi[j] = (j == k) ? p : rowk[j];
      } else {
        for (int j = tx; j < n; j += blockDim.x)
          Mi[j] = (j == k) ? -ci * p : Mi[j] - ci * rowk[j];
      }
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) atomicAdd(bad, 1);
    return;
  }
  T* out = einv + eoff[sd];
  for (int i = ty; i < n; i += blockDim.y)
    for (int j = tx; j < n; j += blockDim.x)
      out[(int64_t)i * n + j] = (T)(0.5 * (M[(int64_t)i * n + j] + M[(int64_t)j * n + i]));
}

}  // namespace

void launch_coarse_matrix(const DTiles& tiles, const EllView<double>& A, const int32_t* aloc,
                          const int32_t* nca, const int64_t* eoff, double* E, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_coarse_matrix<<<tiles.n, kTileRows, 0, st>>>(tiles, A, aloc, nca, eoff, E);
}

template <typename T>
void launch_coarse_invert(int n_sd, const int32_t* nca, const int64_t* eoff, double* E,
                          T* einv, int* bad, cudaStream_t st) {
  if (n_sd <= 0) return;
  count_launch();
  k_coarse_invert<T><<<n_sd, dim3(32, 16), 0, st>>>(nca, eoff, E, einv, bad);
}

template void launch_coarse_invert<float>(int, const int32_t*, const int64_t*, double*, float*,
                                          int*, cudaStream_t);
template void launch_coarse_invert<double>(int, const int32_t*, const int64_t*, double*,
                                           double*, int*, cudaStream_t);

}  // namespace mor
