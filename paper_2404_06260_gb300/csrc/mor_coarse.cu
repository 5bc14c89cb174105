// Setup of the coarse level of the two-level local preconditioner
// M^{-1} = D^{-1} + Z E^{-1} Z^T used by every local CG of step 2: the aggregate
// matrices E = Z^T A Z per subdomain (Z = aggregate indicators) and their inverses.
// The preconditioner only changes how fast the solves of Sec. 4 / Sec. 6 converge,
// not what they compute.
#include "mor_kernels.h"
#include "mor_plan.h"
#include "mor_tc.cuh"

#include <cuda_bf16.h>

#include <algorithm>

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

// ---- E^{-1} by blocked Gauss-Jordan elimination in binary32 ----
// With S = diag(E)^{-1/2} the unit-diagonal W = S E S is inverted in place, pivot block
// by pivot block (kGJ pivots, in order: SPD matrices need no pivoting).  For the pivot
// block K with P = W_KK^{-1}: W_KJ <- P W_KJ (J != K), W_IJ <- W_IJ - W_IK W_KJ
// (I, J != K), W_IK <- -W_IK P (I != K), W_KK <- P.  Then E^{-1} = S W S, symmetrised.
// The coarse level only preconditions the local solves, so binary32 (the working
// precision of the mixed path) is enough for either path: any symmetric positive
// definite E^{-1} leaves the CG solutions unchanged and only moves iteration counts.
constexpr int kGJ = kCoarsePivots;
constexpr int kGJP = kGJ + 1;  // padded shared-memory row

// sc[sd * n_max + a] = E_aa^{-1/2}; W = S E S in binary32.  Block x of grid x rows.
__global__ void k_gj_scale(const int32_t* __restrict__ nca, const int64_t* __restrict__ eoff,
                           const double* __restrict__ E, int n_max, float* __restrict__ W,
                           double* __restrict__ sc, int* bad) {
  const int sd = blockIdx.y, n = nca[sd];
  if (n <= 0) return;
  const double* Eb = E + eoff[sd];
  float* Wb = W + eoff[sd];
  double* s = sc + (int64_t)sd * n_max;
  for (int a = blockIdx.x; a < n; a += gridDim.x) {
    const double da = Eb[(int64_t)a * n + a];
    if (!(da > 0.0)) {
      if (threadIdx.x == 0) atomicAdd(bad, 1);
      continue;
    }
    const double sa = 1.0 / sqrt(da);
    if (threadIdx.x == 0) s[a] = sa;
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
      const double db = Eb[(int64_t)b * n + b];
      const double sb = db > 0.0 ? 1.0 / sqrt(db) : 0.0;
      Wb[(int64_t)a * n + b] = (float)(Eb[(int64_t)a * n + b] * sa * sb);
    }
  }
}

// P = W_KK^{-1} (unblocked Gauss-Jordan in binary64 on the kb x kb pivot block)
__global__ void __launch_bounds__(256)
    k_gj_diag(const int32_t* __restrict__ nca, const int64_t* __restrict__ eoff, int k0,
              const float* __restrict__ W, float* __restrict__ P, int* bad) {
  const int sd = blockIdx.x, n = nca[sd];
  const int kb = min(kGJ, n - k0);
  if (kb <= 0) return;
  __shared__ double a[kGJ][kGJP];
  __shared__ double colk[kGJ], rowk[kGJ];
  __shared__ int fail;
  const int tid = threadIdx.x, nth = blockDim.x;
  const float* Wb = W + eoff[sd];
  if (tid == 0) fail = 0;
  for (int idx = tid; idx < kb * kb; idx += nth) {
    const int i = idx / kb, j = idx - i * kb;
    a[i][j] = Wb[(int64_t)(k0 + i) * n + k0 + j];
  }
  __syncthreads();
  for (int k = 0; k < kb; ++k) {
    for (int i = tid; i < kb; i += nth) {
      colk[i] = a[i][k];
      rowk[i] = a[k][i];
    }
    __syncthreads();
    double d = colk[k];
    if (!(d > 0.0)) {
      if (tid == 0) fail = 1;
      d = 1.0;
    }
    const double p = 1.0 / d;
    for (int idx = tid; idx < kb * kb; idx += nth) {
      const int i = idx / kb, j = idx - i * kb;
      double v;
      if (i == k)
        v = (j == k) ? p : rowk[j] * p;
      else
        v = (j == k) ? -colk[i] * p : a[i][j] - colk[i] * p * rowk[j];
      a[i][j] = v;
    }
    __syncthreads();
  }
  float* Pb = P + (int64_t)sd * kGJ * kGJ;
  for (int idx = tid; idx < kb * kb; idx += nth) {
    const int i = idx / kb, j = idx - i * kb;
    Pb[i * kGJ + j] = (float)a[i][j];
  }
  if (tid == 0 && fail) atomicAdd(bad, 1);
}

// acc[4][4] += As[ty*4 + i][q] * Bs[q][tx*4 + j], q < kb (256 threads: tx = tid % 16,
// ty = tid / 16, a 64 x 64 output tile)
__device__ __forceinline__ void gj_tile_mm(const float (*As)[kGJP], const float (*Bs)[kGJP],
                                           int kb, int ty, int tx, float (&acc)[4][4]) {
  for (int q = 0; q < kb; ++q) {
    float x[4], y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = As[ty * 4 + i][q];
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = Bs[q][tx * 4 + j];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] += x[i] * y[j];
  }
}

// rows [r0, r0 + nr) x columns [c0, c0 + nc) of the n x n block Wb into S (zero-padded)
__device__ __forceinline__ void gj_load(const float* __restrict__ Wb, int n, int r0, int nr,
                                        int c0, int nc, float (*S)[kGJP]) {
  for (int idx = threadIdx.x; idx < kGJ * kGJ; idx += blockDim.x) {
    const int i = idx / kGJ, j = idx - i * kGJ;
    S[i][j] = (i < nr && j < nc) ? Wb[(int64_t)(r0 + i) * n + c0 + j] : 0.0f;
  }
}

// W_KJ <- P W_KJ for the column tiles J != K
__global__ void __launch_bounds__(256)
    k_gj_row(const int32_t* __restrict__ nca, const int64_t* __restrict__ eoff, int k0,
             const float* __restrict__ P, float* __restrict__ W) {
  const int sd = blockIdx.y, n = nca[sd];
  const int kb = min(kGJ, n - k0), j0 = blockIdx.x * kGJ;
  if (kb <= 0 || j0 >= n || j0 == k0) return;
  const int nc = min(kGJ, n - j0);
  __shared__ float As[kGJ][kGJP], Bs[kGJ][kGJP];
  float* Wb = W + eoff[sd];
  const float* Pb = P + (int64_t)sd * kGJ * kGJ;
  for (int idx = threadIdx.x; idx < kGJ * kGJ; idx += blockDim.x) {
    const int i = idx / kGJ, j = idx - i * kGJ;
    As[i][j] = (i < kb && j < kb) ? Pb[i * kGJ + j] : 0.0f;
  }
  gj_load(Wb, n, k0, kb, j0, nc, Bs);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  gj_tile_mm(As, Bs, kb, ty, tx, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty * 4 + i, c = tx * 4 + j;
      if (r < kb && c < nc) Wb[(int64_t)(k0 + r) * n + j0 + c] = acc[i][j];
    }
}

// W_IJ <- W_IJ - W_IK W_KJ for the tiles I, J != K
__global__ void __launch_bounds__(256)
    k_gj_update(const int32_t* __restrict__ nca, const int64_t* __restrict__ eoff, int k0,
                int tiles, float* __restrict__ W) {
  const int sd = blockIdx.y, n = nca[sd];
  const int kb = min(kGJ, n - k0);
  const int i0 = (blockIdx.x / tiles) * kGJ, j0 = (blockIdx.x % tiles) * kGJ;
  if (kb <= 0 || i0 >= n || j0 >= n || i0 == k0 || j0 == k0) return;
  const int nr = min(kGJ, n - i0), nc = min(kGJ, n - j0);
  __shared__ float As[kGJ][kGJP], Bs[kGJ][kGJP];
  float* Wb = W + eoff[sd];
  gj_load(Wb, n, i0, nr, k0, kb, As);
  gj_load(Wb, n, k0, kb, j0, nc, Bs);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  gj_tile_mm(As, Bs, kb, ty, tx, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty * 4 + i, c = tx * 4 + j;
      if (r < nr && c < nc) Wb[(int64_t)(i0 + r) * n + j0 + c] -= acc[i][j];
    }
}

// W_IK <- -W_IK P for the row tiles I != K; W_KK <- P
__global__ void __launch_bounds__(256)
    k_gj_col(const int32_t* __restrict__ nca, const int64_t* __restrict__ eoff, int k0,
             const float* __restrict__ P, float* __restrict__ W) {
  const int sd = blockIdx.y, n = nca[sd];
  const int kb = min(kGJ, n - k0), i0 = blockIdx.x * kGJ;
  if (kb <= 0 || i0 >= n) return;
  float* Wb = W + eoff[sd];
  const float* Pb = P + (int64_t)sd * kGJ * kGJ;
  if (i0 == k0) {
    for (int idx = threadIdx.x; idx < kb * kb; idx += blockDim.x) {
      const int i = idx / kb, j = idx - i * kb;
      Wb[(int64_t)(k0 + i) * n + k0 + j] = Pb[i * kGJ + j];
    }
    return;
  }
  const int nr = min(kGJ, n - i0);
  __shared__ float As[kGJ][kGJP], Bs[kGJ][kGJP];
  gj_load(Wb, n, i0, nr, k0, kb, As);
  for (int idx = threadIdx.x; idx < kGJ * kGJ; idx += blockDim.x) {
    const int i = idx / kGJ, j = idx - i * kGJ;
    Bs[i][j] = (i < kb && j < kb) ? Pb[i * kGJ + j] : 0.0f;
  }
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  float acc[4][4] = {};
  gj_tile_mm(As, Bs, kb, ty, tx, acc);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty * 4 + i, c = tx * 4 + j;
      if (r < nr && c < kb) Wb[(int64_t)(i0 + r) * n + k0 + c] = -acc[i][j];
    }
}

// einv = S (W + W^T) / 2 S in T
template <typename T>
__global__ void k_gj_out(const int32_t* __restrict__ nca, const int64_t* __restrict__ eoff,
                         const float* __restrict__ W, const double* __restrict__ sc, int n_max,
                         T* __restrict__ einv) {
  const int sd = blockIdx.y, n = nca[sd];
  if (n <= 0) return;
  const float* Wb = W + eoff[sd];
  const double* s = sc + (int64_t)sd * n_max;
  T* out = einv + eoff[sd];
  for (int a = blockIdx.x; a < n; a += gridDim.x)
    for (int b = threadIdx.x; b < n; b += blockDim.x) {
      const double w = 0.5 * ((double)Wb[(int64_t)a * n + b] + (double)Wb[(int64_t)b * n + a]);
      out[(int64_t)a * n + b] = (T)(w * (s[a] * s[b]));  // exactly symmetric
    }
}

// the tensor-core operand blocks of E^{-1} (see launch_coarse_tc_pack): one block of
// 256 threads per (subdomain, 128 x 32 block)
__global__ void k_coarse_tc_pack(const int32_t* __restrict__ nca,
                                 const int64_t* __restrict__ eoff,
                                 const float* __restrict__ einv,
                                 const int64_t* __restrict__ etc_off, uint4* out) {
  const int sd = blockIdx.y, n = nca[sd];
  const int nkb = (n + tc::kKB - 1) / tc::kKB;
  const int mt = (n + kCoarseTcM - 1) / kCoarseTcM;
  const int blk = blockIdx.x;
  if (n <= 0 || blk >= mt * nkb) return;
  const int m = blk / nkb, kb = blk - m * nkb;
  const float* E = einv + eoff[sd];
  // 16 KB per block: two planes of 128 x 32 bf16
  __nv_bfloat16* hi = reinterpret_cast<__nv_bfloat16*>(out + (etc_off[sd] + blk) * 1024);
  __nv_bfloat16* lo = hi + kCoarseTcM * tc::kKB;
  for (int idx = threadIdx.x; idx < kCoarseTcM * tc::kKB; idx += blockDim.x) {
    const int r = idx / tc::kKB, k = idx - r * tc::kKB;
    const int a = m * kCoarseTcM + r, b = kb * tc::kKB + k;
    const float v = (a < n && b < n) ? E[(int64_t)a * n + b] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const uint32_t o = tc::kmajor(r, k) >> 1;
    hi[o] = h;
    lo[o] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

}  // namespace

void launch_coarse_tc_pack(int n_sd, int blocks_max, const int32_t* nca, const int64_t* eoff,
                           const float* einv, const int64_t* etc_off, uint4* out,
                           cudaStream_t st) {
  if (n_sd <= 0 || blocks_max <= 0) return;
  count_launch();
  k_coarse_tc_pack<<<dim3(blocks_max, n_sd), 256, 0, st>>>(nca, eoff, einv, etc_off, out);
}

void launch_coarse_matrix(const DTiles& tiles, const EllView<double>& A, const int32_t* aloc,
                          const int32_t* nca, const int64_t* eoff, double* E, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_coarse_matrix<<<tiles.n, kTileRows, 0, st>>>(tiles, A, aloc, nca, eoff, E);
}

template <typename T>
void launch_coarse_invert(int n_sd, int n_max, const int32_t* nca, const int64_t* eoff,
                          const double* E, float* W, float* P, double* sc, T* einv, int* bad,
                          cudaStream_t st) {
  if (n_sd <= 0 || n_max <= 0) return;
  const int rows = std::min(n_max, 64);
  count_launch();
  k_gj_scale<<<dim3(rows, n_sd), 256, 0, st>>>(nca, eoff, E, n_max, W, sc, bad);
  const int tiles = (n_max + kGJ - 1) / kGJ;
  for (int k0 = 0; k0 < n_max; k0 += kGJ) {
    count_launch(4);
    k_gj_diag<<<n_sd, 256, 0, st>>>(nca, eoff, k0, W, P, bad);
    k_gj_row<<<dim3(tiles, n_sd), 256, 0, st>>>(nca, eoff, k0, P, W);
    k_gj_update<<<dim3(tiles * tiles, n_sd), 256, 0, st>>>(nca, eoff, k0, tiles, W);
    k_gj_col<<<dim3(tiles, n_sd), 256, 0, st>>>(nca, eoff, k0, P, W);
  }
  count_launch();
  k_gj_out<T><<<dim3(rows, n_sd), 256, 0, st>>>(nca, eoff, W, sc, n_max, einv);
}

template void launch_coarse_invert<float>(int, int, const int32_t*, const int64_t*,
                                          const double*, float*, float*, double*, float*, int*,
                                          cudaStream_t);
template void launch_coarse_invert<double>(int, int, const int32_t*, const int64_t*,
                                           const double*, float*, float*, double*, double*,
                                           int*, cudaStream_t);

}  // namespace mor
