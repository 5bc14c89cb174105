// Paper-literal weights on the GPU (Sec. 4, Lemma 4.1, Eq. (14)) for subdomains small
// enough for dense factors: batched dense Cholesky factorisations, triangular solves
// and the pieces of the explicit weighted SVD.
//
//   - k_ell_to_dense: scatter a sliced-ELL block into a dense per-subdomain matrix
//     (row-major, leading dimension = its order) with caller-given local indices;
//   - k_potrf_diag / k_potrf_update: right-looking blocked Cholesky A = L L^T in place,
//     64-column panels, batched over subdomains of different orders (Golub & Van Loan
//     Alg. 4.2.2 by blocks);
//   - k_transpose_block: copy of a square block, transposed (the triangular solves
//     walk columns of a factor as contiguous rows of its transpose);
//   - k_trsv_cols: one vector per block: forward (L x = b) or backward (U x = b)
//     substitution, column-oriented;
//   - k_trsv_rows: one row per warp: x R = y with R upper (row-major), for
//     X = Y R_BB^{-1};
//   - k_trmv_upper: y = U z per vector;
//   - k_node_normals: the Gaussian test matrix S of the paper's sketch on B.
// Everything is binary64.
#include "mor_dev.cuh"
#include "mor_kernels.h"

#include <algorithm>

namespace mor {
namespace {

constexpr int kNB = 64;  // Cholesky panel width and update tile

// D[doff[sd] + (rloc[r] - r_sub[sd]) * ld[sd] + (cloc[c] - c_sub[sd])] = A[r, c] for
// the stored entries of rows r in [0, n_rows) whose local row rloc[r] - r_sub[sd] lies
// in [0, r_n[sd]) and whose local column cloc[c] - c_sub[sd] lies in [0, ncols[sd]).
// sd = row_sd[r].
__global__ void k_ell_to_dense(int64_t n_rows, const int32_t* __restrict__ row_sd,
                               const int32_t* __restrict__ rloc,
                               const int32_t* __restrict__ cloc, EllView<double> A,
                               const int32_t* __restrict__ r_sub,
                               const int32_t* __restrict__ r_n,
                               const int32_t* __restrict__ c_sub,
                               const int32_t* __restrict__ ncols,
                               const int32_t* __restrict__ ld, const int64_t* __restrict__ doff,
                               double* __restrict__ D) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const int sd = row_sd[r];
  const int lr = rloc[r] - r_sub[sd];
  if (lr < 0 || lr >= r_n[sd]) return;
  const int w = A.width[r >> 5];
  const int64_t base = doff[sd] + (int64_t)lr * ld[sd];
  for (int j = 0; j < w; ++j) {
    const int64_t at = ell_at(r, j, A.W);
    const int c = A.col[at];
    if (c < 0) continue;
    const int lc = cloc[c] - c_sub[sd];
    if (lc < 0 || lc >= ncols[sd]) continue;
    D[base + lc] = A.val[at];
  }
}

// diagonal block j0 of every subdomain's matrix (order n[sd]) factored in shared
// memory, then the panel below it solved against it: rows i >= j0 + nb satisfy
// L[i, j0:j0+nb] L_dd^T = A[i, j0:j0+nb].  A non-positive pivot sets *bad.
__global__ void __launch_bounds__(256)
    k_potrf_diag(double* D, const int64_t* __restrict__ doff, const int32_t* __restrict__ nn,
                 int j0, int* bad) {
  __shared__ double a[kNB][kNB + 1];
  const int sd = blockIdx.x, n = nn[sd];
  if (j0 >= n) return;
  const int nb = min(kNB, n - j0);
  double* A = D + doff[sd];
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int idx = tid; idx < nb * nb; idx += nth) {
    const int r = idx / nb, c = idx % nb;
    a[r][c] = (c <= r) ? A[(int64_t)(j0 + r) * n + j0 + c] : 0.0;
  }
  __syncthreads();
  for (int c = 0; c < nb; ++c) {
    const double d2 = a[c][c];
    const double d = d2 > 0.0 ? sqrt(d2) : 1.0;
    if (!(d2 > 0.0) && tid == 0) atomicExch(bad, 1);
    __syncthreads();
    for (int r = c + 1 + tid; r < nb; r += nth) a[r][c] /= d;
    if (tid == 0) a[c][c] = d;
    __syncthreads();
    const int m = nb - c - 1;
    for (int idx = tid; idx < m * m; idx += nth) {
      const int r = c + 1 + idx / m, s = c + 1 + idx % m;
      if (s <= r) a[r][s] -= a[r][c] * a[s][c];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * nb; idx += nth) {
    const int r = idx / nb, c = idx % nb;
    A[(int64_t)(j0 + r) * n + j0 + c] = (c <= r) ? a[r][c] : 0.0;
  }
  // panel: forward substitution of each row against L_dd^T
  for (int i = j0 + nb + tid; i < n; i += nth) {
    double* row = A + (int64_t)i * n + j0;
    for (int c = 0; c < nb; ++c) {
      double s = row[c];
      for (int q = 0; q < c; ++q) s -= row[q] * a[c][q];
      row[c] = s / a[c][c];
    }
  }
}

// trailing update of panel j0: A[I, J] -= P_I P_J^T for the 64 x 64 tiles I >= J of the
// rows and columns after the panel (P = the panel's columns); grid (n_sd, tiles)
__global__ void __launch_bounds__(256)
    k_potrf_update(double* D, const int64_t* __restrict__ doff, const int32_t* __restrict__ nn,
                   int j0) {
  extern __shared__ double sm[];
  double* PI = sm;                        // kNB x (kNB + 1)
  double* PJ = sm + kNB * (kNB + 1);
  const int sd = blockIdx.x, n = nn[sd];
  const int t0 = j0 + kNB;
  if (t0 >= n) return;
  const int T = (n - t0 + kNB - 1) / kNB;
  // tile index -> (I, J), I >= J, row-major over the lower triangle of tiles
  const int t = blockIdx.y;
  int I = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  while (I * (I + 1) / 2 > t) --I;
  const int J = t - I * (I + 1) / 2;
  if (I >= T) return;
  double* A = D + doff[sd];
  const int i0 = t0 + I * kNB, c0 = t0 + J * kNB;
  const int tid = threadIdx.y * 16 + threadIdx.x;
  for (int idx = tid; idx < kNB * kNB; idx += 256) {
    const int r = idx / kNB, q = idx % kNB;
    PI[r * (kNB + 1) + q] = (i0 + r < n) ? A[(int64_t)(i0 + r) * n + j0 + q] : 0.0;
    PJ[r * (kNB + 1) + q] = (c0 + r < n) ? A[(int64_t)(c0 + r) * n + j0 + q] : 0.0;
  }
  __syncthreads();
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  const int ty = threadIdx.y, tx = threadIdx.x;
  for (int q = 0; q < kNB; ++q) {
    double xa[4], yb[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) xa[a] = PI[(ty * 4 + a) * (kNB + 1) + q];
#pragma unroll
    for (int b = 0; b < 4; ++b) yb[b] = PJ[(tx * 4 + b) * (kNB + 1) + q];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] += xa[a] * yb[b];
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int r = i0 + ty * 4 + a;
    if (r >= n) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int c = c0 + tx * 4 + b;
      if (c < n && c <= r) A[(int64_t)r * n + c] -= acc[a][b];
    }
  }
}

// Out_sd[r, c] = In_sd[c + s0, r + s0] for r, c < m[sd] (the block starting at (s0, s0)
// with s0 = soff[sd] of an order-n[sd] matrix), lower triangle only of In (upper part
// of the output zero for a lower In block)
__global__ void k_transpose_block(const double* __restrict__ In, const int64_t* __restrict__ ioff,
                                  const int32_t* __restrict__ nn, const int32_t* __restrict__ soff,
                                  const int32_t* __restrict__ mm, double* __restrict__ Out,
                                  const int64_t* __restrict__ ooff, int transpose) {
  const int sd = blockIdx.y, n = nn[sd], s0 = soff[sd], m = mm[sd];
  const double* A = In + ioff[sd];
  double* B = Out + ooff[sd];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)m * m;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / m), c = (int)(idx % m);
    // the lower-triangular source entry (i, j), i >= j
    const int i = transpose ? c : r, j = transpose ? r : c;
    B[idx] = (i >= j) ? A[(int64_t)(i + s0) * n + j + s0] : 0.0;
  }
}

// one vector per block: x = F^{-1} b with F triangular of order n[sd], given through T
// whose row j is column j of F (contiguous).  forward (F lower): x_j = b_j / F_jj, then
// b_l -= F_lj x_j for l > j; backward (F upper): the same for l < j from the last row.
// The vector is column `col` of rows [roff[sd], roff[sd] + n) of X (leading dimension
// ldx), solved in place.  grid (n_sd, columns).
__global__ void __launch_bounds__(256)
    k_trsv_cols(const double* __restrict__ Tm, const int64_t* __restrict__ toff,
                const int32_t* __restrict__ nn, const int32_t* __restrict__ tld,
                const int32_t* __restrict__ tsh, double* X, const int64_t* __restrict__ roff,
                int ldx, const int32_t* __restrict__ ncol, int forward) {
  extern __shared__ double b[];
  const int sd = blockIdx.x, col = blockIdx.y;
  if (col >= ncol[sd]) return;
  const int n = nn[sd], ld = tld[sd], sh = tsh[sd];
  const double* T = Tm + toff[sd] + (int64_t)sh * ld + sh;
  double* x = X + roff[sd] * ldx + col;
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = x[(int64_t)i * ldx];
  __syncthreads();
  for (int s = 0; s < n; ++s) {
    const int j = forward ? s : n - 1 - s;
    const double* tj = T + (int64_t)j * ld;
    const double xj = b[j] / tj[j];
    if (forward) {
      for (int l = j + 1 + threadIdx.x; l < n; l += blockDim.x) b[l] -= tj[l] * xj;
    } else {
      for (int l = threadIdx.x; l < j; l += blockDim.x) b[l] -= tj[l] * xj;
    }
    __syncthreads();
    if (threadIdx.x == 0) b[j] = xj;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[(int64_t)i * ldx] = b[i];
}

// one row per warp: the row y (length m[sd]) of X (rows [roff[sd], roff[sd] + rows[sd]),
// leading dimension ldx) becomes x with x R = y, R upper of order m given row-major
// (x_j = (y_j - sum_{l<j} x_l R_lj) / R_jj, column-oriented over the rows of R:
// x_j = y_j / R_jj, then y_l -= R_jl x_j for l > j)
__global__ void __launch_bounds__(256)
    k_trsv_rows(const double* __restrict__ R, const int64_t* __restrict__ roff_r,
                const int32_t* __restrict__ mm, double* X, const int64_t* __restrict__ roff,
                int ldx, const int* __restrict__ sd_of_warp, const int* __restrict__ row_of_warp,
                int n_warps) {
  extern __shared__ double ysh[];
  const int w = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (w >= n_warps) return;
  const int sd = sd_of_warp[w], row = row_of_warp[w];
  const int m = mm[sd];
  double* y = ysh + (threadIdx.x / 32) * ldx;
  double* xr = X + (roff[sd] + row) * (int64_t)ldx;
  const double* Rm = R + roff_r[sd];
  for (int l = lane; l < m; l += 32) y[l] = xr[l];
  __syncwarp();
  for (int j = 0; j < m; ++j) {
    const double* rj = Rm + (int64_t)j * m;
    const double xj = y[j] / rj[j];
    for (int l = j + 1 + lane; l < m; l += 32) y[l] -= rj[l] * xj;
    __syncwarp();
    if (lane == 0) y[j] = xj;
    __syncwarp();
  }
  for (int l = lane; l < m; l += 32) xr[l] = y[l];
}

// y = U z per vector, U upper of order n[sd] (row-major): y_a = sum_{b >= a} U_ab z_b;
// z = column `col` of rows [roff[sd], +n) of Z, y into the same place of Y
__global__ void __launch_bounds__(256)
    k_trmv_upper(const double* __restrict__ U, const int64_t* __restrict__ uoff,
                 const int32_t* __restrict__ nn, const double* __restrict__ Z, double* Y,
                 const int64_t* __restrict__ roff, int ld, const int32_t* __restrict__ ncol) {
  extern __shared__ double z[];
  const int sd = blockIdx.x, col = blockIdx.y;
  if (col >= ncol[sd]) return;
  const int n = nn[sd];
  const double* Us = U + uoff[sd];
  for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] = Z[(roff[sd] + i) * ld + col];
  __syncthreads();
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const double* ua = Us + (int64_t)a * n;
    double s = 0.0;
    for (int b2 = a; b2 < n; ++b2) s += ua[b2] * z[b2];
    Y[(roff[sd] + a) * ld + col] = s;
  }
}

// S[b, j] of the paper's sketch for the B rows in ascending node order: the first
// normal of Philox(counter (node, j, sd, 1), key = seed); rows [boff[sd], +m[sd]) of
// out (leading dimension ld), columns j < kk[sd]
__global__ void k_node_normals(int n_sd, const int32_t* __restrict__ bnode,
                               const int64_t* __restrict__ boff, const int32_t* __restrict__ mm,
                               const int32_t* __restrict__ kk, int k, uint64_t seed,
                               uint32_t sd_base, double* __restrict__ out, int ld) {
  const int sd = blockIdx.y;
  const int m = mm[sd];
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)m * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(idx / k), j = (int)(idx % k);
    double v = 0.0;
    if (j < kk[sd]) {
      uint32_t c[4] = {(uint32_t)bnode[boff[sd] + r], (uint32_t)j, (uint32_t)sd + sd_base, 1u};
      philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
      float z0, z1;
      box_muller(c[0], c[1], z0, z1);
      v = (double)z0;
    }
    out[(boff[sd] + r) * ld + j] = v;
  }
}

}  // namespace

void launch_ell_to_dense(int64_t n_rows, const int32_t* row_sd, const int32_t* rloc,
                         const int32_t* cloc, const EllView<double>& A, const int32_t* r_sub,
                         const int32_t* r_n, const int32_t* c_sub, const int32_t* ncols,
                         const int32_t* ld, const int64_t* doff, double* D, cudaStream_t st) {
  if (n_rows <= 0) return;
  count_launch();
  k_ell_to_dense<<<(unsigned)((n_rows + 255) / 256), 256, 0, st>>>(
      n_rows, row_sd, rloc, cloc, A, r_sub, r_n, c_sub, ncols, ld, doff, D);
}

void launch_potrf(int n_sd, int n_max, double* D, const int64_t* doff, const int32_t* nn,
                  int* bad, cudaStream_t st) {
  if (n_sd <= 0) return;
  static bool attr = false;
  const size_t sm = sizeof(double) * 2 * kNB * (kNB + 1);
  if (!attr) {
    cudaFuncSetAttribute(k_potrf_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    attr = true;
  }
  for (int j0 = 0; j0 < n_max; j0 += kNB) {
    count_launch();
    k_potrf_diag<<<n_sd, 256, 0, st>>>(D, doff, nn, j0, bad);
    const int T = (n_max - j0 - kNB + kNB - 1) / kNB;
    if (T > 0) {
      count_launch();
      k_potrf_update<<<dim3(n_sd, T * (T + 1) / 2), dim3(16, 16), sm, st>>>(D, doff, nn, j0);
    }
  }
}

void launch_transpose_block(int n_sd, int m_max, const double* In, const int64_t* ioff,
                            const int32_t* nn, const int32_t* soff, const int32_t* mm,
                            double* Out, const int64_t* ooff, int transpose, cudaStream_t st) {
  if (n_sd <= 0 || m_max <= 0) return;
  count_launch();
  const int64_t n = (int64_t)m_max * m_max;
  const unsigned bx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  k_transpose_block<<<dim3(bx, n_sd), 256, 0, st>>>(In, ioff, nn, soff, mm, Out, ooff,
                                                    transpose);
}

void launch_trsv_cols(int n_sd, int n_max, int ncol_max, const double* T, const int64_t* toff,
                      const int32_t* nn, const int32_t* tld, const int32_t* tsh, double* X,
                      const int64_t* roff, int ldx, const int32_t* ncol, int forward,
                      cudaStream_t st) {
  if (n_sd <= 0 || ncol_max <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_trsv_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launch();
  k_trsv_cols<<<dim3(n_sd, ncol_max), 256, sizeof(double) * n_max, st>>>(
      T, toff, nn, tld, tsh, X, roff, ldx, ncol, forward);
}

void launch_trsv_rows(const double* R, const int64_t* roff_r, const int32_t* mm, double* X,
                      const int64_t* roff, int ldx, const int* sd_of_warp,
                      const int* row_of_warp, int n_warps, cudaStream_t st) {
  if (n_warps <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_trsv_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launch();
  const int wpb = 8;
  k_trsv_rows<<<(n_warps + wpb - 1) / wpb, 32 * wpb, sizeof(double) * wpb * ldx, st>>>(
      R, roff_r, mm, X, roff, ldx, sd_of_warp, row_of_warp, n_warps);
}

void launch_trmv_upper(int n_sd, int n_max, int ncol_max, const double* U, const int64_t* uoff,
                       const int32_t* nn, const double* Z, double* Y, const int64_t* roff,
                       int ld, const int32_t* ncol, cudaStream_t st) {
  if (n_sd <= 0 || ncol_max <= 0) return;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_trmv_upper, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launch();
  k_trmv_upper<<<dim3(n_sd, ncol_max), 256, sizeof(double) * n_max, st>>>(U, uoff, nn, Z, Y,
                                                                          roff, ld, ncol);
}

void launch_node_normals(int n_sd, int m_max, const int32_t* bnode, const int64_t* boff,
                         const int32_t* mm, const int32_t* kk, int k, uint64_t seed,
                         uint32_t sd_base, double* out, int ld, cudaStream_t st) {
  if (n_sd <= 0 || m_max <= 0 || k <= 0) return;
  count_launch();
  const int64_t n = (int64_t)m_max * k;
  const unsigned bx = (unsigned)std::min<int64_t>((n + 255) / 256, 1024);
  k_node_normals<<<dim3(bx, n_sd), 256, 0, st>>>(n_sd, bnode, boff, mm, kk, k, seed, sd_base,
                                                 out, ld);
}

}  // namespace mor
