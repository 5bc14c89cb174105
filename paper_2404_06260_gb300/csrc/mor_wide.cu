// Dense per-subdomain linear algebra of step 2 for wide sketches (k up to 511 columns,
// the k_i = floor(M_i / 8) sketch size of Sec. 7.1 and App. C) and for the |B| x |B|
// Gram of the explicit SVD (|B| up to 1024), where the small shared-memory kernels of
// mor_dense.cu do not fit:
//   - tall-skinny Grams X^T Y over the rows of each subdomain, 64 x 64 output tiles,
//     split over row chunks and reduced in chunk order (deterministic);
//   - the symmetric eigensolver: the same threshold cyclic Jacobi as the small kernel
//     (round-robin ordering, Golub & Van Loan Alg. 8.4.1 rotations, Demmel-Veselic
//     threshold) with the matrix and the eigenvectors in global memory, one block of
//     1024 threads per subdomain;
//   - row-block products X M_sd in 128-row x 64-column output tiles.
// Everything is binary64.
#include "mor_kernels.h"

namespace mor {
namespace {

constexpr int kWT = 64;      // output tile of the Gram and of the row product
constexpr int kWRows = 16;   // rows staged per step of the Gram

// part[(sd * S + s)][i * ny + j] = sum over the rows of chunk s of subdomain sd of
// X[r, i] Y[r, j]; block (16, 16), each thread a 4 x 4 patch of the 64 x 64 tile
__global__ void __launch_bounds__(256)
    k_gram_wide(DTiles tl, int S, const double* __restrict__ X, int ldx, int nx,
                const double* __restrict__ Y, int ldy, int ny, double* __restrict__ part) {
  __shared__ double Xs[kWRows][kWT + 1];
  __shared__ double Ys[kWRows][kWT + 1];
  const int sd = blockIdx.x / S, s = blockIdx.x % S;
  const int ntj = (ny + kWT - 1) / kWT;
  const int i0 = (blockIdx.y / ntj) * kWT, j0 = (blockIdx.y % ntj) * kWT;
  const int lo = tl.lo[sd], hi = tl.hi[sd];
  const int nt = hi - lo;
  const int t0 = lo + (int)((int64_t)nt * s / S), t1 = lo + (int)((int64_t)nt * (s + 1) / S);
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  for (int t = t0; t < t1; ++t) {
    const int r0 = tl.r0[t], r1 = tl.r1[t];
    for (int base = r0; base < r1; base += kWRows) {
      const int nr = min(kWRows, r1 - base);
      for (int idx = tid; idx < kWRows * kWT; idx += 256) {
        const int rr = idx / kWT, c = idx % kWT;
        const bool in = rr < nr;
        Xs[rr][c] = (in && i0 + c < nx) ? X[(int64_t)(base + rr) * ldx + i0 + c] : 0.0;
        Ys[rr][c] = (in && j0 + c < ny) ? Y[(int64_t)(base + rr) * ldy + j0 + c] : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int rr = 0; rr < kWRows; ++rr) {
        double xa[4], yb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = Xs[rr][ty * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) yb[b] = Ys[rr][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += xa[a] * yb[b];
      }
      __syncthreads();
    }
  }
  double* P = part + (int64_t)(sd * S + s) * nx * ny;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty * 4 + a, j = j0 + tx * 4 + b;
      if (i < nx && j < ny) P[(int64_t)i * ny + j] = acc[a][b];
    }
}

// G[sd][i * ldg + j] = sum over s of part[(sd * S + s)][i * ny + j], s in order
__global__ void k_gram_wide_reduce(int S, int nx, int ny, const double* __restrict__ part,
                                   double* __restrict__ G, int ldg, int64_t sd_stride) {
  const int sd = blockIdx.y;
  const int64_t n = (int64_t)nx * ny;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n;
       o += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += part[(int64_t)(sd * S + s) * n + o];
    const int i = (int)(o / ny), j = (int)(o % ny);
    G[(int64_t)sd * sd_stride + (int64_t)i * ldg + j] = acc;
  }
}

// threshold cyclic Jacobi of the symmetric part of A_sd (n x n, leading dimension ld),
// a and v are m x m work arrays per subdomain (m = n rounded up to even, n <= 1024).
// evals descending, evecs[r * ld + rank] the matching eigenvectors, zero beyond n.
constexpr int kEigThreads = 1024;
__global__ void __launch_bounds__(kEigThreads)
    k_sym_eig_wide(const double* __restrict__ A, int ld, int n, double* evals, double* evecs,
                   double* work) {
  __shared__ double rc[512], rs[512];
  __shared__ int rp[512], rq[512];
  __shared__ int nrot;
  const int m = n + (n & 1);
  const int sd = blockIdx.x, tid = threadIdx.x, nth = blockDim.x;
  double* a = work + (int64_t)sd * 2 * m * m;
  double* v = a + (int64_t)m * m;
  const double* As = A + (int64_t)sd * ld * ld;
  for (int idx = tid; idx < m * m; idx += nth) {
    const int i = idx / m, j = idx % m;
    a[idx] = (i < n && j < n) ? 0.5 * (As[i * ld + j] + As[j * ld + i]) : 0.0;
    v[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      for (int k = tid; k < m / 2; k += nth) {
        const int x0 = k, x1 = m - 1 - k;
        const int p = (x0 == 0) ? 0 : ((x0 - 1 + round) % (m - 1)) + 1;
        const int q = ((x1 - 1 + round) % (m - 1)) + 1;
        const double apq = a[(int64_t)p * m + q];
        const double app = a[(int64_t)p * m + p], aqq = a[(int64_t)q * m + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 0x1p-52 * sqrt(fabs(app * aqq))) {
          atomicAdd(&nrot, 1);
          const double tau = (aqq - app) / (2.0 * apq);
          double t;
          if (fabs(tau) > 1e150)
            t = 0.5 / tau;
          else
            t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          s = t * c;
        }
        rp[k] = p;
        rq[k] = q;
        rc[k] = c;
        rs[k] = s;
      }
      __syncthreads();
      // rows p, q of A: A <- J^T A
      for (int w = tid; w < (m / 2) * m; w += nth) {
        const int k = w / m, j = w % m;
        const double c = rc[k], s = rs[k];
        if (s == 0.0) continue;
        const int64_t p = rp[k], q = rq[k];
        const double ap = a[p * m + j], aq = a[q * m + j];
        a[p * m + j] = c * ap - s * aq;
        a[q * m + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q of A and V: A <- A J, V <- V J
      for (int w = tid; w < (m / 2) * m; w += nth) {
        const int k = w % (m / 2), i = w / (m / 2);
        const double c = rc[k], s = rs[k];
        if (s == 0.0) continue;
        const int p = rp[k], q = rq[k];
        const int64_t ri = (int64_t)i * m;
        const double ap = a[ri + p], aq = a[ri + q];
        a[ri + p] = c * ap - s * aq;
        a[ri + q] = s * ap + c * aq;
        const double vp = v[ri + p], vq = v[ri + q];
        v[ri + p] = c * vp - s * vq;
        v[ri + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    const int rotated = nrot;
    __syncthreads();
    if (rotated == 0) break;
  }
  double* ev = evals + (int64_t)sd * ld;
  double* V = evecs + (int64_t)sd * ld * ld;
  for (int64_t idx = tid; idx < (int64_t)ld * ld; idx += nth) V[idx] = 0.0;
  for (int i = tid; i < ld; i += nth)
    if (i >= n) ev[i] = 0.0;
  __syncthreads();
  for (int i = tid; i < n; i += nth) {
    const double li = a[(int64_t)i * m + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double lj = a[(int64_t)j * m + j];
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    ev[rank] = li;
    for (int r = 0; r < n; ++r) V[(int64_t)r * ld + rank] = v[(int64_t)r * m + i];
  }
}

// Y[row, j] = sum_l X[row, l] M_sd[l, j] for j < nout, 0 for nout <= j < ldy; block
// (16, 16) over a 128-row x 64-column output tile (each thread 8 rows x 4 columns)
constexpr int kRMRows = 128, kRMK = 16;
__global__ void __launch_bounds__(256)
    k_rowmul_wide(DTiles tl, const double* __restrict__ X, int ldx, int nin,
                  const double* __restrict__ M, int ldm, double* __restrict__ Y, int ldy,
                  int nout) {
  __shared__ double Xs[kRMRows][kRMK + 1];
  __shared__ double Ms[kRMK][kWT + 1];
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int r0 = tl.r0[tile], r1 = tl.r1[tile];
  const int nr = r1 - r0;
  const int j0 = blockIdx.y * kWT;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 16 + tx;
  const double* Msd = M + (int64_t)sd * ldm * ldm;
  double acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  if (j0 < nout) {
    for (int l0 = 0; l0 < nin; l0 += kRMK) {
      for (int idx = tid; idx < kRMRows * kRMK; idx += 256) {
        const int rr = idx / kRMK, l = idx % kRMK;
        Xs[rr][l] = (rr < nr && l0 + l < nin) ? X[(int64_t)(r0 + rr) * ldx + l0 + l] : 0.0;
      }
      for (int idx = tid; idx < kRMK * kWT; idx += 256) {
        const int l = idx / kWT, c = idx % kWT;
        Ms[l][c] = (l0 + l < nin && j0 + c < nout) ? Msd[(int64_t)(l0 + l) * ldm + j0 + c]
                                                   : 0.0;
      }
      __syncthreads();
#pragma unroll 4
      for (int l = 0; l < kRMK; ++l) {
        double mb[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) mb[b] = Ms[l][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          const double xv = Xs[ty * 8 + a][l];
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] += xv * mb[b];
        }
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int rr = ty * 8 + a;
    if (rr >= nr) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int j = j0 + tx * 4 + b;
      if (j < ldy) Y[(int64_t)(r0 + rr) * ldy + j] = (j < nout) ? acc[a][b] : 0.0;
    }
  }
}

}  // namespace

int gram_wide_chunks(int n_sd, int nx, int ny) {
  const int tiles = ((nx + kWT - 1) / kWT) * ((ny + kWT - 1) / kWT);
  int S = (4 * 152 + n_sd * tiles - 1) / (n_sd * tiles);
  return S < 1 ? 1 : (S > 16 ? 16 : S);
}

void launch_gram_wide(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                      const double* Y, int ldy, int ny, double* part, double* G, int ldg,
                      int64_t sd_stride, cudaStream_t st) {
  if (tiles.n <= 0 || n_sd <= 0) return;
  const int S = gram_wide_chunks(n_sd, nx, ny);
  const int nt = ((nx + kWT - 1) / kWT) * ((ny + kWT - 1) / kWT);
  count_launch(2);
  k_gram_wide<<<dim3(n_sd * S, nt), dim3(16, 16), 0, st>>>(tiles, S, X, ldx, nx, Y, ldy, ny,
                                                          part);
  const int64_t n = (int64_t)nx * ny;
  const int bx = (int)((n + 255) / 256 < 64 ? (n + 255) / 256 : 64);
  k_gram_wide_reduce<<<dim3(bx, n_sd), 256, 0, st>>>(S, nx, ny, part, G, ldg, sd_stride);
}

void launch_sym_eig_wide(int n_sd, const double* A, int ld, int n, double* evals,
                         double* evecs, double* work, cudaStream_t st) {
  if (n_sd <= 0) return;
  count_launch();
  k_sym_eig_wide<<<n_sd, kEigThreads, 0, st>>>(A, ld, n, evals, evecs, work);
}

void launch_rowmul_wide(const DTiles& tiles, const double* X, int ldx, int nin,
                        const double* M, int ldm, double* Y, int ldy, int nout,
                        cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_rowmul_wide<<<dim3(tiles.n, (ldy + kWT - 1) / kWT), dim3(16, 16), 0, st>>>(
      tiles, X, ldx, nin, M, ldm, Y, ldy, nout);
}

}  // namespace mor
