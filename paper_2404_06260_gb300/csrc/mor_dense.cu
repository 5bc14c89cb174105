// Small dense per-subdomain linear algebra of step 2 (Sec. 4, Sec. 6): tall-skinny
// Grams X^T Y, the symmetric eigensolver used for the H_i-orthonormalisation, the
// singular values of the projected operator (Eq. (24)) and the diagonal-block update,
// and the k x k right-multiplications that apply their results to row blocks.
#include "mor_kernels.h"

namespace mor {
namespace {

constexpr int kGramThreads = 512;
constexpr int kGramPerThread = 13;  // 512 * 13 >= 80 * 80 outputs
constexpr int kGramRows = 32;

// partial Gram of one row tile, then the last tile of the subdomain reduces the
// partials in tile order (deterministic)
__global__ void __launch_bounds__(kGramThreads)
    k_gram(DTiles tl, const double* __restrict__ X, int ldx, int nx,
           const double* __restrict__ Y, int ldy, int ny, double* part, int* counter,
           double* G, int ldg, int sd_stride) {
  extern __shared__ double sh[];
  double* Xs = sh;
  double* Ys = sh + kGramRows * nx;
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  int tid = threadIdx.x, nth = blockDim.x;
  int nout = nx * ny;
  double acc[kGramPerThread];
#pragma unroll
  for (int m = 0; m < kGramPerThread; ++m) acc[m] = 0.0;
  for (int base = r0; base < r1; base += kGramRows) {
    int nr = min(kGramRows, r1 - base);
    for (int idx = tid; idx < nr * nx; idx += nth) {
      int rr = idx / nx, c = idx % nx;
      Xs[rr * nx + c] = X[(int64_t)(base + rr) * ldx + c];
    }
    for (int idx = tid; idx < nr * ny; idx += nth) {
      int rr = idx / ny, c = idx % ny;
      Ys[rr * ny + c] = Y[(int64_t)(base + rr) * ldy + c];
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kGramPerThread; ++m) {
      int o = tid + m * nth;
      if (o < nout) {
        int i = o / ny, j = o % ny;
        double s = 0.0;
        for (int rr = 0; rr < nr; ++rr) s += Xs[rr * nx + i] * Ys[rr * ny + j];
        acc[m] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int m = 0; m < kGramPerThread; ++m) {
    int o = tid + m * nth;
    if (o < nout) part[(int64_t)tile * nout + o] = acc[m];
  }
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  int lo = tl.lo[sd], hi = tl.hi[sd];
  if (tid == 0) {
    int prev = atomicAdd(counter + sd, 1);
    is_last = (prev == hi - lo - 1);
    if (is_last) counter[sd] = 0;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int o = tid; o < nout; o += nth) {
    double s = 0.0;
    for (int t = lo; t < hi; ++t) s += __ldcg(part + (int64_t)t * nout + o);
    int i = o / ny, j = o % ny;
    G[(int64_t)sd * sd_stride + i * ldg + j] = s;
  }
}

// cyclic Jacobi with the round-robin (circle) ordering: m/2 disjoint rotations per
// round, m-1 rounds per sweep; A <- J^T A J, V <- V J with the symmetric 2x2 Schur
// rotation (Golub & Van Loan, Alg. 8.4.1).  A pair is rotated only while
// |a_pq| > eps sqrt(|a_pp a_qq|) (eps = 2^-52), the threshold that keeps small
// eigenvalues accurate relative to themselves (Demmel & Veselic); the iteration stops
// after a sweep without rotations (at most 40 sweeps).
__global__ void k_sym_eig(const double* __restrict__ A, int ld, int n, double* evals,
                          double* evecs) {
  extern __shared__ double sh[];
  int m = n + (n & 1);
  int lds = m + 1;
  double* a = sh;
  double* v = a + m * lds;
  double* rc = v + m * lds;        // m/2 cosines
  double* rs = rc + m / 2;         // m/2 sines
  double* red = rs + m / 2;        // blockDim.x
  int* rp = reinterpret_cast<int*>(red + blockDim.x);
  int* rq = rp + m / 2;
  int sd = blockIdx.x;
  int tid = threadIdx.x, nth = blockDim.x;
  const double* As = A + (int64_t)sd * ld * ld;
  for (int idx = tid; idx < m * m; idx += nth) {
    int i = idx / m, j = idx % m;
    a[i * lds + j] = (i < n && j < n) ? 0.5 * (As[i * ld + j] + As[j * ld + i]) : 0.0;
    v[i * lds + j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  auto block_sum = [&](double x) -> double {
    red[tid] = x;
    __syncthreads();
    for (int s = nth / 2; s > 0; s >>= 1) {
      if (tid < s) red[tid] += red[tid + s];
      __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
  };
  (void)block_sum;
  __shared__ int nrot;
  for (int sweep = 0; sweep < 40 && m > 1; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int round = 0; round < m - 1; ++round) {
      for (int k = tid; k < m / 2; k += nth) {
        int x0 = k, x1 = m - 1 - k;
        int p = (x0 == 0) ? 0 : ((x0 - 1 + round) % (m - 1)) + 1;
        int q = ((x1 - 1 + round) % (m - 1)) + 1;
        double apq = a[p * lds + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 0x1p-52 * sqrt(fabs(a[p * lds + p] * a[q * lds + q]))) {
          atomicAdd(&nrot, 1);
          double tau = (a[q * lds + q] - a[p * lds + p]) / (2.0 * apq);
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
      for (int w = tid; w < (m / 2) * m; w += nth) {
        int k = w / m, j = w % m;
        double c = rc[k], s = rs[k];
        if (s == 0.0) continue;  // pair not rotated
        int p = rp[k], q = rq[k];
        double ap = a[p * lds + j], aq = a[q * lds + j];
        a[p * lds + j] = c * ap - s * aq;
        a[q * lds + j] = s * ap + c * aq;
      }
      __syncthreads();
      for (int w = tid; w < (m / 2) * m; w += nth) {
        int k = w / m, i = w % m;
        double c = rc[k], s = rs[k];
        if (s == 0.0) continue;
        int p = rp[k], q = rq[k];
        double ap = a[i * lds + p], aq = a[i * lds + q];
        a[i * lds + p] = c * ap - s * aq;
        a[i * lds + q] = s * ap + c * aq;
        double vp = v[i * lds + p], vq = v[i * lds + q];
        v[i * lds + p] = c * vp - s * vq;
        v[i * lds + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
    // every thread reads the count before thread 0 resets it for the next sweep
    const int rotated = nrot;
    __syncthreads();
    if (rotated == 0) break;
  }
  double* ev = evals + (int64_t)sd * ld;
  double* V = evecs + (int64_t)sd * ld * ld;
  for (int idx = tid; idx < ld * ld; idx += nth) V[idx] = 0.0;
  for (int i = tid; i < ld; i += nth)
    if (i >= n) ev[i] = 0.0;
  __syncthreads();
  for (int i = tid; i < n; i += nth) {
    double li = a[i * lds + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double lj = a[j * lds + j];
      if (lj > li || (lj == li && j < i)) ++rank;
    }
    ev[rank] = li;
    for (int r = 0; r < n; ++r) V[r * ld + rank] = v[r * lds + i];
  }
}

__global__ void k_make_M(int mode, const double* __restrict__ evals,
                         const double* __restrict__ evecs, int ld, int n, double rel, int keep,
                         double* M, int* kept, const int32_t* __restrict__ keep_sd) {
  int sd = blockIdx.x;
  const double* ev = evals + (int64_t)sd * ld;
  const double* V = evecs + (int64_t)sd * ld * ld;
  double* Ms = M + (int64_t)sd * ld * ld;
  double l0 = ev[0];
  const int kmax = keep_sd ? min(keep, (int)keep_sd[sd]) : keep;
  // mode 0: eigenvalues above rel * largest; 1: the first kmax; 2: the first kmax above
  // rel; 3 and 4: as 1 and 2; modes 0, 3 and 4 scale column j by ev[j]^(-1/2)
  auto take = [&](int j) -> bool {
    if (mode == 0) return l0 > 0.0 && ev[j] > rel * l0;
    if (mode == 1 || mode == 3) return j < kmax && (mode == 1 || ev[j] > 0.0);
    return j < kmax && ev[j] > rel;
  };
  const bool scaled = mode == 0 || mode >= 3;
  for (int idx = threadIdx.x; idx < ld * ld; idx += blockDim.x) {
    int l = idx / ld, j = idx % ld;
    double val = 0.0;
    if (l < n && j < n && take(j)) val = scaled ? V[l * ld + j] / sqrt(ev[j]) : V[l * ld + j];
    Ms[idx] = val;
  }
  if (threadIdx.x == 0 && kept) {
    int c = 0;
    for (int j = 0; j < n; ++j) c += take(j) ? 1 : 0;
    kept[sd] = c;
  }
}

__global__ void k_rowmul(DTiles tl, const double* __restrict__ X, int ldx, int nin,
                         const double* __restrict__ M, int ldm, double* __restrict__ Y, int ldy,
                         int nout) {
  extern __shared__ double Ms[];
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  int tid = threadIdx.y * blockDim.x + threadIdx.x, nth = blockDim.x * blockDim.y;
  const double* Msd = M + (int64_t)sd * ldm * ldm;
  for (int idx = tid; idx < nin * nout; idx += nth) {
    int l = idx / nout, j = idx % nout;
    Ms[idx] = Msd[l * ldm + j];
  }
  __syncthreads();
  for (int64_t row = r0 + threadIdx.y; row < r1; row += blockDim.y) {
    const double* x = X + row * ldx;
    for (int j = threadIdx.x; j < ldy; j += blockDim.x) {
      double s = 0.0;
      if (j < nout)
        for (int l = 0; l < nin; ++l) s += x[l] * Ms[l * nout + j];
      Y[row * ldy + j] = s;
    }
  }
}

__global__ void k_gather_rows(int64_t n_rows, const int32_t* __restrict__ map,
                              const double* __restrict__ src, int lds, int sc0,
                              double* __restrict__ dst, int ldd, int dc0, int ncols) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_rows * ncols) return;
  int64_t r = idx / ncols;
  int c = (int)(idx % ncols);
  int64_t s = map ? map[r] : r;
  dst[r * ldd + dc0 + c] = src[s * lds + sc0 + c];
}

__global__ void k_scatter_rows(int64_t n_rows, const int32_t* __restrict__ map,
                               const double* __restrict__ src, int lds,
                               double* __restrict__ dst, int ldd, int ncols) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_rows * ncols) return;
  int64_t r = idx / ncols;
  int c = (int)(idx % ncols);
  dst[(int64_t)map[r] * ldd + c] = src[r * lds + c];
}

__global__ void k_set_col(DTiles tl, const double* __restrict__ src, double* dst, int ld,
                          int col) {
  int tile = blockIdx.x;
  for (int64_t r = tl.r0[tile] + threadIdx.x; r < tl.r1[tile]; r += blockDim.x)
    dst[r * ld + col] = src[r];
}

__global__ void k_to_float(int64_t n, const double* __restrict__ src, float* dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

}  // namespace

void launch_gram(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                 const double* Y, int ldy, int ny, double* part, int* counter, double* G,
                 int ldg, cudaStream_t st) {
  (void)n_sd;
  if (tiles.n <= 0) return;
  size_t sm = sizeof(double) * kGramRows * (nx + ny);
  count_launch();
  k_gram<<<tiles.n, kGramThreads, sm, st>>>(tiles, X, ldx, nx, Y, ldy, ny, part, counter, G,
                                           ldg, ldg * ldg);
}

void launch_gram_vec(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                     const double* y, int ldy, double* part, int* counter, double* g, int ldg,
                     cudaStream_t st) {
  (void)n_sd;
  if (tiles.n <= 0) return;
  size_t sm = sizeof(double) * kGramRows * (nx + 1);
  count_launch();
  // the nx x 1 product, rows of stride 1 and ldg per subdomain
  k_gram<<<tiles.n, kGramThreads, sm, st>>>(tiles, X, ldx, nx, y, ldy, 1, part, counter, g, 1,
                                           ldg);
}

void launch_sym_eig(int n_sd, const double* A, int ld, int n, double* evals,
                    double* evecs, cudaStream_t st) {
  if (n_sd <= 0) return;
  int m = n + (n & 1);
  int nth = 256;
  size_t sm = sizeof(double) * (2 * (size_t)m * (m + 1) + m + nth) + sizeof(int) * m;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_sym_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  count_launch();
  k_sym_eig<<<n_sd, nth, sm, st>>>(A, ld, n, evals, evecs);
}

void launch_make_M(int n_sd, int mode, const double* evals, const double* evecs, int ld,
                   int n, double rel, int keep, double* M, int* kept, cudaStream_t st,
                   const int32_t* keep_sd) {
  if (n_sd <= 0) return;
  count_launch();
  k_make_M<<<n_sd, 256, 0, st>>>(mode, evals, evecs, ld, n, rel, keep, M, kept, keep_sd);
}

void launch_rowmul(const DTiles& tiles, const double* X, int ldx, int nin, const double* M,
                   int ldm, double* Y, int ldy, int nout, cudaStream_t st) {
  if (tiles.n <= 0) return;
  size_t sm = sizeof(double) * (size_t)nin * nout;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_rowmul, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    attr = true;
  }
  count_launch();
  k_rowmul<<<tiles.n, dim3(32, 8), sm, st>>>(tiles, X, ldx, nin, M, ldm, Y, ldy, nout);
}

void launch_gather_rows(int64_t n_rows, const int32_t* map, const double* src, int lds,
                        int sc0, double* dst, int ldd, int dc0, int ncols, cudaStream_t st) {
  int64_t n = n_rows * ncols;
  if (n <= 0) return;
  count_launch();
  k_gather_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_rows, map, src, lds, sc0, dst,
                                                             ldd, dc0, ncols);
}

void launch_scatter_rows(int64_t n_rows, const int32_t* map, const double* src, int lds,
                         double* dst, int ldd, int ncols, cudaStream_t st) {
  int64_t n = n_rows * ncols;
  if (n <= 0) return;
  count_launch();
  k_scatter_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_rows, map, src, lds, dst,
                                                              ldd, ncols);
}

void launch_set_col(const DTiles& tiles, const double* src, double* dst, int ld, int col,
                    cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_set_col<<<tiles.n, 128, 0, st>>>(tiles, src, dst, ld, col);
}

void launch_to_float(int64_t n, const double* src, float* dst, cudaStream_t st) {
  if (n <= 0) return;
  count_launch();
  k_to_float<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, src, dst);
}

}  // namespace mor
