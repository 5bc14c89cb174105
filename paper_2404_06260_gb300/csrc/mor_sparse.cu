// Sliced-ELL multi-right-hand-side products and the batched Jacobi-preconditioned CG
// used for every local solve of step 2 (A_II and H^+ systems of Sec. 4 and Sec. 6).
//
// Vectors are row-major blocks [rows x kp] (kp = right-hand sides padded to a multiple
// of 4).  A CUDA block owns one row tile of one subdomain; thread (tx, ty) handles the
// 16-byte column chunk tx of rows r0 + ty, r0 + ty + RB, ...  Every (subdomain, column)
// pair runs its own CG recurrence; per-tile column sums go to a partial array and the
// last tile of a subdomain to finish (atomic ticket) reduces them in tile order, so the
// reductions are deterministic and need no extra launch.
#include "mor_kernels.h"
#include "mor_plan.h"

namespace mor {
namespace {

template <typename T>
struct alignas(16) Pack {
  static constexpr int N = 16 / sizeof(T);
  T v[N];
};

template <typename T>
__device__ __forceinline__ Pack<T> ld(const T* p) {
  return *reinterpret_cast<const Pack<T>*>(p);
}
template <typename T>
__device__ __forceinline__ void st(T* p, const Pack<T>& x) {
  *reinterpret_cast<Pack<T>*>(p) = x;
}

struct Geo {
  int tx, ty, nch, rb, tid, nth;
};
__device__ __forceinline__ Geo geo() {
  Geo g;
  g.tx = threadIdx.x;
  g.ty = threadIdx.y;
  g.nch = blockDim.x;
  g.rb = blockDim.y;
  g.tid = g.ty * g.nch + g.tx;
  g.nth = g.nch * g.rb;
  return g;
}

// shared memory layout: red[nth * N] of T, scratch[nth] doubles, sums[2*kp] doubles,
// then the staged sliced-ELL tile: scol[kTileRows * W] int32, sval[kTileRows * W] T
template <typename T>
struct Smem {
  T* red;
  double* scratch;
  double* sums;
  int32_t* scol;
  T* sval;
};
__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
template <typename T>
__device__ __forceinline__ Smem<T> smem_layout(const Geo& g, int kp, int W) {
  extern __shared__ __align__(16) unsigned char raw[];
  Smem<T> s;
  size_t o = 0;
  s.red = reinterpret_cast<T*>(raw + o);
  o += align16(16 * (size_t)g.nth);
  s.scratch = reinterpret_cast<double*>(raw + o);
  s.sums = s.scratch + g.nth;
  o += align16(sizeof(double) * ((size_t)g.nth + 2 * kp));
  s.scol = reinterpret_cast<int32_t*>(raw + o);
  o += align16(sizeof(int32_t) * (size_t)kTileRows * W);
  s.sval = reinterpret_cast<T*>(raw + o);
  return s;
}
template <typename T>
size_t smem_bytes(int nch, int rb, int kp, int W) {
  size_t nth = (size_t)nch * rb;
  return align16(16 * nth) + align16(sizeof(double) * (nth + 2 * kp)) +
         align16(sizeof(int32_t) * (size_t)kTileRows * W) + sizeof(T) * (size_t)kTileRows * W;
}

// column sums over ty of per-thread N-wide accumulators -> out[tx*N + e] (double)
template <typename T, int N>
__device__ void block_colsum(const Geo& g, const T (&acc)[N], T* red, double* out) {
#pragma unroll
  for (int e = 0; e < N; ++e) red[g.tid * N + e] = acc[e];
  __syncthreads();
  int p2 = 1;
  while (p2 < g.rb) p2 <<= 1;
  for (int s = p2 >> 1; s > 0; s >>= 1) {
    if (g.ty < s && g.ty + s < g.rb)
#pragma unroll
      for (int e = 0; e < N; ++e) red[g.tid * N + e] += red[(g.tid + s * g.nch) * N + e];
    __syncthreads();
  }
  if (g.ty == 0)
#pragma unroll
    for (int e = 0; e < N; ++e) out[g.tx * N + e] = (double)red[g.tx * N + e];
}

__device__ __forceinline__ bool last_block(const Geo& g, int* counter, int sd, int nblk) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (g.tid == 0) {
    int prev = atomicAdd(counter + sd, 1);
    is_last = (prev == nblk - 1);
    if (is_last) counter[sd] = 0;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// sums[c] = sum over tiles lo..hi-1 of part[t*kp + c], fixed order
__device__ void sd_colsums(const Geo& g, const double* part, int kp, int lo, int hi,
                           double* scratch, double* sums) {
  int S = g.nth / kp;
  if (S < 1) S = 1;
  int c = g.tid % kp, sidx = g.tid / kp;
  double acc = 0.0;
  if (sidx < S) {
#pragma unroll 4
    for (int t = lo + sidx; t < hi; t += S) acc += __ldcg(part + (int64_t)t * kp + c);
  }
  scratch[g.tid] = acc;
  __syncthreads();
  for (int cc = g.tid; cc < kp; cc += g.nth) {
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += scratch[q * kp + cc];
    sums[cc] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ void count_active(const Geo& g, const int* done, int sd, int kp,
                                             int* active) {
  __shared__ int cnt;
  if (g.tid == 0) cnt = 0;
  __syncthreads();
  for (int c = g.tid; c < kp; c += g.nth)
    if (!done[sd * kp + c]) atomicAdd(&cnt, 1);
  __syncthreads();
  if (g.tid == 0) active[sd] = cnt;
}

// ---------------------------------------------------------------------------------
// Sliced-ELL products on a row tile.  The tile's slots (column index and value) are
// first staged in shared memory with coalesced loads (consecutive threads take
// consecutive rows of one slot), which takes the index load off the critical path of
// the gathers.  Thread (tx, ty) then computes the 16-byte column chunk tx of rows
// ty, ty + RB, ...: eight slots are gathered (predicated, independent loads) before
// their multiply-adds.  k_spmm: Y = A X.  k_cg_spmm_pq: q = A p with the column sums
// of p.q.  k_residual64: r = b - A x with the column sums of r.r.
template <typename T>
__device__ __forceinline__ void stage_tile(const Geo& g, int r0, int nrows,
                                           const EllView<T>& A, int32_t* scol, T* sval) {
  const int W = A.W;
  const bool full = nrows == kTileRows;  // full tiles: slot and row by shifts
  for (int idx = g.tid; idx < nrows * W; idx += g.nth) {
    int j, rr;
    if (full) {
      j = idx / kTileRows;  // kTileRows is a power of two: compiles to a shift
      rr = idx & (kTileRows - 1);
    } else {
      j = idx / nrows;
      rr = idx - j * nrows;
    }
    int64_t r = (int64_t)r0 + rr;
    int32_t c = -1;
    T v = T(0);
    if (j < A.width[r >> 5]) {
      int64_t at = ell_at(r, j, W);
      c = A.col[at];
      v = A.val[at];
    }
    scol[rr * W + j] = c;
    sval[rr * W + j] = v;
  }
}

template <typename T>
__device__ __forceinline__ Pack<T> spmm_row(int rr, int w, int W, int tx, const int32_t* scol,
                                            const T* sval, const T* __restrict__ X, int kp) {
  constexpr int N = Pack<T>::N;
  constexpr int U = 8;
  Pack<T> acc;
#pragma unroll
  for (int e = 0; e < N; ++e) acc.v[e] = T(0);
  const int32_t* cr = scol + rr * W;
  const T* vr = sval + rr * W;
  for (int j0 = 0; j0 < w; j0 += U) {
    Pack<T> xv[U];
    T av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int j = j0 + u;
      int32_t c = (j < w) ? cr[j] : -1;
      av[u] = (j < w) ? vr[j] : T(0);
      if (c >= 0) {
        xv[u] = ld(X + (int64_t)c * kp + tx * N);
      } else {
#pragma unroll
        for (int e = 0; e < N; ++e) xv[u].v[e] = T(0);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < N; ++e) acc.v[e] += av[u] * xv[u].v[e];
  }
  return acc;
}

template <typename T>
__global__ void k_spmm(DTiles tl, EllView<T> A, const T* __restrict__ X, T* __restrict__ Y,
                       int kp) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, A.W);
  const int tile = blockIdx.x;
  const int r0 = tl.r0[tile], r1 = tl.r1[tile];
  stage_tile(g, r0, r1 - r0, A, sm.scol, sm.sval);
  __syncthreads();
  for (int rr = g.ty; rr < r1 - r0; rr += g.rb) {
    int64_t row = r0 + rr;
    st(Y + row * kp + g.tx * N,
       spmm_row(rr, A.width[row >> 5], A.W, g.tx, sm.scol, sm.sval, X, kp));
  }
}

// binary64 residual row: A x and sum_j |a_ij x_j| in one pass over the staged slots
__device__ __forceinline__ void spmm_row_res(int rr, int w, int W, int tx, const int32_t* scol,
                                             const double* sval, const double* __restrict__ X,
                                             int kp, Pack<double>& acc, Pack<double>& aabs) {
  constexpr int N = Pack<double>::N;
  constexpr int U = 8;
#pragma unroll
  for (int e = 0; e < N; ++e) acc.v[e] = aabs.v[e] = 0.0;
  const int32_t* cr = scol + rr * W;
  const double* vr = sval + rr * W;
  for (int j0 = 0; j0 < w; j0 += U) {
    Pack<double> xv[U];
    double av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      int j = j0 + u;
      int32_t c = (j < w) ? cr[j] : -1;
      av[u] = (j < w) ? vr[j] : 0.0;
      if (c >= 0) {
        xv[u] = ld(X + (int64_t)c * kp + tx * N);
      } else {
#pragma unroll
        for (int e = 0; e < N; ++e) xv[u].v[e] = 0.0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int e = 0; e < N; ++e) {
        double t = av[u] * xv[u].v[e];
        acc.v[e] += t;
        aabs.v[e] += fabs(t);
      }
  }
}

template <typename T>
__global__ void k_cg_spmm_pq(DTiles tl, EllView<T> A, const T* __restrict__ p,
                             T* __restrict__ q, int kp, CgState s) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, A.W);
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int r0 = tl.r0[tile], r1 = tl.r1[tile];
  stage_tile(g, r0, r1 - r0, A, sm.scol, sm.sval);
  __syncthreads();
  T acc[N];
#pragma unroll
  for (int e = 0; e < N; ++e) acc[e] = T(0);
  for (int rr = g.ty; rr < r1 - r0; rr += g.rb) {
    int64_t row = r0 + rr;
    Pack<T> qv = spmm_row(rr, A.width[row >> 5], A.W, g.tx, sm.scol, sm.sval, p, kp);
    int64_t o = row * kp + g.tx * N;
    st(q + o, qv);
    Pack<T> pv = ld(p + o);
#pragma unroll
    for (int e = 0; e < N; ++e) acc[e] += pv.v[e] * qv.v[e];
  }
  block_colsum<T, N>(g, acc, sm.red, s.part1 + (int64_t)tile * kp);
  const int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part1, kp, lo, hi, sm.scratch, sm.sums);
  for (int c = g.tid; c < kp; c += g.nth) {
    int i = sd * kp + c;
    double a = 0.0;
    if (!s.done[i]) {
      double pq = sm.sums[c];
      if (pq > 0.0)
        a = s.rz[i] / pq;
      else
        s.done[i] = 1;  // breakdown (p = 0 or indefinite): stop this column
    }
    s.alpha[i] = a;
  }
}

template <bool kFloor>
__global__ void k_residual64(DTiles tl, EllView<double> A, const double* __restrict__ b,
                             const double* __restrict__ x, double* __restrict__ r, int kp,
                             int nc, int ncn, double rtol2, int first, RefineState s) {
  constexpr int N = 2;
  Geo g = geo();
  Smem<double> sm = smem_layout<double>(g, kp, A.W);
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int r0 = tl.r0[tile], r1 = tl.r1[tile];
  stage_tile(g, r0, r1 - r0, A, sm.scol, sm.sval);
  __syncthreads();
  double acc[N] = {0.0, 0.0}, aca[N] = {0.0, 0.0};
  for (int rr = g.ty; rr < r1 - r0; rr += g.rb) {
    int64_t row = r0 + rr;
    Pack<double> ax, aabs;
    if constexpr (kFloor)
      spmm_row_res(rr, A.width[row >> 5], A.W, g.tx, sm.scol, sm.sval, x, kp, ax, aabs);
    else
      ax = spmm_row(rr, A.width[row >> 5], A.W, g.tx, sm.scol, sm.sval, x, kp);
    int64_t o = row * kp + g.tx * N;
    Pack<double> bv = ld(b + o), rv;
#pragma unroll
    for (int e = 0; e < N; ++e) {
      rv.v[e] = bv.v[e] - ax.v[e];
      acc[e] += rv.v[e] * rv.v[e];
      if constexpr (kFloor) {
        double f = aabs.v[e] + fabs(bv.v[e]);
        aca[e] += f * f;
      }
    }
    st(r + o, rv);
  }
  block_colsum<double, N>(g, acc, sm.red, s.part + (int64_t)tile * kp);
  if constexpr (kFloor) {
    __syncthreads();
    block_colsum<double, N>(g, aca, sm.red, s.part2 + (int64_t)tile * kp);
  }
  const int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part, kp, lo, hi, sm.scratch, sm.sums);
  if constexpr (kFloor) {
    sd_colsums(g, s.part2, kp, lo, hi, sm.scratch, sm.sums + kp);
    for (int c = g.tid; c < kp; c += g.nth) s.oaa[sd * kp + c] = sm.sums[kp + c];
  }
  __shared__ int cnt, nfl;
  __shared__ double bref;
  if (g.tid == 0) {
    cnt = 0;
    nfl = 0;
    double m = 0.0;
    if (first)
      for (int c = 0; c < ncn; ++c) m = fmax(m, sm.sums[c]);
    bref = m;
  }
  __syncthreads();
  // attainable accuracy: the rounding error of the binary64 residual of a binary64 x is
  // about u || |A| |x| + |b| ||_2 (u = 2^-53); a residual below kResidualFloor times that
  // is rounding noise, so the column stops there even if rtol is not reached.  The
  // reference (oaa, squared) is refreshed only by the kFloor sweeps; it is a scale,
  // and zero (no floor test) until the first of them
  const double fl2 = (kResidualFloor * 0x1p-53) * (kResidualFloor * 0x1p-53);
  for (int c = g.tid; c < kp; c += g.nth) {
    int i = sd * kp + c;
    double rr = sm.sums[c];
    if (first) {
      s.obb[i] = (c < ncn) ? bref : rr;
      s.oaa[i] = 0.0;
    }
    s.orr[i] = rr;
    bool by_rtol = rr <= rtol2 * s.obb[i];
    bool by_floor = rr <= fl2 * s.oaa[i];
    bool done = (c >= nc) || !(s.obb[i] > 0.0) || by_rtol || by_floor;
    s.scale[i] = done ? 0.0 : 1.0 / sqrt(rr);
    if (!done) atomicAdd(&cnt, 1);
    if (c < nc && s.obb[i] > 0.0 && !by_rtol && by_floor) atomicAdd(&nfl, 1);
  }
  __syncthreads();
  if (g.tid == 0) {
    s.active[sd] = cnt;
    s.nfloor[sd] = nfl;
  }
}

template <typename T>
__global__ void k_cg_init(DTiles tl, const T* __restrict__ b, T* x, T* r, T* p,
                          const T* __restrict__ dinv, int kp, int nc, int ncn, CgState s) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  T arz[N], arr[N];
#pragma unroll
  for (int e = 0; e < N; ++e) arz[e] = arr[e] = T(0);
  Pack<T> zero;
#pragma unroll
  for (int e = 0; e < N; ++e) zero.v[e] = T(0);
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> bv = ld(b + o), pv;
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      pv.v[e] = d * bv.v[e];
      arz[e] += bv.v[e] * pv.v[e];
      arr[e] += bv.v[e] * bv.v[e];
    }
    st(x + o, zero);
    st(r + o, bv);
    st(p + o, pv);
  }
  block_colsum<T, N>(g, arz, sm.red, s.part1 + (int64_t)tile * kp);
  __syncthreads();
  block_colsum<T, N>(g, arr, sm.red, s.part2 + (int64_t)tile * kp);
  int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part1, kp, lo, hi, sm.scratch, sm.sums);
  sd_colsums(g, s.part2, kp, lo, hi, sm.scratch, sm.sums + kp);
  __shared__ double bref;
  if (g.tid == 0) {
    double m = 0.0;
    for (int c = 0; c < ncn; ++c) m = fmax(m, sm.sums[kp + c]);
    bref = m;
  }
  __syncthreads();
  for (int c = g.tid; c < kp; c += g.nth) {
    int i = sd * kp + c;
    double bb = sm.sums[kp + c];
    s.rz[i] = sm.sums[c];
    s.bb[i] = (c < ncn) ? bref : bb;
    s.rr[i] = bb;
    s.done[i] = (c >= nc || !(bb > 0.0)) ? 1 : 0;
    s.alpha[i] = 0.0;
    s.beta[i] = 0.0;
  }
  if (g.tid == 0) s.iters[sd] = 0;
  __syncthreads();
  count_active(g, s.done, sd, kp, s.active);
}


template <typename T>
__global__ void k_cg_update_xr(DTiles tl, T* x, T* r, const T* __restrict__ p,
                               const T* __restrict__ q, const T* __restrict__ dinv, int kp,
                               double tol2, CgState s) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  T al[N];
#pragma unroll
  for (int e = 0; e < N; ++e) al[e] = (T)s.alpha[sd * kp + g.tx * N + e];
  T arr[N], arz[N];
#pragma unroll
  for (int e = 0; e < N; ++e) arr[e] = arz[e] = T(0);
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> xv = ld(x + o), rv = ld(r + o), pv = ld(p + o), qv = ld(q + o);
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      xv.v[e] += al[e] * pv.v[e];
      rv.v[e] -= al[e] * qv.v[e];
      arr[e] += rv.v[e] * rv.v[e];
      arz[e] += rv.v[e] * (d * rv.v[e]);
    }
    st(x + o, xv);
    st(r + o, rv);
  }
  block_colsum<T, N>(g, arr, sm.red, s.part1 + (int64_t)tile * kp);
  __syncthreads();
  block_colsum<T, N>(g, arz, sm.red, s.part2 + (int64_t)tile * kp);
  int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part1, kp, lo, hi, sm.scratch, sm.sums);
  sd_colsums(g, s.part2, kp, lo, hi, sm.scratch, sm.sums + kp);
  for (int c = g.tid; c < kp; c += g.nth) {
    int i = sd * kp + c;
    double be = 0.0;
    s.rr[i] = sm.sums[c];
    if (!s.done[i]) {
      double rr = sm.sums[c], rzn = sm.sums[kp + c];
      if (rr <= tol2 * s.bb[i] || !(s.rz[i] > 0.0)) {
        s.done[i] = 1;
      } else {
        be = rzn / s.rz[i];
        s.rz[i] = rzn;
      }
    }
    s.beta[i] = be;
  }
  __syncthreads();
  count_active(g, s.done, sd, kp, s.active);
  if (g.tid == 0 && s.active[sd] > 0) s.iters[sd] += 1;
}

template <typename T>
__global__ void k_cg_update_p(DTiles tl, const T* __restrict__ r, T* p,
                              const T* __restrict__ dinv, int kp, CgState s) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  T be[N];
#pragma unroll
  for (int e = 0; e < N; ++e) be[e] = (T)s.beta[sd * kp + g.tx * N + e];
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> rv = ld(r + o), pv = ld(p + o);
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) pv.v[e] = d * rv.v[e] + be[e] * pv.v[e];
    st(p + o, pv);
  }
}

__global__ void k_count_active(int n_sd, const int* active, int* out) {
  __shared__ int tot;
  if (threadIdx.x == 0) tot = 0;
  __syncthreads();
  int a = 0;
  for (int i = threadIdx.x; i < n_sd; i += blockDim.x) a += active[i];
  atomicAdd(&tot, a);
  __syncthreads();
  if (threadIdx.x == 0) *out = tot;
}


__global__ void k_zero_rows(DTiles tl, double* x, int kp) {
  Geo g = geo();
  int tile = blockIdx.x;
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb)
    for (int c = g.tx; c < kp; c += g.nch) x[row * kp + c] = 0.0;
}

// residual replacement: rT = (T) r64 (the true residual), rz recomputed from it, and
// each column's done flag taken from the binary64 convergence test (scale == 0)
// Columns the recursion had declared converged but the binary64 test reopens, and
// columns whose true residual norm exceeds drift x the recursive one, restart from
// p = D^{-1} r: their stored direction belongs to a much smaller residual.
template <typename T>
__global__ void k_cg_replace(DTiles tl, const double* __restrict__ r64, T* __restrict__ rT,
                             T* __restrict__ pT, const T* __restrict__ dinv, int kp,
                             double drift2, CgState s, RefineState rs) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  bool restart[N];
#pragma unroll
  for (int e = 0; e < N; ++e) {
    int i = sd * kp + g.tx * N + e;
    // reopened, or the recursion drifted from the true residual (a stale direction
    // would make the next step length meaningless)
    restart[e] = rs.scale[i] != 0.0 && (s.done[i] || rs.orr[i] > drift2 * s.rr[i]);
  }
  T arz[N];
#pragma unroll
  for (int e = 0; e < N; ++e) arz[e] = T(0);
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> rv, pv = ld(pT + o);
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      rv.v[e] = (T)r64[o + e];
      arz[e] += rv.v[e] * (d * rv.v[e]);
      if (restart[e]) pv.v[e] = d * rv.v[e];
    }
    st(rT + o, rv);
    st(pT + o, pv);
  }
  block_colsum<T, N>(g, arz, sm.red, s.part1 + (int64_t)tile * kp);
  int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part1, kp, lo, hi, sm.scratch, sm.sums);
  for (int c = g.tid; c < kp; c += g.nth) {
    int i = sd * kp + c;
    s.rz[i] = sm.sums[c];
    s.bb[i] = rs.obb[i];
    s.done[i] = (rs.scale[i] == 0.0) ? 1 : 0;
    s.alpha[i] = 0.0;
    s.beta[i] = 0.0;
  }
  __syncthreads();
  count_active(g, s.done, sd, kp, s.active);
}

// x64 += xT; xT = 0
template <typename T>
__global__ void k_accum_reset(DTiles tl, T* __restrict__ xT, double* __restrict__ x64, int kp) {
  Geo g = geo();
  int tile = blockIdx.x;
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb)
    for (int c = g.tx; c < kp; c += g.nch) {
      int64_t o = row * kp + c;
      x64[o] += (double)xT[o];
      xT[o] = T(0);
    }
}

// rT = (T) src
template <typename T>
__global__ void k_cast(DTiles tl, const double* __restrict__ src, T* __restrict__ dst, int kp) {
  Geo g = geo();
  int tile = blockIdx.x;
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb)
    for (int c = g.tx; c < kp; c += g.nch) dst[row * kp + c] = (T)src[row * kp + c];
}

template <typename T>
dim3 block_of(int kp) {
  int nch = kp / Pack<T>::N;
  int rb = 256 / nch;
  if (rb < 1) rb = 1;
  return dim3(nch, rb);
}

}  // namespace

template <typename T>
void set_smem_attr(const void* fn) {
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
}

template <typename T>
void launch_spmm(const DTiles& tiles, const EllView<T>& A, const T* X, T* Y, int kp,
                 cudaStream_t st) {
  if (tiles.n <= 0) return;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_spmm<T>);
    attr = true;
  }
  dim3 bl = block_of<T>(kp);
  count_launch();
  k_spmm<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, A.W), st>>>(tiles, A, X, Y, kp);
}

template <typename T>
void launch_cg_init(const DTiles& tiles, const T* b, T* x, T* r, T* p, const T* dinv,
                    int kp, int nc, int ncn, const CgState& s, cudaStream_t st) {
  if (tiles.n <= 0) return;
  dim3 bl = block_of<T>(kp);
  count_launch();
  k_cg_init<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, 0), st>>>(tiles, b, x, r, p, dinv,
                                                                      kp, nc, ncn, s);
}

template <typename T>
void launch_cg_step(const DTiles& tiles, const EllView<T>& A, T* x, T* r, T* p, T* q,
                    const T* dinv, int kp, double tol2, const CgState& s, cudaStream_t st,
                    const cudaEvent_t* ev) {
  if (tiles.n <= 0) return;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T>);
    attr = true;
  }
  dim3 bl = block_of<T>(kp);
  count_launch(3);
  if (ev) cudaEventRecord(ev[0], st);
  k_cg_spmm_pq<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, A.W), st>>>(tiles, A, p, q, kp,
                                                                           s);
  if (ev) cudaEventRecord(ev[1], st);
  k_cg_update_xr<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, 0), st>>>(tiles, x, r, p, q,
                                                                           dinv, kp, tol2, s);
  if (ev) cudaEventRecord(ev[2], st);
  k_cg_update_p<T><<<tiles.n, bl, 0, st>>>(tiles, r, p, dinv, kp, s);
  if (ev) cudaEventRecord(ev[3], st);
}

void launch_count_active(int n_sd, const int* active, int* out, cudaStream_t st) {
  count_launch();
  k_count_active<<<1, 256, 0, st>>>(n_sd, active, out);
}

void launch_residual64(const DTiles& tiles, const EllView<double>& A, const double* b64,
                       const double* x64, double* r64, int kp, int nc, int ncn, double rtol2,
                       int first, bool floor_ref, const RefineState& s, cudaStream_t st) {
  if (tiles.n <= 0) return;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<double>((const void*)k_residual64<false>);
    set_smem_attr<double>((const void*)k_residual64<true>);
    attr = true;
  }
  dim3 bl = block_of<double>(kp);
  size_t sm = smem_bytes<double>(bl.x, bl.y, kp, A.W);
  count_launch();
  if (floor_ref && !first)
    k_residual64<true><<<tiles.n, bl, sm, st>>>(tiles, A, b64, x64, r64, kp, nc, ncn, rtol2,
                                                first, s);
  else
    k_residual64<false><<<tiles.n, bl, sm, st>>>(tiles, A, b64, x64, r64, kp, nc, ncn, rtol2,
                                                 first, s);
}

template <typename T>
void launch_cg_replace(const DTiles& tiles, const double* r64, T* rT, T* pT, const T* dinv,
                       int kp, double drift, const CgState& s, const RefineState& rs,
                       cudaStream_t st) {
  if (tiles.n <= 0) return;
  dim3 bl = block_of<T>(kp);
  count_launch();
  k_cg_replace<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, 0), st>>>(
      tiles, r64, rT, pT, dinv, kp, drift * drift, s, rs);
}

template <typename T>
void launch_accum_reset(const DTiles& tiles, T* xT, double* x64, int kp, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_accum_reset<T><<<tiles.n, dim3(32, 8), 0, st>>>(tiles, xT, x64, kp);
}

template <typename T>
void launch_cast(const DTiles& tiles, const double* src, T* dst, int kp, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_cast<T><<<tiles.n, dim3(32, 8), 0, st>>>(tiles, src, dst, kp);
}

template void launch_cg_replace<float>(const DTiles&, const double*, float*, float*,
                                       const float*, int, double, const CgState&,
                                       const RefineState&, cudaStream_t);
template void launch_cg_replace<double>(const DTiles&, const double*, double*, double*,
                                        const double*, int, double, const CgState&,
                                        const RefineState&, cudaStream_t);
template void launch_accum_reset<float>(const DTiles&, float*, double*, int, cudaStream_t);
template void launch_accum_reset<double>(const DTiles&, double*, double*, int, cudaStream_t);
template void launch_cast<float>(const DTiles&, const double*, float*, int, cudaStream_t);
template void launch_cast<double>(const DTiles&, const double*, double*, int, cudaStream_t);

void launch_zero_rows(const DTiles& tiles, double* x, int kp, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_zero_rows<<<tiles.n, dim3(32, 8), 0, st>>>(tiles, x, kp);
}

template void launch_spmm<float>(const DTiles&, const EllView<float>&, const float*, float*,
                                 int, cudaStream_t);
template void launch_spmm<double>(const DTiles&, const EllView<double>&, const double*,
                                  double*, int, cudaStream_t);
template void launch_cg_init<float>(const DTiles&, const float*, float*, float*, float*,
                                    const float*, int, int, int, const CgState&, cudaStream_t);
template void launch_cg_init<double>(const DTiles&, const double*, double*, double*, double*,
                                     const double*, int, int, int, const CgState&,
                                     cudaStream_t);
template void launch_cg_step<float>(const DTiles&, const EllView<float>&, float*, float*,
                                    float*, float*, const float*, int, double, const CgState&,
                                    cudaStream_t, const cudaEvent_t*);
template void launch_cg_step<double>(const DTiles&, const EllView<double>&, double*, double*,
                                     double*, double*, const double*, int, double,
                                     const CgState&, cudaStream_t, const cudaEvent_t*);
}  // namespace mor
