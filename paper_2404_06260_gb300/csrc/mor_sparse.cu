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
#include "mor_tc.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>
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

// two consecutive slots of one row of a staged sliced-ELL tile: values first, so that a
// binary32 record is one 16-byte shared-memory load
template <typename T>
struct alignas(16) Slot2 {
  T v[2];
  int32_t c[2];
};

// shared memory layout: red[nth * N] of T, scratch[nth] doubles, sums[2*kp] doubles,
// then the staged sliced-ELL tile: slots[((W + 1) / 2) * kTileRows] pair records,
// pair-major (record h of row rr at h * kTileRows + rr)
template <typename T>
struct Smem {
  T* red;
  double* scratch;
  double* sums;
  Slot2<T>* slots;
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
  s.slots = reinterpret_cast<Slot2<T>*>(raw + o);
  return s;
}
template <typename T>
__host__ __device__ __forceinline__ size_t smem_bytes(int nch, int rb, int kp, int W) {
  size_t nth = (size_t)nch * rb;
  return align16(16 * nth) + align16(sizeof(double) * (nth + 2 * kp)) +
         sizeof(Slot2<T>) * (size_t)kTileRows * ((W + 1) / 2);
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

// sums[c] = sum over tiles lo..hi-1 of part[t*kp + c], fixed order.  Columns are taken
// in groups of at most nth; within a group S = nth / group threads share a column.
__device__ void sd_colsums(const Geo& g, const double* part, int kp, int lo, int hi,
                           double* scratch, double* sums) {
  for (int c0 = 0; c0 < kp; c0 += g.nth) {
    const int cw = min(kp - c0, g.nth);
    const int S = g.nth / cw;
    const int c = c0 + g.tid % cw, sidx = g.tid / cw;
    double acc = 0.0;
    if (sidx < S) {
#pragma unroll 4
      for (int t = lo + sidx; t < hi; t += S) acc += __ldcg(part + (int64_t)t * kp + c);
    }
    scratch[g.tid] = acc;
    __syncthreads();
    for (int cc = g.tid; cc < cw; cc += g.nth) {
      double s = 0.0;
      for (int q = 0; q < S; ++q) s += scratch[q * cw + cc];
      sums[c0 + cc] = s;
    }
    __syncthreads();
  }
}

// CG coefficients: binary64 state with a binary32 copy
__device__ __forceinline__ void set_coef(double* c64, float* c32, int i, double v) {
  c64[i] = v;
  c32[i] = (float)v;
}
// the N coefficients of pack tx of subdomain sd in the working precision
template <typename T>
__device__ __forceinline__ Pack<T> coef_pack(const double* c64, const float* c32, int sd,
                                             int kp, int tx) {
  constexpr int N = Pack<T>::N;
  if constexpr (sizeof(T) == 4) {
    return ld(reinterpret_cast<const T*>(c32) + sd * kp + tx * N);
  } else {
    return ld(reinterpret_cast<const T*>(c64) + sd * kp + tx * N);
  }
}

// the N columns of pack tx of subdomain sd have all converged (their work can be skipped:
// converged columns have alpha = 0 and are reset at the next residual replacement)
template <typename T>
__device__ __forceinline__ bool pack_done(const CgState& s, int sd, int kp, int tx) {
  constexpr int N = Pack<T>::N;
  const int* d = s.done + sd * kp + tx * N;
  bool all = true;
#pragma unroll
  for (int e = 0; e < N; ++e) all = all && d[e] != 0;
  return all;
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
// consecutive rows of one slot pair), which takes the index load off the critical path
// of the gathers; a row's slots 2h and 2h + 1 form one record, so one shared load feeds
// two gathers.  Thread (tx, ty) then computes the 16-byte column chunk tx of rows
// ty, ty + RB, ...: the slots of a batch are gathered (predicated, independent loads)
// before their multiply-adds, which run in slot order.  k_spmm: Y = A X.
// k_cg_spmm_pq: q = A p with the column sums of p.q.  k_residual64: r = b - A x with
// the column sums of r.r.
template <typename T>
__device__ __forceinline__ void stage_tile(const Geo& g, int r0, int nrows,
                                           const EllView<T>& A, Slot2<T>* slots) {
  const int W = A.W, W2 = (W + 1) / 2;
  const bool full = nrows == kTileRows;  // full tiles: pair and row by shifts
  for (int idx = g.tid; idx < nrows * W2; idx += g.nth) {
    int h, rr;
    if (full) {
      h = idx / kTileRows;  // kTileRows is a power of two: compiles to a shift
      rr = idx & (kTileRows - 1);
    } else {
      h = idx / nrows;
      rr = idx - h * nrows;
    }
    int64_t r = (int64_t)r0 + rr;
    const int w = A.width[r >> 5];
    Slot2<T> rec;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      int j = 2 * h + u;
      rec.c[u] = -1;
      rec.v[u] = T(0);
      if (j < w) {
        int64_t at = ell_at(r, j, W);
        rec.c[u] = A.col[at];
        rec.v[u] = A.val[at];
      }
    }
    slots[h * kTileRows + rr] = rec;
  }
}

// row rr of the staged tile (slice width w) times X: column chunk tx.  R records (2 R
// slots) are gathered per batch before their multiply-adds, which run in slot order
// (the sum is the same for every R).
template <typename T, int R = 1>
__device__ __forceinline__ Pack<T> spmm_row(int rr, int w, int tx, const Slot2<T>* slots,
                                            const T* __restrict__ X, int kp) {
  constexpr int N = Pack<T>::N;
  Pack<T> acc;
#pragma unroll
  for (int e = 0; e < N; ++e) acc.v[e] = T(0);
  const int w2 = (w + 1) >> 1;
  for (int h0 = 0; h0 < w2; h0 += R) {
    Slot2<T> rec[R];
    Pack<T> xv[2 * R];
#pragma unroll
    for (int g = 0; g < R; ++g) {
      if (h0 + g < w2) {
        rec[g] = slots[(h0 + g) * kTileRows + rr];
      } else {
        rec[g].c[0] = rec[g].c[1] = -1;
        rec[g].v[0] = rec[g].v[1] = T(0);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (rec[g].c[u] >= 0) {
          xv[2 * g + u] = ld(X + (int64_t)rec[g].c[u] * kp + tx * N);
        } else {
#pragma unroll
          for (int e = 0; e < N; ++e) xv[2 * g + u].v[e] = T(0);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < R; ++g)
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int e = 0; e < N; ++e) acc.v[e] += rec[g].v[u] * xv[2 * g + u].v[e];
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
  stage_tile(g, r0, r1 - r0, A, sm.slots);
  __syncthreads();
  for (int rr = g.ty; rr < r1 - r0; rr += g.rb) {
    int64_t row = r0 + rr;
    st(Y + row * kp + g.tx * N,
       spmm_row(rr, A.width[row >> 5], g.tx, sm.slots, X, kp));
  }
}

// binary64 residual row: A x and sum_j |a_ij x_j| in one pass over the staged slots
// (batches of four records, eight slots)
__device__ __forceinline__ void spmm_row_res(int rr, int w, int tx, const Slot2<double>* slots,
                                             const double* __restrict__ X, int kp,
                                             Pack<double>& acc, Pack<double>& aabs) {
  constexpr int N = Pack<double>::N;
  constexpr int H = 4;
#pragma unroll
  for (int e = 0; e < N; ++e) acc.v[e] = aabs.v[e] = 0.0;
  const int w2 = (w + 1) >> 1;
  for (int h0 = 0; h0 < w2; h0 += H) {
    Pack<double> xv[2 * H];
    double av[2 * H];
#pragma unroll
    for (int hh = 0; hh < H; ++hh) {
      Slot2<double> rec;
      if (h0 + hh < w2) {
        rec = slots[(h0 + hh) * kTileRows + rr];
      } else {
        rec.c[0] = rec.c[1] = -1;
        rec.v[0] = rec.v[1] = 0.0;
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        av[2 * hh + u] = rec.v[u];
        if (rec.c[u] >= 0) {
          xv[2 * hh + u] = ld(X + (int64_t)rec.c[u] * kp + tx * N);
        } else {
#pragma unroll
          for (int e = 0; e < N; ++e) xv[2 * hh + u].v[e] = 0.0;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 2 * H; ++u)
#pragma unroll
      for (int e = 0; e < N; ++e) {
        double t = av[u] * xv[u].v[e];
        acc.v[e] += t;
        aabs.v[e] += fabs(t);
      }
  }
}

// at most TH threads per block; 40 registers leave room for 1536 threads per SM (six
// blocks of 256, twelve of 128).  R: records gathered per batch (spmm_row)
template <typename T, int R = 1, int TH = 256>
__global__ void __launch_bounds__(TH, 1536 / TH)
    k_cg_spmm_pq(DTiles tl, EllView<T> A, const T* __restrict__ p, T* __restrict__ q, int kp,
                 CgState s) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, A.W);
  const int tile = blockIdx.x, sd = tl.sd[tile];
  if (s.active[sd] == 0) return;  // every column of this subdomain has converged
  const int r0 = tl.r0[tile], r1 = tl.r1[tile];
  stage_tile(g, r0, r1 - r0, A, sm.slots);
  __syncthreads();
  T acc[N];
#pragma unroll
  for (int e = 0; e < N; ++e) acc[e] = T(0);
  const int rend = pack_done<T>(s, sd, kp, g.tx) ? 0 : r1 - r0;
  for (int rr = g.ty; rr < rend; rr += g.rb) {
    int64_t row = r0 + rr;
    Pack<T> qv = spmm_row<T, R>(rr, A.width[row >> 5], g.tx, sm.slots, p, kp);
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
      // exact line search along p: alpha = p.r / p.Ap (equals r.z / p.Ap in exact CG,
      // and stays a descent step after a residual replacement kept p)
      double pq = sm.sums[c];
      if (pq > 0.0)
        a = s.pr[i] / pq;
      else
        s.done[i] = 1;  // breakdown (p = 0 or indefinite): stop this column
    }
    set_coef(s.alpha, s.alpha32, i, a);
  }
}

template <bool kFloor>
__global__ void k_residual64(DTiles tl, EllView<double> A, const double* __restrict__ b,
                             const double* __restrict__ x, double* __restrict__ r, int kp,
                             int nc, int ncn, double rtol2, int first, RefineState s,
                             const double* __restrict__ anorm) {
  constexpr int N = 2;
  Geo g = geo();
  Smem<double> sm = smem_layout<double>(g, kp, A.W);
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int r0 = tl.r0[tile], r1 = tl.r1[tile];
  stage_tile(g, r0, r1 - r0, A, sm.slots);
  __syncthreads();
  double acc[N] = {0.0, 0.0}, aca[N] = {0.0, 0.0}, axx[N] = {0.0, 0.0};
  for (int rr = g.ty; rr < r1 - r0; rr += g.rb) {
    int64_t row = r0 + rr;
    Pack<double> ax, aabs;
    {
      Pack<double> xo = ld(x + row * kp + g.tx * N);
#pragma unroll
      for (int e = 0; e < N; ++e) axx[e] += xo.v[e] * xo.v[e];
    }
    if constexpr (kFloor)
      spmm_row_res(rr, A.width[row >> 5], g.tx, sm.slots, x, kp, ax, aabs);
    else
      ax = spmm_row(rr, A.width[row >> 5], g.tx, sm.slots, x, kp);
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
  __syncthreads();
  block_colsum<double, N>(g, axx, sm.red, s.part3 + (int64_t)tile * kp);
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
    __syncthreads();
  }
  sd_colsums(g, s.part3, kp, lo, hi, sm.scratch, sm.sums + kp);
  for (int c = g.tid; c < kp; c += g.nth) s.xx[sd * kp + c] = sm.sums[kp + c];
  __shared__ int cnt, nfl, nnear;
  __shared__ double bref;
  if (g.tid == 0) {
    cnt = 0;
    nfl = 0;
    nnear = 0;
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
    // || |A| |x| + |b| || <= ||A||_inf ||x|| + ||b|| (A symmetric): a column above
    // that bound's rounding level cannot stop on the floor test, so the reference
    // needs refreshing only when some open column is below it
    if (!done && !first) {
      double bnd = anorm[sd] * sqrt(s.xx[i]) + sqrt(s.obb[i]);
      if (rr <= fl2 * bnd * bnd) atomicAdd(&nnear, 1);
    }
  }
  __syncthreads();
  if (g.tid == 0) {
    s.active[sd] = cnt;
    s.nfloor[sd] = nfl;
    s.nnear[sd] = nnear;
  }
}

// ---------------------------------------------------------------------------------
// Restriction r_c = Z^T r on a row tile: aggregates are contiguous runs of rows, so the
// rows of one thread (increasing) change aggregate rarely; each thread keeps a running
// sum and adds it to the tile's slot (aggregate - aggregate of the first row) in shared
// memory when its aggregate changes.  The tile's slots then go to cpart in order.
template <typename T>
__device__ __forceinline__ T* slot_smem(const Geo& g, int kp) {
  extern __shared__ __align__(16) unsigned char raw[];
  return reinterpret_cast<T*>(raw + align16(smem_bytes<T>(g.nch, g.rb, kp, 0)));
}
size_t slot_smem_bytes(size_t base, int kp, size_t tsz) {
  return align16(base) + (size_t)kMaxSlots * kp * tsz;
}

template <typename T>
struct RestrictAcc {
  static constexpr int N = Pack<T>::N;
  int cur = -1;
  T acc[N];
  __device__ __forceinline__ void flush(T* cs, int kp, int tx) {
    if (cur >= 0)
#pragma unroll
      for (int e = 0; e < N; ++e) atomicAdd(&cs[cur * kp + tx * N + e], acc[e]);
  }
  __device__ __forceinline__ void add(T* cs, int kp, int tx, int slot, const Pack<T>& v) {
    if (slot != cur) {
      flush(cs, kp, tx);
      cur = slot;
#pragma unroll
      for (int e = 0; e < N; ++e) acc[e] = T(0);
    }
#pragma unroll
    for (int e = 0; e < N; ++e) acc[e] += v.v[e];
  }
};

template <typename T>
__device__ __forceinline__ void slots_zero(const Geo& g, T* cs, int nsl, int kp) {
  for (int i = g.tid; i < nsl * kp; i += g.nth) cs[i] = T(0);
}
template <typename T>
__device__ __forceinline__ void slots_store(const Geo& g, const T* cs, int nsl, int kp,
                                            T* dst) {
  for (int i = g.tid; i < nsl * kp; i += g.nth) dst[i] = cs[i];
}

// x = 0, r = b, the fine r.z = b.D^{-1}b, ||b||^2 and the restriction of b; the coarse
// kernel (INIT) then sets rz and the p update forms p = M^{-1} b
template <typename T>
__global__ void k_cg_init(DTiles tl, const T* __restrict__ b, T* x, T* r,
                          const T* __restrict__ dinv, int kp, int nc, int ncn, CgState s,
                          Coarse<T> co) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  const bool coarse = co.aloc != nullptr;
  T* cs = slot_smem<T>(g, kp);
  int a0 = 0, nsl = 0;
  if (coarse) {
    a0 = co.aloc[r0];
    nsl = co.aloc[r1 - 1] - a0 + 1;
    slots_zero(g, cs, nsl, kp);
    __syncthreads();
  }
  RestrictAcc<T> ra;
  T arz[N], arr[N];
#pragma unroll
  for (int e = 0; e < N; ++e) arz[e] = arr[e] = T(0);
  Pack<T> zero;
#pragma unroll
  for (int e = 0; e < N; ++e) zero.v[e] = T(0);
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> bv = ld(b + o);
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      arz[e] += bv.v[e] * (d * bv.v[e]);
      arr[e] += bv.v[e] * bv.v[e];
    }
    if (coarse) ra.add(cs, kp, g.tx, co.aloc[row] - a0, bv);
    st(x + o, zero);
    st(r + o, bv);
  }
  if (coarse) {
    ra.flush(cs, kp, g.tx);
    __syncthreads();
    slots_store(g, cs, nsl, kp, co.cpart + co.toff[tile] * kp);
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
    s.rzf[i] = sm.sums[c];
    s.bb[i] = (c < ncn) ? bref : bb;
    s.rr[i] = bb;
    s.done[i] = (c >= nc || !(bb > 0.0)) ? 1 : 0;
    set_coef(s.alpha, s.alpha32, i, 0.0);
    set_coef(s.beta, s.beta32, i, 0.0);
    set_coef(s.gam, s.gam32, i, 1.0);
  }
  if (g.tid == 0) s.iters[sd] = 0;
  __syncthreads();
  count_active(g, s.done, sd, kp, s.active);
}

// x += alpha p, r -= alpha q; ||r||^2, the fine r.z = r.D^{-1}r and the restriction of
// the new r; the coarse kernel (STEP) completes r.M^{-1}r, beta and the done flags.
// 48 registers (binary32) leave room for five blocks per SM; six cost spills.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 4)
    k_cg_update_xr(DTiles tl, T* x, T* r, const T* __restrict__ p, const T* __restrict__ q,
                   const T* __restrict__ dinv, int kp, CgState s, Coarse<T> co) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  if (s.active[sd] == 0) return;
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  const bool coarse = co.aloc != nullptr;
  T* cs = slot_smem<T>(g, kp);
  int a0 = 0, nsl = 0;
  if (coarse) {
    a0 = co.aloc[r0];
    nsl = co.aloc[r1 - 1] - a0 + 1;
    slots_zero(g, cs, nsl, kp);
    __syncthreads();
  }
  RestrictAcc<T> ra;
  const int64_t rend = pack_done<T>(s, sd, kp, g.tx) ? r0 : r1;
  const Pack<T> alp = coef_pack<T>(s.alpha, s.alpha32, sd, kp, g.tx);
  T al[N];
#pragma unroll
  for (int e = 0; e < N; ++e) al[e] = alp.v[e];
  T arr[N], arz[N];
#pragma unroll
  for (int e = 0; e < N; ++e) arr[e] = arz[e] = T(0);
  for (int64_t row = r0 + g.ty; row < rend; row += g.rb) {
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
    if (coarse) ra.add(cs, kp, g.tx, co.aloc[row] - a0, rv);
    st(x + o, xv);
    st(r + o, rv);
  }
  if (coarse) {
    ra.flush(cs, kp, g.tx);
    __syncthreads();
    slots_store(g, cs, nsl, kp, co.cpart + co.toff[tile] * kp);
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
    s.rr[i] = sm.sums[c];
    s.rzf[i] = sm.sums[kp + c];
  }
}

constexpr int kCoarseCols = 16;
enum { kCoarseInit = 0, kCoarseStep = 1, kCoarseReplace = 2 };

// The last block of a subdomain in the coarse kernels: r.M^{-1}r = fine part + the
// nrb row blocks' parts of r_c.y_c (in order); mode STEP: the convergence test on the
// recursive residual, beta and gam, the work counts (cw: columns per chunk, each open
// chunk reads E^{-1} once) and the active count; INIT / REPLACE: rz only.
template <typename T>
__device__ void coarse_finish(const Geo& g, const DTiles& tl, int sd, int kp, int cw, int nrb,
                              double tol2, int mode, CgState& s, const Coarse<T>& co) {
  constexpr int PN = Pack<T>::N;
  const int nchunk = (kp + cw - 1) / cw;
  // the subdomain's columns: open packs before the update (the sparse product and the
  // x/r update of this step worked on them), the test and beta, open packs after
  __shared__ int open_pre, open_post, chunks_open;
  const bool count = s.work && mode == kCoarseStep;
  if (g.tid == 0) open_pre = open_post = chunks_open = 0;
  __syncthreads();
  if (count) {
    for (int pk = g.tid; pk * PN < kp; pk += g.nth) {
      bool open = false;
      for (int e = 0; e < PN; ++e) open = open || !s.done[sd * kp + pk * PN + e];
      if (open) atomicAdd(&open_pre, 1);
    }
    for (int ch = g.tid; ch < nchunk; ch += g.nth) {
      bool open = false;
      for (int j = 0; j < cw && ch * cw + j < kp; ++j) open = open || !s.done[sd * kp + ch * cw + j];
      if (open) atomicAdd(&chunks_open, 1);
    }
  }
  __syncthreads();
  for (int c = g.tid; c < kp; c += g.nth) {
    const int i = sd * kp + c;
    double cd = 0.0;
    if (co.dpart)
      for (int r = 0; r < nrb; ++r) cd += __ldcg(co.dpart + ((int64_t)sd * nrb + r) * kp + c);
    const double rzn = s.rzf[i] + cd;
    if (mode == kCoarseStep) {
      double be = 0.0;
      if (!s.done[i]) {
        if (s.rr[i] <= tol2 * s.bb[i] || !(s.rz[i] > 0.0)) {
          s.done[i] = 1;
        } else {
          be = rzn / s.rz[i];
          s.rz[i] = rzn;
        }
      }
      set_coef(s.beta, s.beta32, i, be);
      set_coef(s.gam, s.gam32, i, 1.0);
    } else {
      s.rz[i] = rzn;
    }
  }
  if (mode != kCoarseStep) return;
  __syncthreads();
  if (count) {
    for (int pk = g.tid; pk * PN < kp; pk += g.nth) {
      bool open = false;
      for (int e = 0; e < PN; ++e) open = open || !s.done[sd * kp + pk * PN + e];
      if (open) atomicAdd(&open_post, 1);
    }
    __syncthreads();
    if (g.tid == 0) {
      // work counts of the algorithmic-bytes model
      const int nsd = tl.n_sd;
      const unsigned long long rows = (unsigned long long)s.sd_rows[sd];
      const unsigned long long nc = co.aloc ? (unsigned long long)co.nca[sd] : 0ull;
      atomicAdd(s.work + sd, (unsigned long long)s.sd_nnz[sd]);
      atomicAdd(s.work + nsd + sd, (unsigned long long)open_pre * rows);
      atomicAdd(s.work + 2 * nsd + sd, (unsigned long long)open_post * rows);
      if (nc) atomicAdd(s.work + 3 * nsd + sd, (unsigned long long)chunks_open * nc * nc);
    }
  }
  count_active(g, s.done, sd, kp, s.active);
  if (g.tid == 0 && s.active[sd] > 0) s.iters[sd] += 1;
}

// Coarse level of one subdomain in SIMT arithmetic (grid: x = row block x column chunk,
// y = subdomain).  Block (rb, chunk) forms r_c = Z^T r for the chunk's kCoarseCols
// columns from the tile partials, then rows [rb R, (rb + 1) R) of y_c = E^{-1} r_c
// (stored for the p update), R = kCoarseThreads kCoarseRpt with kCoarseRpt rows per
// thread (1 up to 256 aggregates, else 2), and their part of r_c.y_c.  The last block
// of the subdomain (atomic ticket) adds the parts in row-block order, r.M^{-1}r = fine
// part + r_c.y_c, and in mode STEP takes the convergence test on the recursive residual
// and beta = (r.z)_new / (r.z)_old; INIT / REPLACE: rz only (beta and gam come from the
// init / replacement kernel).  Without a coarse level y_c = 0.  The blocks of one row
// block are adjacent in the grid, so the chunks read its E^{-1} rows from L2 after the
// first.
constexpr int kCoarseThreads = 256;
constexpr size_t kCoarseRedBytes = sizeof(double) * (kCoarseThreads / 32) * kCoarseCols;
template <typename T, int kCoarseRpt>  // rows of y_c per thread
__global__ void __launch_bounds__(kCoarseThreads)
    k_cg_coarse(DTiles tl, int kp, double tol2, int mode, CgState s, Coarse<T> co) {
  constexpr int kCoarseRows = kCoarseThreads * kCoarseRpt;
  constexpr int CW = kCoarseCols;
  constexpr int PN = Pack<T>::N;
  Geo g = geo();
  extern __shared__ __align__(16) unsigned char raw[];
  T* rc = reinterpret_cast<T*>(raw);  // round_up(n, 8) x CW
  // rc holds round_up(n_max, 8) rows (the product reads whole groups of 8)
  const int n_max8 = co.aloc ? (co.n_max + 7) & ~7 : 0;
  double* red = reinterpret_cast<double*>(raw + align16(sizeof(T) * n_max8 * CW));
  const int sd = blockIdx.y;
  const int nchunk = (kp + CW - 1) / CW;
  const int chunk = blockIdx.x % nchunk, rbk = blockIdx.x / nchunk;
  const int nrb = gridDim.x / nchunk;
  const int c0 = chunk * CW, ncol = min(CW, kp - c0);
  const int cw = CW;
  if (s.active[sd] == 0) return;
  // a chunk whose columns have all converged needs no coarse product
  bool chunk_open = false;
  for (int j = 0; j < ncol; ++j) chunk_open = chunk_open || !s.done[sd * kp + c0 + j];
  const int n = (co.aloc && chunk_open) ? co.nca[sd] : 0;
  const int a_lo = rbk * kCoarseRows, a_hi = min(n, a_lo + kCoarseRows);
  double dl[CW];
#pragma unroll
  for (int j = 0; j < CW; ++j) dl[j] = 0.0;
  if (a_lo < n) {
    const int a0 = co.aoff[sd];
    // r_c = Z^T r: one (aggregate, pack) pair per thread step, summed over the tiles
    // holding the aggregate (kp and c0 are multiples of the pack width).  Rows
    // n .. round_up(n, 8) are zero: the product runs in steps of 8.
    const int n8 = (n + 7) & ~7, cwp = CW / PN;
    for (int idx = g.tid; idx < n8 * cwp; idx += g.nth) {
      const int a = idx / cwp, pk = idx - a * cwp;
      Pack<T> v;
#pragma unroll
      for (int e = 0; e < PN; ++e) v.v[e] = T(0);
      if (a < n && pk * PN < ncol) {
        const int ga = a0 + a;
        const int t0 = co.tfirst[ga], tn = co.tcount[ga];
        for (int t = t0; t < t0 + tn; ++t) {
          const int slot = a - co.aloc[tl.r0[t]];
          Pack<T> pv = ld(co.cpart + (co.toff[t] + slot) * kp + c0 + pk * PN);
#pragma unroll
          for (int e = 0; e < PN; ++e) v.v[e] += pv.v[e];
        }
      }
      st(rc + a * CW + pk * PN, v);
    }
    __syncthreads();
    // rows a_lo + tid + kCoarseThreads i, i < kCoarseRpt, one thread each
    if (a_lo + g.tid < a_hi) {
      // E^{-1} is symmetric: row a is read as column a, coalesced across the block;
      // each element feeds the CW multiply-adds of the chunk, the r_c pieces (broadcast
      // shared loads) feed the kCoarseRpt rows of the thread, and eight columns of
      // loads are issued before their multiply-adds
      const T* Eb = co.einv + co.eoff[sd];
      int ra[kCoarseRpt];
      bool rv[kCoarseRpt];
#pragma unroll
      for (int i = 0; i < kCoarseRpt; ++i) {
        ra[i] = a_lo + g.tid + kCoarseThreads * i;
        rv[i] = ra[i] < a_hi;
      }
      T acc[kCoarseRpt][CW];
#pragma unroll
      for (int i = 0; i < kCoarseRpt; ++i)
#pragma unroll
        for (int j = 0; j < CW; ++j) acc[i][j] = T(0);
      for (int b0 = 0; b0 < n; b0 += 8) {
        T e[8][kCoarseRpt];
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
          for (int i = 0; i < kCoarseRpt; ++i)
            e[u][i] = (b0 + u < n && rv[i]) ? Eb[(int64_t)(b0 + u) * n + ra[i]] : T(0);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const T* rb = rc + (b0 + u) * CW;
#pragma unroll
          for (int h = 0; h < CW; h += PN) {
            Pack<T> xv = ld(rb + h);
#pragma unroll
            for (int i = 0; i < kCoarseRpt; ++i)
#pragma unroll
              for (int e2 = 0; e2 < PN; ++e2) acc[i][h + e2] += e[u][i] * xv.v[e2];
          }
        }
      }
#pragma unroll
      for (int i = 0; i < kCoarseRpt; ++i) {
        if (!rv[i]) continue;
        T* yo = co.yc + (int64_t)(a0 + ra[i]) * kp + c0;
#pragma unroll
        for (int j = 0; j < CW; ++j) {
          if (j < ncol) yo[j] = acc[i][j];
          dl[j] += (double)acc[i][j] * (double)rc[ra[i] * CW + j];
        }
      }
    }
  }
  // this block's part of r_c.y_c per column: rows summed within each warp (fixed
  // shuffle tree), then the warps in order
  {
    const int lane = g.tid & 31, wid = g.tid >> 5;
#pragma unroll
    for (int j = 0; j < CW; ++j) {
      double v = dl[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wid * CW + j] = v;
    }
    __syncthreads();
    if (g.tid < ncol && co.dpart) {
      double t = 0.0;
      for (int w = 0; w < g.nth / 32; ++w) t += red[w * CW + g.tid];
      co.dpart[((int64_t)sd * nrb + rbk) * kp + c0 + g.tid] = t;
    }
  }
  if (!last_block(g, s.counter, sd, gridDim.x)) return;
  coarse_finish<T>(g, tl, sd, kp, cw, nrb, tol2, mode, s, co);
}

// The coarse product of the binary32 path on the tensor cores, y_c = E^{-1} r_c for
// every column (NP = kp rounded up to 16, at most 128), in two kernels.
// k_coarse_rc_pack forms r_c = Z^T r per 32-aggregate block from the tile partials and
// stores it as bf16 high and low planes in the K-major operand layout (row = column of
// r_c).  k_cg_coarse_tc then runs block (m, sd): rows [128 m, 128 m + 128) of y_c as
// one tcgen05 MMA tile with its FP32 accumulator in TMEM, A = E^{-1} (launch_coarse_tc_
// pack) and B = r_c streamed through kTcStages shared-memory stages by cp.async, and
// three products hi.hi + hi.lo + lo.hi per block (about 16 significant bits of each
// factor; the dropped lo.lo term is below 2^-16 of a product, under the binary32
// accumulation error of a 1,000-term sum).  One thread issues the MMAs and commits them
// to the stage's mbarrier; a stage is refilled once its MMAs are done, and every wait
// is bounded (a timeout sets co.tc_err and ends the block after its MMAs drain).  The
// epilogue reads the accumulator rows (tcgen05.ld, one row per thread), stores y_c and
// this block's part of r_c.y_c; the last block of the subdomain finishes as in
// k_cg_coarse.
constexpr int kTcThreads = 128;  // one thread per accumulator row (TMEM lane)
constexpr int kTcStages = 4;
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}
// r_c pack (aggregate a of subdomain sd, columns 4 pk .. 4 pk + 3), zero outside n, kp
__device__ __forceinline__ Pack<float> restrict_pack(const DTiles& tl, const Coarse<float>& co,
                                                     int a0, int n, int kp, int a, int pk) {
  Pack<float> v;
#pragma unroll
  for (int e = 0; e < 4; ++e) v.v[e] = 0.0f;
  if (a < n && 4 * pk < kp) {
    const int ga = a0 + a;
    const int t0 = co.tfirst[ga], tn = co.tcount[ga];
    for (int t = t0; t < t0 + tn; ++t) {
      const int slot = a - co.aloc[tl.r0[t]];
      const Pack<float> pv = ld(co.cpart + (co.toff[t] + slot) * kp + 4 * pk);
#pragma unroll
      for (int e = 0; e < 4; ++e) v.v[e] += pv.v[e];
    }
  }
  return v;
}
// an open column of subdomain sd (the coarse product is skipped without one)
__device__ __forceinline__ bool any_open_column(const CgState& s, int sd, int kp) {
  bool open = false;
  for (int c = 0; c < kp; ++c) open = open || !s.done[sd * kp + c];
  return open;
}

// block (kb, sd): r_c of aggregates 32 kb .. 32 kb + 31 into co.rcb at co.rcb_off[sd] + kb
__global__ void __launch_bounds__(kTcThreads)
    k_coarse_rc_pack(DTiles tl, int kp, int NP, CgState s, Coarse<float> co) {
  const int sd = blockIdx.y, kb = blockIdx.x;
  if (s.active[sd] == 0 || !any_open_column(s, sd, kp)) return;
  const int n = co.nca[sd];
  if (kb * tc::kKB >= n) return;
  const int a0 = co.aoff[sd];
  __nv_bfloat16* bh = co.rcb + (co.rcb_off[sd] + kb) * (int64_t)(2 * NP * tc::kKB);
  __nv_bfloat16* bl = bh + NP * tc::kKB;
  const int npk = NP / 4;
  for (int idx = threadIdx.x; idx < tc::kKB * npk; idx += blockDim.x) {
    const int k = idx / npk, pk = idx - k * npk;
    const Pack<float> v = restrict_pack(tl, co, a0, n, kp, kb * tc::kKB + k, pk);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      __nv_bfloat16 h, l;
      split_bf16(v.v[e], h, l);
      const uint32_t o = tc::kmajor(4 * pk + e, k) >> 1;
      bh[o] = h;
      bl[o] = l;
    }
  }
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}

__global__ void __launch_bounds__(kTcThreads)
    k_cg_coarse_tc(DTiles tl, int kp, int NP, double tol2, int mode, CgState s,
                   Coarse<float> co) {
  constexpr int KB = tc::kKB;
  constexpr int A_PLANE = kCoarseTcM * KB * 2;  // bytes
  extern __shared__ __align__(128) unsigned char smem[];
  const int B_PLANE = NP * KB * 2;
  const int STAGE = 2 * A_PLANE + 2 * B_PLANE;  // A hi, A lo, B hi, B lo
  double* red = reinterpret_cast<double*>(smem + kTcStages * STAGE);  // 4 warps x NP
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar[kTcStages];
  __shared__ int s_ok;
  Geo g = geo();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int sd = blockIdx.y, mt = blockIdx.x, nmt = gridDim.x;
  if (s.active[sd] == 0) return;
  const int n = (co.aloc && any_open_column(s, sd, kp)) ? co.nca[sd] : 0;
  const int a_lo = mt * kCoarseTcM;
  for (int c = tid; c < 4 * NP; c += kTcThreads) red[c] = 0.0;
  if (a_lo < n) {
    const int a0 = co.aoff[sd];
    const int nkb = (n + KB - 1) / KB;
    const unsigned char* Ag =
        reinterpret_cast<const unsigned char*>(co.etc + (co.etc_off[sd] + (int64_t)mt * nkb) * 1024);
    const unsigned char* Bg =
        reinterpret_cast<const unsigned char*>(co.rcb + co.rcb_off[sd] * (int64_t)(2 * NP * KB));
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    // block kb's operands into stage stg: 16-byte asynchronous copies, one group
    auto issue = [&](int kb, int stg) {
      if (kb < nkb) {
        const uint32_t sa = s0 + (uint32_t)(stg * STAGE);
        const unsigned char* ga = Ag + (int64_t)kb * (2 * A_PLANE);
        for (int i = tid; i < 2 * A_PLANE / 16; i += kTcThreads)
          cp_async16(sa + 16 * i, ga + 16 * i);
        const unsigned char* gb = Bg + (int64_t)kb * (2 * B_PLANE);
        for (int i = tid; i < 2 * B_PLANE / 16; i += kTcThreads)
          cp_async16(sa + 2 * A_PLANE + 16 * i, gb + 16 * i);
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    uint32_t ncols = 32;
    while (ncols < (uint32_t)NP) ncols <<= 1;
    if (warp == 0) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                   ::"r"(dst), "r"(ncols));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
      for (int q = 0; q < kTcStages; ++q) {
        const uint32_t mq = (uint32_t)__cvta_generic_to_shared(&mbar[q]);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mq), "r"(1));
      }
      asm volatile("fence.mbarrier_init.release.cluster;");
      s_ok = 1;
    }
    for (int q = 0; q < kTcStages - 1; ++q) issue(q, q);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    const uint32_t idesc = tc::instr_desc(kCoarseTcM, NP);
    uint32_t ph = 0;  // bit q: parity of the next completion of stage q's mbarrier
    bool ok = true;
    int last = -1;  // stage of the last committed MMAs
    for (int kb = 0; kb < nkb && ok; ++kb) {
      const int stg = kb % kTcStages;
      // block kb's copies are done (at most kTcStages - 2 newer groups pending)
      asm volatile("cp.async.wait_group %0;" ::"n"(kTcStages - 2) : "memory");
      asm volatile("fence.proxy.async.shared::cta;");
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;");
      if (tid == 0) {
        const uint32_t sa = s0 + (uint32_t)(stg * STAGE);
        const int pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};  // hi.hi, hi.lo, lo.hi
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
          for (int ks = 0; ks < KB / 16; ++ks) {
            const uint64_t ad =
                tc::smem_desc(sa + (uint32_t)(pa[q] * A_PLANE + ks * 256), 128, (KB / 8) * 128);
            const uint64_t bd = tc::smem_desc(
                sa + (uint32_t)(2 * A_PLANE + pb[q] * B_PLANE + ks * 256), 128, (KB / 8) * 128);
            const uint32_t en = (kb == 0 && q == 0 && ks == 0) ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tbase),
                "l"(ad), "l"(bd), "r"(idesc), "r"(en));
          }
        const uint32_t mq = (uint32_t)__cvta_generic_to_shared(&mbar[stg]);
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                mq));
      }
      __syncwarp();
      last = stg;
      // refill the stage of block kb - 1 (block kb + kTcStages - 1) once its MMAs are done
      if (kb >= 1) {
        const int ps = (kb - 1) % kTcStages;
        const uint32_t mq = (uint32_t)__cvta_generic_to_shared(&mbar[ps]);
        if (tc::mbar_wait(mq, (ph >> ps) & 1u, co.tc_budget)) {
          ph ^= 1u << ps;
        } else {
          atomicExch(co.tc_err, 1);
          s_ok = 0;
        }
      }
      issue(kb + kTcStages - 1, (kb + kTcStages - 1) % kTcStages);
      __syncthreads();
      ok = s_ok != 0;
    }
    // the last block's MMAs (the others were waited for before their refills)
    if (ok && last >= 0) {
      const uint32_t mq = (uint32_t)__cvta_generic_to_shared(&mbar[last]);
      if (tc::mbar_wait(mq, (ph >> last) & 1u, co.tc_budget)) {
        ph ^= 1u << last;
      } else {
        atomicExch(co.tc_err, 1);
        s_ok = 0;
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    ok = s_ok != 0;
    if (ok) {
      // epilogue: row a of the tile is TMEM lane a = thread tid; eight columns per load
      const int a = a_lo + tid;
      for (int c0 = 0; c0 < NP; c0 += 8) {
        uint32_t r[8];
        const uint32_t ta = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
              "=r"(r[6]), "=r"(r[7])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        double dl[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) dl[e] = 0.0;
        if (a < n) {
          float* yo = co.yc + (int64_t)(a0 + a) * kp;
#pragma unroll
          for (int h = 0; h < 8; h += 4) {
            const Pack<float> rp = restrict_pack(tl, co, a0, n, kp, a, (c0 + h) / 4);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c = c0 + h + e;
              const float y = __uint_as_float(r[h + e]);
              if (c < kp) yo[c] = y;
              dl[h + e] = (double)y * (double)rp.v[e];
            }
          }
        }
        // rows summed within the warp (fixed shuffle tree), one partial per warp
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          double v = dl[e];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
          if (lane == 0) red[warp * NP + c0 + e] = v;
        }
      }
    } else if (last >= 0) {
      // a wait ran out: wait once more (bounded) for the stages' pending MMAs, so that
      // they drain before the TMEM is released
      for (int q = 0; q < kTcStages; ++q) {
        const uint32_t mq = (uint32_t)__cvta_generic_to_shared(&mbar[q]);
        tc::mbar_wait(mq, (ph >> q) & 1u, co.tc_budget);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                   "r"(ncols));
  }
  __syncthreads();
  // this block's part of r_c.y_c per column, warps in order
  for (int c = tid; c < kp; c += kTcThreads) {
    double t = 0.0;
    for (int w = 0; w < kTcThreads / 32; ++w) t += red[w * NP + c];
    co.dpart[((int64_t)sd * nmt + mt) * kp + c] = t;
  }
  if (!last_block(g, s.counter, sd, nmt)) return;
  coarse_finish<float>(g, tl, sd, kp, kp, nmt, tol2, mode, s, co);
}

// p = gam (D^{-1} r + Z y_c) + beta p (p is not read where beta = 0), and p.r of the
// new direction for the next step length
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 6 : 4)
    k_cg_update_p(DTiles tl, const T* __restrict__ r, T* p, const T* __restrict__ dinv, int kp,
                  CgState s, Coarse<T> co) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  if (s.active[sd] == 0) return;
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  const int64_t rend = pack_done<T>(s, sd, kp, g.tx) ? r0 : r1;
  const bool coarse = co.aloc != nullptr;
  const int64_t a0 = coarse ? co.aoff[sd] : 0;
  const Pack<T> bep = coef_pack<T>(s.beta, s.beta32, sd, kp, g.tx);
  const Pack<T> gap = coef_pack<T>(s.gam, s.gam32, sd, kp, g.tx);
  T be[N], ga[N];
  bool needp = false;
#pragma unroll
  for (int e = 0; e < N; ++e) {
    be[e] = bep.v[e];
    ga[e] = gap.v[e];
    needp = needp || be[e] != T(0);
  }
  T apr[N];
#pragma unroll
  for (int e = 0; e < N; ++e) apr[e] = T(0);
  for (int64_t row = r0 + g.ty; row < rend; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> rv = ld(r + o), pv, yv;
    if (needp) pv = ld(p + o);
    if (coarse) yv = ld(co.yc + (a0 + co.aloc[row]) * kp + g.tx * N);
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      T z = d * rv.v[e];
      if (coarse) z += yv.v[e];
      T v = ga[e] * z;
      if (be[e] != T(0)) v += be[e] * pv.v[e];
      pv.v[e] = v;
      apr[e] += v * rv.v[e];
    }
    st(p + o, pv);
  }
  block_colsum<T, N>(g, apr, sm.red, s.part1 + (int64_t)tile * kp);
  int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part1, kp, lo, hi, sm.scratch, sm.sums);
  for (int c = g.tid; c < kp; c += g.nth) s.pr[sd * kp + c] = sm.sums[c];
}

// out[0] = sum of active, out[1] = sum of second (if not null)
__global__ void k_count_active(int n_sd, const int* active, const int* second, int* out) {
  __shared__ int tot, tot2;
  if (threadIdx.x == 0) tot = tot2 = 0;
  __syncthreads();
  int a = 0, b = 0;
  for (int i = threadIdx.x; i < n_sd; i += blockDim.x) {
    a += active[i];
    if (second) b += second[i];
  }
  atomicAdd(&tot, a);
  atomicAdd(&tot2, b);
  __syncthreads();
  if (threadIdx.x == 0) {
    out[0] = tot;
    out[1] = tot2;
  }
}


__global__ void k_zero_rows(DTiles tl, double* x, int kp) {
  Geo g = geo();
  int tile = blockIdx.x;
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb)
    for (int c = g.tx; c < kp; c += g.nch) x[row * kp + c] = 0.0;
}

// residual replacement: rT = (T) r64 (the true residual), the fine r.z and the
// restriction of it, each column's done flag from the binary64 convergence test
// (scale == 0).  Columns the recursion had declared converged but the binary64 test
// reopens, and columns whose true residual norm exceeds drift x the recursive one,
// restart from p = M^{-1} r (their stored direction belongs to a much smaller
// residual: gam = 1, beta = 0); the others keep p (gam = 0, beta = 1).  The coarse
// kernel (REPLACE) then sets rz and the p update applies gam and beta.
template <typename T>
__global__ void k_cg_replace(DTiles tl, const double* __restrict__ r64, T* __restrict__ rT,
                             const T* __restrict__ dinv, int kp, double drift2, CgState s,
                             RefineState rs, Coarse<T> co) {
  constexpr int N = Pack<T>::N;
  Geo g = geo();
  Smem<T> sm = smem_layout<T>(g, kp, 0);
  int tile = blockIdx.x, sd = tl.sd[tile];
  int r0 = tl.r0[tile], r1 = tl.r1[tile];
  const bool coarse = co.aloc != nullptr;
  T* cs = slot_smem<T>(g, kp);
  int a0 = 0, nsl = 0;
  if (coarse) {
    a0 = co.aloc[r0];
    nsl = co.aloc[r1 - 1] - a0 + 1;
    slots_zero(g, cs, nsl, kp);
    __syncthreads();
  }
  RestrictAcc<T> ra;
  T arz[N];
#pragma unroll
  for (int e = 0; e < N; ++e) arz[e] = T(0);
  for (int64_t row = r0 + g.ty; row < r1; row += g.rb) {
    int64_t o = row * kp + g.tx * N;
    Pack<T> rv;
    T d = dinv[row];
#pragma unroll
    for (int e = 0; e < N; ++e) {
      rv.v[e] = (T)r64[o + e];
      arz[e] += rv.v[e] * (d * rv.v[e]);
    }
    if (coarse) ra.add(cs, kp, g.tx, co.aloc[row] - a0, rv);
    st(rT + o, rv);
  }
  if (coarse) {
    ra.flush(cs, kp, g.tx);
    __syncthreads();
    slots_store(g, cs, nsl, kp, co.cpart + co.toff[tile] * kp);
  }
  block_colsum<T, N>(g, arz, sm.red, s.part1 + (int64_t)tile * kp);
  int lo = tl.lo[sd], hi = tl.hi[sd];
  if (!last_block(g, s.counter, sd, hi - lo)) return;
  sd_colsums(g, s.part1, kp, lo, hi, sm.scratch, sm.sums);
  for (int c = g.tid; c < kp; c += g.nth) {
    int i = sd * kp + c;
    // reopened, or the recursion drifted from the true residual (a stale direction
    // would make the next step length meaningless)
    bool restart = rs.scale[i] != 0.0 && (s.done[i] || rs.orr[i] > drift2 * s.rr[i]);
    bool done = rs.scale[i] == 0.0;
    s.rzf[i] = sm.sums[c];
    s.bb[i] = rs.obb[i];
    s.done[i] = done ? 1 : 0;
    set_coef(s.alpha, s.alpha32, i, 0.0);
    set_coef(s.beta, s.beta32, i, (done || restart) ? 0.0 : 1.0);
    set_coef(s.gam, s.gam32, i, (done || restart) ? 1.0 : 0.0);
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

// per subdomain: max over its rows of sum_j |a_ij| (nonnegative doubles order like
// their bit patterns, so an integer atomicMax is exact); out zeroed by the caller
__global__ void k_row_abs_max(DTiles tl, EllView<double> A, unsigned long long* out) {
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int64_t row = tl.r0[tile] + (int64_t)threadIdx.x;
  double sum = 0.0;
  if (row < tl.r1[tile]) {
    const int w = A.width[row >> 5];
    for (int j = 0; j < w; ++j) {
      int64_t at = ell_at(row, j, A.W);
      if (A.col[at] >= 0) sum += fabs(A.val[at]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) sum = fmax(sum, __shfl_xor_sync(0xFFFFFFFFu, sum, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out + sd, (unsigned long long)__double_as_longlong(sum));
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
dim3 block_of(int kp, int threads = 256) {
  int nch = kp / Pack<T>::N;
  int rb = threads / nch;
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
size_t slot_kernel_smem(dim3 bl, int kp) {
  return slot_smem_bytes(smem_bytes<T>(bl.x, bl.y, kp, 0), kp, sizeof(T));
}

template <typename T>
void launch_coarse_then_p(const DTiles& tiles, int n_sd, const T* r, T* p, const T* dinv,
                          int kp, double tol2, int mode, const CgState& s, const Coarse<T>& co,
                          cudaStream_t st, const cudaEvent_t* ev_mid) {
  static bool attr = false;
  if (!attr) {
    const int mx = (int)(align16(sizeof(T) * kMaxAgg * kCoarseCols) + kCoarseRedBytes);
    cudaFuncSetAttribute((const void*)k_cg_coarse<T, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute((const void*)k_cg_coarse<T, 2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    attr = true;
  }
  const int n_max = co.aloc ? co.n_max : 0;
  dim3 bl = block_of<T>(kp);
  count_launch(2);
  if constexpr (sizeof(T) == 4) {
    if (co.etc) {
      // tensor-core product: one block per 128 rows of y_c and subdomain, every column
      const int NP = (kp + 15) & ~15;
      const size_t smt = (size_t)kTcStages * (2 * (kCoarseTcM * tc::kKB * 2) +
                                              2 * NP * tc::kKB * 2) +
                         sizeof(double) * 4 * NP;
      static bool attr_tc = false;
      if (!attr_tc) {
        cudaFuncSetAttribute((const void*)k_cg_coarse_tc,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_tc = true;
      }
      const int nmt = std::max(1, (n_max + kCoarseTcM - 1) / kCoarseTcM);
      const int nkb = std::max(1, (n_max + tc::kKB - 1) / tc::kKB);
      count_launch();
      k_coarse_rc_pack<<<dim3(nkb, n_sd), kTcThreads, 0, st>>>(tiles, kp, NP, s, co);
      k_cg_coarse_tc<<<dim3(nmt, n_sd), kTcThreads, smt, st>>>(tiles, kp, NP, tol2, mode, s,
                                                                co);
      if (ev_mid) cudaEventRecord(*ev_mid, st);
      k_cg_update_p<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, 0), st>>>(tiles, r, p,
                                                                             dinv, kp, s, co);
      return;
    }
  }
  const size_t sm = align16(sizeof(T) * ((n_max + 7) & ~7) * kCoarseCols) + kCoarseRedBytes;
  const int rows = n_max > kCoarseThreads ? 2 * kCoarseThreads : kCoarseThreads;
  const int nrb = std::max(1, (n_max + rows - 1) / rows);
  const int nchunk = (kp + kCoarseCols - 1) / kCoarseCols;
  dim3 grid(nrb * nchunk, n_sd);
  if (rows > kCoarseThreads)
    k_cg_coarse<T, 2><<<grid, kCoarseThreads, sm, st>>>(tiles, kp, tol2, mode, s, co);
  else
    k_cg_coarse<T, 1><<<grid, kCoarseThreads, sm, st>>>(tiles, kp, tol2, mode, s, co);
  if (ev_mid) cudaEventRecord(*ev_mid, st);
  k_cg_update_p<T><<<tiles.n, bl, smem_bytes<T>(bl.x, bl.y, kp, 0), st>>>(tiles, r, p, dinv,
                                                                         kp, s, co);
}

template <typename T>
void launch_cg_init(const DTiles& tiles, const T* b, T* x, T* r, T* p, const T* dinv,
                    int kp, int nc, int ncn, const CgState& s, const Coarse<T>& co,
                    cudaStream_t st) {
  if (tiles.n <= 0) return;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cg_init<T>);
    attr = true;
  }
  dim3 bl = block_of<T>(kp);
  count_launch();
  k_cg_init<T><<<tiles.n, bl, slot_kernel_smem<T>(bl, kp), st>>>(tiles, b, x, r, dinv, kp, nc,
                                                                  ncn, s, co);
  launch_coarse_then_p<T>(tiles, tiles.n_sd, r, p, dinv, kp, 0.0, kCoarseInit, s, co, st,
                          nullptr);
}

// ---- autotuner of the sparse product: four launch configurations of k_cg_spmm_pq
// (1 or 2 records per gather batch, blocks of 256 or 128 threads), timed on the first
// product of each (precision, column count, slot width) the process meets, the fastest
// kept for the rest of the process.  The product is a pure function of p (q, its
// column sums and the step length are rewritten), so timing it on live data changes
// no result.
constexpr int kSpmmVariants = 4;
template <typename T>
void launch_spmm_pq_variant(int v, const DTiles& tiles, const EllView<T>& A, const T* p, T* q,
                            int kp, const CgState& s, cudaStream_t st) {
  const int th = (v & 2) ? 128 : 256;
  dim3 bl = block_of<T>(kp, th);
  const size_t sm = smem_bytes<T>(bl.x, bl.y, kp, A.W);
  switch (v) {
    case 0: k_cg_spmm_pq<T, 1, 256><<<tiles.n, bl, sm, st>>>(tiles, A, p, q, kp, s); break;
    case 1: k_cg_spmm_pq<T, 2, 256><<<tiles.n, bl, sm, st>>>(tiles, A, p, q, kp, s); break;
    case 2: k_cg_spmm_pq<T, 1, 128><<<tiles.n, bl, sm, st>>>(tiles, A, p, q, kp, s); break;
    default: k_cg_spmm_pq<T, 2, 128><<<tiles.n, bl, sm, st>>>(tiles, A, p, q, kp, s); break;
  }
}

struct TuneEntry {
  int wide, kp, W, variant;
  float ms[kSpmmVariants];
};
std::mutex g_tune_mu;
std::vector<TuneEntry> g_tune;
bool g_tune_on = true;

template <typename T>
int spmm_variant(const DTiles& tiles, const EllView<T>& A, const T* p, T* q, int kp,
                 const CgState& s, cudaStream_t st) {
  const int wide = sizeof(T) == 8 ? 1 : 0;
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& e : g_tune)
    if (e.wide == wide && e.kp == kp && e.W == A.W) return e.variant;
  if (!g_tune_on || kp / Pack<T>::N > 128) return 0;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 1, 256>);
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 2, 256>);
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 1, 128>);
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 2, 128>);
    attr = true;
  }
  TuneEntry e{wide, kp, A.W, 0, {0, 0, 0, 0}};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (int v = 0; v < kSpmmVariants; ++v) {
    launch_spmm_pq_variant<T>(v, tiles, A, p, q, kp, s, st);  // warm-up
    cudaEventRecord(a, st);
    for (int rep = 0; rep < 3; ++rep) launch_spmm_pq_variant<T>(v, tiles, A, p, q, kp, s, st);
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    e.ms[v] = t / 3.0f;
    count_launch(4);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  for (int v = 1; v < kSpmmVariants; ++v)
    if (e.ms[v] < e.ms[e.variant]) e.variant = v;
  g_tune.push_back(e);
  return e.variant;
}

template <typename T>
void launch_cg_step(const DTiles& tiles, const EllView<T>& A, T* x, T* r, T* p, T* q,
                    const T* dinv, int kp, double tol2, const CgState& s, const Coarse<T>& co,
                    cudaStream_t st, const cudaEvent_t* ev) {
  if (tiles.n <= 0) return;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 1, 256>);
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 2, 256>);
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 1, 128>);
    set_smem_attr<T>((const void*)k_cg_spmm_pq<T, 2, 128>);
    set_smem_attr<T>((const void*)k_cg_update_xr<T>);
    attr = true;
  }
  dim3 bl = block_of<T>(kp);
  const int variant = spmm_variant<T>(tiles, A, p, q, kp, s, st);
  count_launch(2);
  if (ev) cudaEventRecord(ev[0], st);
  launch_spmm_pq_variant<T>(variant, tiles, A, p, q, kp, s, st);
  if (ev) cudaEventRecord(ev[1], st);
  k_cg_update_xr<T><<<tiles.n, bl, slot_kernel_smem<T>(bl, kp), st>>>(tiles, x, r, p, q, dinv,
                                                                       kp, s, co);
  if (ev) cudaEventRecord(ev[2], st);
  launch_coarse_then_p<T>(tiles, tiles.n_sd, r, p, dinv, kp, tol2, kCoarseStep, s, co, st,
                          ev ? &ev[3] : nullptr);
  if (ev) cudaEventRecord(ev[4], st);
}

void launch_count_active(int n_sd, const int* active, int* out, cudaStream_t st,
                         const int* second) {
  count_launch();
  k_count_active<<<1, 256, 0, st>>>(n_sd, active, second, out);
}

void launch_residual64(const DTiles& tiles, const EllView<double>& A, const double* b64,
                       const double* x64, double* r64, int kp, int nc, int ncn, double rtol2,
                       int first, bool floor_ref, const double* anorm, const RefineState& s,
                       cudaStream_t st) {
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
                                                first, s, anorm);
  else
    k_residual64<false><<<tiles.n, bl, sm, st>>>(tiles, A, b64, x64, r64, kp, nc, ncn, rtol2,
                                                 first, s, anorm);
}

template <typename T>
void launch_cg_replace(const DTiles& tiles, const double* r64, T* rT, T* pT, const T* dinv,
                       int kp, double drift, const CgState& s, const RefineState& rs,
                       const Coarse<T>& co, cudaStream_t st) {
  if (tiles.n <= 0) return;
  static bool attr = false;
  if (!attr) {
    set_smem_attr<T>((const void*)k_cg_replace<T>);
    attr = true;
  }
  dim3 bl = block_of<T>(kp);
  count_launch();
  k_cg_replace<T><<<tiles.n, bl, slot_kernel_smem<T>(bl, kp), st>>>(
      tiles, r64, rT, dinv, kp, drift * drift, s, rs, co);
  launch_coarse_then_p<T>(tiles, tiles.n_sd, rT, pT, dinv, kp, 0.0, kCoarseReplace, s, co, st,
                          nullptr);
}

template <typename T>
void launch_accum_reset(const DTiles& tiles, T* xT, double* x64, int kp, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_accum_reset<T><<<tiles.n, dim3(32, 8), 0, st>>>(tiles, xT, x64, kp);
}

// out[sd] += stored entries of the rows of each tile of sd (one thread per row)
__global__ void k_count_sd_nnz(DTiles tl, EllView<double> A, unsigned long long* out) {
  const int tile = blockIdx.x, sd = tl.sd[tile];
  const int64_t row = tl.r0[tile] + (int64_t)threadIdx.x;
  unsigned long long c = 0;
  if (row < tl.r1[tile]) {
    const int w = A.width[row >> 5];
    for (int j = 0; j < w; ++j) c += A.col[ell_at(row, j, A.W)] >= 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out + sd, c);
}

void launch_count_sd_nnz(const DTiles& tiles, const EllView<double>& A, int64_t* out,
                         cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_count_sd_nnz<<<tiles.n, kTileRows, 0, st>>>(tiles, A, (unsigned long long*)out);
}

void launch_row_abs_max(const DTiles& tiles, const EllView<double>& A, double* out,
                        cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_row_abs_max<<<tiles.n, kTileRows, 0, st>>>(tiles, A, (unsigned long long*)out);
}

template <typename T>
void launch_cast(const DTiles& tiles, const double* src, T* dst, int kp, cudaStream_t st) {
  if (tiles.n <= 0) return;
  count_launch();
  k_cast<T><<<tiles.n, dim3(32, 8), 0, st>>>(tiles, src, dst, kp);
}

template void launch_cg_replace<float>(const DTiles&, const double*, float*, float*,
                                       const float*, int, double, const CgState&,
                                       const RefineState&, const Coarse<float>&, cudaStream_t);
template void launch_cg_replace<double>(const DTiles&, const double*, double*, double*,
                                        const double*, int, double, const CgState&,
                                        const RefineState&, const Coarse<double>&,
                                        cudaStream_t);
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
                                    const float*, int, int, int, const CgState&,
                                    const Coarse<float>&, cudaStream_t);
template void launch_cg_init<double>(const DTiles&, const double*, double*, double*, double*,
                                     const double*, int, int, int, const CgState&,
                                     const Coarse<double>&, cudaStream_t);
template void launch_cg_step<float>(const DTiles&, const EllView<float>&, float*, float*,
                                    float*, float*, const float*, int, double, const CgState&,
                                    const Coarse<float>&, cudaStream_t, const cudaEvent_t*);
template void launch_cg_step<double>(const DTiles&, const EllView<double>&, double*, double*,
                                     double*, double*, const double*, int, double,
                                     const CgState&, const Coarse<double>&, cudaStream_t,
                                     const cudaEvent_t*);
void autotune_enable(bool on) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune_on = on;
}

void autotune_reset() {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tune.clear();
}

int autotune_entries(int64_t* out, int max_entries) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  const int n = (int)g_tune.size();
  for (int i = 0; i < n && i < max_entries; ++i) {
    const TuneEntry& e = g_tune[i];
    int64_t* o = out + 8 * (int64_t)i;
    o[0] = e.wide;
    o[1] = e.kp;
    o[2] = e.W;
    o[3] = e.variant;
    for (int v = 0; v < kSpmmVariants; ++v) o[4 + v] = (int64_t)(1e3 * e.ms[v]);  // us
  }
  return n;
}

}  // namespace mor
