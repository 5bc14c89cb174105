// Tensor-core Grams for the mixed-precision path (Sec. 6: the H_i-orthonormalisation
// X^T H_i X, the weighted Gram G_B of Eq. (24) and the interface blocks Q_i^T A_0 Q_j of
// Eq. (23)) on tcgen05 with accumulators in TMEM.
//
// Arithmetic: every binary64 operand column c is scaled by 2^(7 - e_c), e_c the binary
// exponent of its largest entry in the block's rows, rounded to 28 bits and split into
// four integer slices, x = 2^(e_c - 7) sum_t s_t 2^(-7t) with s_0 in [-128, 128], s_t in
// [-64, 64] (t > 0).  Each slice is an integer, exact in bf16.  The products s_t s'_u of one
// slice order d = t + u (t + u <= 3, ten pairs) are summed by kind::f16 MMAs (bf16
// operands) into one FP32 accumulator per order; every product and every partial sum
// over 256 rows is an integer below 2^24, so the FP32 accumulation is exact.  Every 256
// rows the accumulators are read (tcgen05.ld), combined in binary64 with their scales
// 2^(e_i + e_j - 7(d + 2)) and added to the block's binary64 partial.  The result
// carries the slicing error only, about 2^-28 relative to the product of the column
// maxima: column by column, so columns of small norm keep their relative accuracy (the
// Gram is graded like its columns).  This is the error-free splitting of Ozaki et al.
// (Numer. Algorithms 59, 2012) with integer slices.
//
// Layout: one block of 128 threads per (batch item, row chunk); the A operand holds the
// X columns as its M = 128 rows (zero-padded), B the Y columns (N = ny rounded up to 16),
// both K-major without swizzle: 8 x 8 core matrices of 128 bytes, 128 bytes apart along K
// (leading byte offset) and 512 bytes apart along M / N (stride byte offset, K = 32 rows
// per block).  One elected thread issues the MMAs; tcgen05.commit signals an mbarrier
// whose waits are bounded (a timeout sets *err and ends the block after its MMAs drain).
#include <cuda_bf16.h>

#include <algorithm>

#include "mor_kernels.h"
#include "mor_tc.cuh"

namespace mor {
namespace {

constexpr int kKB = tc::kKB;   // rows per MMA block (two K = 16 steps)
constexpr int kNS = 4;         // slices per value
constexpr int kM = 128;        // MMA M
constexpr int kFlush = 8;      // blocks between accumulator flushes (256 rows)

using tc::instr_desc;
using tc::kmajor;
using tc::mbar_wait;
using tc::smem_desc;

// the four slices of x * 2^(7 - e) into column c, row k of the four slice planes.  The
// slicing is integer work on the bits of x (GB300's binary64 rate is low): with
// x = +-m 2^(E - 1075) (m the 53-bit significand), N = round(x 2^(28 - e)) =
// round(m / 2^sh), sh = e - 28 - E + 1075 >= 25 because |x| < 2^e; then N =
// s_0 2^21 + s_1 2^14 + s_2 2^7 + s_3 with each s_t rounded off the remainder, so
// s_0 in [-128, 128] and s_1, s_2, s_3 in [-64, 64].  Subnormals count as zero.
__device__ __forceinline__ void put_slices(__nv_bfloat16* plane, uint32_t plane_bytes, int c,
                                           int k, double x, int e) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  int n = 0;
  if (E != 0) {
    const long long m = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = (e - 28) - (E - 1075);
    const long long q = sh >= 62 ? 0 : ((m + (1LL << (sh - 1))) >> sh);
    n = b < 0 ? -(int)q : (int)q;
  }
  int sl[kNS];
  sl[0] = (n + (1 << 20)) >> 21;
  int r = n - (sl[0] << 21);
  sl[1] = (r + (1 << 13)) >> 14;
  r -= sl[1] << 14;
  sl[2] = (r + (1 << 6)) >> 7;
  sl[3] = r - (sl[2] << 7);
  const uint32_t o = kmajor(c, k);
#pragma unroll
  for (int t = 0; t < kNS; ++t) plane[(t * plane_bytes + o) >> 1] = __int2bfloat16_rn(sl[t]);
}

// binary exponent e with |x| < 2^e (the biased exponent minus 1022), 0 for zero and
// subnormal x
__device__ __forceinline__ int exponent_of(double x) {
  const int E = (int)((__double_as_longlong(x) >> 52) & 0x7FF);
  return E == 0 ? 0 : E - 1022;
}

// Rows of item b: [rlo[b], rhi[b]), split into S chunks (one block each); rows are rows
// of X and Y (gather = false), or entries of a pair list: X row xrow[e] scaled by w[e],
// Y row yrow[e].
template <bool kGather>
__global__ void __launch_bounds__(128)
    k_tc_gram(const int64_t* __restrict__ rlo, const int64_t* __restrict__ rhi, int S,
              const double* __restrict__ X, int ldx,
              int nx, const double* __restrict__ Y, int ldy, int ny, int NP,
              const int32_t* __restrict__ xrow, const int32_t* __restrict__ yrow,
              const double* __restrict__ w, double* __restrict__ part, long long budget,
              int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Bs = As + kNS * kM * kKB;
  __shared__ uint32_t tmem_base;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ int ex[kM], ey[kM];
  __shared__ int s_ok;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int item = blockIdx.x / S, s = blockIdx.x % S;
  const int64_t lo = rlo[item], hi = rhi[item];
  const int64_t ra = lo + (hi - lo) * s / S, rb = lo + (hi - lo) * (s + 1) / S;
  double* P = part + (int64_t)blockIdx.x * nx * ny;
  // binary64 partial of this block, zero
  for (int idx = tid; idx < nx * ny; idx += 128) P[idx] = 0.0;
  // column exponents over the block's rows (coalesced sweeps, integer maxima); -1100
  // marks a column without a normal entry
  ex[tid] = -1100;
  ey[tid] = -1100;
  __syncthreads();
  {
    const int64_t nr = rb - ra;
    for (int64_t idx = tid; idx < nr * nx; idx += 128) {
      const int64_t e = ra + idx / nx;
      const int c = (int)(idx % nx);
      const double v = kGather ? w[e] * X[(int64_t)xrow[e] * ldx + c] : X[e * ldx + c];
      if (v != 0.0) atomicMax(&ex[c], exponent_of(v));
    }
    for (int64_t idx = tid; idx < nr * ny; idx += 128) {
      const int64_t e = ra + idx / ny;
      const int c = (int)(idx % ny);
      const double v = Y[(kGather ? (int64_t)yrow[e] : e) * ldy + c];
      if (v != 0.0) atomicMax(&ey[c], exponent_of(v));
    }
  }
  __syncthreads();
  if (ex[tid] == -1100) ex[tid] = 0;
  if (ey[tid] == -1100) ey[tid] = 0;
  // TMEM: four FP32 accumulators of NP columns (power of two >= 32 columns allocated)
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(kNS * NP)) ncols <<= 1;
  if (warp == 0) {
    const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&tmem_base);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(dst), "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_ok = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tbase = tmem_base;
  const uint32_t idesc = instr_desc(kM, NP);
  const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(As);
  const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(Bs);
  const uint32_t a_plane = kM * kKB * 2, b_plane = (uint32_t)NP * kKB * 2;
  uint32_t phase = 0;
  int in_acc = 0;
  const int64_t nblk = (rb - ra + kKB - 1) / kKB;
  bool ok = true;
  // the padding rows of the operands (X columns nx..127, Y columns ny..NP-1) stay zero
  for (int idx = tid; idx < kKB * (kM - nx); idx += 128)
    put_slices(As, a_plane, nx + idx / kKB, idx % kKB, 0.0, 0);
  for (int idx = tid; idx < kKB * (NP - ny); idx += 128)
    put_slices(Bs, b_plane, ny + idx / kKB, idx % kKB, 0.0, 0);
  for (int64_t blk = 0; blk < nblk && ok; ++blk) {
    const int64_t e0 = ra + blk * kKB;
    for (int idx = tid; idx < kKB * nx; idx += 128) {
      const int k = idx / nx, c = idx % nx;
      const int64_t e = e0 + k;
      double v = 0.0;
      if (e < rb) v = kGather ? w[e] * X[(int64_t)xrow[e] * ldx + c] : X[e * ldx + c];
      put_slices(As, a_plane, c, k, v, ex[c]);
    }
    for (int idx = tid; idx < kKB * ny; idx += 128) {
      const int k = idx / ny, c = idx % ny;
      const int64_t e = e0 + k;
      double v = 0.0;
      if (e < rb) v = Y[(kGather ? (int64_t)yrow[e] : e) * ldy + c];
      put_slices(Bs, b_plane, c, k, v, ey[c]);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      for (int d = 0; d < kNS; ++d) {
        const uint32_t tacc = tbase + (uint32_t)(d * NP);
        bool first = in_acc == 0;
        for (int t = 0; t <= d; ++t)
          for (int ks = 0; ks < kKB / 16; ++ks) {
            const uint64_t ad = smem_desc(a0 + t * a_plane + ks * 256, 128, (kKB / 8) * 128);
            const uint64_t bd =
                smem_desc(b0 + (d - t) * b_plane + ks * 256, 128, (kKB / 8) * 128);
            const uint32_t en = first ? 0u : 1u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tacc),
                "l"(ad), "l"(bd), "r"(idesc), "r"(en));
            first = false;
          }
      }
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              mb));
    }
    __syncwarp();
    if (mbar_wait(mb, phase, budget)) {
      phase ^= 1u;
    } else {
      atomicExch(err, 1);
      s_ok = 0;
    }
    __syncthreads();
    ok = s_ok != 0;
    ++in_acc;
    if (ok && (in_acc == kFlush || blk == nblk - 1)) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int i = tid;  // output row = TMEM lane
      for (int c0 = 0; c0 < NP; c0 += 8) {
        double tmp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int d = 0; d < kNS; ++d) {
          uint32_t r[8];
          const uint32_t ta = tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * NP + c0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7])
              : "r"(ta));
          asm volatile("tcgen05.wait::ld.sync.aligned;");
          const double sc = ldexp(1.0, -7 * (d + 2));
#pragma unroll
          for (int e = 0; e < 8; ++e) tmp[e] += sc * (double)__uint_as_float(r[e]);
        }
        if (i < nx)
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = c0 + e;
            if (j < ny) P[(int64_t)i * ny + j] += ldexp(tmp[e], ex[i] + ey[j]);
          }
      }
      in_acc = 0;
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();
    }
  }
  if (!ok) {
    // a wait ran out: wait once more (bounded) for the pending phase, so that the
    // issued MMAs drain before the TMEM is released
    mbar_wait(mb, phase, budget);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                 "r"(ncols));
}

// G[item][i * ldg + j] = sum over s of part[(item * S + s)][i * ny + j], in order
__global__ void k_tc_reduce(int S, int nx, int ny, const double* __restrict__ part, double* G,
                            int ldg, int64_t stride) {
  const int item = blockIdx.y;
  const int n = nx * ny;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < n; o += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < S; ++s) acc += part[((int64_t)item * S + s) * n + o];
    G[(int64_t)item * stride + (int64_t)(o / ny) * ldg + (o % ny)] = acc;
  }
}

// pair blocks: Bij = G, Bji = G^T (kq x kq, zero beyond nx = ny)
__global__ void k_tc_pairs_out(int n_pairs, int kq, const double* __restrict__ G, double* blocks) {
  const int p = blockIdx.x;
  const double* g = G + (int64_t)p * kq * kq;
  double* Bij = blocks + (int64_t)(2 * p) * kq * kq;
  double* Bji = blocks + (int64_t)(2 * p + 1) * kq * kq;
  for (int o = threadIdx.x; o < kq * kq; o += blockDim.x) {
    const int i = o / kq, j = o % kq;
    Bij[o] = g[o];
    Bji[j * kq + i] = g[o];
  }
}

// rows of subdomain sd in a tile set: its tiles cover [r0 of the first, r1 of the last)
__global__ void k_tiles_range(DTiles tl, int64_t* rlo, int64_t* rhi) {
  const int sd = blockIdx.x * blockDim.x + threadIdx.x;
  if (sd >= tl.n_sd) return;
  const int a = tl.lo[sd], b = tl.hi[sd];
  rlo[sd] = a < b ? tl.r0[a] : 0;
  rhi[sd] = a < b ? tl.r1[b - 1] : 0;
}

size_t tc_smem(int NP) { return (size_t)kNS * (kM + NP) * kKB * 2; }

}  // namespace

int tc_gram_chunks(int n_items) {
  int S = (4 * 152 + n_items - 1) / n_items;
  return S < 1 ? 1 : (S > 16 ? 16 : S);
}

void launch_tc_gram(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                    const double* Y, int ldy, int ny, double* part, int64_t* range, double* G,
                    int ldg, int64_t stride, long long budget, int* err, cudaStream_t st) {
  // range: 2 * n_sd entries (row starts, then row ends)
  if (tiles.n <= 0 || n_sd <= 0) return;
  const int NP = ((ny + 15) / 16) * 16;
  const int S = tc_gram_chunks(n_sd);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_smem(128));
    attr = true;
  }
  count_launch(3);
  // the row range of each subdomain: its tiles are contiguous rows
  k_tiles_range<<<(n_sd + 255) / 256, 256, 0, st>>>(tiles, range, range + n_sd);
  k_tc_gram<false><<<n_sd * S, 128, tc_smem(NP), st>>>(range, range + n_sd, S, X, ldx, nx, Y,
                                                      ldy, ny, NP, nullptr, nullptr, nullptr,
                                                      part, budget, err);
  k_tc_reduce<<<dim3(std::max(1, std::min(64, (nx * ny + 255) / 256)), n_sd), 256, 0, st>>>(
      S, nx, ny, part, G, ldg, stride);
}

void launch_tc_pair_blocks(int n_pairs, const int64_t* pair_ptr, const int32_t* urow,
                           const int32_t* vrow, const double* aval, const double* Q, int kq,
                           double* part, double* G, double* blocks, long long budget, int* err,
                           cudaStream_t st) {
  if (n_pairs <= 0) return;
  const int NP = ((kq + 15) / 16) * 16;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gram<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_smem(128));
    attr = true;
  }
  count_launch(3);
  k_tc_gram<true><<<n_pairs, 128, tc_smem(NP), st>>>(pair_ptr, pair_ptr + 1, 1, Q, kq, kq, Q,
                                                    kq, kq, NP, urow, vrow, aval, part, budget,
                                                    err);
  k_tc_reduce<<<dim3(std::max(1, std::min(64, (kq * kq + 255) / 256)), n_pairs), 256, 0, st>>>(
      1, kq, kq, part, G, kq, (int64_t)kq * kq);
  k_tc_pairs_out<<<n_pairs, 256, 0, st>>>(n_pairs, kq, G, blocks);
}

void launch_tc_gram_rows(int64_t rows, const double* X, int ldx, int nx, const double* Y,
                         int ldy, int ny, double* part, int64_t* range, double* G,
                         long long budget, int* err, cudaStream_t st) {
  const int NP = ((ny + 15) / 16) * 16;
  const int S = 1;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tc_gram<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)tc_smem(128));
    attr = true;
  }
  const int64_t hr[2] = {0, rows};
  cudaMemcpyAsync(range, hr, sizeof(hr), cudaMemcpyHostToDevice, st);
  count_launch(2);
  k_tc_gram<false><<<S, 128, tc_smem(NP), st>>>(range, range + 1, S, X, ldx, nx, Y, ldy, ny,
                                               NP, nullptr, nullptr, nullptr, part, budget,
                                               err);
  k_tc_reduce<<<dim3(std::max(1, std::min(64, (nx * ny + 255) / 256)), 1), 256, 0, st>>>(
      S, nx, ny, part, G, ny, (int64_t)nx * ny);
}

}  // namespace mor
