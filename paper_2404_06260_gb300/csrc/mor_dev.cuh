// Device-side building blocks shared by the CUDA translation units of libmor:
// sliced-ELL indexing, row tiles, P1 element geometry, and the counter-based Gaussian
// generator of the sketch.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mor {

// (row r, slot j) of a fixed-stride sliced ELL with stride W (slices of 32 rows)
__host__ __device__ __forceinline__ int64_t ell_at(int64_t r, int j, int W) {
  return (r >> 5) * (int64_t)(32 * W) + (int64_t)j * 32 + (r & 31);
}

struct DTiles {
  int n = 0;
  int n_sd = 0;                 // subdomains (lo/hi length)
  const int32_t* sd = nullptr;
  const int32_t* r0 = nullptr;
  const int32_t* r1 = nullptr;
  const int32_t* lo = nullptr;  // per subdomain first tile
  const int32_t* hi = nullptr;  // per subdomain end tile
};

// ---- P1 tetrahedron (Sec. 2): barycentric gradients and volume -------------------
// J = [x1-x0, x2-x0, x3-x0]; rows of J^{-1} are (e1 x e2, e2 x e0, e0 x e1) / det J.
__device__ __forceinline__ bool tet_gradients(const double* __restrict__ xyz,
                                              const int32_t* __restrict__ tets, int64_t t,
                                              double G[4][3], double& vol) {
  int32_t v0 = tets[4 * t], v1 = tets[4 * t + 1], v2 = tets[4 * t + 2], v3 = tets[4 * t + 3];
  double e[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double x0 = xyz[3 * (int64_t)v0 + i];
    e[0][i] = xyz[3 * (int64_t)v1 + i] - x0;
    e[1][i] = xyz[3 * (int64_t)v2 + i] - x0;
    e[2][i] = xyz[3 * (int64_t)v3 + i] - x0;
  }
  double c[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double* p = e[(a + 1) % 3];
    const double* q = e[(a + 2) % 3];
    c[a][0] = p[1] * q[2] - p[2] * q[1];
    c[a][1] = p[2] * q[0] - p[0] * q[2];
    c[a][2] = p[0] * q[1] - p[1] * q[0];
  }
  double det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
  double inv = 1.0 / det;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G[1][i] = c[0][i] * inv;
    G[2][i] = c[1][i] * inv;
    G[3][i] = c[2][i] * inv;
    G[0][i] = -(G[1][i] + G[2][i] + G[3][i]);
  }
  vol = det / 6.0;
  return det > 0.0;
}

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ---- Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) ---------------------------
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0;
    uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// ---- Box-Muller in binary32 with a fixed sequence of correctly rounded operations --
// ln u = e ln2 + 2 s (1 + s^2/3 + s^4/5 + s^6/7 + s^8/9), s = (m-1)/(m+1), u = m 2^e,
// m in [sqrt(2)/2, sqrt(2)]; sin/cos: Taylor degree 9/10 on [0, pi/4] after an exact
// octant reduction.  Only _rn intrinsics, so no contraction into FMA: any other
// implementation of the same sequence draws bit-identical normals.
__device__ __forceinline__ float bm_uniform(uint32_t x) {
  return __fmul_rn((float)((x >> 9) * 2u + 1u), 5.9604644775390625e-08f);  // 2^-24
}

__device__ __forceinline__ float bm_ln(float u) {
  const float kLn2 = 0x1.62e430p-1f, kSqrt2 = 0x1.6a09e6p+0f;
  uint32_t bits = __float_as_uint(u);
  int e = (int)((bits >> 23) & 0xFFu) - 127;
  float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
  if (m > kSqrt2) {
    m = __fmul_rn(m, 0.5f);
    e += 1;
  }
  float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  float s2 = __fmul_rn(s, s);
  float p = 0x1.c71c72p-4f;
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.24924ap-3f);
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.99999ap-3f);
  p = __fadd_rn(__fmul_rn(p, s2), 0x1.555556p-2f);
  p = __fadd_rn(__fmul_rn(p, s2), 1.0f);
  float lnm = __fmul_rn(__fadd_rn(s, s), p);
  return __fadd_rn(__fmul_rn((float)e, kLn2), lnm);
}

__device__ __forceinline__ void bm_sincos_2pi(float u, float& c, float& s) {
  float t = __fmul_rn(u, 8.0f);
  float q = floorf(t);
  float f = __fsub_rn(t, q);
  int qi = (int)q;
  float g = (qi & 1) ? __fsub_rn(1.0f, f) : f;
  float th = __fmul_rn(g, 0x1.921fb6p-1f);
  float th2 = __fmul_rn(th, th);
  float sp = 0x1.71de3ap-19f;
  sp = __fadd_rn(__fmul_rn(sp, th2), -0x1.a01a02p-13f);
  sp = __fadd_rn(__fmul_rn(sp, th2), 0x1.111112p-7f);
  sp = __fadd_rn(__fmul_rn(sp, th2), -0x1.555556p-3f);
  sp = __fmul_rn(sp, th2);
  float sn = __fadd_rn(th, __fmul_rn(th, sp));
  float cp = -0x1.27e4fcp-22f;
  cp = __fadd_rn(__fmul_rn(cp, th2), 0x1.a01a02p-16f);
  cp = __fadd_rn(__fmul_rn(cp, th2), -0x1.6c16c2p-10f);
  cp = __fadd_rn(__fmul_rn(cp, th2), 0x1.555556p-5f);
  cp = __fadd_rn(__fmul_rn(cp, th2), -0.5f);
  float cs = __fadd_rn(__fmul_rn(cp, th2), 1.0f);
  bool swap = (qi == 1) || (qi == 2) || (qi == 5) || (qi == 6);
  c = swap ? sn : cs;
  s = swap ? cs : sn;
  if (qi >= 2 && qi <= 5) c = -c;
  if (qi >= 4) s = -s;
}

__device__ __forceinline__ void box_muller(uint32_t x1, uint32_t x2, float& z0, float& z1) {
  float r = __fsqrt_rn(__fmul_rn(-2.0f, bm_ln(bm_uniform(x1))));
  float c, s;
  bm_sincos_2pi(bm_uniform(x2), c, s);
  z0 = __fmul_rn(r, c);
  z1 = __fmul_rn(r, s);
}

// four standard normals xi_T[0..3] for (element T, column j, subdomain i): counter
// (T, j, i, 0), key = seed
__device__ __forceinline__ void field_normals(uint32_t T, uint32_t j, uint32_t i,
                                              uint64_t seed, float z[4]) {
  uint32_t c[4] = {T, j, i, 0u};
  philox4x32_10(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
  box_muller(c[0], c[1], z[0], z[1]);
  box_muller(c[2], c[3], z[2], z[3]);
}

// Bounded wait of one thread until *gen differs from `seen` (a grid barrier's
// generation counter, or any flag another block or the host sets).  It gives up after
// `budget` clock cycles, or as soon as *err is non-zero (another block gave up), sets
// *err to 1 when it is the one that ran out, and returns false; true when the flag
// moved.  The caller's block then leaves its kernel, so no wait is unbounded.
__device__ __forceinline__ bool bounded_wait(const volatile unsigned* gen, unsigned seen,
                                             volatile int* err, long long budget) {
  const long long t0 = clock64();
  while (*gen == seen) {
    if (*err) return false;
    if (clock64() - t0 > budget) {
      atomicExch((int*)err, 1);
      return false;
    }
    __nanosleep(100);
  }
  return true;
}

// Grid-wide barrier of a cooperative launch (all blocks co-resident) with bounded
// waits: arrivals count on *count; the last one resets it and advances *gen.  Returns
// false (for every thread of the block) when the block gave up waiting.
__device__ __forceinline__ bool grid_barrier(unsigned* count, volatile unsigned* gen,
                                             volatile int* err, long long budget) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned seen = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(count, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
      ok = 1;
    } else {
      ok = bounded_wait(gen, seen, err, budget) ? 1 : 0;
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace mor
