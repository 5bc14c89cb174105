// P1 assembly, the field-sketch right-hand side, sliced-ELL extraction, energy norm and
// interface coupling values (Sec. 2, Sec. 4, Sec. 6 steps 2 and 3).
#include "mor_kernels.h"

namespace mor {

__global__ void k_assemble(int64_t n_rows, const int64_t* __restrict__ inc_ptr,
                           const int32_t* __restrict__ inc_tet,
                           const uint32_t* __restrict__ inc_code, int W,
                           const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                           const double* __restrict__ kappa, int h1w, double* valA,
                           double* valH, double* load, int* err) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  double bl = 0.0;
  for (int64_t q = inc_ptr[r]; q < inc_ptr[r + 1]; ++q) {
    int32_t t = inc_tet[q];
    uint32_t code = inc_code[q];
    int a = code & 3u;
    double G[4][3], vol;
    if (!tet_gradients(xyz, tets, t, G, vol)) {
      atomicExch(err, 1);
      return;
    }
    double kap = kappa[t];
    double hk = h1w ? kap : 1.0;  // weight of the gradient part of the H1 form
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      uint32_t slot = (code >> (2 + 7 * b)) & 127u;
      if (slot == 127u) continue;
      double g = dot3(G[a], G[b]) * vol;
      int64_t at = ell_at(r, (int)slot, W);
      valA[at] += kap * g;
      valH[at] += hk * g + vol * (a == b ? 0.1 : 0.05);
    }
    bl += 0.25 * vol;
  }
  load[r] = bl;
}

void launch_assemble(int64_t n_rows, const int64_t* inc_ptr, const int32_t* inc_tet,
                     const uint32_t* inc_code, int W, const double* xyz, const int32_t* tets,
                     const double* kappa, int h1_weighted, double* valA, double* valH,
                     double* load, int* err, cudaStream_t st) {
  if (n_rows <= 0) return;
  int bs = 128;
  count_launch();
  k_assemble<<<(unsigned)((n_rows + bs - 1) / bs), bs, 0, st>>>(
      n_rows, inc_ptr, inc_tet, inc_code, W, xyz, tets, kappa, h1_weighted, valA, valH, load,
      err);
}

// element H1 matrix H_T = w_T |T| grad.grad + |T|(1 + d_ab)/20 (w_T = k_T when the H1
// form is weighted, else 1) and its lower Cholesky factor
// L_T (H_T = L_T L_T^T), once per element: the 10 entries L[a][b], b <= a, at
// a(a+1)/2 + b, each split into binary32 hi + lo (hi = fl32(L), lo = fl32(L - hi)), so
// the sketch sums can run in double-binary32 arithmetic
__global__ void k_elem_chol(int64_t n_tets, const double* __restrict__ xyz,
                            const int32_t* __restrict__ tets, const double* __restrict__ kappa,
                            int h1w, float2* __restrict__ lsplit) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n_tets) return;
  double G[4][3], vol;
  tet_gradients(xyz, tets, (int32_t)t, G, vol);
  const double hk = h1w ? kappa[t] : 1.0;
  double H[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
      H[i][j] = hk * dot3(G[i], G[j]) * vol + vol * (i == j ? 0.1 : 0.05);
  double L[4][4] = {};
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    double d = H[j][j];
#pragma unroll
    for (int l = 0; l < j; ++l) d -= L[j][l] * L[j][l];
    L[j][j] = sqrt(d);
#pragma unroll
    for (int i = j + 1; i < 4; ++i) {
      double v = H[i][j];
#pragma unroll
      for (int l = 0; l < j; ++l) v -= L[i][l] * L[j][l];
      L[i][j] = v / L[j][j];
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b <= a; ++b) {
      float hi = (float)L[a][b];
      float lo = (float)(L[a][b] - (double)hi);
      lsplit[10 * t + a * (a + 1) / 2 + b] = make_float2(hi, lo);
    }
}

void launch_elem_chol(int64_t n_tets, const double* xyz, const int32_t* tets,
                      const double* kappa, int h1_weighted, float2* lsplit, cudaStream_t st) {
  if (n_tets <= 0) return;
  int bs = 256;
  count_launch();
  k_elem_chol<<<(unsigned)((n_tets + bs - 1) / bs), bs, 0, st>>>(n_tets, xyz, tets, kappa,
                                                                 h1_weighted, lsplit);
}

// (hi, lo) += x, the rounding error of hi + x kept in lo (Knuth's two-sum)
__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
  float s = hi + x;
  float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// one thread per (row, column), consecutive threads taking consecutive columns of a
// row: out[r, j] = sum over incident elements T of
// (L_T xi_T[:, j])[a(r)].  The Gaussian draws are binary32 (bit-exact Box-Muller); the
// products and sums run in double-binary32 arithmetic (about 2^-48 relative), the same in
// every solve precision, so every precision sketches with the same test matrix W
__global__ void k_sketch_rhs(int64_t row0, int64_t n_rows, const int32_t* __restrict__ row_sd,
                             const int64_t* __restrict__ inc_ptr,
                             const int32_t* __restrict__ inc_tet,
                             const uint32_t* __restrict__ inc_code,
                             const float2* __restrict__ lsplit, int k, uint64_t seed,
                             uint32_t sd_base, double* __restrict__ out, int ld,
                             const int32_t* __restrict__ k_sd) {
  // one thread per (row, column): consecutive threads take consecutive columns of a
  // row (coalesced stores; the threads of a row read the same incidence entries)
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= n_rows * (int64_t)k) return;
  const int64_t w = idx / k;
  const int j = (int)(idx - w * k);
  int64_t r = row0 + w;
  uint32_t sd = (uint32_t)row_sd[r];
  const uint32_t sd_id = sd + sd_base;  // the subdomain's id in the whole batch
  int64_t q0 = inc_ptr[r], q1 = inc_ptr[r + 1];
  const int kk = k_sd ? min(k, (int)k_sd[sd]) : k;
  if (j >= kk) {
    out[r * ld + j] = 0.0;
  } else {
    float hi = 0.f, lo = 0.f;
    for (int64_t q = q0; q < q1; ++q) {
      float z[4];
      const uint32_t t = (uint32_t)inc_tet[q];
      field_normals(t, (uint32_t)j, sd_id, seed, z);
      const int a = inc_code[q] & 3u;
      const float2* La = lsplit + 10 * (int64_t)t + a * (a + 1) / 2;
      for (int b = 0; b <= a; ++b) {
        const float2 l = La[b];
        const float p = l.x * z[b];
        const float e = fmaf(l.x, z[b], -p);  // l.x z[b] = p + e exactly
        df_add(hi, lo, p);
        lo += e + l.y * z[b];
      }
    }
    out[r * ld + j] = (double)hi + (double)lo;
  }
}

void launch_sketch_rhs(int64_t row0, int64_t n_rows, const int32_t* row_sd,
                       const int64_t* inc_ptr, const int32_t* inc_tet,
                       const uint32_t* inc_code, const float2* lsplit, int k, uint64_t seed,
                       uint32_t sd_base, double* out, int ld, cudaStream_t st,
                       const int32_t* k_sd) {
  if (n_rows <= 0) return;
  int bs = 256;
  unsigned grid = (unsigned)((n_rows * (int64_t)k + bs - 1) / bs);
  count_launch();
  k_sketch_rhs<<<grid, bs, 0, st>>>(row0, n_rows, row_sd, inc_ptr, inc_tet, inc_code, lsplit,
                                    k, seed, sd_base, out, ld, k_sd);
}

// one thread per destination row; warps cover whole slices so the slice width is a
// warp maximum
__global__ void k_extract(int64_t n_dst, const int32_t* __restrict__ row_src,
                          const uint8_t* __restrict__ row_cls, int row_want,
                          const int32_t* __restrict__ src_col,
                          const int32_t* __restrict__ src_width, int Wsrc,
                          const double* __restrict__ src_val,
                          const int32_t* __restrict__ col_map,
                          const uint8_t* __restrict__ col_cls, int col_want, double drop_rel,
                          int Wdst, int32_t* dst_width, int32_t* dst_col, double* dst_val,
                          float* dst_val32, double* dinv64, float* dinv32) {
  int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int cnt = 0;
  double diag = 0.0;
  if (r < n_dst) {
    int64_t s = row_src ? row_src[r] : r;
    bool take = (row_cls == nullptr) || (row_cls[s] == row_want);
    if (take) {
      int w = src_width[s >> 5];
      double dsrc = 0.0;
      for (int j = 0; j < w; ++j) {
        int64_t at = ell_at(s, j, Wsrc);
        if (src_col[at] == (int32_t)s) dsrc = src_val[at];
      }
      for (int j = 0; j < w; ++j) {
        int64_t at = ell_at(s, j, Wsrc);
        int32_t c = src_col[at];
        if (c < 0) continue;
        if (col_cls && col_cls[c] != col_want) continue;
        int32_t cm = col_map ? col_map[c] : c;
        if (cm < 0) continue;
        double v = src_val[at];
        if (drop_rel >= 0.0 && c != (int32_t)s && fabs(v) <= drop_rel * fabs(dsrc)) continue;
        if (cnt < Wdst) {
          int64_t d = ell_at(r, cnt, Wdst);
          dst_col[d] = cm;
          dst_val[d] = v;
          if (dst_val32) dst_val32[d] = (float)v;
        }
        if (c == (int32_t)s) diag = v;
        ++cnt;
      }
    }
    if (dinv64) dinv64[r] = diag != 0.0 ? 1.0 / diag : 0.0;
    if (dinv32) dinv32[r] = diag != 0.0 ? (float)(1.0 / diag) : 0.0f;
  }
  unsigned mask = __ballot_sync(0xFFFFFFFFu, true);
  int mx = __reduce_max_sync(mask, cnt);
  if ((threadIdx.x & 31) == 0 && r < n_dst) dst_width[r >> 5] = mx < Wdst ? mx : Wdst;
}

void launch_extract(int64_t n_dst, const int32_t* row_src, const uint8_t* row_cls,
                    int row_want, const int32_t* src_col, const int32_t* src_width, int Wsrc,
                    const double* src_val, const int32_t* col_map, const uint8_t* col_cls,
                    int col_want, double drop_rel, int Wdst, int32_t* dst_width,
                    int32_t* dst_col, double* dst_val, float* dst_val32, double* dinv64,
                    float* dinv32, cudaStream_t st) {
  if (n_dst <= 0) return;
  int bs = 256;  // multiple of 32: warps align with slices
  count_launch();
  k_extract<<<(unsigned)((n_dst + bs - 1) / bs), bs, 0, st>>>(
      n_dst, row_src, row_cls, row_want, src_col, src_width, Wsrc, src_val, col_map, col_cls,
      col_want, drop_rel, Wdst, dst_width, dst_col, dst_val, dst_val32, dinv64, dinv32);
}

__global__ void k_energy(int64_t n_tets, const double* __restrict__ xyz,
                         const int32_t* __restrict__ tets, const double* __restrict__ kappa,
                         const double* __restrict__ u1, const double* __restrict__ u2,
                         double* partials) {
  __shared__ double red[256];
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e = 0.0;
  if (t < n_tets) {
    double G[4][3], vol;
    tet_gradients(xyz, tets, t, G, vol);
    double d[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int32_t v = tets[4 * t + a];
      d[a] = u1[v] - (u2 ? u2[v] : 0.0);
    }
    double g[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i) g[i] += d[a] * G[a][i];
    e = kappa[t] * vol * dot3(g, g);
  }
  red[threadIdx.x] = e;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_partials(int64_t n, const double* __restrict__ p, double* out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += 256) s += p[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

void launch_energy(int64_t n_tets, const double* xyz, const int32_t* tets,
                   const double* kappa, const double* u1, const double* u2,
                   double* partials, double* out, cudaStream_t st) {
  int64_t nb = (n_tets + 255) / 256;
  count_launch();
  k_energy<<<(unsigned)nb, 256, 0, st>>>(n_tets, xyz, tets, kappa, u1, u2, partials);
  count_launch();
  k_sum_partials<<<1, 256, 0, st>>>(nb, partials, out);
}

__global__ void k_iface_vals(int64_t n_e, const int32_t* __restrict__ unode,
                             const int32_t* __restrict__ vnode,
                             const int64_t* __restrict__ n2t_ptr,
                             const int32_t* __restrict__ n2t, const double* __restrict__ xyz,
                             const int32_t* __restrict__ tets,
                             const double* __restrict__ kappa, double* val) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  int32_t u = unode[e], v = vnode[e];
  double acc = 0.0;
  for (int64_t q = n2t_ptr[u]; q < n2t_ptr[u + 1]; ++q) {
    int32_t t = n2t[q];
    int au = -1, av = -1;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int32_t w = tets[4 * (int64_t)t + a];
      if (w == u) au = a;
      if (w == v) av = a;
    }
    if (av < 0) continue;
    double G[4][3], vol;
    tet_gradients(xyz, tets, t, G, vol);
    acc += kappa[t] * vol * dot3(G[au], G[av]);
  }
  val[e] = acc;
}

void launch_iface_vals(int64_t n_e, const int32_t* unode, const int32_t* vnode,
                       const int64_t* n2t_ptr, const int32_t* n2t, const double* xyz,
                       const int32_t* tets, const double* kappa, double* val,
                       cudaStream_t st) {
  if (n_e <= 0) return;
  int bs = 256;
  count_launch();
  k_iface_vals<<<(unsigned)((n_e + bs - 1) / bs), bs, 0, st>>>(n_e, unode, vnode, n2t_ptr,
                                                                n2t, xyz, tets, kappa, val);
}

}  // namespace mor
