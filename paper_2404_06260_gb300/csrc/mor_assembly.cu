// P1 assembly, the field-sketch right-hand side, sliced-ELL extraction, energy norm and
// interface coupling values (Sec. 2, Sec. 4, Sec. 6 steps 2 and 3).
#include "mor_kernels.h"

namespace mor {

__global__ void k_assemble(int64_t n_rows, const int64_t* __restrict__ inc_ptr,
                           const int32_t* __restrict__ inc_tet,
                           const uint32_t* __restrict__ inc_code, int W,
                           const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                           const double* __restrict__ kappa, double* valA, double* valH,
                           double* load, int* err) {
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
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      uint32_t slot = (code >> (2 + 7 * b)) & 127u;
      if (slot == 127u) continue;
      double g = dot3(G[a], G[b]) * vol;
      int64_t at = ell_at(r, (int)slot, W);
      valA[at] += kap * g;
      valH[at] += g + vol * (a == b ? 0.1 : 0.05);
    }
    bl += 0.25 * vol;
  }
  load[r] = bl;
}

void launch_assemble(int64_t n_rows, const int64_t* inc_ptr, const int32_t* inc_tet,
                     const uint32_t* inc_code, int W, const double* xyz, const int32_t* tets,
                     const double* kappa, double* valA, double* valH, double* load,
                     int* err, cudaStream_t st) {
  if (n_rows <= 0) return;
  int bs = 128;
  count_launch();
  k_assemble<<<(unsigned)((n_rows + bs - 1) / bs), bs, 0, st>>>(
      n_rows, inc_ptr, inc_tet, inc_code, W, xyz, tets, kappa, valA, valH, load, err);
}

// element H1 matrix and its 4x4 Cholesky factor; row a of L into lrow[4q..4q+3]
__global__ void k_elem_lrow(int64_t n_inc, const int32_t* __restrict__ inc_tet,
                            const uint32_t* __restrict__ inc_code,
                            const double* __restrict__ xyz, const int32_t* __restrict__ tets,
                            double* __restrict__ lrow) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n_inc) return;
  int32_t t = inc_tet[q];
  int a = inc_code[q] & 3u;
  double G[4][3], vol;
  tet_gradients(xyz, tets, t, G, vol);
  double H[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) H[i][j] = dot3(G[i], G[j]) * vol + vol * (i == j ? 0.1 : 0.05);
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
  for (int b = 0; b < 4; ++b) lrow[4 * q + b] = (b <= a) ? L[a][b] : 0.0;
}

void launch_elem_lrow(int64_t n_inc, const int32_t* inc_tet, const uint32_t* inc_code,
                      const double* xyz, const int32_t* tets, double* lrow, cudaStream_t st) {
  if (n_inc <= 0) return;
  int bs = 256;
  count_launch();
  k_elem_lrow<<<(unsigned)((n_inc + bs - 1) / bs), bs, 0, st>>>(n_inc, inc_tet, inc_code,
                                                                 xyz, tets, lrow);
}

// one warp per row, lanes over columns.  The Gaussian draws are binary32 (bit-exact
// Box-Muller); the sums over element incidences are binary64 whatever the solve
// precision, so every precision sketches with the same test matrix W
__global__ void k_sketch_rhs(int64_t row0, int64_t n_rows, const int32_t* __restrict__ row_sd,
                             const int64_t* __restrict__ inc_ptr,
                             const int32_t* __restrict__ inc_tet,
                             const double* __restrict__ lrow, int k, uint64_t seed,
                             double* __restrict__ out, int ld,
                             const int32_t* __restrict__ k_sd) {
  int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (w >= n_rows) return;
  int64_t r = row0 + w;
  uint32_t sd = (uint32_t)row_sd[r];
  int64_t q0 = inc_ptr[r], q1 = inc_ptr[r + 1];
  const int kk = k_sd ? min(k, (int)k_sd[sd]) : k;
  for (int j = lane + kk; j < k; j += 32) out[r * ld + j] = 0.0;
  for (int j = lane; j < kk; j += 32) {
    double acc = 0.0;
    for (int64_t q = q0; q < q1; ++q) {
      float z[4];
      field_normals((uint32_t)inc_tet[q], (uint32_t)j, sd, seed, z);
      const double* L = lrow + 4 * q;
      acc += L[0] * (double)z[0] + L[1] * (double)z[1] + L[2] * (double)z[2] +
             L[3] * (double)z[3];
    }
    out[r * ld + j] = acc;
  }
}

void launch_sketch_rhs(int64_t row0, int64_t n_rows, const int32_t* row_sd,
                       const int64_t* inc_ptr, const int32_t* inc_tet,
                       const uint32_t* inc_code, const double* lrow, int k, uint64_t seed,
                       double* out, int ld, cudaStream_t st, const int32_t* k_sd) {
  (void)inc_code;
  if (n_rows <= 0) return;
  int bs = 256;
  unsigned grid = (unsigned)((n_rows * 32 + bs - 1) / bs);
  count_launch();
  k_sketch_rhs<<<grid, bs, 0, st>>>(row0, n_rows, row_sd, inc_ptr, inc_tet, lrow, k, seed, out,
                                    ld, k_sd);
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
