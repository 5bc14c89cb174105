// Host launchers of the libmor CUDA kernels (one declaration per kernel family).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "mor_dev.cuh"

#include <cuda_bf16.h>

namespace mor {

// host-side count of kernel launches issued by the library (every launcher adds its
// launches before enqueuing them)
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(int n = 1) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

// record a failure for mor_last_error (thread-local) and return code
int set_error(int code, const std::string& msg);

// ---------------- assembly (mor_assembly.cu) ----------------
// Row-gather P1 assembly (Sec. 2, Sec. 4): for every row the element contributions
// of its incident elements are summed in incidence order (deterministic): stiffness
// k_T |T| grad(l_a).grad(l_b) into valA, H1 form w_T |T| grad.grad + |T|(1+d_ab)/20
// into valH (w_T = k_T if h1_weighted, else 1), load |T|/4 into load[row].  err is set
// to 1 on det <= 0.
void launch_assemble(int64_t n_rows, const int64_t* inc_ptr, const int32_t* inc_tet,
                     const uint32_t* inc_code, int W, const double* xyz, const int32_t* tets,
                     const double* kappa, int h1_weighted, double* valA, double* valH,
                     double* load, int* err, cudaStream_t st);

// Lower Cholesky factor L_T of every element's H1 matrix (the element factors of the
// field sketch, L L^T = H^+; gradient part weighted by k_T if h1_weighted):
// lsplit[10 t + a(a+1)/2 + b] = L[a][b] (b <= a) as binary32 hi + lo.
void launch_elem_chol(int64_t n_tets, const double* xyz, const int32_t* tets,
                      const double* kappa, int h1_weighted, float2* lsplit, cudaStream_t st);

// out[r, j] = sum over incident elements T of (L_T xi_T[:, j])[a(r)], j < k_sd[row_sd[r]]
// (or j < k when k_sd is null), zero for the other j < k, for rows [row0, row0 + n_rows);
// xi from Philox counter (T, j, sd_base + row_sd[r], 0) (sd_base: the batch id of the
// plan's first subdomain); products and sums in double-binary32.
void launch_sketch_rhs(int64_t row0, int64_t n_rows, const int32_t* row_sd,
                       const int64_t* inc_ptr, const int32_t* inc_tet,
                       const uint32_t* inc_code, const float2* lsplit, int k, uint64_t seed,
                       uint32_t sd_base, double* out, int ld, cudaStream_t st,
                       const int32_t* k_sd);

// Extract a sliced-ELL matrix from an assembled pattern: destination row r takes source
// row s = row_src ? row_src[r] : r when row_cls is null or row_cls[s] == row_want;
// an entry (s, c) is kept when (col_cls null or col_cls[c] == col_want), col_map is
// null or col_map[c] >= 0, and |v| > drop_rel |v_ss| (drop_rel < 0 keeps all).
// The kept columns are col_map[c] (or c).  Writes slice widths, columns, binary64 and
// optional binary32 values, and optional inverse diagonals (Jacobi preconditioner).
void launch_extract(int64_t n_dst, const int32_t* row_src, const uint8_t* row_cls,
                    int row_want, const int32_t* src_col, const int32_t* src_width, int Wsrc,
                    const double* src_val, const int32_t* col_map, const uint8_t* col_cls,
                    int col_want, double drop_rel, int Wdst, int32_t* dst_width,
                    int32_t* dst_col, double* dst_val, float* dst_val32, double* dinv64,
                    float* dinv32, cudaStream_t st);

// sum_T d_T^T K_T d_T, d = u1 - u2 (u2 may be null), over all elements; deterministic
// two-level reduction into *out (device).  partials: ceil(n_tets/256) doubles.
void launch_energy(int64_t n_tets, const double* xyz, const int32_t* tets,
                   const double* kappa, const double* u1, const double* u2,
                   double* partials, double* out, cudaStream_t st);

// A[u, v] = sum over elements containing u and v of k_T |T| grad(l_u).grad(l_v)
void launch_iface_vals(int64_t n_e, const int32_t* unode, const int32_t* vnode,
                       const int64_t* n2t_ptr, const int32_t* n2t, const double* xyz,
                       const int32_t* tets, const double* kappa, double* val,
                       cudaStream_t st);

// ---------------- sparse products and batched CG (mor_sparse.cu) ----------------
struct CgState {
  double *rz, *bb, *alpha, *beta;  // n_sd x kp
  double* rr;                       // n_sd x kp: recursive ||r||^2 after the last update
  double* rzf;                      // n_sd x kp: r^T D^{-1} r (the fine part of r^T M^{-1} r)
  double* gam;                      // n_sd x kp: p = gam z + beta p in the p update
  double* pr;                       // n_sd x kp: p.r after the p update (the step length
                                    // is the exact line search alpha = p.r / p.Ap)
  float *alpha32, *beta32, *gam32;  // n_sd x kp: binary32 copies written beside alpha,
                                    // beta, gam (binary32 kernels load them as packs)
  int* done;                        // n_sd x kp
  double *part1, *part2;            // n_tiles x kp
  int* counter;                     // n_sd
  int* iters;                       // n_sd
  int* active;                      // n_sd: active columns after the last update
  // work counters of the algorithmic-bytes model, kept by the coarse kernel (once per
  // subdomain and step; null: not counted): work[k * n_sd + sd] with k = [0] stored
  // entries read by the sparse product, [1] (row, open pack) pairs of the sparse
  // product and the x/r update, [2] those of the p update, [3] E^{-1} entries read.
  // sd_rows / sd_nnz: rows and stored entries of each subdomain for the current solve.
  unsigned long long* work;
  const int32_t* sd_rows;
  const int64_t* sd_nnz;
};

// Coarse level of the two-level additive preconditioner M^{-1} = D^{-1} + Z E^{-1} Z^T
// of the local solves.  Z has one indicator column per aggregate: a contiguous run of
// rows of one subdomain (rows are in Morton order, so a run is a spatial box);
// E = Z^T A Z per subdomain, inverted once per matrix.  With aloc = null the
// preconditioner is D^{-1} alone.
constexpr int kMaxSlots = 32;  // aggregates meeting one row tile (host-enforced)
constexpr int kMaxAgg = 1024;  // aggregates per subdomain and matrix (host-enforced)
constexpr int kCoarseRowsMin = 256;  // fewest rows of E^{-1} per block of the SIMT coarse product
template <typename T>
struct Coarse {
  const int32_t* aloc = nullptr;    // per P row: aggregate index within its subdomain
  const int32_t* aoff = nullptr;    // per subdomain: first global aggregate id
  const int32_t* nca = nullptr;     // per subdomain: aggregates of this matrix (<= kMaxAgg)
  const int32_t* tfirst = nullptr;  // per global aggregate: first tile holding its rows
  const int32_t* tcount = nullptr;  // per global aggregate: tiles holding its rows
  const int64_t* toff = nullptr;    // per tile: first row of its partials (n_tiles + 1)
  const int64_t* eoff = nullptr;    // per subdomain: offset of its nca x nca block
  const T* einv = nullptr;          // E^{-1} blocks, symmetric, row-major
  T* cpart = nullptr;               // toff[n_tiles] x kp restriction partials
  T* yc = nullptr;                  // global aggregates x kp: E^{-1} Z^T r
  double* dpart = nullptr;          // n_sd x row blocks x kp: partial r_c . y_c
  int n_max = 0;                    // largest nca
  // binary32 path with the tensor-core product (null: binary32 / binary64 SIMT):
  // E^{-1} as bf16 hi / lo planes in tcgen05 operand blocks (launch_coarse_tc_pack),
  // the first block of each subdomain, and the flag a timed-out wait sets
  const uint4* etc = nullptr;
  const int64_t* etc_off = nullptr;
  // r_c of every step as bf16 high and low planes, 2 x NP x 32 per 32-aggregate block
  // (NP = kp rounded up to 16), the first block of each subdomain at rcb_off[sd]
  __nv_bfloat16* rcb = nullptr;
  const int64_t* rcb_off = nullptr;
  int* tc_err = nullptr;
  long long tc_budget = 0;
};

template <typename T>
struct EllView {
  const int32_t* width;
  const int32_t* col;
  const T* val;
  int W;
};

// Y = A X on the rows of `tiles` (kp columns, row stride kp).
template <typename T>
void launch_spmm(const DTiles& tiles, const EllView<T>& A, const T* X, T* Y, int kp,
                 cudaStream_t st);

// Preconditioned CG (Jacobi, or two-level with a Coarse level), independent per
// (subdomain, column); one step = 4 kernels (sparse product with p.q, x/r update with
// the fine r.z and the restriction, coarse solve with beta, p update).  Columns
// c < ncn of a subdomain measure convergence against the largest ||b_c|| among them
// (block-normwise); the others against their own ||b_c||.
template <typename T>
void launch_cg_init(const DTiles& tiles, const T* b, T* x, T* r, T* p, const T* dinv,
                    int kp, int nc, int ncn, const CgState& s, const Coarse<T>& co,
                    cudaStream_t st);
// ev (null or 5 events) is recorded before the sparse product and after each of the
// four kernels of the step.
template <typename T>
void launch_cg_step(const DTiles& tiles, const EllView<T>& A, T* x, T* r, T* p, T* q,
                    const T* dinv, int kp, double tol2, const CgState& s,
                    const Coarse<T>& co, cudaStream_t st, const cudaEvent_t* ev = nullptr);
// out[0] = sum of active[0..n_sd), out[1] = sum of second (0 if null); out has 2 ints
void launch_count_active(int n_sd, const int* active, int* out, cudaStream_t st,
                         const int* second = nullptr);

// binary64 residual: r64 = b64 - A64 x64 with per-column norms; scale = 1/||r64|| for
// columns with ||r64|| > rtol ||b64|| (0 = converged); first = 1 records ||b64||.
struct RefineState {
  double *obb, *orr, *scale;  // n_sd x kp
  double* oaa;                // n_sd x kp: || |A| |x| + |b| ||^2 at the last refresh
  double *part, *part2, *part3;  // n_tiles x kp
  int* counter;               // n_sd
  int* active;                // n_sd
  int* nfloor;                // n_sd: columns stopped by the attainable-accuracy test
  int* nnear;                 // n_sd: open columns within reach of that test
  double* xx;                 // n_sd x kp: ||x64||^2 of the last residual sweep
};
// a binary64 residual below kResidualFloor * 2^-53 * || |A| |x| + |b| ||_2 is rounding
// noise of its own evaluation; launch_residual64 stops such columns
constexpr double kResidualFloor = 4.0;
// r64 = b - A x64 per column, the binary64 convergence test (rtol, or the rounding level
// of the residual itself), done flags in s.scale; first = 1 also fixes the references
// from b (x64 = 0).  floor_ref = true refreshes the rounding-level reference
// || |A| |x| + |b| || (one extra binary64 add per product).  s.nnear counts the open
// columns whose residual is within the rounding level of the bound
// anorm[sd] ||x|| + ||b|| (anorm = max row sum of |A|; ||x|| of this sweep).
void launch_residual64(const DTiles& tiles, const EllView<double>& A, const double* b64,
                       const double* x64, double* r64, int kp, int nc, int ncn, double rtol2,
                       int first, bool floor_ref, const double* anorm, const RefineState& s,
                       cudaStream_t st);
// out[sd] += stored entries in the rows of the tiles of sd (out zeroed by the caller)
void launch_count_sd_nnz(const DTiles& tiles, const EllView<double>& A, int64_t* out,
                         cudaStream_t st);
// anorm[sd] = max over the rows of tiles in sd of sum_j |a_ij| (anorm zeroed by caller)
void launch_row_abs_max(const DTiles& tiles, const EllView<double>& A, double* anorm,
                        cudaStream_t st);
void launch_zero_rows(const DTiles& tiles, double* x, int kp, cudaStream_t st);
// residual replacement of the CG recursion: rT = (T) r64, rz recomputed, done flags from
// the binary64 convergence test of launch_residual64 (scale == 0 means converged);
// reopened columns restart with pT = M^{-1} rT
template <typename T>
void launch_cg_replace(const DTiles& tiles, const double* r64, T* rT, T* pT, const T* dinv,
                       int kp, double drift, const CgState& s, const RefineState& rs,
                       const Coarse<T>& co, cudaStream_t st);

// ---------------- coarse level setup (mor_coarse.cu) ----------------
// E[sd][a][b] += A[i][j] over the stored entries of the rows of tiles, a = aloc[i],
// b = aloc[j] (entries with a or b >= nca[sd] are skipped); E zeroed by the caller.
void launch_coarse_matrix(const DTiles& tiles, const EllView<double>& A, const int32_t* aloc,
                          const int32_t* nca, const int64_t* eoff, double* E, cudaStream_t st);
// einv = E^{-1} of every SPD block E[sd] (nca[sd] <= n_max), symmetrised, in T: blocked
// Gauss-Jordan elimination without pivoting on the diagonally scaled block in binary32.
// Workspace: W [eoff[n_sd] floats], P [n_sd x 64 x 64 floats], sc [n_sd x n_max
// doubles].  bad[0] counts blocks with a non-positive diagonal entry or pivot.
template <typename T>
void launch_coarse_invert(int n_sd, int n_max, const int32_t* nca, const int64_t* eoff,
                          const double* E, float* W, float* P, double* sc, T* einv, int* bad,
                          cudaStream_t st);
constexpr int kCoarsePivots = 64;  // pivot block of launch_coarse_invert
// E^{-1} of every subdomain as tcgen05 A-operand blocks for y_c = E^{-1} r_c: block
// (m * nkb + kb) of subdomain sd (at etc_off[sd], 16 KB each, nkb = ceil(n / 32)) holds
// E^{-1}[128 m + r][32 kb + k] (zero outside n) split into a bf16 high part and the
// bf16 rounding of the remainder, two K-major planes of 128 x 32.
constexpr int kCoarseTcM = 128;  // rows of y_c per tensor-core block (the MMA M)
void launch_coarse_tc_pack(int n_sd, int blocks_max, const int32_t* nca, const int64_t* eoff,
                           const float* einv, const int64_t* etc_off, uint4* out,
                           cudaStream_t st);
// x64 += xT, xT = 0
template <typename T>
void launch_accum_reset(const DTiles& tiles, T* xT, double* x64, int kp, cudaStream_t st);
// dst = (T) src on the rows of tiles
template <typename T>
void launch_cast(const DTiles& tiles, const double* src, T* dst, int kp, cudaStream_t st);

// ---------------- dense per-subdomain kernels (mor_dense.cu) ----------------
// G[sd] = X^T Y over the rows of tiles: nx x ny with row stride ldg and subdomain
// stride ldg*ldg (also for nx = ny = 1).  part: n_tiles x nx x ny doubles.
void launch_gram(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                 const double* Y, int ldy, int ny, double* part, int* counter, double* G,
                 int ldg, cudaStream_t st);
// x_sd^T y per subdomain for one column y: g[sd * ldg + i] (ldg >= nx)
void launch_gram_vec(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                     const double* y, int ldy, double* part, int* counter, double* g,
                     int ldg, cudaStream_t st);
// symmetric eigensolver (cyclic Jacobi, parallel ordering) per subdomain on the
// leading n x n block of A[sd] (stride ld); evals descending (n_sd x ld), evecs
// columns (n_sd x ld x ld).
void launch_sym_eig(int n_sd, const double* A, int ld, int n, double* evals,
                    double* evecs, cudaStream_t st);
// M[sd] from an eigen-decomposition: mode 0: V_j / sqrt(l_j) for l_j > rel * l_0 (else 0
// column); mode 1: V_j for j < keep (or j < keep_sd[sd]); mode 2: V_j for l_j > rel
// (absolute), j < keep and j < keep_sd[sd]; kept[sd] = number of nonzero columns.
void launch_make_M(int n_sd, int mode, const double* evals, const double* evecs, int ld,
                   int n, double rel, int keep, double* M, int* kept, cudaStream_t st,
                   const int32_t* keep_sd = nullptr);
// Y[r, j] = sum_{l < nin} X[r, l] M[sd(r)][l, j] for j < nout; columns nout..ldy-1 of Y
// are zeroed.
void launch_rowmul(const DTiles& tiles, const double* X, int ldx, int nin, const double* M,
                   int ldm, double* Y, int ldy, int nout, cudaStream_t st);
// dst[r, dc0 + c] = src[map[r], sc0 + c] (map null: r), c < ncols
// wide-sketch versions (k up to 511 columns, mor_wide.cu): the Gram needs a partial
// buffer of n_sd * gram_wide_chunks(n_sd, nx, ny) * nx * ny doubles, the eigensolver a
// work buffer of n_sd * 2 * m * m doubles (m = n rounded up to even, n <= 1024)
int gram_wide_chunks(int n_sd, int nx, int ny);
void launch_gram_wide(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                      const double* Y, int ldy, int ny, double* part, double* G, int ldg,
                      int64_t sd_stride, cudaStream_t st);
void launch_sym_eig_wide(int n_sd, const double* A, int ld, int n, double* evals,
                         double* evecs, double* work, cudaStream_t st);
void launch_rowmul_wide(const DTiles& tiles, const double* X, int ldx, int nin,
                        const double* M, int ldm, double* Y, int ldy, int nout,
                        cudaStream_t st);
// paper-literal weights (mor_explicit.cu): dense per-subdomain factors
void launch_ell_to_dense(int64_t n_rows, const int32_t* row_sd, const int32_t* rloc,
                         const int32_t* cloc, const EllView<double>& A, const int32_t* r_sub,
                         const int32_t* r_n, const int32_t* c_sub, const int32_t* ncols,
                         const int32_t* ld, const int64_t* doff, double* D, cudaStream_t st);
void launch_potrf(int n_sd, int n_max, double* D, const int64_t* doff, const int32_t* nn,
                  int* bad, cudaStream_t st);
void launch_transpose_block(int n_sd, int m_max, const double* In, const int64_t* ioff,
                            const int32_t* nn, const int32_t* soff, const int32_t* mm,
                            double* Out, const int64_t* ooff, int transpose, cudaStream_t st);
void launch_trsv_cols(int n_sd, int n_max, int ncol_max, const double* T, const int64_t* toff,
                      const int32_t* nn, const int32_t* tld, const int32_t* tsh, double* X,
                      const int64_t* roff, int ldx, const int32_t* ncol, int forward,
                      cudaStream_t st);
void launch_trsv_rows(const double* R, const int64_t* roff_r, const int32_t* mm, double* X,
                      const int64_t* roff, int ldx, const int* sd_of_warp,
                      const int* row_of_warp, int n_warps, cudaStream_t st);
void launch_trmv_upper(int n_sd, int n_max, int ncol_max, const double* U, const int64_t* uoff,
                       const int32_t* nn, const double* Z, double* Y, const int64_t* roff,
                       int ld, const int32_t* ncol, cudaStream_t st);
void launch_node_normals(int n_sd, int m_max, const int32_t* bnode, const int64_t* boff,
                         const int32_t* mm, const int32_t* kk, int k, uint64_t seed,
                         uint32_t sd_base, double* out, int ld, cudaStream_t st);
// tensor-core Grams (mor_tc.cu), columns nx, ny <= 128: partial buffers of
// n_items * tc_gram_chunks(n_items) * nx * ny doubles, range of 2 * n_items int64, err
// set when a bounded wait ran out
int tc_gram_chunks(int n_items);
void launch_tc_gram(const DTiles& tiles, int n_sd, const double* X, int ldx, int nx,
                    const double* Y, int ldy, int ny, double* part, int64_t* range, double* G,
                    int ldg, int64_t stride, long long budget, int* err, cudaStream_t st);
void launch_tc_pair_blocks(int n_pairs, const int64_t* pair_ptr, const int32_t* urow,
                           const int32_t* vrow, const double* aval, const double* Q, int kq,
                           double* part, double* G, double* blocks, long long budget, int* err,
                           cudaStream_t st);
void launch_tc_gram_rows(int64_t rows, const double* X, int ldx, int nx, const double* Y,
                         int ldy, int ny, double* part, int64_t* range, double* G,
                         long long budget, int* err, cudaStream_t st);
// autotuner of the sparse product (mor_sparse.cu)
void autotune_enable(bool on);
void autotune_reset();
int autotune_entries(int64_t* out, int max_entries);
void launch_gather_rows(int64_t n_rows, const int32_t* map, const double* src, int lds,
                        int sc0, double* dst, int ldd, int dc0, int ncols, cudaStream_t st);
// dst[map[r], c] = src[r, c]
void launch_scatter_rows(int64_t n_rows, const int32_t* map, const double* src, int lds,
                         double* dst, int ldd, int ncols, cudaStream_t st);
// dst[r, col] = src[r] for the rows of tiles
void launch_set_col(const DTiles& tiles, const double* src, double* dst, int ld, int col,
                    cudaStream_t st);
void launch_to_float(int64_t n, const double* src, float* dst, cudaStream_t st);

// ---------------- reduced system (mor_reduced.cu) ----------------
// K~_ij = sum_e a_e Q[u_e]^T Q[v_e] per interface pair; block 2p = (i, j), 2p+1 = (j, i)
void launch_pair_blocks(int n_pairs, const int64_t* pair_ptr, const int32_t* urow,
                        const int32_t* vrow, const double* aval, const double* Q, int kq,
                        double* blocks, cudaStream_t st);
struct RcgState {
  double *x, *r, *p, *q;    // dim
  double* part;             // n_sd x 2
  int* counter;             // 1
  double* scal;             // [0] rz, [1] bb, [2] alpha, [3] beta, [4] rr
  int* flag;                // [0] done, [1] iterations
};
// the reduced CG in one cooperative launch with bounded grid-barrier waits; returns the
// grid size, or -1 when a cooperative launch is not possible.  sync: 3 zeroed words.
int launch_rcg_persistent(int n_sd, int kq, const int32_t* nbr_ptr, const int32_t* nbr_sd,
                          const int32_t* nbr_blk, const double* blocks, const double* bt,
                          double tol2, int max_iter, const RcgState& s, unsigned* sync,
                          long long budget, cudaStream_t st);
void launch_wait_unset_flag(unsigned* sync, long long budget, int* status, cudaStream_t st);
void launch_rcg_init(int n_sd, int kq, const double* bt, const RcgState& s,
                     cudaStream_t st);
void launch_rcg_step(int n_sd, int kq, const int32_t* nbr_ptr, const int32_t* nbr_sd,
                     const int32_t* nbr_blk, const double* blocks, double tol2,
                     const RcgState& s, cudaStream_t st);
void launch_lift(int64_t n_o, const int32_t* o_node, const int32_t* o_sd, const double* Q,
                 int kq, const double* x, double* u, cudaStream_t st);

}  // namespace mor
