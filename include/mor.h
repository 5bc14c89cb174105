/*
 * mor.h -- C ABI of the GB300 localized model-order-reduction library (libmor).
 *
 * Method: "Distributed finite element solution using model order reduction"
 * (Gustafsson, Hannukainen, Kohonen).  The library runs the data-parallel part of the
 * paper's three-step framework (Sec. 6) on one GPU:
 *   step 1  mor_build_subdomains  overlapping subdomains and r-hop extensions (Sec. 3,
 *                                 Sec. 6 step 1, Sec. 7.1 "r-hops")
 *   step 2  mor_build_bases       optimal local bases (Sec. 4, Sec. 6 step 2 and
 *                                 "Randomized numerical linear algebra")
 *   step 3  mor_project           Q^T A Q by the interface-only product (Eq. (23), Sec. 6
 *                                 step 3), then mor_solve_reduced (diagonally
 *                                 preconditioned CG on the reduced system, Sec. 6 step 3)
 * plus mor_lift (u~ = sum_i S_i Q_i x_i, Eq. (11) with Def. 3.1) and mor_energy_norm.
 *
 * Model problem: -div(k grad u) = 1 in Omega, u = 0 on the boundary, P1 tetrahedra
 * (Sec. 2; a per-element coefficient k as in Sec. 7.2).
 *
 * Conventions
 *   - Return value: MOR_OK (0) or a negative MOR_ERR_* code; mor_last_error() gives a
 *     thread-local message for the last failing call on the calling thread.
 *   - Pointers marked [host] are read only during the call.  Pointers marked [device]
 *     are CUDA device pointers owned by the caller; those given to
 *     mor_build_subdomains must stay valid until the handle is freed.
 *   - Handles are opaque, owned by the library and released by mor_free_*.  They own
 *     their device memory.
 *   - stream: a cudaStream_t (NULL = legacy default stream).  Every call enqueues its
 *     GPU work on that stream and returns after its own status is known (the call
 *     synchronizes the stream when it needs a device-side status).
 *   - Index arrays are int32 in row-major layout; floating point is IEEE binary64
 *     unless stated otherwise.
 */
#ifndef MOR_H
#define MOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MOR_OK 0
#define MOR_ERR_ARG (-1)            /* invalid argument or size                        */
#define MOR_ERR_BAD_MESH (-2)       /* element with non-positive volume, bad index     */
#define MOR_ERR_OOM (-3)            /* device or host allocation failed                */
#define MOR_ERR_NOT_CONVERGED (-4)  /* an iterative solve hit max_iter (results kept)  */
#define MOR_ERR_TIMEOUT (-5)        /* a bounded device-side wait ran out (the kernel
                                       returned; the CUDA context stays usable)       */
#define MOR_ERR_CUDA (-6)           /* CUDA runtime or launch error                    */
#define MOR_ERR_STATE (-7)          /* handle used in the wrong state                  */

#define MOR_FP64 0   /* every local solve, Gram and eigensolve in binary64             */
#define MOR_MIXED 1  /* binary32 CG recursions with binary64 residual replacement;
                        binary64 small dense factorisations and reduced solve           */

typedef struct mor_subdomains_s mor_subdomains;
typedef struct mor_bases_s mor_bases;
typedef struct mor_reduced_s mor_reduced;

/* A P1 tetrahedral mesh.  Host copies drive the index construction of step 1; device
 * copies feed the numeric kernels.  Elements must be positively oriented
 * (det[x1-x0, x2-x0, x3-x0] > 0); otherwise MOR_ERR_BAD_MESH. */
typedef struct {
  int64_t n_nodes;
  int64_t n_tets;
  const int32_t* tets;       /* [host]   n_tets x 4 vertex ids                          */
  const uint8_t* dirichlet;  /* [host]   n_nodes, 1 = node on the Dirichlet boundary    */
  const double* xyz_dev;     /* [device] n_nodes x 3 coordinates                        */
  const int32_t* tets_dev;   /* [device] n_tets x 4, same content as tets               */
  const double* kappa_dev;   /* [device] n_tets coefficient k_T > 0                     */
} mor_mesh;

/* Step 1 (Sec. 3, Sec. 6 step 1, Sec. 7.1).  owner[host, n_nodes] labels every node with
 * its subdomain 0..n_sub-1 (the graph partition; every label must occur).  For each
 * subdomain i: P_i = owned nodes; omega_i = elements touching P_i; the extension
 * T_i^+ = elements touching the r_hops-hop ball of P_i in the edge graph of the mesh;
 * I = free nodes of T_i^+ all of whose elements lie in T_i^+, B = its other free nodes.
 * r_hops >= 1, or r_hops = -1 for a per-subdomain rule r_i = max(1, round(|P_i|^(1/3)/2))
 * (about half the subdomain width, so the extension roughly doubles its diameter,
 * Sec. 7.1).  The mesh's device arrays are referenced, not copied. */
int mor_build_subdomains(const mor_mesh* mesh, const int32_t* owner, int32_t r_hops,
                         void* stream, mor_subdomains** out);

/* A P1 tetrahedral mesh with every array in host memory (pinned memory makes the
 * copies faster; pageable memory works too). */
typedef struct {
  int64_t n_nodes;
  int64_t n_tets;
  const int32_t* tets;       /* [host] n_tets x 4 vertex ids                            */
  const uint8_t* dirichlet;  /* [host] n_nodes, 1 = node on the Dirichlet boundary      */
  const double* xyz;         /* [host] n_nodes x 3 coordinates                          */
  const double* kappa;       /* [host] n_tets coefficient k_T > 0                       */
} mor_mesh_host;

/* Step 1 from host arrays: as mor_build_subdomains (wave_subdomains = 0) or
 * mor_build_subdomains_streamed (wave_subdomains > 0), but the library copies the
 * coordinates, connectivity and coefficient to the device itself, on `stream`, into
 * memory owned by the handle (freed by mor_free_subdomains).  The host arrays are only
 * read during the call. */
int mor_build_subdomains_host(const mor_mesh_host* mesh, const int32_t* owner,
                              int32_t r_hops, int32_t wave_subdomains, void* stream,
                              mor_subdomains** out);

/* Step 1 for meshes whose per-subdomain structures do not fit at once (the 440^3
 * cube of 8000 subdomains: ~6e8 extended rows).  Builds and keeps only the global part
 * (owned DOFs, interface entries, node -> element incidence) plus host copies of the
 * mesh connectivity, Dirichlet flags and coordinates.  mor_build_bases then builds the
 * per-subdomain part in waves of wave_subdomains consecutive subdomains and runs each
 * wave on the device in turn; mor_project, mor_solve_reduced, mor_lift and
 * mor_energy_norm work as for mor_build_subdomains.  mor_subdomains_counts reports
 * only the owned DOFs and r_i (other entries -1); mor_subdomains_indices and
 * mor_debug_sketch_rhs return MOR_ERR_STATE.  The paper has no counterpart (its
 * workers each build one subdomain, Sec. 6). */
int mor_build_subdomains_streamed(const mor_mesh* mesh, const int32_t* owner, int32_t r_hops,
                                  int32_t wave_subdomains, void* stream,
                                  mor_subdomains** out);

/* Sizes of step 1.  counts[host, n_sub x 7] receives per subdomain
 * {|I|, |B|, |omega dofs|, |owned dofs|, |T_i^+|, |omega_i elements|, r_i}; n_sub_out
 * may be NULL.  Pass counts = NULL to query n_sub only. */
int mor_subdomains_counts(const mor_subdomains* h, int32_t* n_sub_out, int64_t* counts);

/* Copy one index list of subdomain `sub` (global node ids, ascending) into out[host]:
 * which = 0 I, 1 B, 2 omega dofs, 3 owned dofs, 4 T_i^+ element ids,
 * 5 omega_i element ids.  The length is the matching entry of mor_subdomains_counts. */
int mor_subdomains_indices(const mor_subdomains* h, int32_t sub, int32_t which,
                           int32_t* out);

#define MOR_SKETCH_FIELD 0 /* W = ((H^+)^{-1} L xi)_B, L L^T = H^+ element-wise       */
#define MOR_SKETCH_PAPER 1 /* W = R_BB^{-1} S, S Gaussian on B, R_BB from a dense
                              Cholesky factor of H^+ in [I; B] order (Sec. 6, Lemma 4.1);
                              subdomains with |I| + |B| <= 6144, one-shot plans        */

typedef struct {
  int32_t rank;        /* m: singular vectors kept per subdomain (fixed-rank mode)      */
  int32_t oversample;  /* p: k = m + p sketch columns (Halko et al., App. B)           */
  const int32_t* ranks; /* [host, n_sub] per-subdomain m_i replacing `rank` (may be NULL):
                          subdomain i sketches k_i = m_i + p columns                    */
  double eps;          /* > 0: tolerance mode (Eq. (15)): keep the sigma_j > eps among
                          the k_i computed, instead of the first m_i                    */
  uint64_t seed;       /* Philox-4x32-10 key of the Gaussian draws                      */
  int32_t precision;   /* MOR_FP64 or MOR_MIXED                                         */
  int32_t sketch;      /* MOR_SKETCH_FIELD or MOR_SKETCH_PAPER                          */
  double cg_rtol;      /* every local solve: ||b - A x||_2 <= cg_rtol ||b||_2 per column,
                          residual measured in binary64.  A column also stops when its
                          residual is below 4 u || |A| |x| + |b| ||_2 (u = 2^-53), the
                          rounding level of the binary64 residual itself: with high
                          coefficient contrast a small cg_rtol can lie below it        */
  int32_t max_iter;    /* CG iterations per local solve                                 */
  int32_t replace_every; /* the CG residual is replaced by the binary64 residual
                          b - A x every replace_every iterations (rounded to a multiple
                          of 8) and whenever the recursion reports convergence         */
  int32_t normwise;    /* 1: the lifting columns of a subdomain share one reference,
                          the largest right-hand side of its block (the weighted SVD
                          needs the block accurate normwise); 0: each column is
                          measured against its own right-hand side.  The load column
                          u_0 is always measured against its own.                       */
  double drift_restart; /* at a replacement, a column whose true residual norm exceeds
                          drift_restart x its recursive one restarts from p = D^{-1} r
                          (its search direction no longer matches the residual)       */
  double sketch_rtol;  /* tolerance of the sketch solve W = ((H^+)^{-1} L xi)_B; W only
                          has to be a Gaussian-like test matrix, so it may be loose
                          (<= 0: use cg_rtol)                                           */
  double tau;          /* diagonal-block update: drop eigen-directions of
                          V^T A_ii V below tau * largest                                */
  double orth_tol;     /* Gram orthonormalisation: drop directions below
                          orth_tol * largest Gram eigenvalue                             */
  int32_t coarse_rows; /* local preconditioner: > 0 adds a coarse level to Jacobi,
                          M^{-1} = D^{-1} + Z E^{-1} Z^T with Z the indicators of
                          spatial aggregates of about coarse_rows rows (runs of the
                          Morton-ordered rows of a subdomain, at most 1024 per
                          subdomain) and E = Z^T A Z inverted per subdomain; 0: Jacobi
                          only; < 0 (default): 35 in MOR_MIXED, 300 in MOR_FP64 (the
                          coarse product runs in the working precision).  Changes
                          iteration counts, not the solutions.                        */
  int32_t h1_weighted; /* 0: the H1 inner product of H_i and H^+ is the unweighted
                          int grad w . grad v + w v of Sec. 4 (as printed); 1: its
                          gradient part is weighted by the coefficient k, a variant for
                          high contrast (the paper analyses k = 1, Sec. 7.3)           */
  int32_t sketch_div;  /* > 0: subdomain i sketches k_i = max(1, floor(M_i / sketch_div))
                          columns, M_i = |B_i| (the paper's k_i = floor(M_i / 8) with
                          sketch_div = 8, Sec. 7.1 and App. C); needs eps > 0 (tolerance
                          mode) and a one-shot plan; k_i <= 511.  0: k_i = m_i + p.    */
  int32_t sub_begin;   /* streamed plans only: build the bases of subdomains            */
  int32_t sub_end;     /* [sub_begin, sub_end) and leave the others empty (kept 0, Q and
                          b~ zero), e.g. one GPU's share of a multi-GPU run or a sampled
                          check; sub_end <= 0 means all.  The draws of a subdomain do
                          not depend on the range.  One-shot plans require the whole
                          range (MOR_ERR_ARG otherwise).                                */
  int32_t tc_gram;     /* MOR_MIXED: 1 (default) forms the H_i-Grams and G_B on the
                          tensor cores (tcgen05, exact 7-bit bf16 slices: entry (i, j)
                          off by at most about 2^-28 rows max|X_i| max|Y_j|), and the
                          coarse-level product E^{-1} r_c of the local solves for up to
                          128 columns (bf16 high and low parts of both factors, three
                          products, FP32 accumulators); 2 also
                          forms the interface blocks of Eq. (23) there, whose error is
                          then relative to the largest a_e-weighted entry of a column
                          (at 1e4 coefficient contrast it moves x^T K~ x away from the
                          lifted energy by about 1e-5 relative); 0 keeps all of them
                          in binary64 SIMT.  V^T A V (the diagonal-block update) and
                          MOR_FP64 always use binary64.  Other values: MOR_ERR_ARG.   */
  int32_t explicit_svd; /* 1: the explicit weighted SVD of Eq. (14) instead of the
                          randomized one: dense Cholesky factors of A_II, H_i and H^+
                          (R_i, R_BB, Lemma 4.1), Z_i = C_i A_II^{-1} A_IB, and the
                          singular vectors of R_i Z_i R_BB^{-1} (|B| <= 1024,
                          |I| + |B| <= 6144, one-shot plans); rank / eps select the
                          kept directions, sketch and oversample are not used          */
} mor_basis_opts;

/* Fill opts with defaults (rank 8, oversample 5, seed 0, MOR_MIXED, cg_rtol 1e-9,
 * max_iter 20000, replace_every 40, normwise 1, drift_restart 1.5, sketch_rtol 0,
 * tau 1e-12, orth_tol 1e-14, coarse_rows -1, h1_weighted 0, sketch_div 0, sub_begin 0,
 * sub_end 0, tc_gram 1, explicit_svd 0). */
int mor_basis_opts_default(mor_basis_opts* opts);

/* Step 2 for every subdomain in one batch (Sec. 4, Sec. 6 step 2, Eq. (24)):
 * assemble A_II, A_IB, H^+ on T_i^+ and H_i, A[P_i,P_i] on omega_i; solve
 * A_II u_0 = b_I; sketch W (k columns, field mode); X = C_i A_II^{-1} A_IB W;
 * orthonormalise X in the H_i inner product (R_i X^ = Qh); T = A_BI A_II^{-1} C_i^T H_i X^;
 * G_B = T^T S_B^{-1} T with S_B^{-1} T from a solve with H^+ (Lemma 4.1), which equals
 * B B^T for the matrix B of Eq. (24); eig(G_B) gives sigma_j^2 and the rotation of the
 * top `rank` directions; V = D_i [u_0, X^ U_m]; Q_i = V W Lambda^{-1/2} from
 * eig(V^T A[P_i,P_i] V) (so Q_i^T A_ii Q_i = I); b~_i = Q_i^T b[P_i].
 * Returns MOR_ERR_NOT_CONVERGED (with the bases still built) if a local solve stopped
 * at max_iter. */
int mor_build_bases(const mor_subdomains* sd, const mor_basis_opts* opts, void* stream,
                    mor_bases** out);

/* Sizes of step 2: *kq = columns stored per subdomain (>= max kept + 1, multiple of 4,
 * at most 128),
 * *k = the largest sketch width k_i; kept[host, n_sub] = basis columns kept per
 * subdomain (may be NULL); *total_kept = sum of kept (may be NULL). */
int mor_bases_info(const mor_bases* h, int32_t* kq, int32_t* k, int32_t* kept,
                   int64_t* total_kept);

/* sigma[host, n_sub x k]: the singular values of B (Eq. (24)) per subdomain, descending
 * (zeros beyond k_i). */
int mor_bases_sigma(const mor_bases* h, double* sigma);

/* R_BB of subdomain `sub` (Lemma 4.1: the trailing |B| x |B| block of the upper
 * Cholesky factor of H^+ in [I; B] order, B in ascending node order) into
 * out[host, |B| x |B|], row-major; only for bases built with MOR_SKETCH_PAPER or
 * explicit_svd (MOR_ERR_STATE otherwise). */
int mor_bases_get_rbb(const mor_bases* h, int32_t sub, double* out);

/* Q_i of subdomain `sub` into out[host, |owned| x kq] (row-major; rows = owned dofs in
 * ascending node order, columns beyond kept[sub] are zero). */
int mor_bases_get_Q(const mor_bases* h, int32_t sub, double* out);

/* b~ for all subdomains into out[host, n_sub x kq]. */
int mor_bases_get_bt(const mor_bases* h, double* out);

/* Solver statistics of the last mor_build_bases: stats[host, 8] =
 * {iterations of the four local solves (sketch, forward, adjoint, H^+), residual
 * replacements (sum), columns not converged, columns that stopped on the
 * attainable-accuracy test instead of cg_rtol, 0}; summed over the waves of a
 * streamed plan. */
int mor_bases_stats(const mor_bases* h, int64_t* stats);

/* Step 3a (Eq. (23), Sec. 6 step 3): K~ with identity diagonal blocks (from step 2) and
 * off-diagonal blocks K~_ij = Q_i^T A_0[P_i, P_j] Q_j, A_0 assembled on the interface
 * elements omega_0 only, iterating over neighbouring pairs. */
int mor_project(const mor_subdomains* sd, const mor_bases* b, void* stream,
                mor_reduced** out);

/* Reduced system sizes: *dim = n_sub * kq, *n_blocks = stored off-diagonal blocks. */
int mor_reduced_info(const mor_reduced* h, int64_t* dim, int64_t* n_blocks);

/* Dense copy of K~ into out[host, dim x dim] (for small systems; MOR_ERR_ARG if
 * dim > 20000). */
int mor_reduced_dense(const mor_reduced* h, double* out);

typedef struct {
  int32_t iterations;
  int32_t converged;     /* 1 if ||b~ - K~ x|| <= rtol ||b~||                          */
  double rel_residual;   /* final ||b~ - K~ x|| / ||b~|| (recursive residual)          */
  double energy;         /* E = b~^T x                                                  */
} mor_solve_info;

/* Step 3b: K~ x = b~ by CG with the diagonal (= identity) preconditioner, binary64.
 * x_dev [device, dim] is written.  info may be NULL.  The whole iteration runs in one
 * cooperative launch (blocks over the block rows of K~, grid barriers between the
 * phases of an iteration); every barrier wait is bounded by the wait budget
 * (mor_set_wait_budget), and a wait that runs out ends the kernel with
 * MOR_ERR_TIMEOUT instead of hanging.  Where a cooperative launch is not possible the
 * same iteration runs as three launches per step. */
int mor_solve_reduced(const mor_reduced* h, double rtol, int32_t max_iter, void* stream,
                      double* x_dev, mor_solve_info* info);

/* mor_solve_reduced without any allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library allocate device memory, such as a
 * host application whose device memory is owned by its own allocator or memory pool,
 * or a time-critical loop that cannot afford cudaMalloc's implicit device-wide
 * synchronization.  It runs the same CG iteration as mor_solve_reduced and makes no
 * call to cudaMalloc, cudaFree or any allocating routine.
 *
 * Inputs [device, caller-owned]: the block-sparse reduced matrix as in mor_project:
 *   nbr_ptr_dev[n_sub + 1], nbr_sub_dev[], nbr_blk_dev[] list, per block row i, its
 *   off-diagonal blocks (neighbour subdomain, block index); blocks_dev holds
 *   kq x kq row-major blocks; the diagonal blocks are the identity and are not stored.
 *   bt_dev[n_sub * kq] is the reduced load.
 * Output [device, caller-owned]: x_dev[n_sub * kq].  info [host] may be NULL.
 * Work space: a fixed device array inside the library (1,703,952 doubles = 13.6 MB:
 * the three CG vectors plus partial sums).  It is placed on a device when the
 * library's device code for this entry point is loaded there (with CUDA's default lazy
 * module loading: during the first call on that device) and stays until the process
 * exits.  Limits: n_sub * kq <= 524288 and n_sub <= 65536; larger systems are rejected
 * with MOR_ERR_ARG and a message.
 * Set-up: the first call on a device (and the first after that device's context was
 * reset) looks up the array's device address with that device current and keeps it.
 * That first call loads the module, which may allocate and synchronize inside the
 * CUDA runtime: make it once at initialisation, before any stream capture.  Later
 * calls on that device allocate nothing.
 * The call waits for its stream every 16 iterations to read the convergence flag, and
 * at the end to read the residual and energy.
 * Every call shares the one array and leaves its contents behind; the call clears the
 * state that must start at zero.  Calls whose GPU work overlaps (for example on two
 * streams, or two host threads) race on the array: serialise them.
 * Returns MOR_OK, MOR_ERR_NOT_CONVERGED (x holds the last iterate), MOR_ERR_ARG or
 * MOR_ERR_CUDA. */
int mor_solve_reduced_noalloc(int32_t n_sub, int32_t kq, const int32_t* nbr_ptr_dev,
                              const int32_t* nbr_sub_dev, const int32_t* nbr_blk_dev,
                              const double* blocks_dev, const double* bt_dev, double rtol,
                              int32_t max_iter, void* stream, double* x_dev,
                              mor_solve_info* info);

/* Budget of every bounded device-side wait (grid barriers of mor_solve_reduced, the
 * mbarrier waits of the tensor-core kernels), in seconds of the GPU's SM clock
 * (default 1 s; a wait normally lasts microseconds), between 1 ms and 3600 s
 * (MOR_ERR_ARG otherwise): a tensor-core kernel whose wait ran out waits once more, with
 * the same budget, for its MMAs in flight before it releases its tensor memory.
 * Process-wide, not thread-safe.  The paper has no counterpart. */
int mor_set_wait_budget(double seconds);

/* Test of the timeout path: one thread waits, with the given budget in seconds, on a
 * device flag that nothing sets.  *timed_out [host] = 1 when the wait ran out and the
 * kernel returned (the expected outcome), 0 otherwise; returns MOR_ERR_TIMEOUT in the
 * first case and MOR_OK in the second.  Allocates 16 bytes of device memory for the
 * flag.  The paper has no counterpart. */
int mor_debug_wait_timeout(double seconds, int32_t* timed_out);

/* u~ = sum_i S_i Q_i x_i on all nodes (zero on the Dirichlet boundary):
 * x_dev [device, dim], u_dev [device, n_nodes]. */
int mor_lift(const mor_subdomains* sd, const mor_bases* b, const double* x_dev,
             double* u_dev, void* stream);

/* ||u1 - u2||_A = sqrt(sum_T (u1-u2)_T^T K_T (u1-u2)_T) over all elements; u1_dev,
 * u2_dev [device, n_nodes]; u2_dev may be NULL (then ||u1||_A).  *out [host]. */
int mor_energy_norm(const mor_subdomains* sd, const double* u1_dev, const double* u2_dev,
                    double* out, void* stream);

/* Host-only check of step 1 (no device needed; mesh arrays on the host, xyz may be
 * NULL): builds the one-shot plan of mor_build_subdomains, the global plan and the
 * waves of wave_subdomains of mor_build_subdomains_streamed, and the coarse-level
 * aggregates for coarse_rows.  out[host, 8] = {n_sub, extended rows, waves, wave rows /
 * patterns / incidences / maps that differ from the one-shot plan, aggregate violations
 * (not contiguous, not I-then-B, above the cap), most aggregates meeting one row tile,
 * most aggregates of one subdomain, owned DOFs}.  The paper has no counterpart. */
int mor_debug_plan_check(int64_t n_nodes, int64_t n_tets, const int32_t* tets,
                         const uint8_t* dirichlet, const int32_t* owner, const double* xyz,
                         int32_t r_hops, int32_t wave_subdomains, int32_t coarse_rows,
                         int64_t* out);

/* Debug/parity access: the field-sketch right-hand side L xi of subdomain `sub`
 * (rows I then B, k columns, row-major) into out[host, (|I|+|B|) x k], computed by the
 * same kernel mor_build_bases uses (binary32 Gaussian draws, binary64 element factors
 * and sums, in every precision). */
int mor_debug_sketch_rhs(const mor_subdomains* sd, const mor_basis_opts* opts,
                         int32_t sub, double* out, void* stream);

/* Debug/parity access: G = X^T Y on the tensor cores, as the mixed path computes its
 * Grams (tcgen05 MMAs on exact 7-bit bf16 slices, FP32 accumulators in TMEM, binary64
 * combination; see mor_basis_opts.tc_gram).  X_dev [device, rows x nx], Y_dev [device,
 * rows x ny] row-major binary64, nx, ny <= 128; G_dev [device, nx x ny] is written.
 * Allocates its work space.  The paper has no counterpart (its contractions are
 * binary64). */
int mor_debug_tc_gram(int64_t rows, int32_t nx, int32_t ny, const double* X_dev,
                      const double* Y_dev, double* G_dev, void* stream);

/* Debug/parity access: the inverse that the coarse level of the local preconditioner
 * takes of every aggregate matrix E = Z^T A Z (mor_basis_opts.coarse_rows): blocked
 * Gauss-Jordan elimination without pivoting on diag(E)^{-1/2} E diag(E)^{-1/2} in
 * binary32, symmetrised.  E_dev [device, n x n] symmetric positive definite binary64,
 * 1 <= n <= 1024; Einv_dev [device, n x n] is written.  MOR_ERR_ARG on a non-positive
 * diagonal entry or pivot.  Allocates its work space.  The paper has no counterpart (its
 * local solves are direct). */
int mor_debug_coarse_inverse(int32_t n, const double* E_dev, double* Einv_dev, void* stream);

/* Kernel timing for the roofline: when enabled, the four kernels of every local CG
 * step of mor_build_bases are bracketed by CUDA events on the launching stream.
 * mor_profile_query fills out[host, 4] = {launches, total milliseconds, algorithmic
 * bytes moved, 0} accumulated since the last reset for `family` = 2 * kind + wide,
 * kind 0 = sparse product q = A p with the p.q column sums, 1 = x/r update with the
 * r.r and fine r.z sums and the restriction Z^T r, 2 = p update with the
 * prolongation and the p.r sums, 3 = coarse solve E^{-1} Z^T r; wide 0 = binary32,
 * 1 = binary64 (families 0..7).  Algorithmic bytes count the work actually done
 * (subdomains and 16-byte column packs whose columns have all converged are skipped):
 * every stored nonzero (value + column index) of an active subdomain's sparse
 * product, and every element of an open pack the kernel must read or write once (the
 * coarse kernel: its E^{-1} blocks once per open 16-column chunk); diagonal,
 * aggregate-index and coarse-correction reads are not counted.  Process-wide state,
 * not thread-safe. */
int mor_profile_enable(int32_t on);
int mor_profile_reset(void);
int mor_profile_query(int32_t family, double* out);

/* Autotuner of the local solves' sparse product q = A p (with the p.q sums): the first
 * product of each (precision, column count, slot width) the process meets is timed in
 * four launch configurations (1 or 2 slot records gathered per batch, blocks of 256 or
 * 128 threads; CUDA events, three launches each after one warm-up) and the fastest is
 * used from then on.  All four give the same bits.  mor_autotune(0) turns tuning off
 * (the first configuration is used where nothing is cached), mor_autotune(-1) clears the
 * cache.  mor_autotune_report fills out[host, 8 x max_entries] with {binary64, columns,
 * slot width, chosen configuration, microseconds of configurations 0..3} per entry and
 * *n with the entry count.  Process-wide, not thread-safe.  The paper has no
 * counterpart. */
int mor_autotune(int32_t on);
int mor_autotune_report(int64_t* out, int32_t max_entries, int32_t* n);

/* Number of CUDA kernels this library has launched in the process so far
 * (host-side counter), into *out. */
int mor_kernel_launches(int64_t* out);

void mor_free_subdomains(mor_subdomains* h);
void mor_free_bases(mor_bases* h);
void mor_free_reduced(mor_reduced* h);
const char* mor_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MOR_H */
