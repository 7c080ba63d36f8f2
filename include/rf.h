/*
 * rf.h — C ABI of the GB300 (sm_103a) LIMEX stage solver for incompressible,
 * immiscible two-phase (water / DNAPL) flow in heterogeneous porous media.
 *
 * The method is that of "A highly scalable numerical framework for reservoir
 * simulation on UG4 platform" (arXiv 2506.04763):
 *   - vertex-centred finite volumes (Sec. 3.1, Eqs. dsW, dpN) with fully
 *     upwinded relative permeabilities (Sec. 3.2, Eqs. up_krw, up_krn),
 *     gravity, capillary pressure, and the p_dmin interface condition between
 *     materials of different entry pressure (Sec. 3.3, Eqs. pdmin, hSw,
 *     krn_ip, krw_ip);
 *   - the linearly implicit Euler / LIMEX stage (M - tau J) du = tau F with the
 *     exact Jacobian J = F_u and extrapolation (Sec. 4);
 *   - BiCGSTAB preconditioned by geometric multigrid (Sec. 5, setup paragraph).
 * Primary unknowns per vertex are (p_w, S_n), interleaved.
 *
 * Conventions shared by every entry point
 *   Grid: structured box of n[0] x n[1] (x n[2]) vertices, spacing h.  Vertex
 *     v = i + n0*(j + n1*k) (x fastest); cell c = i + (n0-1)*(j + (n1-1)*k).
 *     Multigrid coarsening needs n[a]-1 divisible by 2 per level.
 *   Vectors: double, length 2*nv, u[2v] = p_w (Pa), u[2v+1] = S_n; residual
 *     F[2v] water mass balance, F[2v+1] NAPL mass balance (kg/s).
 *   Pointers: every array argument may be HOST or DEVICE memory (the library
 *     asks the CUDA driver which); device buffers are used in place.  State
 *     and solution vectors in page-locked host memory (cudaHostAlloc, or
 *     cudaHostRegister with mapping) are read and written by the library's
 *     kernels directly over the CPU-GPU interconnect; other host buffers
 *     are staged through device memory inside the call.  All inputs stay
 *     owned by the caller and are only borrowed for the call.
 *   Streams: every call is ordered on the given cudaStream_t (NULL = legacy
 *     default stream).  Calls that return numbers on the host (info structs,
 *     host outputs) synchronise that stream before returning.
 *   Errors: argument errors return RF_EINVAL synchronously; CUDA failures
 *     RF_ECUDA; device-detected conditions (non-convergence, breakdown,
 *     non-finite values) are returned once the stream has been synchronised.
 *     rf_last_error() gives a one-line message for the calling thread.
 *   Memory: all device memory of a grid comes from the rf_allocator given to
 *     rf_grid_create (cudaMalloc/cudaFree when it is NULL) and is released by
 *     rf_grid_destroy.  There is no CPU fallback: every step runs on the GPU.
 */
#ifndef RF_H
#define RF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RF_OK = 0,
  RF_EINVAL = 1,      /* bad argument (checked before any GPU work)          */
  RF_ENOMEM = 2,      /* the allocator returned NULL                          */
  RF_ECUDA = 3,       /* a CUDA runtime call failed                           */
  RF_ENOTCONV = 4,    /* linear solve hit max_it before reaching rtol         */
  RF_EBREAKDOWN = 5,  /* BiCGSTAB breakdown that a restart did not cure       */
  RF_ENONFINITE = 6,  /* NaN/Inf met in the state, residual or iteration      */
  RF_ETIMEOUT = 7     /* a bounded device wait gave up                        */
} rf_status;

typedef struct rf_grid rf_grid;

/* Device allocator: alloc(bytes, stream, ctx) -> device pointer or NULL;
 * free(ptr, bytes, stream, ctx).  NULL allocator = cudaMalloc / cudaFree. */
typedef struct {
  void* (*alloc)(size_t bytes, void* stream, void* ctx);
  void (*free)(void* ptr, size_t bytes, void* stream, void* ctx);
  void* ctx;
} rf_allocator;

/* dim = 2 or 3; n = vertices per axis (n[2] = 1 in 2D); h = spacing (m);
 * g = gravity vector (m/s^2), e.g. (0, -9.81, 0) in 2D. */
typedef struct { int dim; int64_t n[3]; double h[3]; double g[3]; } rf_grid_desc;

/* Densities (kg/m^3) and viscosities (Pa s) of water (w) and DNAPL (n). */
typedef struct { double rho_w, rho_n, mu_w, mu_n; } rf_fluids;

/* Brooks-Corey residual saturations and pore-size index (uniform), and per
 * cell permeability K (m^2), porosity phi and entry pressure p_d (Pa), each
 * of length (n0-1)(n1-1)(n2-1) (2D: (n0-1)(n1-1)).  Copied at creation. */
typedef struct { double S_wr, S_nr, lambda; const double *K, *phi, *pd; } rf_materials;

/* Boundary data, per vertex (copied at creation): dir_pw[v] = 1 makes the
 * water-balance row of v the algebraic equation 0 = pw_dir[v] - p_w (Dirichlet
 * p_w); q_in[2v+a] is a mass source of phase a (kg/s; Neumann inflow).  Any
 * pointer may be NULL (no Dirichlet vertices / no sources). */
typedef struct { const uint8_t* dir_pw; const double* pw_dir; const double* q_in; } rf_bc;

enum { RF_SMOOTH_JACOBI = 0, RF_SMOOTH_GS8 = 1 };
enum { RF_PREC_FP64 = 0, RF_PREC_FP32 = 1, RF_PREC_FP16 = 2 };

/* Multigrid options.  nlevels: vertex-nested levels (coarsened while possible,
 * at most this many); smoother: damped point-block Jacobi or multicolour
 * (4 colours 2D / 8 colours 3D) block Gauss-Seidel; nu1/nu2 pre/post sweeps;
 * omega: Jacobi damping; precision: storage and arithmetic of the
 * preconditioner (FP64; FP32; FP16 storage of the finest level's matrix
 * with per-block-row FP32 scales, FP32 storage on the coarser levels, FP32
 * arithmetic throughout).  The coarsest level is solved exactly in FP64.
 * autotune = 1 times candidate thread-block sizes (64..512) for each level's
 * smoothing and residual kernels during the set-up and keeps the fastest
 * (cached per level shape for the process, and in the file named by the
 * environment variable RF_TUNE_CACHE, one JSON object per line). */
typedef struct { int nlevels, smoother, nu1, nu2; double omega; int precision; int autotune; } rf_gmg_opts;

/* Stop when the TRUE FP64 residual |b - A x|_2 <= rtol |b|_2.  outer selects
 * the arithmetic of the two operator applications inside each iteration:
 * RF_OUTER_FP64 (FP64 J), or RF_OUTER_DF32 (J split once into FP32 hi + lo,
 * |J - hi - lo| <= 2^-48 |J|, exact FP32 products via FMA, compensated FP32
 * sums; only with an FP32/FP16 preconditioner, whose outputs are exact FP32).
 * The convergence decision always uses the FP64 true residual. */
enum { RF_OUTER_FP64 = 0, RF_OUTER_DF32 = 1 };
typedef struct { double rtol; int max_it; int outer; } rf_solve_opts;
typedef struct { int iterations; double relres; int status; int restarts; } rf_solve_info;

/* LIMEX step options: kappa columns (n_j = 1..kappa, one shared Jacobian),
 * error tolerance tol, safety factor rho, step factor bounds. */
typedef struct {
  int kappa; double tol, rho, fac_min, fac_max;
  rf_gmg_opts gmg; rf_solve_opts solve;
} rf_limex_opts;
typedef struct { double eps, H_new; int accepted, solves, iterations, status; } rf_limex_info;

/* Create a grid: validates the description, copies materials and boundary
 * data to the device and precomputes p_dmin,i = min of p_d over the elements
 * around vertex i (Eq. pdmin) and the lumped pore volume (Phi V)_i. */
rf_status rf_grid_create(const rf_grid_desc* desc, const rf_fluids* fluids, const rf_materials* mat,
                         const rf_bc* bc, const rf_allocator* alloc, void* stream, rf_grid** out);
void rf_grid_destroy(rf_grid* g);

/* Number of vertices of the grid (0 if g is NULL). */
int64_t rf_grid_nv(const rf_grid* g);

/* Assemble at state u [2nv]: F(u) into F_out (may be NULL) and, when
 * want_jacobian, the exact Jacobian J = F_u (27 or 9 2x2 blocks per vertex,
 * FP64) and the lumped mass matrix M (vertex-diagonal) kept inside the grid.
 * Sec. 3 (Eqs. dsW, dpN, up_krw, up_krn, hSw, krn_ip, krw_ip), Sec. 4 (J=F_u). */
rf_status rf_assemble(rf_grid* g, const double* u, int want_jacobian, double* F_out, void* stream);

/* Discretisation variants (bits; 0, the default, is the scheme of Sec. 3):
 * RF_SCHEME_SHAT_STORAGE: the storage of each sub-control volume b_i^j uses
 *   the interface saturation S hat of Eq. (hSw) (Sec. 3.3 applies it "as
 *   well" beyond k_rn); M becomes diag(d m / d S_n) with the S hat slopes and
 *   the storage is no longer linear in S_n.
 * RF_SCHEME_DARCY_UPWIND: the whole water flux, capillary-diffusion part
 *   included, is upwinded by the sign of the Darcy velocity u_w . n, the
 *   scheme Sec. 3.2 sets its own against; the NAPL flux is unchanged.
 * Changing the scheme drops the assembled Jacobian and multigrid set-up.
 * RF_EINVAL for unknown bits. */
#define RF_SCHEME_SHAT_STORAGE 1
#define RF_SCHEME_DARCY_UPWIND 2
rf_status rf_grid_set_scheme(rf_grid* g, int scheme);

/* Per-medium relative permeabilities (Sec. 6, Case 2, Table "Parameters for
 * Case-2": each of the two media has its own polynomial k_rw and k_rn).
 * laws (host, 6 doubles per law, nlaws <= RF_MAX_KR_LAWS) holds rows
 * {kind, a_w, n_w, a_n, b_n, c_n}:
 *   RF_KR_BROOKS_COREY: the grid's Brooks-Corey laws (other entries unused);
 *   RF_KR_POLY: k_rw = a_w S^n_w, k_rn = a_n (1 - b_n S)^2 (1 - c_n S^2)
 *     while 1 - b_n S > 0 and 1 - c_n S^2 > 0, and k_rn = 0 from the first of
 *     those roots on; S = S_e clamped to [0, 1], derivatives 0 outside
 *     (0, 1); n_w a whole number 1..8, a_w, a_n >= 0.
 * cell_law (host, one byte per cell in natural cell order) names each cell's
 * law.  Every face of a cell uses that cell's law for the upwinded k_rw
 * (Eq. krw_ip), the k_rw of the capillary term and k_rn of S hat (Eq.
 * krn_ip).  Capillary pressure stays Brooks-Corey with the cell's p_d.
 * nlaws = 0 returns to Brooks-Corey everywhere.  Both arrays are copied
 * (synchronously on `stream`); the assembled Jacobian and the multigrid
 * set-up are dropped.  RF_EINVAL for a bad count, kind or coefficient, a cell
 * naming a missing law, or device pointers; RF_ENOMEM if the device copy
 * cannot be allocated. */
#define RF_MAX_KR_LAWS 4
#define RF_KR_BROOKS_COREY 0
#define RF_KR_POLY 1
rf_status rf_grid_set_kr_laws(rf_grid* g, int nlaws, const double* laws, const uint8_t* cell_law, void* stream);

/* Build the multigrid hierarchy for the stage matrices A_j = shift[j] M - J,
 * j < nshift <= 4 (shift = 1/h_j), from the last assembled J, M: Galerkin
 * coarse operators P^T A P with trilinear P (FP64), the preconditioner copies
 * in the chosen precision, block-diagonal inverses and the coarsest inverse. */
rf_status rf_gmg_setup(rf_grid* g, const double* shifts, int nshift, const rf_gmg_opts* opts, void* stream);

/* Solve A_shift x = b by BiCGSTAB right-preconditioned with one V-cycle per
 * application, x0 = 0.  b, x: [2nv].  info (host, may be NULL) receives the
 * iteration count, the true relative residual and the status. */
rf_status rf_solve(rf_grid* g, int shift, const double* b, double* x, const rf_solve_opts* opts,
                   rf_solve_info* info, void* stream);

/* One LIMEX step of size H from state u (in/out [2nv]): assembly of J, M at
 * u, multigrid setup for the kappa shifts n_j/H, the columns of linearly
 * implicit Euler steps (each an rf_solve), Aitken-Neville extrapolation, the
 * scaled error estimate and the step-size proposal (q = 2).  u is replaced by
 * the extrapolated state only when the step is accepted (eps <= tol).
 * The columns are independent until the extrapolation.  On grids of at most
 * 4M vertices (or as the environment variable RF_LIMEX_CONCURRENT=1/0 says)
 * they run at the same time, each on its own stream and host thread, with
 * vectors of their own and the operators shared. The results are bitwise
 * those of running the columns in turn. */
rf_status rf_limex_step(rf_grid* g, double* u, double H, const rf_limex_opts* opts, rf_limex_info* info,
                        void* stream);

/* One LIMEX step for each of nprob independent problems (an ensemble of
 * realisations on grids of any sizes), run concurrently: every grid works on
 * its own stream with its own captured iteration graphs, and up to
 * max_concurrent host workers (<= 0: min(nprob, 16)) keep the GPU fed while
 * each waits for its convergence checks.  grids[i], u[i] (in/out), H[i] and
 * opts[i] (an array of nprob options, e.g. with per-grid level counts) as in
 * rf_limex_step; infos[i] receives each problem's result (status included).
 * Ordered after `stream`; `stream` waits for all problems.  Returns the first
 * non-OK status in problem order (all problems are attempted). */
rf_status rf_limex_step_batched(rf_grid* const* grids, double* const* u, const double* H, int nprob,
                                const rf_limex_opts* opts, rf_limex_info* infos, int max_concurrent, void* stream);

/* Adaptive LIMEX integration under the step control of Sec. 4: repeated
 * rf_limex_step calls from t = 0 on state u (in/out).  Before each step H =
 * min(H, t_end - t) when t_end > 0 (the last step lands on t_end).  An
 * accepted step advances t by H and replaces u; a rejected one keeps u and is
 * retried with the proposed smaller H.  The next H is the step's proposal
 * H_new, but not larger than H after a step accepted right after a rejection
 * when hold_after_reject (a common safeguard; the paper states no rule), and
 * at most H_max when H_max > 0.  Stops after max_steps accepted steps (when >
 * 0) or at t_end (when > 0), whichever comes first.  RF_ENOTCONV after more
 * than max_rejects rejections; a step's own failure is returned as is (u then
 * holds the last accepted state).  hist (host, may be NULL when hist_cap = 0)
 * receives {H, eps, accepted} per attempted step, for at most hist_cap steps;
 * info (host, may be NULL) the totals. */
typedef struct {
  rf_limex_opts step;
  double t_end, H_max;
  int max_steps, max_rejects, hold_after_reject;
} rf_limex_run_opts;
typedef struct { double t, H_next; int accepted, rejected, solves, iterations, steps, status; } rf_limex_run_info;
rf_status rf_limex_run(rf_grid* g, double* u, double H0, const rf_limex_run_opts* opts, rf_limex_run_info* info,
                       double* hist, int hist_cap, void* stream);

/* One implicit Euler step of size H solved by Newton's method — the fixed-step
 * scheme the paper compares LIMEX with (Sec. 6, Case 4, Table case4_2; Newton
 * tolerances 1e-8 absolute / 1e-6 relative there).  Finds u with
 *   R(u) = F(u) - (m(u) - m(u_old)) / H = 0
 * (m the storage of Eqs. (dsW),(dpN); no storage in Dirichlet p_w rows) by
 * Newton iterations (M(u_k)/H - J(u_k)) d = R(u_k), u_{k+1} = u_k + d: each
 * iteration assembles J, M and F at u_k, rebuilds the multigrid hierarchy
 * (opts->gmg) and solves with BiCGSTAB (opts->solve).  Converged when
 * ||R||_2 <= atol or ||R||_2 <= rtol ||R(u_old)||_2.  u [2nv] (host or device)
 * is updated in place only on success; info (host, may be NULL) receives the
 * Newton and linear iteration counts and the first and last residual norms.
 * max_ls > 0 damps each correction by backtracking: lambda = 1, 1/2, ... (at
 * most max_ls halvings, one residual evaluation each) until ||R(u + lambda d)||
 * <= (1 - 1e-4 lambda) ||R(u)||, else the last lambda is kept.
 * RF_ENOTCONV when max_newton iterations do not converge; a linear solver
 * failure is returned as is. */
typedef struct { double atol, rtol; int max_newton; rf_gmg_opts gmg; rf_solve_opts solve; int max_ls; } rf_ie_opts;
typedef struct { int newton, linear; double res0, res; rf_status status; } rf_ie_info;
rf_status rf_ie_step(rf_grid* g, double* u, double H, const rf_ie_opts* opts, rf_ie_info* info, void* stream);

/* Total phase masses (kg) of state u [2nv] with the lumped storage of Eqs.
 * (dsW),(dpN): mass_out[0] = sum_i rho_w (Phi V)_i (1 - S_n,i), mass_out[1] =
 * sum_i rho_n (Phi V)_i S_n,i (host array of 2; synchronises the stream);
 * with RF_SCHEME_SHAT_STORAGE each sub-control volume's S hat saturation.
 * Each linearly implicit Euler stage changes the NAPL mass by exactly h times
 * its sources plus the linear solve's residual, so the difference between two
 * states checks discrete mass conservation. */
rf_status rf_phase_mass(rf_grid* g, const double* u, double* mass_out, void* stream);

/* ---- test and inspection hooks (host buffers, natural vertex order) ---- */

/* Copy out J as [nv][nb][4] (entries (w,p_w),(w,S_n),(n,p_w),(n,S_n)) and the
 * mass diagonal as [nv][2] (dm_w/dS_n, dm_n/dS_n); either may be NULL. */
rf_status rf_export_jacobian(rf_grid* g, double* J_host, double* mdiag_host, void* stream);

/* Copy out the Jacobian block rows [count][nb][4] and mass diagonals
 * [count][2] of the listed vertices (natural indices, host array) — for
 * sampled checks on grids too large to export whole. */
rf_status rf_export_rows(rf_grid* g, const int64_t* vertices, int count, double* J_rows_host,
                         double* mdiag_host, void* stream);

/* Copy out the multigrid operator of `level` for shift index `shift` as
 * [nv_l][nb][4] in FP64 (the Galerkin product as computed; level 0 is
 * shift*M - J); dims_out[3] receives the level's vertex counts. */
rf_status rf_export_level(rf_grid* g, int level, int shift, double* A_host, int64_t dims_out[3], void* stream);

enum {
  RF_OP_SPMV = 0,        /* out = A_shift in0 on the fine grid, FP64            */
  RF_OP_VCYCLE = 1,      /* out = V-cycle(in0) (fine grid, preconditioner)      */
  RF_OP_SMOOTH = 2,      /* out = one smoother sweep at `level`: b = in0, x = in1
                            (Jacobi; forward colour sweep for GS)               */
  RF_OP_RESIDUAL = 3,    /* out = in0 - A_level in1 at `level`                  */
  RF_OP_RESTRICT = 4,    /* out (level+1) = P^T in0 (level)                     */
  RF_OP_PROLONG = 5,     /* out (level) = in1 (level) + P in0 (level+1)         */
  RF_OP_COARSE = 6       /* out = A_coarsest^-1 in0                             */
};
/* Apply one preconditioner building block with the precision of the current
 * hierarchy (inputs are rounded to it); vectors are [2 nv_level] doubles. */
rf_status rf_apply(rf_grid* g, int op, int level, int shift, const double* in0, const double* in1,
                   double* out, void* stream);

/* Per-kernel-class timing (inspection hook).  While enabled, the library
 * brackets each launch group of a class with CUDA events on the launching
 * stream and accounts the group's ALGORITHMIC bytes (every matrix entry and
 * every vector element counted once per launch).  rf_profile(g, 1) clears and
 * starts, rf_profile(g, 0) stops; rf_profile_read synchronises the device and
 * returns, for class cls, the summed event time (ms), launches and bytes. */
enum {
  RF_PROF_SPMV64 = 0,     /* outer FP64 operator applications (fused with dots)  */
  RF_PROF_SMOOTH_FINE,    /* smoother sweeps on the finest level                 */
  RF_PROF_RESID_FINE,     /* residual on the finest level                        */
  RF_PROF_TRANSFER,       /* restrictions and prolongations, all levels          */
  RF_PROF_COARSE_LEVELS,  /* smoothing/residual on levels >= 1, coarsest solve   */
  RF_PROF_VECTOR,         /* BiCGSTAB vector updates and reduction finalisation  */
  RF_PROF_NCLASS
};
rf_status rf_profile(rf_grid* g, int enable);
rf_status rf_profile_read(rf_grid* g, int cls, double* ms, int64_t* launches, double* bytes);

/* ---- allocation-free entry point (the paper has no counterpart) ----
 * For callers that cannot call cudaMalloc: applications whose device memory is
 * owned entirely by another allocator (a framework's caching pool, a fixed
 * budget) and latency-critical code that must not pay for cudaMalloc/cudaFree,
 * which may synchronise the device.  Inverts a dense FP64 N x N matrix
 * (row-major, DEVICE pointers A and Ainv, caller-owned; A is not modified) by
 * LU with partial pivoting, as the multigrid set-up does for the coarsest
 * operator, and allocates nothing: the LU factors, pivots and status live in
 * a static device array of RF_NOALLOC_MAX_N^2 * 8 bytes plus a little (about
 * 2 MiB), reserved on every GPU that loads the library until the process
 * exits.  Calls share the array: calls that overlap on the GPU race and must
 * be serialised by the caller.  Every call reads the status word back and
 * synchronises `stream`, so no call can be captured into a CUDA graph: on a
 * stream that is capturing it returns RF_EINVAL before enqueuing anything.
 * Returns RF_EINVAL for N outside [1, RF_NOALLOC_MAX_N] or for pointers that
 * are not device (or managed) memory of the current device, RF_ENONFINITE for
 * a singular matrix or one with non-finite entries. */
#define RF_NOALLOC_MAX_N 512
rf_status rf_dense_inverse_noalloc(int N, const double* A, double* Ainv, void* stream);

/* FP64 fused multiply-add throughput of the current GPU (FMA per second),
 * timed with CUDA events on `stream`: 8 independent FMA chains per thread, 8
 * blocks of 256 threads per SM.  The roofline denominator of the kernels that
 * the FP64 pipe, not HBM, bounds (outer operator, vector updates, assembly).
 * Synchronises `stream`. */
rf_status rf_fp64_fma_rate(void* stream, double* fma_per_s);

/* Kernels launched by this library in this process so far. */
int64_t rf_launch_count(void);

/* Check of the bounded grid barrier that the cooperative V-cycle tail
 * (environment RF_TAIL_NV) separates its phases with: one cooperative launch
 * of every block that fits on the GPU at once passes `rounds` barriers.  With
 * extra = 1 each barrier expects one block more than there are, so no barrier
 * completes: every wait gives up after limit_s seconds and the call returns
 * RF_ETIMEOUT with the context still usable.  blocks_out (host, may be NULL)
 * receives the launch's block count.  RF_EINVAL unless 1 <= rounds <= 10^6,
 * extra is 0 or 1 and 0 < limit_s <= 10; RF_ECUDA if the launch fails.
 * Synchronous on `stream`.  The barrier: the last block to arrive resets the
 * arrival count and publishes the next generation; the others poll the
 * generation (with the global timer bounding the wait). */
rf_status rf_barrier_check(int rounds, int extra, double limit_s, int* blocks_out, void* stream);
const char* rf_status_string(rf_status s);
const char* rf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
