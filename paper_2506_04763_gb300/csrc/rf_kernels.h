// rf_kernels.h — launchers exported by the kernel translation units to the
// host driver (driver.cu).  Plain C++ types only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "rf_common.cuh"

namespace rf {

// discretisation variants (bits of PhysParams::scheme)
enum { SCHEME_SHAT_STORAGE = 1, SCHEME_DARCY_UPWIND = 2 };

struct PhysParams {
  double rho_w, rho_n, mu_w, mu_n, S_wr, S_nr, lambda;
  double h[3], g[3];
  int scheme;
};

struct AsmArrays {
  const double* u;                 // [2nv] parity-split
  double *Se, *pn, *pc, *dpc, *krw, *dkrw;  // [nv] scratch
  const double *pdmin, *phiv;      // [nv]
  const double *K, *pd, *phi;      // per cell
  double vol;                      // cell volume
  const uint8_t* dir;              // [nv]
  const double* pw_dir;            // [nv]
  const double* q_in;              // [2nv] or null
  const uint8_t* law;              // per cell: index of its k_r law, or null (Brooks-Corey everywhere)
  const double* kr_tab;            // [RF_MAX_KR_LAWS][6] law table (with law)
  double* F;                       // [2nv]
  double* J;                       // [nb][nv][4] or null
  double* mdiag;                   // [2nv] or null
};

// assemble.cu
void launch_vertex_setup(const Dims& d, const double* pd, const double* phi, double vol, double* pdmin,
                         double* phiv, void* s);
void launch_perm_to_p(const Dims& d, const double* nat, double* out, void* s);
void launch_perm_from_p(const Dims& d, const double* pl, double* nat, void* s);
void launch_perm_bytes_to_p(const Dims& d, const uint8_t* nat, uint8_t* out, void* s);
void launch_perm_scalar_to_p(const Dims& d, const double* nat, double* out, void* s);
cudaError_t launch_assemble(const Dims& d, const PhysParams& pp, const AsmArrays& a, bool want_j, void* s);
// S hat storage variant: sw[p] = sum over the sub-control volumes of p of Phi |b| S_w (S hat)
void launch_storage_sw(const Dims& d, const PhysParams& pp, const double* u, const double* pdmin,
                       const double* phi, const double* pd, double vol, double* sw, void* s);

// ---- multigrid level operators (levelops.cu) ----
enum StoreKind { STORE_F64 = 0, STORE_F32 = 1, STORE_F16 = 2 };
// stencil blocks stored per row: FP16 rows are stored in block pairs (an odd
// count gets an empty slot)
inline int stored_blocks(int kind, int nb) { return kind == STORE_F16 ? (nb + 1) & ~1 : nb; }

// One level's operator as seen by the smoothing / residual kernels.
struct LevelOp {
  Dims d;
  Nbr nb;
  int kind;              // StoreKind of the blocks (and T = double for F64, float otherwise)
  bool fine;             // true: blocks hold J and A = shift*M - J with M = mdiag;
                         // false: blocks hold A itself
  const void* A;         // [nb][nv] blocks of 4
  const float* scale;    // F16: [nv][4] per-entry-position row scales
  const double* mdiag;   // fine: [2nv] (dm_w/dS_n, dm_n/dS_n)
  double shift;          // fine: 1/h_j
  const void* Dinv;      // [nv][4] inverse diagonal blocks (T)
  const uint8_t* dmask;  // [nv]
  int block = 256;       // threads per block of the smoothing / residual kernels (autotuned)
  bool batched = false;  // smoothing / residual kernels issue 9 blocks' loads per round trip
  uint32_t nomask = 0;   // always 0: a stencil skip mask the compiler cannot fold (see apply_row)
};

// Vectors are T2 pointers to the first interior element of padded buffers.
void launch_residual(const LevelOp& L, const void* b, const void* x, void* r, void* s);
void launch_jacobi(const LevelOp& L, const void* b, const void* xin, void* xout, double omega, bool zero_x,
                   void* s);
// zero_start: x holds no data yet (first forward sweep of a V-cycle); blocks that
// reach colours not yet visited in this sweep are skipped and x need not be cleared.
// flip: the sweep's first colour launch walks the grid from its far end
// (consecutive colour launches alternate their direction; see levelops.cu)
void launch_gs_sweep(const LevelOp& L, const void* b, void* x, bool forward, bool zero_start, void* s,
                     bool flip = false);
void launch_restrict(const LevelOp& F, const LevelOp& C, const void* rf, void* bc, void* s);
void launch_prolong(const LevelOp& F, const LevelOp& C, const void* xc, void* xf, void* s);
void launch_coarse_solve(const LevelOp& C, const double* Ainv, const void* b, void* x, void* s);

// The V-cycle below a size threshold, run by one thread-block cluster.
#define TAIL_THREADS 256
struct TailLevel {
  LevelOp op;                 // coarse-level operator (blocks hold A)
  void *x, *b, *r, *t;        // level vectors (T2, padded)
};
struct TailParams {
  int first, coarsest;        // levels first .. coarsest (coarsest solved exactly)
  int smoother, nu1, nu2;
  double omega;
  uint32_t zmask[8];          // first-sweep skip masks per colour
  const double* Ainv;         // coarsest inverse, N x N
  int N;
  // cooperative form only: barrier words {count, generation}, the flag a
  // barrier that gave up sets (a Krylov scalar slot), and the wait limit
  unsigned* bar;
  double* status;
  long long limit_ns;
  // shared-memory form (k_vcycle_tail_sm, sm_bytes > 0): CTA r of the
  // cluster's sm_cs keeps the stencil blocks and D^-1 of its x-lines
  // L = r + sm_cs * i (i < sm_lines[l]) of every level below the coarsest,
  // level l's blocks from float4 sm_base[l] on, block b of local row lr at
  // sm_base[l] + b * sm_rows[l] + lr, D^-1 after the last block
  int sm_bytes, sm_cs;
  int sm_lines[RF_MAXL], sm_rows[RF_MAXL], sm_base[RF_MAXL];
  TailLevel L[RF_MAXL];
};
int tail_cluster_size(int kind, int nb);
void fill_tail_masks(TailParams& P, int dim);
cudaError_t launch_vcycle_tail(const TailParams& P, int kind, int nb, int csize, void* s);
// the shared-memory form (FP32 levels, GS smoother): fills P.sm_* for cluster
// size csize and returns true if it fits and can be co-scheduled
bool tail_sm_plan(TailParams& P, int nb, int csize);
cudaError_t launch_vcycle_tail_sm(const TailParams& P, int nb, void* s);
// the same V-cycle as one cooperative launch of `blocks` blocks (coop_tail_blocks: all that fit at once)
int coop_tail_blocks(int kind, int nb);
cudaError_t launch_vcycle_coop(const TailParams& P, int kind, int nb, int blocks, void* s);
// `rounds` bounded grid barriers over all co-resident blocks, each expecting `extra` more arrivals
// than there are blocks; *passed counts the (block, round) passes, *status = 1 if a wait gave up
cudaError_t launch_barrier_check(unsigned* bar, int rounds, int extra, double* status, long long limit_ns,
                                 unsigned* passed, int* blocks_out, void* s);

// set-up kernels (levelops.cu)
void launch_galerkin_axis(int axis, const Dims& din, const uint8_t* dmf, const double* Jin, const double* Min,
                          const double* mdiag, const Dims& dout, const uint8_t* dmc, double* Jout, double* Mout,
                          void* s);
void launch_coarse_mask(const Dims& df, const uint8_t* dmf, const Dims& dc, uint8_t* dmc, void* s);
// pack A = shift*M - J (coarse: from Jc/Mc; fine: keep J, only Dinv) into storage `kind`; write Dinv
void launch_pack_level(const Dims& d, bool fine, const double* J, const double* M, const double* mdiag,
                       double shift, int kind, void* A_out, float* scale_out, void* Dinv_out, void* s);
void launch_dense_coarsest(const Dims& d, const Nbr& nb, const double* Jc, const double* Mc,
                           const double* mdiag, bool fine, double shift, double* D, void* s);
cudaError_t launch_dense_inverse(int N, double* D, double* Ainv, int* piv, double* work, int* status,
                                 void* s);
// nmat (<= RF_MAXSHIFT) independent inverses at once, one CTA each for the LU:
// D = nmat consecutive N x N matrices (overwritten), piv = nmat x N, status = nmat
struct InvOut { double* Ainv[RF_MAXSHIFT]; };
cudaError_t launch_dense_inverse_batched(int N, int nmat, double* D, double* const* Ainv, int* piv, int* status,
                                         void* s);
void launch_export_level(const Dims& d, bool fine, const double* J, const double* M, const double* mdiag,
                         double shift, double* A_nat, void* s);
void launch_gather_rows(const Dims& d, const double* J, const double* mdiag, const int64_t* verts, int count,
                        double* Jout, double* mout, void* s);
void launch_cast_f64_to_f32(const double* in, float* out, int64_t n, void* s);
void launch_cast_f32_to_f64(const float* in, double* out, int64_t n, void* s);

// ---- Krylov (krylov.cu) ----
struct KrylovVecs {
  double2 *x, *r, *rh, *p, *v, *s, *t;   // FP64, parity-split (x and p padded not required)
  void *y, *z;                            // preconditioned vectors (T2, padded)
  double2 *y64, *z64;                     // FP64 copies read by the outer operator (padded)
  void *p_lo, *s_lo;                      // preconditioner inputs (T2)
  double* partial;                        // reduction partials [8][max_blocks]
  double* scal;                           // device scalars (see krylov.cu)
};
int krylov_blocks(int64_t nv);
// outer operator: y = (shift*M - J) x with J FP64, x FP64 or FP32 (x_is_f32)
void launch_spmv64(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                   const void* x, bool x_is_f32, double2* y, void* s);
void launch_bicg_init(int64_t nv, const double2* b, KrylovVecs& K, double rtol, void* s);
void launch_bicg_p(int64_t nv, KrylovVecs& K, bool lo_is_f32, bool first, void* s);
void launch_bicg_v(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                   KrylovVecs& K, bool y_is_f32, void* s);
void launch_bicg_s(int64_t nv, KrylovVecs& K, bool lo_is_f32, void* s);
// double-FP32 outer operator (FP32 operands y, z; J as FP32 hi/lo pairs)
void launch_split_df(const Dims& d, const double* J, float* Jdf, void* s);
void launch_bicg_v_df(const Dims& d, const Nbr& nb, const float* Jdf, const double* mdiag, double shift,
                      KrylovVecs& K, void* s);
void launch_bicg_t_df(const Dims& d, const Nbr& nb, const float* Jdf, const double* mdiag, double shift,
                      KrylovVecs& K, void* s);
void launch_bicg_t(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                   KrylovVecs& K, bool z_is_f32, void* s);
void launch_bicg_xr(int64_t nv, KrylovVecs& K, bool yz_is_f32, void* s);
void launch_true_residual(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                          const double2* b, KrylovVecs& K, void* s);
void launch_restart(int64_t nv, KrylovVecs& K, void* s);
void launch_axpy_pairs(int64_t nv, double2* u, const double2* du, void* s);

// sw (may be null): per-vertex water pore volume sum Phi |b| S_w; null: phiv (1 - S_n)
void launch_phase_mass(int64_t nv, double rho_w, double rho_n, const double* phiv, const double* u, const double* sw,
                       double* out2, double* partial, void* s);

// implicit Euler Newton residual R = F - (m(u) - m(u_old))/H (sw, sw_old: S hat storage, else null)
// and ||R||^2 into out1[0]
void launch_ie_residual(int64_t nv, const double* F, const double* u, const double* u_old, const double* mdiag,
                        const double* sw, const double* sw_old, const uint8_t* dir, double rho_w, double rho_n,
                        double inv_h, double* R, double* out1, double* partial, void* s);

void launch_axpby_pairs(int64_t nv, double* out, const double* a, const double2* d, double lam, void* s);

// ---- batched execution: several systems of one level shape per launch ----
// The systems of a batch (the active LIMEX columns of a step, the members of an
// ensemble with equal grids) run in lock-step: every launch below serves all
// of them, one system per blockIdx.y (or, for the finest level of systems that
// share one Jacobian, all of them per thread, the matrix read once).  Each
// system computes exactly what its own single-system launch would, in the same
// order, so results are bitwise those of solving the systems one by one.  A
// system whose Krylov scalar slot RF_SCAL_DONE is set has finished: its
// blocks return at once and its data stay as they are.
#define RF_MAXSYS 64
constexpr int RF_SCAL_DONE = 15;
// set to 1 by a cooperative V-cycle tail whose barrier wait gave up (read by
// the host with the iteration's scalars)
constexpr int RF_SCAL_TAIL = 16;
struct SysLevel {                  // one system's operands of a batched level launch
  const void* A;                   // blocks (coarse solve: the FP64 inverse)
  const float* scale;              // FP16 row scales
  const void* Dinv;
  const double* mdiag;
  const uint8_t* dmask;            // (transfers: the fine level's mask)
  const uint8_t* dmask_c;          // (transfers: the coarse level's mask)
  double shift;
  const double* scal;              // the system's Krylov scalars
  const void* in0;
  const void* in1;
  void* out;
};
struct SysBatch {
  int n;
  SysLevel s[RF_MAXSYS];
};
void launch_residual_b(const LevelOp& L, const SysBatch& B, void* s);
void launch_jacobi_b(const LevelOp& L, const SysBatch& B, double omega, bool zero_x, void* s);
void launch_gs_sweep_b(const LevelOp& L, const SysBatch& B, bool forward, bool zero_start, void* s,
                       bool flip = false);
void launch_restrict_b(const LevelOp& F, const LevelOp& C, const SysBatch& B, void* s);
void launch_prolong_b(const LevelOp& F, const LevelOp& C, const SysBatch& B, void* s);
void launch_coarse_solve_b(const LevelOp& C, const SysBatch& B, void* s);
void launch_cast_f32_to_f64_b(int64_t n, const SysBatch& B, void* s);
// finest level of systems that share J: consecutive groups of `share` (1..4)
// systems of B (B.n a multiple of it) use one matrix, FP16 scales and mass
// diagonal, those of the group's first system; a thread reads each block once
// per vertex for all systems of its group (blockIdx.y = group)
void launch_residual_shared(const LevelOp& L, const SysBatch& B, int share, void* s);
void launch_jacobi_shared(const LevelOp& L, const SysBatch& B, int share, double omega, bool zero_x, void* s);
void launch_gs_sweep_shared(const LevelOp& L, const SysBatch& B, int share, bool forward, bool zero_start, void* s,
                            bool flip = false);

struct SysKrylov {                 // one system of a batched BiCGSTAB iteration
  KrylovVecs K;
  const double* J;                 // FP64 Jacobian of the outer operator
  const double* mdiag;
  double shift;
};
struct KBatch {
  int n;
  SysKrylov s[RF_MAXSYS];
};
void launch_bicg_p_b(int64_t nv, const KBatch& B, bool lo_is_f32, void* s);
void launch_bicg_s_b(int64_t nv, const KBatch& B, bool lo_is_f32, void* s);
void launch_bicg_xr_b(int64_t nv, const KBatch& B, bool yz_is_f32, void* s);
// outer operator with the fused dots; share > 1: consecutive groups of `share`
// (<= 4) systems use one J (that of the group's first system), read once
void launch_bicg_v_b(const Dims& d, const Nbr& nb, const KBatch& B, int share, void* s);
void launch_bicg_t_b(const Dims& d, const Nbr& nb, const KBatch& B, int share, void* s);
// copy scalar slots [0, 16) of every system into out[16 * system]
void launch_gather_scalars(const KBatch& B, double* out, void* s);

// ---- LIMEX (krylov.cu) ----
void launch_extrapolate(int64_t n2, int kappa, double* T, void* s);
void launch_error_norms(const Dims& d, const double* h, const double* Tkk, const double* Tkk1, double* out4,
                        double* partial, void* s);

}  // namespace rf
