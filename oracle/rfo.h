/*
 * rfo — the ORACLE: a plain, slow, FP64 CPU restatement of the discrete
 * two-phase flow model, the BiCGSTAB + geometric-multigrid stage solver and the
 * LIMEX step of "A highly scalable numerical framework for reservoir simulation
 * on UG4 platform" (arXiv 2506.04763).
 *
 * This is TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA library; the two meet only through the data formats
 * below, which both sides implement on their own.
 *
 * Data formats (natural lexicographic order, x fastest):
 *   vertex  v = i + nx*(j + ny*k)           cell c = i + (nx-1)*(j + (ny-1)*k)
 *   state   u[2v+0] = p_w (Pa), u[2v+1] = S_n
 *   residual F[2v+0] = water equation (kg/s), F[2v+1] = NAPL equation
 *   stencil block b = (dx+1) + 3(dy+1) [+ 9(dz+1) in 3D]; nb = 9 (2D) or 27 (3D)
 *   2x2 block entries e: 0=(w,p_w) 1=(w,S_n) 2=(n,p_w) 3=(n,S_n)
 *   matrix  A[(v*nb + b)*4 + e]   (blocks reaching outside the grid are zero)
 *   mass    mdiag[2v+0] = d m_w/d S_n, mdiag[2v+1] = d m_n/d S_n  (M is
 *           vertex-diagonal and its p_w column is zero)
 */
#ifndef RFO_H
#define RFO_H
#include <stddef.h>

typedef struct {
  int dim;             /* 2 or 3 */
  int n[3];            /* vertices per axis (n[2] = 1 in 2D) */
  double h[3];         /* mesh spacing per axis (m) */
  double g[3];         /* gravity vector (m/s^2) */
  double rho_w, rho_n, mu_w, mu_n;
  double S_wr, S_nr, lambda;       /* Brooks-Corey parameters (uniform) */
  const double* K;     /* per cell permeability (m^2) */
  const double* phi;   /* per cell porosity */
  const double* pd;    /* per cell entry pressure (Pa) */
  const unsigned char* dir;  /* per vertex: 1 = Dirichlet p_w (may be NULL) */
  const double* pw_dir;      /* per vertex Dirichlet value (used where dir=1) */
  const double* q_in;        /* per vertex [2] mass source kg/s (may be NULL) */
  int scheme;                /* RFO_SCHEME_* bits; 0 = the discretisation of Sec. 3 */
  /* Per-medium relative permeabilities (Sec. 6, Case 2 gives each of its two
   * media its own polynomial k_rw, k_rn).  nlaws = 0 (and cell_law NULL):
   * the Brooks-Corey laws everywhere.  Otherwise kr_laws[6m .. 6m+5] =
   * {kind, a_w, n_w, a_n, b_n, c_n} for law m < nlaws and cell_law[c] < nlaws
   * names the law of cell c; kind RFO_KR_BROOKS_COREY uses the Brooks-Corey
   * laws, RFO_KR_POLY the polynomial laws of rfo_kr_law.  Capillary pressure
   * stays Brooks-Corey with the cell's p_d. */
  int nlaws;
  const double* kr_laws;
  const unsigned char* cell_law;
} rfo_model;
enum { RFO_KR_BROOKS_COREY = 0, RFO_KR_POLY = 1 };

/* Discretisation variants (bits of rfo_model.scheme):
 *   RFO_SCHEME_SHAT_STORAGE: the storage term of sub-control volume b_i^j uses
 *     the interface saturation S hat_{w,i,N} of Eq. (hSw) instead of the vertex
 *     saturation (Sec. 3.3 asks for Eq. (hSw) "as well" beyond k_rn).
 *   RFO_SCHEME_DARCY_UPWIND: the water flux is upwinded as a whole by the sign
 *     of its Darcy velocity u_w . n (phase-potential upwinding, the scheme
 *     Sec. 3.2 contrasts with its own), i.e. the capillary-diffusion part is
 *     upwinded too. The NAPL flux is unchanged (u_n and v_n share their sign). */
enum { RFO_SCHEME_SHAT_STORAGE = 1, RFO_SCHEME_DARCY_UPWIND = 2 };

/* ---- threads: OpenMP threads of the per-vertex loops (results do not depend
 * on the count; see rfo.c) ---- */
void rfo_set_threads(int n);
int rfo_get_threads(void);

/* ---- constitutive laws (Brooks-Corey; interface condition) ---- */
void rfo_brooks_corey(const rfo_model* m, double Se, double out[6]);
/* out = {krw, dkrw/dSe, krn, dkrn/dSe, J, dJ/dSe} */
void rfo_shat(const rfo_model* m, double Se, double pd_cell, double pdmin, double out[2]);
/* out = {S_e hat, d S_e hat / d S_e} */
void rfo_kr_law(const rfo_model* m, int cell, double Se, double out[4]);
/* relative permeabilities of cell's medium: out = {krw, dkrw/dSe, krn, dkrn/dSe}.
 * RFO_KR_POLY (S = S_e clamped to [0, 1], derivatives 0 outside (0, 1)):
 *   k_rw = a_w S^n_w (n_w a whole number, 1..8),
 *   k_rn = a_n (1 - b_n S)^2 (1 - c_n S^2) while both 1 - b_n S and
 *   1 - c_n S^2 are positive, and 0 from the first of their roots on (the
 *   NAPL is immobile there). */

/* ---- spatial discretisation ---- */
void rfo_pdmin(const rfo_model* m, double* pdmin);   /* [nv] */
void rfo_phiv(const rfo_model* m, double* phiv);     /* [nv] */
void rfo_assemble(const rfo_model* m, const double* u, double* F, double* J, double* mdiag);
/* J, mdiag may be NULL (residual only) */
void rfo_storage(const rfo_model* m, const double* u, double* mass);
/* mass[2v] = m_w,i, mass[2v+1] = m_n,i (kg): the storage terms of Eqs. (dsW),(dpN) */

/* ---- algebra on the stencil format ---- */
void rfo_make_A(int nv, int nb, const double* J, const double* mdiag, double shift, double* A);
void rfo_spmv(int dim, const int n[3], const double* A, const double* x, double* y);
void rfo_residual(int dim, const int n[3], const double* A, const double* b, const double* x, double* r);
void rfo_jacobi(int dim, const int n[3], const double* A, const double* b, const double* xin,
                double* xout, double omega);
void rfo_gs_sweep(int dim, const int n[3], const double* A, const double* b, double* x, int forward);
void rfo_restrict(int dim, const int nf[3], const unsigned char* dmf, const int nc[3],
                  const unsigned char* dmc, const double* rf, double* bc);
void rfo_prolong_add(int dim, const int nf[3], const unsigned char* dmf, const int nc[3],
                     const unsigned char* dmc, const double* xc, double* xf);
void rfo_galerkin(int dim, const int nf[3], const unsigned char* dmf, const double* Af,
                  const int nc[3], const unsigned char* dmc, double* Ac);
int  rfo_lu_factor(int N, double* LU, int* piv);
void rfo_lu_solve(int N, const double* LU, const int* piv, double* x);

/* ---- geometric multigrid ---- */
typedef struct rfo_gmg rfo_gmg;
enum { RFO_JACOBI = 0, RFO_GS8 = 1 };
rfo_gmg* rfo_gmg_create(int dim, const int n[3], const double* A0, const unsigned char* dmask,
                        int nlevels, int smoother, int nu1, int nu2, double omega);
void rfo_gmg_free(rfo_gmg* g);
int  rfo_gmg_nlevels(const rfo_gmg* g);
void rfo_gmg_level_dims(const rfo_gmg* g, int level, int n[3]);
void rfo_gmg_level_matrix(const rfo_gmg* g, int level, double* A);
void rfo_gmg_vcycle(rfo_gmg* g, const double* b, double* x);

/* ---- FP32 emulation of the V-cycle (float storage and accumulation; the
 * hierarchy of g rounded to float, the coarsest level solved in double) ---- */
typedef struct rfo_gmg32 rfo_gmg32;
rfo_gmg32* rfo_gmg32_create(const rfo_gmg* g);
void rfo_gmg32_free(rfo_gmg32* h);
void rfo_gmg32_vcycle(rfo_gmg32* h, const float* b, float* x);

/* ---- BiCGSTAB, right-preconditioned by one V-cycle (g may be NULL) ---- */
int rfo_bicgstab(int dim, const int n[3], const double* A, rfo_gmg* g, const double* b, double* x,
                 double rtol, int maxit, int* iters, double* relres);

/* ---- LIMEX ---- */
void rfo_extrapolate(int kappa, const int* nseq, int len, const double* T1, double* Tkk, double* Tkk1);
double rfo_h1_seminorm2(int dim, const int n[3], const double* h, const double* q, int stride);
double rfo_lumped_l2norm2(int dim, const int n[3], const double* h, const double* q, int stride);
typedef struct {
  int kappa; double tol, rho, fac_min, fac_max;
  int nlevels, smoother, nu1, nu2; double omega;
  double rtol; int maxit;
} rfo_limex_opts;
typedef struct { double eps, H_new; int accepted, solves, iterations; } rfo_limex_info;
int rfo_limex_step(const rfo_model* m, const double* u0, double H, const rfo_limex_opts* o,
                   double* u_out, rfo_limex_info* info);

/* ---- adaptive LIMEX integration: repeated steps under the step control of
 * Sec. 4.  From t = 0: H = min(H, t_end - t) when t_end > 0; one step; if it
 * is accepted t += H, else the state stays; the next H is the step's proposal
 * H_new, not larger than H after a step accepted right after a rejection
 * when hold_after_reject (a safeguard; the paper states no rule), and at
 * most H_max when H_max > 0.  Stops after max_steps accepted steps (> 0) or
 * at t_end (> 0), whichever comes first; returns 1 after more than
 * max_rejects rejections, else the last step's status.  hist (may be NULL)
 * receives per attempted step {H, eps, accepted} for at most hist_cap steps. */
typedef struct {
  rfo_limex_opts step;
  double t_end, H_max;
  int max_steps, max_rejects, hold_after_reject;
} rfo_limex_run_opts;
typedef struct { double t, H_next; int accepted, rejected, solves, iterations, steps; } rfo_limex_run_info;
int rfo_limex_run(const rfo_model* m, const double* u0, double H0, const rfo_limex_run_opts* o, double* u_out,
                  rfo_limex_run_info* info, double* hist, int hist_cap);

/* ---- implicit Euler + Newton (the comparison scheme of Sec. 6, Case 4) ----
 * Solves R(u) = F(u) - (m(u) - m(u_old))/H = 0 (storage m of rfo_storage;
 * Dirichlet p_w rows have no storage) by Newton: (M(u_k)/H - J(u_k)) d = R(u_k),
 * u_{k+1} = u_k + d, each linear system by BiCGSTAB + GMG to rtol.  Stops when
 * ||R||_2 <= atol or ||R||_2 <= rtol_newton ||R(u_old)||_2 (Sec. 6: 1e-8 / 1e-6).
 * With max_ls > 0 each Newton correction is damped by backtracking: lambda =
 * 1, 1/2, ... (at most max_ls halvings) until ||R(u + lambda d)|| <= (1 -
 * 1e-4 lambda) ||R(u)||; if no lambda passes, the last one is taken.
 * Returns 0, or 1 if Newton did not converge in max_newton iterations, or the
 * linear solver's status; on failure u_out = u_old. */
typedef struct {
  double atol, rtol; int max_newton;
  int nlevels, smoother, nu1, nu2; double omega;
  double lin_rtol; int lin_maxit;
  int max_ls;
} rfo_ie_opts;
typedef struct { int newton, linear; double res0, res; } rfo_ie_info;
int rfo_ie_step(const rfo_model* m, const double* u_old, double H, const rfo_ie_opts* o, double* u_out,
                rfo_ie_info* info);

#endif
