/*
 * rfo.c — ORACLE (test infrastructure; see rfo.h).  Plain FP64 C, written from
 * the paper's model and method; compiled with -ffp-contract=off so that no
 * multiply-add is fused behind the reader's back.  Everything is a loop over
 * the natural grid; nothing is blocked, fused or reordered beyond what the
 * definitions state.
 *
 * Paper sections followed (arXiv 2506.04763):
 *   Sec. 2, Eqs. (m),(u),(S),(pc): phase mass balance, extended Darcy law,
 *       closure relations; Eqs. (sW),(pN),(vW),(vN): the split with the
 *       capillary-diffusion term separated out of the convective velocities.
 *   Sec. 3.1, Eqs. (dsW),(dpN): vertex-centred finite volumes on the dual mesh,
 *       lumped storage at the vertex, sub-control-volume-face (SCVF) fluxes at
 *       the face midpoint x_M.
 *   Sec. 3.2, Eqs. (up_krw),(up_krn): full upwinding of the relative
 *       permeabilities by the sign of v_alpha . n (tie >= 0 -> own vertex).
 *   Sec. 3.3, Eqs. (pdmin),(hSw),(krn_ip),(krw_ip): p_dmin interface
 *       condition, S hat per sub-control volume, applied to k_rn only.
 *   Sec. 4: linearly implicit Euler (M - tau J) du = tau F with the exact
 *       Jacobian J = F_u, extrapolation, step-size control with q = 2, the
 *       scaled norm alpha |grad p|^2 + beta |S|^2.
 *   Sec. 5 (setup paragraph): BiCGSTAB preconditioned by geometric multigrid.
 *
 * Readings where the paper is silent are listed in the repository's design
 * notes and restated at each use below.
 *
 * Threads: loops whose iterations write disjoint outputs and read nothing
 * another iteration writes (per-vertex rows of a mat-vec, a Jacobi sweep, one
 * colour of the multicolour sweep, a transfer, an elementwise vector update)
 * carry a plain "omp parallel for".  Each output is then computed by exactly
 * the same operations in the same order as in a serial run, so results are
 * bitwise independent of the thread count.  Sums over the whole grid (inner
 * products, norms) and the element and Galerkin loops, which add into shared
 * rows, stay serial.
 */
#include "rfo.h"
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

static int nverts(const int n[3]) { return n[0] * n[1] * n[2]; }

void rfo_set_threads(int n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

int rfo_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
static int nblk(int dim) { return dim == 3 ? 27 : 9; }
static int blk_index(int dx, int dy, int dz) { return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1); }
/* In 2D dz is always 0, so the 2D index (dx+1)+3(dy+1) is blk_index - 9. */
static int blk(int dim, int dx, int dy, int dz) { return dim == 3 ? blk_index(dx, dy, dz) : blk_index(dx, dy, 0) - 9; }
static int centre(int dim) { return dim == 3 ? 13 : 4; }

/* ------------------------------------------------------------------------ */
/* Constitutive laws.  The paper names Brooks-Corey with lambda = 2 (Case 3-5
 * tables) without printing it; the standard Brooks-Corey-Burdine form is used:
 *   S_e = (S_w - S_wr)/(1 - S_wr - S_nr), k_rw = S_e^((2+3l)/l),
 *   k_rn = (1-S_e)^2 (1 - S_e^((2+l)/l)), p_c = p_d J(S_e), J = S_e^(-1/l).
 * Reading: k_r use S_e clamped to [0,1] (zero derivative outside); J is
 * continued linearly (C^1) below S_e = 0.01 and above S_e = 1.             */
static void jpow(double lam, double S, double* J, double* dJ) {
  if (lam == 2.0) {
    double r = sqrt(S);
    *J = 1.0 / r;
    *dJ = -0.5 / (S * r);
  } else {
    *J = pow(S, -1.0 / lam);
    *dJ = (-1.0 / lam) * pow(S, -1.0 / lam - 1.0);
  }
}

static void leverett(double lam, double Se, double* J, double* dJ) {
  const double s0 = 0.01;
  if (Se < s0) {
    double j0, d0;
    jpow(lam, s0, &j0, &d0);
    *J = j0 + d0 * (Se - s0);
    *dJ = d0;
  } else if (Se > 1.0) {
    *J = 1.0 + (-1.0 / lam) * (Se - 1.0);
    *dJ = -1.0 / lam;
  } else {
    jpow(lam, Se, J, dJ);
  }
}

void rfo_brooks_corey(const rfo_model* m, double Se, double out[6]) {
  const double lam = m->lambda;
  const double Sc = Se < 0.0 ? 0.0 : (Se > 1.0 ? 1.0 : Se);
  const int inside = (Se > 0.0 && Se < 1.0);
  double krw, dkrw, krn, dkrn;
  if (lam == 2.0) {
    double s2 = Sc * Sc, om = 1.0 - Sc;
    krw = s2 * s2;
    dkrw = inside ? 4.0 * s2 * Sc : 0.0;
    krn = om * om * (1.0 - s2);
    dkrn = inside ? (-2.0 * om * (1.0 - s2) - 2.0 * Sc * om * om) : 0.0;
  } else {
    double ew = (2.0 + 3.0 * lam) / lam, en = (2.0 + lam) / lam;
    double om = 1.0 - Sc, sa = pow(Sc, en);
    krw = pow(Sc, ew);
    dkrw = inside ? ew * pow(Sc, ew - 1.0) : 0.0;
    krn = om * om * (1.0 - sa);
    dkrn = inside ? (-2.0 * om * (1.0 - sa) - en * om * om * pow(Sc, en - 1.0)) : 0.0;
  }
  out[0] = krw; out[1] = dkrw; out[2] = krn; out[3] = dkrn;
  leverett(lam, Se, &out[4], &out[5]);
}

/* Relative permeabilities of the medium of a cell.  The polynomial laws are
 * those of Sec. 6, Table "Parameters for Case-2" (k_rw,1 = 1.831 S_e^4,
 * k_rn,1 = 0.75 (1 - 1.25 S_e)^2 (1 - 1.652 S_e^2); k_rw,2 = 0.4687 S_e^2,
 * k_rn,2 = 0.25 (1 - 1.25 S_e)^2) written with free coefficients.  Printed as
 * they are, both k_rn turn negative (law 1) or rise again (law 2) past their
 * first root below S_e = 1; k_rn is taken as 0 from that root on.          */
void rfo_kr_law(const rfo_model* m, int cell, double Se, double out[4]) {
  const double* L = (m->nlaws > 0 && m->cell_law) ? m->kr_laws + 6 * m->cell_law[cell] : NULL;
  if (!L || L[0] == RFO_KR_BROOKS_COREY) {
    double bc[6];
    rfo_brooks_corey(m, Se, bc);
    out[0] = bc[0]; out[1] = bc[1]; out[2] = bc[2]; out[3] = bc[3];
    return;
  }
  const double aw = L[1], an = L[3], bn = L[4], cn = L[5];
  const int nw = (int)L[2];
  const double S = Se < 0.0 ? 0.0 : (Se > 1.0 ? 1.0 : Se);
  const int inside = (Se > 0.0 && Se < 1.0);
  double p = 1.0;                      /* S^(n_w - 1) */
  for (int t = 1; t < nw; ++t) p = p * S;
  out[0] = aw * (p * S);
  out[1] = inside ? (aw * nw) * p : 0.0;
  const double r = 1.0 - bn * S, q = 1.0 - cn * (S * S);
  if (r > 0.0 && q > 0.0) {
    out[2] = an * (r * r) * q;
    out[3] = inside ? an * (-2.0 * bn * r * q - 2.0 * cn * S * (r * r)) : 0.0;
  } else {
    out[2] = 0.0;
    out[3] = 0.0;
  }
}

/* Eq. (hSw): the effective saturation seen by vertex i inside an element of
 * entry pressure p_d.  Case 1: p_d = p_dmin,i -> S_i.  Otherwise p_d J(S) =
 * p_dmin J(S_i) gives S = (p_d/p_dmin)^lambda S_i, capped at the residual-NAPL
 * saturation (S_e = 1) when p_d >= p_dmin J(S_i) (case 2, which is the
 * branch taken at equality).                                               */
void rfo_shat(const rfo_model* m, double Se, double pdc, double pdmin, double out[2]) {
  if (pdc == pdmin) { out[0] = Se; out[1] = 1.0; return; }
  double r = pdc / pdmin;
  double rl = (m->lambda == 2.0) ? r * r : pow(r, m->lambda);
  double t = rl * Se;
  if (t >= 1.0) { out[0] = 1.0; out[1] = 0.0; }
  else { out[0] = t; out[1] = rl; }
}

/* ------------------------------------------------------------------------ */
/* Eq. (pdmin): minimum entry pressure over the sub-control volumes of b_i,
 * i.e. over all elements around vertex i.  Precomputed once.               */
void rfo_pdmin(const rfo_model* m, double* pdmin) {
  const int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  const int cx = nx - 1, cy = ny - 1, cz = (m->dim == 3) ? nz - 1 : 1;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double best = INFINITY;
        for (int c2 = 0; c2 < (m->dim == 3 ? 2 : 1); ++c2)
          for (int c1 = 0; c1 < 2; ++c1)
            for (int c0 = 0; c0 < 2; ++c0) {
              int ci = i - c0, cj = j - c1, ck = (m->dim == 3) ? k - c2 : 0;
              if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
              double p = m->pd[ci + cx * (cj + cy * ck)];
              if (p < best) best = p;
            }
        pdmin[i + nx * (j + ny * k)] = best;
      }
}

/* Lumped storage weight (Phi V)_i = sum over elements e around i of
 * Phi_e |e| / 2^d  (Eq. (dsW): storage evaluated at the vertex).          */
void rfo_phiv(const rfo_model* m, double* phiv) {
  const int nx = m->n[0], ny = m->n[1], nz = m->n[2];
  const int cx = nx - 1, cy = ny - 1, cz = (m->dim == 3) ? nz - 1 : 1;
  double vol = m->h[0] * m->h[1] * (m->dim == 3 ? m->h[2] : 1.0);
  double frac = (m->dim == 3) ? 0.125 : 0.25;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        double s = 0.0;
        for (int c2 = 0; c2 < (m->dim == 3 ? 2 : 1); ++c2)
          for (int c1 = 0; c1 < 2; ++c1)
            for (int c0 = 0; c0 < 2; ++c0) {
              int ci = i - c0, cj = j - c1, ck = (m->dim == 3) ? k - c2 : 0;
              if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
              s += m->phi[ci + cx * (cj + cy * ck)] * vol * frac;
            }
        phiv[i + nx * (j + ny * k)] = s;
      }
}

/* Sum over the sub-control volumes b_i^j of vertex v (one per element j around
 * it) of Phi_j |b_i^j| times, for want = 0, the water saturation of b_i^j and,
 * for want = 1, d S hat_e / d S_e (Eq. (hSw)).  With the S hat storage variant
 * the water saturation of b_i^j is S_wr + S hat_e (1 - S_wr - S_nr).        */
static double storage_weight(const rfo_model* m, const double* pdmin, double Se, int v, int want) {
  const int nx = m->n[0], ny = m->n[1];
  const int cx = nx - 1, cy = ny - 1, cz = (m->dim == 3) ? m->n[2] - 1 : 1;
  const int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
  const double vol = m->h[0] * m->h[1] * (m->dim == 3 ? m->h[2] : 1.0);
  const double frac = (m->dim == 3) ? 0.125 : 0.25;
  const double den = 1.0 - m->S_wr - m->S_nr;
  double s = 0.0;
  for (int c2 = 0; c2 < (m->dim == 3 ? 2 : 1); ++c2)
    for (int c1 = 0; c1 < 2; ++c1)
      for (int c0 = 0; c0 < 2; ++c0) {
        int ci = i - c0, cj = j - c1, ck = (m->dim == 3) ? k - c2 : 0;
        if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
        const int cell = ci + cx * (cj + cy * ck);
        double sh[2];
        rfo_shat(m, Se, m->pd[cell], pdmin[v], sh);
        const double w = m->phi[cell] * vol * frac;
        s += w * (want ? sh[1] : m->S_wr + sh[0] * den);
      }
  return s;
}

/* Storage terms m_w,i and m_n,i of Eqs. (dsW),(dpN): rho_alpha times the sum
 * over b_i^j of Phi_j |b_i^j| S_alpha.  The discretisation of Sec. 3 uses the
 * vertex saturation in every b_i^j; the S hat storage variant uses S hat.   */
void rfo_storage(const rfo_model* m, const double* u, double* mass) {
  const int nv = nverts(m->n);
  const double den = 1.0 - m->S_wr - m->S_nr;
  double* pdmin = malloc(sizeof(double) * nv);
  double* phiv = malloc(sizeof(double) * nv);
  rfo_pdmin(m, pdmin);
  rfo_phiv(m, phiv);
  for (int v = 0; v < nv; ++v) {
    const double Sn = u[2 * v + 1];
    if (m->scheme & RFO_SCHEME_SHAT_STORAGE) {
      const double Se = (1.0 - Sn - m->S_wr) / den;
      const double sw = storage_weight(m, pdmin, Se, v, 0);   /* sum Phi |b| S_w */
      mass[2 * v] = m->rho_w * sw;
      mass[2 * v + 1] = m->rho_n * (phiv[v] - sw);
    } else {
      mass[2 * v] = m->rho_w * (phiv[v] * (1.0 - Sn));
      mass[2 * v + 1] = m->rho_n * (phiv[v] * Sn);
    }
  }
  free(pdmin); free(phiv);
}

/* ------------------------------------------------------------------------ */
/* Assembly of F(u), J = F_u and M.  Loop over elements; inside each element
 * over its d*2^(d-1) sub-control-volume faces (one per element edge a->b,
 * a = lower corner along the edge's axis k).  For each face:
 *   A_f = prod_{m != k} h_m/2, x_M = face centre (1/2 along k, 1/4 from the
 *   a side in the other axes).
 *   G(q) = d/dx_k of the Q1 interpolant at x_M
 *        = (sum over the element edges parallel to k of w (q_hi - q_lo)) / h_k,
 *        w = prod_{m != k} (3/4 on a's side, 1/4 opposite).
 *   With p_n = p_w + p_c at vertices (p_c,i = p_dmin,i J(S_e,i)):
 *     T_w = -K A_f (G(p_n) - rho_w g_k),  T_n = -K A_f (G(p_n) - rho_n g_k),
 *     T_c = -K A_f G(p_c).
 *   Mass fluxes a->b (Eqs. (dsW),(dpN) in the upwind form):
 *     F_w = rho_w [ lam_w(S_up(T_w)) T_w - lam_w(S_w(x_M)) T_c ]
 *     F_n = rho_n lam_n(S hat_up(T_n), e) T_n
 *   with lam = k_r/mu and "up" = a if T >= 0 else b (Eqs. (up_krw),(up_krn)).
 *   The capillary-diffusion mobility is not upwinded (Sec. 3.2) and is taken
 *   at x_M from the Q1-interpolated saturation.  S hat (Eq. (hSw)) enters
 *   k_rn only (Eqs. (krn_ip),(krw_ip)).
 * Residual F_i = -(sum of mass fluxes out of b_i) + q_in,i; storage is the
 * left-hand side M u' (Sec. 4).  Dirichlet p_w rows become the algebraic
 * equation 0 = p_dir - p_w (M row 0, J row -e).                            */
void rfo_assemble(const rfo_model* m, const double* u, double* F, double* J, double* mdiag) {
  const int dim = m->dim, nx = m->n[0], ny = m->n[1], nz = m->n[2];
  const int nv = nx * ny * nz, nb = nblk(dim);
  const int cx = nx - 1, cy = ny - 1, cz = (dim == 3) ? nz - 1 : 1;
  const int ncorner = 1 << dim, nedge = 1 << (dim - 1);
  const double den = 1.0 - m->S_wr - m->S_nr;

  double* pdmin = malloc(sizeof(double) * nv);
  double* Se = malloc(sizeof(double) * nv);
  double* pn = malloc(sizeof(double) * nv);
  double* pc = malloc(sizeof(double) * nv);
  double* dpc = malloc(sizeof(double) * nv);
  rfo_pdmin(m, pdmin);
#pragma omp parallel for schedule(static)
  for (int v = 0; v < nv; ++v) {
    double bc[6];
    Se[v] = (1.0 - u[2 * v + 1] - m->S_wr) / den;
    rfo_brooks_corey(m, Se[v], bc);
    pc[v] = pdmin[v] * bc[4];
    dpc[v] = -(pdmin[v] * bc[5]) / den;   /* d p_c / d S_n */
    pn[v] = u[2 * v] + pc[v];
  }

  for (int v = 0; v < 2 * nv; ++v) F[v] = m->q_in ? m->q_in[v] : 0.0;
  if (J) memset(J, 0, sizeof(double) * (size_t)nv * nb * 4);

  for (int ck = 0; ck < cz; ++ck)
    for (int cj = 0; cj < cy; ++cj)
      for (int ci = 0; ci < cx; ++ci) {
        const int cell = ci + cx * (cj + cy * ck);
        const double Kc = m->K[cell], pdc = m->pd[cell];
        int vq[8], qoff[8][3];
        double krn_h[8], dkrn_h[8], krw_c[8], dkrw_c[8];
        for (int q = 0; q < ncorner; ++q) {
          qoff[q][0] = q & 1; qoff[q][1] = (q >> 1) & 1; qoff[q][2] = (q >> 2) & 1;
          int vi = ci + qoff[q][0], vj = cj + qoff[q][1], vk = (dim == 3) ? ck + qoff[q][2] : 0;
          vq[q] = vi + nx * (vj + ny * vk);
          double sh[2], kr[4];
          rfo_shat(m, Se[vq[q]], pdc, pdmin[vq[q]], sh);
          rfo_kr_law(m, cell, sh[0], kr);
          krn_h[q] = kr[2];
          dkrn_h[q] = kr[3] * sh[1] * (-1.0 / den);  /* d k_rn(S hat) / d S_n */
          /* k_rw of the corner's S_w with this cell's law (Eq. krw_ip): the
           * vertex value when one law holds everywhere */
          rfo_kr_law(m, cell, Se[vq[q]], kr);
          krw_c[q] = kr[0];
          dkrw_c[q] = -kr[1] / den;                   /* d k_rw / d S_n */
        }
        for (int k = 0; k < dim; ++k) {
          int oth[2], no = 0;
          for (int mm = 0; mm < dim; ++mm) if (mm != k) oth[no++] = mm;
          double Af = 1.0;
          for (int t = 0; t < no; ++t) Af = Af * (m->h[oth[t]] * 0.5);
          const double KA = Kc * Af;
          for (int e = 0; e < nedge; ++e) {
            int o[2] = {e & 1, (e >> 1) & 1};
            int a = 0;
            for (int t = 0; t < no; ++t) a |= o[t] << oth[t];
            const int b = a | (1 << k);
            /* gradient along k at x_M, canonical edge order e' = 0..nedge-1 */
            double gpn = 0.0, gpc = 0.0, gpw = 0.0;
            for (int e2 = 0; e2 < nedge; ++e2) {
              int o2[2] = {e2 & 1, (e2 >> 1) & 1};
              double w = 1.0;
              int a2 = 0;
              for (int t = 0; t < no; ++t) {
                w = w * (o2[t] == o[t] ? 0.75 : 0.25);
                a2 |= o2[t] << oth[t];
              }
              int b2 = a2 | (1 << k);
              gpn = gpn + w * (pn[vq[b2]] - pn[vq[a2]]);
              gpc = gpc + w * (pc[vq[b2]] - pc[vq[a2]]);
              gpw = gpw + w * (u[2 * vq[b2]] - u[2 * vq[a2]]);
            }
            gpn = gpn / m->h[k];
            gpc = gpc / m->h[k];
            gpw = gpw / m->h[k];
            /* Q1 interpolation weights at x_M, and the saturation there */
            double wM[8], SeM = 0.0;
            for (int q = 0; q < ncorner; ++q) {
              double w = 0.5;
              for (int t = 0; t < no; ++t) w = w * (qoff[q][oth[t]] == o[t] ? 0.75 : 0.25);
              wM[q] = w;
              SeM = SeM + w * Se[vq[q]];
            }
            const double Tw = -KA * (gpn - m->rho_w * m->g[k]);
            const double Tn = -KA * (gpn - m->rho_n * m->g[k]);
            const double Tc = -KA * gpc;
            /* Darcy-velocity upwinding of the whole water flux (scheme variant):
             * T_pw = -K A_f (G(p_w) - rho_w g_k), equal to T_w - T_c up to rounding */
            const int darcy = (m->scheme & RFO_SCHEME_DARCY_UPWIND) != 0;
            const double Tpw = -KA * (gpw - m->rho_w * m->g[k]);
            const int uw = darcy ? ((Tpw >= 0.0) ? a : b) : ((Tw >= 0.0) ? a : b);
            const int un = (Tn >= 0.0) ? a : b;
            double bcM[4];
            rfo_kr_law(m, cell, SeM, bcM);
            const double lw_up = krw_c[uw] / m->mu_w;
            const double lwM = bcM[0] / m->mu_w;
            const double ln_up = krn_h[un] / m->mu_n;
            const double Fw = darcy ? m->rho_w * (lw_up * Tpw) : m->rho_w * (lw_up * Tw - lwM * Tc);
            const double Fn = m->rho_n * (ln_up * Tn);
            F[2 * vq[a]] -= Fw; F[2 * vq[a] + 1] -= Fn;
            F[2 * vq[b]] += Fw; F[2 * vq[b] + 1] += Fn;
            if (!J) continue;
            const double dlw_up = dkrw_c[uw] / m->mu_w;
            const double dlwM_dSeM = bcM[1] / m->mu_w;
            const double dln_up = dkrn_h[un] / m->mu_n;
            for (int q = 0; q < ncorner; ++q) {
              /* d G / d q_q: +-w/h_k, sign + on the b side of the edge */
              double w = 1.0;
              for (int t = 0; t < no; ++t) w = w * (qoff[q][oth[t]] == o[t] ? 0.75 : 0.25);
              const double gq = (qoff[q][k] ? w : -w) / m->h[k];
              const double dT = -KA * gq;
              const double dlwM = wM[q] * dlwM_dSeM * (-1.0 / den);
              double d[4];
              d[0] = m->rho_w * lw_up * dT;
              d[1] = m->rho_w * ((q == uw ? dlw_up * Tw : 0.0) + lw_up * dT * dpc[vq[q]]
                                 - dlwM * Tc - lwM * dT * dpc[vq[q]]);
              d[2] = m->rho_n * ln_up * dT;
              d[3] = m->rho_n * ((q == un ? dln_up * Tn : 0.0) + ln_up * dT * dpc[vq[q]]);
              if (darcy) {   /* T_pw depends on p_w only */
                d[1] = m->rho_w * (q == uw ? dlw_up * Tpw : 0.0);
              }
              for (int side = 0; side < 2; ++side) {
                const int r = side ? b : a;
                const double sg = side ? 1.0 : -1.0;
                int bi = blk(dim, qoff[q][0] - qoff[r][0], qoff[q][1] - qoff[r][1],
                             qoff[q][2] - qoff[r][2]);
                double* Jb = J + ((size_t)vq[r] * nb + bi) * 4;
                for (int t = 0; t < 4; ++t) Jb[t] += sg * d[t];
              }
            }
          }
        }
      }

  double* phiv = malloc(sizeof(double) * nv);
  rfo_phiv(m, phiv);
  if (m->scheme & RFO_SCHEME_SHAT_STORAGE) {
    /* S hat storage: d m_n,i / d S_n,i = rho_n sum_j Phi_j |b_i^j| d S hat_e / d S_e
     * (S_n of b_i^j is 1 - S_wr - S hat_e (1 - S_wr - S_nr)); kept in phiv */
    for (int v = 0; v < nv; ++v) phiv[v] = storage_weight(m, pdmin, Se[v], v, 1);
  }
  for (int v = 0; v < nv; ++v) {
    int dirv = m->dir ? m->dir[v] : 0;
    if (mdiag) {
      mdiag[2 * v] = dirv ? 0.0 : -m->rho_w * phiv[v];
      mdiag[2 * v + 1] = m->rho_n * phiv[v];
    }
    if (!dirv) continue;
    F[2 * v] = m->pw_dir[v] - u[2 * v];
    if (J) {
      for (int bi = 0; bi < nb; ++bi) {
        J[((size_t)v * nb + bi) * 4 + 0] = 0.0;
        J[((size_t)v * nb + bi) * 4 + 1] = 0.0;
      }
      J[((size_t)v * nb + centre(dim)) * 4 + 0] = -1.0;
    }
  }
  free(phiv); free(pdmin); free(Se); free(pn); free(pc); free(dpc);
}

/* ------------------------------------------------------------------------ */
/* Stage matrix A = shift*M - J, shift = 1/h_j (Sec. 4: (M - tau J) du = tau F
 * divided by tau).                                                          */
void rfo_make_A(int nv, int nb, const double* J, const double* mdiag, double shift, double* A) {
  const int c = (nb == 27) ? 13 : 4;
#pragma omp parallel for schedule(static)
  for (size_t t = 0; t < (size_t)nv * nb * 4; ++t) A[t] = -J[t];
  for (int v = 0; v < nv; ++v) {
    A[((size_t)v * nb + c) * 4 + 1] += shift * mdiag[2 * v];
    A[((size_t)v * nb + c) * 4 + 3] += shift * mdiag[2 * v + 1];
  }
}

/* (A x)_v accumulated block by block over the stencil; skip_centre leaves out
 * the diagonal block. */
static void row_apply(int dim, const int n[3], const double* A, const double* x, int i, int j, int k,
                      int skip_centre, double out[2]) {
  const int nb = nblk(dim), v = i + n[0] * (j + n[1] * k);
  double s0 = 0.0, s1 = 0.0;
  for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int ii = i + dx, jj = j + dy, kk = k + dz;
        if (ii < 0 || ii >= n[0] || jj < 0 || jj >= n[1] || kk < 0 || kk >= n[2]) continue;
        if (skip_centre && dx == 0 && dy == 0 && dz == 0) continue;
        const double* a = A + ((size_t)v * nb + blk(dim, dx, dy, dz)) * 4;
        const double* xv = x + 2 * (ii + n[0] * (jj + n[1] * kk));
        s0 += a[0] * xv[0] + a[1] * xv[1];
        s1 += a[2] * xv[0] + a[3] * xv[1];
      }
  out[0] = s0; out[1] = s1;
}

void rfo_spmv(int dim, const int n[3], const double* A, const double* x, double* y) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        double s[2];
        row_apply(dim, n, A, x, i, j, k, 0, s);
        int v = i + n[0] * (j + n[1] * k);
        y[2 * v] = s[0]; y[2 * v + 1] = s[1];
      }
}

void rfo_residual(int dim, const int n[3], const double* A, const double* b, const double* x, double* r) {
  rfo_spmv(dim, n, A, x, r);
  const int N = 2 * nverts(n);
#pragma omp parallel for schedule(static)
  for (int t = 0; t < N; ++t) r[t] = b[t] - r[t];
}

/* 2x2 diagonal-block inverse applied to s. */
static void dsolve(const double* a, const double s[2], double y[2]) {
  double det = a[0] * a[3] - a[1] * a[2];
  y[0] = (a[3] * s[0] - a[1] * s[1]) / det;
  y[1] = (a[0] * s[1] - a[2] * s[0]) / det;
}

/* Damped point-block Jacobi: x_out = x_in + omega D^-1 (b - A x_in). */
void rfo_jacobi(int dim, const int n[3], const double* A, const double* b, const double* xin,
                double* xout, double omega) {
  const int nb = nblk(dim);
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int v = i + n[0] * (j + n[1] * k);
        double s[2], r[2], y[2];
        row_apply(dim, n, A, xin, i, j, k, 0, s);
        r[0] = b[2 * v] - s[0]; r[1] = b[2 * v + 1] - s[1];
        dsolve(A + ((size_t)v * nb + centre(dim)) * 4, r, y);
        xout[2 * v] = xin[2 * v] + omega * y[0];
        xout[2 * v + 1] = xin[2 * v + 1] + omega * y[1];
      }
}

/* Multi-colour block Gauss-Seidel: colour = (i%2) + 2(j%2) [+ 4(k%2)]; the
 * 2^d colours are swept in increasing (forward) or decreasing order.
 * Vertices of one colour do not couple through a 3^d stencil, so the order
 * within a colour is immaterial.  x_v <- D_v^-1 (b_v - sum_{w != v} A_vw x_w). */
void rfo_gs_sweep(int dim, const int n[3], const double* A, const double* b, double* x, int forward) {
  const int nb = nblk(dim), ncol = 1 << dim;
  for (int cc = 0; cc < ncol; ++cc) {
    int col = forward ? cc : ncol - 1 - cc;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          if (((i & 1) | ((j & 1) << 1) | ((k & 1) << 2)) != col) continue;
          int v = i + n[0] * (j + n[1] * k);
          double s[2], r[2];
          row_apply(dim, n, A, x, i, j, k, 1, s);
          r[0] = b[2 * v] - s[0]; r[1] = b[2 * v + 1] - s[1];
          dsolve(A + ((size_t)v * nb + centre(dim)) * 4, r, x + 2 * v);
        }
  }
}

/* Trilinear (bilinear) prolongation per component on the vertex-nested
 * hierarchy (coarse vertex I sits at fine 2I); weight prod_axis (1 if the
 * fine offset is 0, 1/2 if it is +-1).  Reading: Dirichlet p_w unknowns are
 * not in the correction space, so component 0 weights vanish whenever the
 * fine or the coarse vertex is Dirichlet.  Restriction is the transpose.  */
static double pweight(int dim, int fi, int fj, int fk, int I, int J, int K) {
  int d[3] = {fi - 2 * I, fj - 2 * J, fk - 2 * K};
  double w = 1.0;
  for (int t = 0; t < dim; ++t) {
    if (d[t] == 0) continue;
    if (d[t] == 1 || d[t] == -1) w *= 0.5;
    else return 0.0;
  }
  return w;
}

void rfo_restrict(int dim, const int nf[3], const unsigned char* dmf, const int nc[3],
                  const unsigned char* dmc, const double* rf, double* bc) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int K = 0; K < nc[2]; ++K)
    for (int J = 0; J < nc[1]; ++J)
      for (int I = 0; I < nc[0]; ++I) {
        int vc = I + nc[0] * (J + nc[1] * K);
        double s0 = 0.0, s1 = 0.0;
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int fi = 2 * I + dx, fj = 2 * J + dy, fk = (dim == 3) ? 2 * K + dz : 0;
              if (fi < 0 || fi >= nf[0] || fj < 0 || fj >= nf[1] || fk < 0 || fk >= nf[2]) continue;
              int vf = fi + nf[0] * (fj + nf[1] * fk);
              double w = pweight(dim, fi, fj, fk, I, J, (dim == 3) ? K : 0);
              if (!(dmf[vf] || dmc[vc])) s0 += w * rf[2 * vf];
              s1 += w * rf[2 * vf + 1];
            }
        bc[2 * vc] = s0; bc[2 * vc + 1] = s1;
      }
}

void rfo_prolong_add(int dim, const int nf[3], const unsigned char* dmf, const int nc[3],
                     const unsigned char* dmc, const double* xc, double* xf) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int fk = 0; fk < nf[2]; ++fk)
    for (int fj = 0; fj < nf[1]; ++fj)
      for (int fi = 0; fi < nf[0]; ++fi) {
        int vf = fi + nf[0] * (fj + nf[1] * fk);
        double s0 = 0.0, s1 = 0.0;
        for (int K = fk / 2; K <= (fk + 1) / 2; ++K)
          for (int J = fj / 2; J <= (fj + 1) / 2; ++J)
            for (int I = fi / 2; I <= (fi + 1) / 2; ++I) {
              if (I >= nc[0] || J >= nc[1] || K >= nc[2]) continue;
              double w = pweight(dim, fi, fj, fk, I, J, K);
              if (w == 0.0) continue;
              int vc = I + nc[0] * (J + nc[1] * K);
              if (!(dmf[vf] || dmc[vc])) s0 += w * xc[2 * vc];
              s1 += w * xc[2 * vc + 1];
            }
        xf[2 * vf] += s0; xf[2 * vf + 1] += s1;
      }
}

/* Galerkin coarse operator A_c = P^T A P, written as the triple sum over
 * fine rows i, their stencil neighbours j and the coarse parents I of i and
 * J of j.  Coarse Dirichlet p_w rows/columns vanish through the masked P; the
 * row is then made the identity, like the fine Dirichlet rows.             */
void rfo_galerkin(int dim, const int nf[3], const unsigned char* dmf, const double* Af,
                  const int nc[3], const unsigned char* dmc, double* Ac) {
  const int nb = nblk(dim), nvc = nverts(nc);
  memset(Ac, 0, sizeof(double) * (size_t)nvc * nb * 4);
  for (int fk = 0; fk < nf[2]; ++fk)
    for (int fj = 0; fj < nf[1]; ++fj)
      for (int fi = 0; fi < nf[0]; ++fi) {
        int vi = fi + nf[0] * (fj + nf[1] * fk);
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int gi = fi + dx, gj = fj + dy, gk = fk + dz;
              if (gi < 0 || gi >= nf[0] || gj < 0 || gj >= nf[1] || gk < 0 || gk >= nf[2]) continue;
              int vj = gi + nf[0] * (gj + nf[1] * gk);
              const double* a = Af + ((size_t)vi * nb + blk(dim, dx, dy, dz)) * 4;
              for (int K = fk / 2; K <= (fk + 1) / 2; ++K)
                for (int J = fj / 2; J <= (fj + 1) / 2; ++J)
                  for (int I = fi / 2; I <= (fi + 1) / 2; ++I) {
                    double wi = pweight(dim, fi, fj, fk, I, J, K);
                    if (wi == 0.0) continue;
                    int vI = I + nc[0] * (J + nc[1] * K);
                    for (int K2 = gk / 2; K2 <= (gk + 1) / 2; ++K2)
                      for (int J2 = gj / 2; J2 <= (gj + 1) / 2; ++J2)
                        for (int I2 = gi / 2; I2 <= (gi + 1) / 2; ++I2) {
                          double wj = pweight(dim, gi, gj, gk, I2, J2, K2);
                          if (wj == 0.0) continue;
                          int vJ = I2 + nc[0] * (J2 + nc[1] * K2);
                          double* c = Ac + ((size_t)vI * nb + blk(dim, I2 - I, J2 - J, K2 - K)) * 4;
                          for (int al = 0; al < 2; ++al)
                            for (int be = 0; be < 2; ++be) {
                              double pa = (al == 0 && (dmf[vi] || dmc[vI])) ? 0.0 : wi;
                              double pb = (be == 0 && (dmf[vj] || dmc[vJ])) ? 0.0 : wj;
                              c[2 * al + be] += pa * a[2 * al + be] * pb;
                            }
                        }
                  }
            }
      }
  for (int v = 0; v < nvc; ++v)
    if (dmc[v]) Ac[((size_t)v * nb + centre(dim)) * 4 + 0] = 1.0;
}

/* Dense LU with partial pivoting (row-major N x N), the textbook algorithm. */
int rfo_lu_factor(int N, double* LU, int* piv) {
  for (int c = 0; c < N; ++c) piv[c] = c;   /* defined even if a zero pivot stops the factorisation */
  for (int c = 0; c < N; ++c) {
    int p = c;
    double best = fabs(LU[(size_t)c * N + c]);
    for (int r = c + 1; r < N; ++r)
      if (fabs(LU[(size_t)r * N + c]) > best) { best = fabs(LU[(size_t)r * N + c]); p = r; }
    piv[c] = p;
    if (best == 0.0) return -1;
    if (p != c)
      for (int t = 0; t < N; ++t) {
        double tmp = LU[(size_t)c * N + t]; LU[(size_t)c * N + t] = LU[(size_t)p * N + t]; LU[(size_t)p * N + t] = tmp;
      }
    for (int r = c + 1; r < N; ++r) {
      double l = LU[(size_t)r * N + c] / LU[(size_t)c * N + c];
      LU[(size_t)r * N + c] = l;
      for (int t = c + 1; t < N; ++t) LU[(size_t)r * N + t] -= l * LU[(size_t)c * N + t];
    }
  }
  return 0;
}

void rfo_lu_solve(int N, const double* LU, const int* piv, double* x) {
  for (int c = 0; c < N; ++c) {
    int p = piv[c];
    if (p != c) { double t = x[c]; x[c] = x[p]; x[p] = t; }
  }
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < r; ++c) x[r] -= LU[(size_t)r * N + c] * x[c];
  for (int r = N - 1; r >= 0; --r) {
    for (int c = r + 1; c < N; ++c) x[r] -= LU[(size_t)r * N + c] * x[c];
    x[r] /= LU[(size_t)r * N + r];
  }
}

/* ------------------------------------------------------------------------ */
/* Geometric multigrid V(nu1,nu2) on the vertex-nested hierarchy with Galerkin
 * coarse operators and a dense LU on the coarsest level.                   */
#define RFO_MAXL 16
struct rfo_gmg {
  int dim, nl, smoother, nu1, nu2;
  double omega;
  int n[RFO_MAXL][3];
  double* A[RFO_MAXL];
  unsigned char* dm[RFO_MAXL];
  double *x[RFO_MAXL], *b[RFO_MAXL], *r[RFO_MAXL];
  double* lu; int* piv; int N;
};

rfo_gmg* rfo_gmg_create(int dim, const int n[3], const double* A0, const unsigned char* dmask,
                        int nlevels, int smoother, int nu1, int nu2, double omega) {
  rfo_gmg* g = calloc(1, sizeof(rfo_gmg));
  const int nb = nblk(dim);
  g->dim = dim; g->smoother = smoother; g->nu1 = nu1; g->nu2 = nu2; g->omega = omega;
  for (int t = 0; t < 3; ++t) g->n[0][t] = n[t];
  int nl = 1;
  while (nl < nlevels && nl < RFO_MAXL) {
    int ok = 1, nn[3];
    for (int t = 0; t < 3; ++t) {
      int m = g->n[nl - 1][t];
      if (t >= dim) { nn[t] = 1; continue; }
      if ((m - 1) % 2 != 0 || m < 3) ok = 0;
      nn[t] = (m - 1) / 2 + 1;
    }
    if (!ok) break;
    for (int t = 0; t < 3; ++t) g->n[nl][t] = nn[t];
    ++nl;
  }
  g->nl = nl;
  for (int l = 0; l < nl; ++l) {
    int nv = nverts(g->n[l]);
    g->A[l] = malloc(sizeof(double) * (size_t)nv * nb * 4);
    g->dm[l] = malloc(nv);
    g->x[l] = calloc(2 * nv, sizeof(double));
    g->b[l] = calloc(2 * nv, sizeof(double));
    g->r[l] = calloc(2 * nv, sizeof(double));
  }
  memcpy(g->A[0], A0, sizeof(double) * (size_t)nverts(n) * nb * 4);
  for (int v = 0; v < nverts(n); ++v) g->dm[0][v] = dmask ? dmask[v] : 0;
  for (int l = 1; l < nl; ++l) {
    const int* nc = g->n[l];
    for (int K = 0; K < nc[2]; ++K)
      for (int J = 0; J < nc[1]; ++J)
        for (int I = 0; I < nc[0]; ++I) {
          int fk = (dim == 3) ? 2 * K : 0;
          g->dm[l][I + nc[0] * (J + nc[1] * K)] = g->dm[l - 1][2 * I + g->n[l - 1][0] * (2 * J + g->n[l - 1][1] * fk)];
        }
    rfo_galerkin(dim, g->n[l - 1], g->dm[l - 1], g->A[l - 1], nc, g->dm[l], g->A[l]);
  }
  /* dense coarsest operator */
  const int* nc = g->n[nl - 1];
  int nvc = nverts(nc), N = 2 * nvc;
  g->N = N;
  g->lu = calloc((size_t)N * N, sizeof(double));
  g->piv = malloc(sizeof(int) * N);
  for (int K = 0; K < nc[2]; ++K)
    for (int J = 0; J < nc[1]; ++J)
      for (int I = 0; I < nc[0]; ++I) {
        int v = I + nc[0] * (J + nc[1] * K);
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int ii = I + dx, jj = J + dy, kk = K + dz;
              if (ii < 0 || ii >= nc[0] || jj < 0 || jj >= nc[1] || kk < 0 || kk >= nc[2]) continue;
              int w = ii + nc[0] * (jj + nc[1] * kk);
              const double* a = g->A[nl - 1] + ((size_t)v * nb + blk(dim, dx, dy, dz)) * 4;
              for (int al = 0; al < 2; ++al)
                for (int be = 0; be < 2; ++be) g->lu[(size_t)(2 * v + al) * N + 2 * w + be] = a[2 * al + be];
            }
      }
  rfo_lu_factor(N, g->lu, g->piv);
  return g;
}

void rfo_gmg_free(rfo_gmg* g) {
  if (!g) return;
  for (int l = 0; l < g->nl; ++l) { free(g->A[l]); free(g->dm[l]); free(g->x[l]); free(g->b[l]); free(g->r[l]); }
  free(g->lu); free(g->piv); free(g);
}
int rfo_gmg_nlevels(const rfo_gmg* g) { return g->nl; }
void rfo_gmg_level_dims(const rfo_gmg* g, int level, int n[3]) { for (int t = 0; t < 3; ++t) n[t] = g->n[level][t]; }
void rfo_gmg_level_matrix(const rfo_gmg* g, int level, double* A) {
  memcpy(A, g->A[level], sizeof(double) * (size_t)nverts(g->n[level]) * nblk(g->dim) * 4);
}

static void smooth(rfo_gmg* g, int l, int nsweep, int pre) {
  const int* n = g->n[l];
  int nv = nverts(n);
  for (int s = 0; s < nsweep; ++s) {
    if (g->smoother == RFO_JACOBI) {
      rfo_jacobi(g->dim, n, g->A[l], g->b[l], g->x[l], g->r[l], g->omega);
      memcpy(g->x[l], g->r[l], sizeof(double) * 2 * nv);
    } else {
      rfo_gs_sweep(g->dim, n, g->A[l], g->b[l], g->x[l], pre);
    }
  }
}

static void vcycle(rfo_gmg* g, int l) {
  const int* n = g->n[l];
  int nv = nverts(n);
  if (l == g->nl - 1) {
    memcpy(g->x[l], g->b[l], sizeof(double) * 2 * nv);
    rfo_lu_solve(g->N, g->lu, g->piv, g->x[l]);
    return;
  }
  memset(g->x[l], 0, sizeof(double) * 2 * nv);
  smooth(g, l, g->nu1, 1);
  rfo_residual(g->dim, n, g->A[l], g->b[l], g->x[l], g->r[l]);
  rfo_restrict(g->dim, n, g->dm[l], g->n[l + 1], g->dm[l + 1], g->r[l], g->b[l + 1]);
  vcycle(g, l + 1);
  rfo_prolong_add(g->dim, n, g->dm[l], g->n[l + 1], g->dm[l + 1], g->x[l + 1], g->x[l]);
  smooth(g, l, g->nu2, 0);
}

void rfo_gmg_vcycle(rfo_gmg* g, const double* b, double* x) {
  int nv = nverts(g->n[0]);
  memcpy(g->b[0], b, sizeof(double) * 2 * nv);
  vcycle(g, 0);
  memcpy(x, g->x[0], sizeof(double) * 2 * nv);
}

/* ------------------------------------------------------------------------ */
/* FP32 emulation of the multigrid V-cycle: the same hierarchy, smoother and
 * schedule as rfo_gmg_vcycle, with every level matrix and vector stored in
 * float and every sum accumulated in float, as a reference for a
 * preconditioner run in single precision.  The inverse 2x2 diagonal blocks are
 * the float roundings of the double inverses of the double blocks; the
 * coarsest level is solved in double (the LU of rfo_gmg_create) and rounded
 * back to float.                                                            */
struct rfo_gmg32 {
  const rfo_gmg* g;
  float* A[RFO_MAXL];
  float* Dinv[RFO_MAXL];
  float *x[RFO_MAXL], *b[RFO_MAXL], *r[RFO_MAXL], *t[RFO_MAXL];
  double* xc;
};

static void row_apply32(int dim, const int n[3], const float* A, const float* x, int i, int j, int k,
                        int skip_centre, float out[2]) {
  const int nb = nblk(dim), v = i + n[0] * (j + n[1] * k);
  float s0 = 0.0f, s1 = 0.0f;
  for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int ii = i + dx, jj = j + dy, kk = k + dz;
        if (ii < 0 || ii >= n[0] || jj < 0 || jj >= n[1] || kk < 0 || kk >= n[2]) continue;
        if (skip_centre && dx == 0 && dy == 0 && dz == 0) continue;
        const float* a = A + ((size_t)v * nb + blk(dim, dx, dy, dz)) * 4;
        const float* xv = x + 2 * (ii + n[0] * (jj + n[1] * kk));
        s0 += a[0] * xv[0] + a[1] * xv[1];
        s1 += a[2] * xv[0] + a[3] * xv[1];
      }
  out[0] = s0; out[1] = s1;
}

static void residual32(int dim, const int n[3], const float* A, const float* b, const float* x, float* r) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int v = i + n[0] * (j + n[1] * k);
        float s[2];
        row_apply32(dim, n, A, x, i, j, k, 0, s);
        r[2 * v] = b[2 * v] - s[0];
        r[2 * v + 1] = b[2 * v + 1] - s[1];
      }
}

static void dinv32(const float* D, const float r[2], float y[2]) {
  y[0] = D[0] * r[0] + D[1] * r[1];
  y[1] = D[2] * r[0] + D[3] * r[1];
}

static void jacobi32(int dim, const int n[3], const float* A, const float* Dinv, const float* b, const float* xin,
                     float* xout, float omega) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int v = i + n[0] * (j + n[1] * k);
        float s[2], r[2], y[2];
        row_apply32(dim, n, A, xin, i, j, k, 0, s);
        r[0] = b[2 * v] - s[0]; r[1] = b[2 * v + 1] - s[1];
        dinv32(Dinv + 4 * (size_t)v, r, y);
        xout[2 * v] = xin[2 * v] + omega * y[0];
        xout[2 * v + 1] = xin[2 * v + 1] + omega * y[1];
      }
}

static void gs32(int dim, const int n[3], const float* A, const float* Dinv, const float* b, float* x, int forward) {
  const int ncol = 1 << dim;
  for (int cc = 0; cc < ncol; ++cc) {
    int col = forward ? cc : ncol - 1 - cc;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < n[2]; ++k)
      for (int j = 0; j < n[1]; ++j)
        for (int i = 0; i < n[0]; ++i) {
          if (((i & 1) | ((j & 1) << 1) | ((k & 1) << 2)) != col) continue;
          int v = i + n[0] * (j + n[1] * k);
          float s[2], r[2];
          row_apply32(dim, n, A, x, i, j, k, 1, s);
          r[0] = b[2 * v] - s[0]; r[1] = b[2 * v + 1] - s[1];
          dinv32(Dinv + 4 * (size_t)v, r, x + 2 * v);
        }
  }
}

static void restrict32(int dim, const int nf[3], const unsigned char* dmf, const int nc[3], const unsigned char* dmc,
                       const float* rf, float* bc) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int K = 0; K < nc[2]; ++K)
    for (int J = 0; J < nc[1]; ++J)
      for (int I = 0; I < nc[0]; ++I) {
        int vc = I + nc[0] * (J + nc[1] * K);
        float s0 = 0.0f, s1 = 0.0f;
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int fi = 2 * I + dx, fj = 2 * J + dy, fk = (dim == 3) ? 2 * K + dz : 0;
              if (fi < 0 || fi >= nf[0] || fj < 0 || fj >= nf[1] || fk < 0 || fk >= nf[2]) continue;
              int vf = fi + nf[0] * (fj + nf[1] * fk);
              float w = (float)pweight(dim, fi, fj, fk, I, J, (dim == 3) ? K : 0);
              if (!(dmf[vf] || dmc[vc])) s0 += w * rf[2 * vf];
              s1 += w * rf[2 * vf + 1];
            }
        bc[2 * vc] = s0; bc[2 * vc + 1] = s1;
      }
}

static void prolong_add32(int dim, const int nf[3], const unsigned char* dmf, const int nc[3],
                          const unsigned char* dmc, const float* xc, float* xf) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int fk = 0; fk < nf[2]; ++fk)
    for (int fj = 0; fj < nf[1]; ++fj)
      for (int fi = 0; fi < nf[0]; ++fi) {
        int vf = fi + nf[0] * (fj + nf[1] * fk);
        float s0 = 0.0f, s1 = 0.0f;
        for (int K = fk / 2; K <= (fk + 1) / 2; ++K)
          for (int J = fj / 2; J <= (fj + 1) / 2; ++J)
            for (int I = fi / 2; I <= (fi + 1) / 2; ++I) {
              if (I >= nc[0] || J >= nc[1] || K >= nc[2]) continue;
              float w = (float)pweight(dim, fi, fj, fk, I, J, K);
              if (w == 0.0f) continue;
              int vc = I + nc[0] * (J + nc[1] * K);
              if (!(dmf[vf] || dmc[vc])) s0 += w * xc[2 * vc];
              s1 += w * xc[2 * vc + 1];
            }
        xf[2 * vf] += s0; xf[2 * vf + 1] += s1;
      }
}

rfo_gmg32* rfo_gmg32_create(const rfo_gmg* g) {
  rfo_gmg32* h = calloc(1, sizeof(rfo_gmg32));
  const int nb = nblk(g->dim), c = centre(g->dim);
  h->g = g;
  for (int l = 0; l < g->nl; ++l) {
    const size_t nv = (size_t)nverts(g->n[l]);
    h->A[l] = malloc(sizeof(float) * nv * nb * 4);
    h->Dinv[l] = malloc(sizeof(float) * nv * 4);
    for (size_t t = 0; t < nv * nb * 4; ++t) h->A[l][t] = (float)g->A[l][t];
    for (size_t v = 0; v < nv; ++v) {
      const double* a = g->A[l] + (v * nb + c) * 4;
      const double det = a[0] * a[3] - a[1] * a[2];
      h->Dinv[l][4 * v] = (float)(a[3] / det);
      h->Dinv[l][4 * v + 1] = (float)(-a[1] / det);
      h->Dinv[l][4 * v + 2] = (float)(-a[2] / det);
      h->Dinv[l][4 * v + 3] = (float)(a[0] / det);
    }
    h->x[l] = calloc(2 * nv, sizeof(float));
    h->b[l] = calloc(2 * nv, sizeof(float));
    h->r[l] = calloc(2 * nv, sizeof(float));
    h->t[l] = calloc(2 * nv, sizeof(float));
  }
  h->xc = malloc(sizeof(double) * g->N);
  return h;
}

void rfo_gmg32_free(rfo_gmg32* h) {
  if (!h) return;
  for (int l = 0; l < h->g->nl; ++l) {
    free(h->A[l]); free(h->Dinv[l]); free(h->x[l]); free(h->b[l]); free(h->r[l]); free(h->t[l]);
  }
  free(h->xc);
  free(h);
}

static void smooth32(rfo_gmg32* h, int l, int nsweep, int pre) {
  const rfo_gmg* g = h->g;
  const int* n = g->n[l];
  const int nv = nverts(n);
  for (int s = 0; s < nsweep; ++s) {
    if (g->smoother == RFO_JACOBI) {
      jacobi32(g->dim, n, h->A[l], h->Dinv[l], h->b[l], h->x[l], h->t[l], (float)g->omega);
      memcpy(h->x[l], h->t[l], sizeof(float) * 2 * nv);
    } else {
      gs32(g->dim, n, h->A[l], h->Dinv[l], h->b[l], h->x[l], pre);
    }
  }
}

static void vcycle32(rfo_gmg32* h, int l) {
  const rfo_gmg* g = h->g;
  const int* n = g->n[l];
  const int nv = nverts(n);
  if (l == g->nl - 1) {
    for (int q = 0; q < 2 * nv; ++q) h->xc[q] = (double)h->b[l][q];
    rfo_lu_solve(g->N, g->lu, g->piv, h->xc);
    for (int q = 0; q < 2 * nv; ++q) h->x[l][q] = (float)h->xc[q];
    return;
  }
  memset(h->x[l], 0, sizeof(float) * 2 * nv);
  smooth32(h, l, g->nu1, 1);
  residual32(g->dim, n, h->A[l], h->b[l], h->x[l], h->r[l]);
  restrict32(g->dim, n, g->dm[l], g->n[l + 1], g->dm[l + 1], h->r[l], h->b[l + 1]);
  vcycle32(h, l + 1);
  prolong_add32(g->dim, n, g->dm[l], g->n[l + 1], g->dm[l + 1], h->x[l + 1], h->x[l]);
  smooth32(h, l, g->nu2, 0);
}

void rfo_gmg32_vcycle(rfo_gmg32* h, const float* b, float* x) {
  const int nv = nverts(h->g->n[0]);
  memcpy(h->b[0], b, sizeof(float) * 2 * nv);
  vcycle32(h, 0);
  memcpy(x, h->x[0], sizeof(float) * 2 * nv);
}

/* ------------------------------------------------------------------------ */
/* BiCGSTAB (van der Vorst), right-preconditioned, x0 = 0.  Converged when the
 * TRUE residual satisfies |b - A x| <= rtol |b|; when the recursive residual
 * passes but the true one does not, the iteration restarts from the current
 * x (r = b - A x, r_hat = r).                                              */
static double dot(int N, const double* a, const double* b) {
  double s = 0.0;
  for (int t = 0; t < N; ++t) s += a[t] * b[t];
  return s;
}

int rfo_bicgstab(int dim, const int n[3], const double* A, rfo_gmg* g, const double* b, double* x,
                 double rtol, int maxit, int* iters, double* relres) {
  const int N = 2 * nverts(n);
  double *r = malloc(sizeof(double) * N), *rh = malloc(sizeof(double) * N), *p = calloc(N, sizeof(double));
  double *v = calloc(N, sizeof(double)), *y = malloc(sizeof(double) * N), *s = malloc(sizeof(double) * N);
  double *z = malloc(sizeof(double) * N), *t = malloc(sizeof(double) * N);
  for (int q = 0; q < N; ++q) { x[q] = 0.0; r[q] = b[q]; rh[q] = b[q]; }
  double bn = sqrt(dot(N, b, b));
  int it = 0, status = 1;
  double rel = 0.0;
  if (bn == 0.0) { status = 0; goto done; }
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  for (it = 1; it <= maxit; ++it) {
    double rho = dot(N, rh, r);
    double beta = (rho / rho_old) * (alpha / omega);
#pragma omp parallel for schedule(static)
    for (int q = 0; q < N; ++q) p[q] = r[q] + beta * (p[q] - omega * v[q]);
    if (g) rfo_gmg_vcycle(g, p, y); else memcpy(y, p, sizeof(double) * N);
    rfo_spmv(dim, n, A, y, v);
    alpha = rho / dot(N, rh, v);
    /* Breakdown <r_hat, v> = 0 (a reading: the paper names BiCGSTAB only):
     * no BiCG half step (alpha = 0, so x and r stay finite), and a restart
     * from the current x after the minimal-residual half step below. */
    const int broke = !isfinite(alpha);
    if (broke) alpha = 0.0;
#pragma omp parallel for schedule(static)
    for (int q = 0; q < N; ++q) s[q] = r[q] - alpha * v[q];
    if (g) rfo_gmg_vcycle(g, s, z); else memcpy(z, s, sizeof(double) * N);
    rfo_spmv(dim, n, A, z, t);
    double tt = dot(N, t, t);
    omega = (tt > 0.0) ? dot(N, t, s) / tt : 0.0;
#pragma omp parallel for schedule(static)
    for (int q = 0; q < N; ++q) { x[q] += alpha * y[q] + omega * z[q]; r[q] = s[q] - omega * t[q]; }
    rho_old = rho;
    /* the next <r_hat, r> vanishing is a breakdown as well */
    int restart = !(omega != 0.0) || !isfinite(omega) || broke || !(dot(N, rh, r) != 0.0);
    if (sqrt(dot(N, r, r)) <= rtol * bn || restart) {
      rfo_residual(dim, n, A, b, x, r);
      rel = sqrt(dot(N, r, r)) / bn;
      if (rel <= rtol) { status = 0; break; }
      if (!isfinite(rel)) { status = 2; break; }
      memcpy(rh, r, sizeof(double) * N);
      memset(p, 0, sizeof(double) * N); memset(v, 0, sizeof(double) * N);
      rho_old = alpha = omega = 1.0;
    }
  }
  if (status != 0) {
    rfo_residual(dim, n, A, b, x, r);
    rel = sqrt(dot(N, r, r)) / bn;
    if (it > maxit) it = maxit;
  }
done:
  if (iters) *iters = it;
  if (relres) *relres = rel;
  free(r); free(rh); free(p); free(v); free(y); free(s); free(z); free(t);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Aitken-Neville extrapolation of the linearly implicit Euler columns
 * (Deuflhard's LIMEX; the paper uses it without printing the table):
 *   T_{j,k+1} = T_{j,k} + (T_{j,k} - T_{j-1,k}) / (n_j/n_{j-k} - 1).
 * Returns the final entry T_kk and the subdiagonal T_{k,k-1}.               */
void rfo_extrapolate(int kappa, const int* nseq, int len, const double* T1, double* Tkk, double* Tkk1) {
  double* T = malloc(sizeof(double) * (size_t)kappa * kappa * len);
#define TT(j, k) (T + ((size_t)(j) * kappa + (k)) * len)
  for (int j = 0; j < kappa; ++j) {
    memcpy(TT(j, 0), T1 + (size_t)j * len, sizeof(double) * len);
    for (int k = 1; k <= j; ++k) {
      double f = (double)nseq[j] / (double)nseq[j - k] - 1.0;
      for (int q = 0; q < len; ++q) TT(j, k)[q] = TT(j, k - 1)[q] + (TT(j, k - 1)[q] - TT(j - 1, k - 1)[q]) / f;
    }
  }
  memcpy(Tkk, TT(kappa - 1, kappa - 1), sizeof(double) * len);
  memcpy(Tkk1, TT(kappa - 1, kappa > 1 ? kappa - 2 : 0), sizeof(double) * len);
#undef TT
  free(T);
}

/* |grad q|^2 integrated over the domain for the Q1 interpolant, by 2-point
 * Gauss per axis (exact: each squared partial derivative is at most
 * quadratic in every variable).                                             */
double rfo_h1_seminorm2(int dim, const int n[3], const double* h, const double* q, int stride) {
  const double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  const int cx = n[0] - 1, cy = n[1] - 1, cz = (dim == 3) ? n[2] - 1 : 1;
  const int nc = 1 << dim;
  double vol = h[0] * h[1] * (dim == 3 ? h[2] : 1.0), total = 0.0;
  for (int ck = 0; ck < cz; ++ck)
    for (int cj = 0; cj < cy; ++cj)
      for (int ci = 0; ci < cx; ++ci) {
        double qv[8];
        for (int c = 0; c < nc; ++c) {
          int vi = ci + (c & 1), vj = cj + ((c >> 1) & 1), vk = (dim == 3) ? ck + ((c >> 2) & 1) : 0;
          qv[c] = q[(size_t)stride * (vi + n[0] * (vj + n[1] * vk))];
        }
        for (int gq = 0; gq < nc; ++gq) {
          double xi[3] = {gp[gq & 1], gp[(gq >> 1) & 1], gp[(gq >> 2) & 1]};
          double g2 = 0.0;
          for (int k = 0; k < dim; ++k) {
            double d = 0.0;
            for (int c = 0; c < nc; ++c) {
              double w = ((c >> k) & 1) ? 1.0 : -1.0;
              for (int mm = 0; mm < dim; ++mm)
                if (mm != k) w *= ((c >> mm) & 1) ? xi[mm] : 1.0 - xi[mm];
              d += w * qv[c];
            }
            d /= h[k];
            g2 += d * d;
          }
          total += g2 * vol / nc;
        }
      }
  return total;
}

/* Lumped L2 norm squared: sum_i V_i q_i^2 with V_i the dual-cell volume. */
double rfo_lumped_l2norm2(int dim, const int n[3], const double* h, const double* q, int stride) {
  double s = 0.0, vol = h[0] * h[1] * (dim == 3 ? h[2] : 1.0);
  for (int k = 0; k < n[2]; ++k)
    for (int j = 0; j < n[1]; ++j)
      for (int i = 0; i < n[0]; ++i) {
        int cnt = 0;
        for (int c = 0; c < (1 << dim); ++c) {
          int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = (dim == 3) ? k - ((c >> 2) & 1) : 0;
          if (ci >= 0 && ci < n[0] - 1 && cj >= 0 && cj < n[1] - 1 && ck >= 0 && ck < (dim == 3 ? n[2] - 1 : 1)) ++cnt;
        }
        double qq = q[(size_t)stride * (i + n[0] * (j + n[1] * k))];
        s += cnt * vol / (1 << dim) * qq * qq;
      }
  return s;
}

/* One LIMEX step (Sec. 4): kappa linearly implicit Euler columns with the
 * harmonic step-number sequence n_j = j and ONE Jacobian J(u0), M(u0):
 *   column j: h_j = H/n_j; u <- u0; n_j times: (M/h_j - J) du = F(u), u += du.
 * Extrapolated T_kk is the result, delta = T_kk - T_{k,k-1} the error.
 * Reading of the scaled norm: eps^2 = (alpha |grad dp_w|^2 + beta |dS_n|^2)/2
 * with alpha = 1/|grad p_w(T_kk)|^2, beta = 1/(|S_n(T_kk)|^2 + 1e-4 |Omega|).
 * Step control with q = 2: H_new = H clip((rho TOL/eps)^(1/3), fac_min, fac_max). */
int rfo_limex_step(const rfo_model* m, const double* u0, double H, const rfo_limex_opts* o,
                   double* u_out, rfo_limex_info* info) {
  const int dim = m->dim, nv = nverts(m->n), nb = nblk(dim), N = 2 * nv, kap = o->kappa;
  double* J = malloc(sizeof(double) * (size_t)nv * nb * 4);
  double* A = malloc(sizeof(double) * (size_t)nv * nb * 4);
  double* md = malloc(sizeof(double) * N);
  double* F0 = malloc(sizeof(double) * N);
  double* F = malloc(sizeof(double) * N);
  double* du = malloc(sizeof(double) * N);
  double* T1 = malloc(sizeof(double) * (size_t)kap * N);
  double* Tkk = malloc(sizeof(double) * N);
  double* Tkk1 = malloc(sizeof(double) * N);
  int* nseq = malloc(sizeof(int) * kap);
  unsigned char* dm = calloc(nv, 1);
  if (m->dir) memcpy(dm, m->dir, nv);
  rfo_assemble(m, u0, F0, J, md);
  int status = 0, solves = 0, iters_total = 0;
  for (int j = 0; j < kap; ++j) {
    nseq[j] = j + 1;
    double shift = (double)nseq[j] / H;
    rfo_make_A(nv, nb, J, md, shift, A);
    rfo_gmg* g = rfo_gmg_create(dim, m->n, A, dm, o->nlevels, o->smoother, o->nu1, o->nu2, o->omega);
    double* U = T1 + (size_t)j * N;
    memcpy(U, u0, sizeof(double) * N);
    for (int k = 0; k < nseq[j]; ++k) {
      if (k == 0) memcpy(F, F0, sizeof(double) * N);
      else rfo_assemble(m, U, F, NULL, NULL);
      int it = 0; double rr = 0.0;
      int st = rfo_bicgstab(dim, m->n, A, g, F, du, o->rtol, o->maxit, &it, &rr);
      if (st != 0) status = st;
      ++solves; iters_total += it;
      for (int q = 0; q < N; ++q) U[q] += du[q];
    }
    rfo_gmg_free(g);
  }
  rfo_extrapolate(kap, nseq, N, T1, Tkk, Tkk1);
  for (int q = 0; q < N; ++q) du[q] = Tkk[q] - Tkk1[q];
  double vol = 1.0;
  for (int t = 0; t < dim; ++t) vol *= (m->n[t] - 1) * m->h[t];
  double a = 1.0 / (rfo_h1_seminorm2(dim, m->n, m->h, Tkk, 2) + 1e-30);
  double b = 1.0 / (rfo_lumped_l2norm2(dim, m->n, m->h, Tkk + 1, 2) + 1e-4 * vol);
  double e2 = a * rfo_h1_seminorm2(dim, m->n, m->h, du, 2) + b * rfo_lumped_l2norm2(dim, m->n, m->h, du + 1, 2);
  double eps = sqrt(e2 / 2.0);
  double fac = (eps > 0.0) ? pow(o->rho * o->tol / eps, 1.0 / 3.0) : o->fac_max;
  if (fac > o->fac_max) fac = o->fac_max;
  if (fac < o->fac_min) fac = o->fac_min;
  int acc = (eps <= o->tol);
  memcpy(u_out, acc ? Tkk : u0, sizeof(double) * N);
  if (info) { info->eps = eps; info->H_new = H * fac; info->accepted = acc; info->solves = solves; info->iterations = iters_total; }
  free(J); free(A); free(md); free(F0); free(F); free(du); free(T1); free(Tkk); free(Tkk1); free(nseq); free(dm);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Adaptive integration with the step control of Sec. 4 (see rfo.h).        */
int rfo_limex_run(const rfo_model* m, const double* u0, double H0, const rfo_limex_run_opts* o, double* u_out,
                  rfo_limex_run_info* info, double* hist, int hist_cap) {
  const int N = 2 * nverts(m->n);
  double* u = malloc(sizeof(double) * N);
  double* un = malloc(sizeof(double) * N);
  memcpy(u, u0, sizeof(double) * N);
  double t = 0.0, H = H0;
  int acc = 0, rej = 0, solves = 0, iters = 0, steps = 0, status = 0, last_rejected = 0;
  for (;;) {
    if (o->max_steps > 0 && acc >= o->max_steps) break;
    if (o->t_end > 0.0 && !(t < o->t_end * (1.0 - 1e-12))) break;
    if (o->t_end > 0.0 && H > o->t_end - t) H = o->t_end - t;
    rfo_limex_info si;
    status = rfo_limex_step(m, u, H, &o->step, un, &si);
    solves += si.solves;
    iters += si.iterations;
    if (hist && steps < hist_cap) {
      hist[3 * steps] = H;
      hist[3 * steps + 1] = si.eps;
      hist[3 * steps + 2] = si.accepted;
    }
    ++steps;
    if (status != 0) break;
    double Hn = si.H_new;
    if (si.accepted) {
      memcpy(u, un, sizeof(double) * N);
      t += H;
      ++acc;
      if (o->hold_after_reject && last_rejected && Hn > H) Hn = H;
      last_rejected = 0;
    } else {
      ++rej;
      last_rejected = 1;
      if (rej > o->max_rejects) { status = 1; break; }
    }
    H = (o->H_max > 0.0 && Hn > o->H_max) ? o->H_max : Hn;
  }
  memcpy(u_out, u, sizeof(double) * N);
  if (info) {
    info->t = t; info->H_next = H; info->accepted = acc; info->rejected = rej;
    info->solves = solves; info->iterations = iters; info->steps = steps;
  }
  free(u); free(un);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Implicit Euler with Newton's method, the fixed-step scheme the paper sets
 * LIMEX against (Sec. 6, Case 4; nonlinear tolerances 1e-8 abs / 1e-6 rel).
 * One step: find u with F(u) - (m(u) - m(u_old))/H = 0, where m is the
 * storage (rfo_storage) and F the flux residual (rfo_assemble); Dirichlet p_w
 * rows keep their algebraic equation.  The Newton matrix is M(u_k)/H - J(u_k)
 * with M = dm/dS_n from the assembly.                                      */
/* R = F(u) - (m(u) - m_old)/H with no storage in Dirichlet p_w rows; returns ||R||_2 */
static double ie_residual(const rfo_model* m, const unsigned char* dm, const double* u, const double* m_old,
                          double H, const double* F, double* mk, double* R) {
  const int nv = nverts(m->n);
  rfo_storage(m, u, mk);
  double s2 = 0.0;
  for (int v = 0; v < nv; ++v) {
    for (int a = 0; a < 2; ++a) {
      const int q = 2 * v + a;
      const int storage = !(a == 0 && dm[v]);
      R[q] = F[q] - (storage ? (mk[q] - m_old[q]) / H : 0.0);
      s2 += R[q] * R[q];
    }
  }
  return sqrt(s2);
}

int rfo_ie_step(const rfo_model* m, const double* u_old, double H, const rfo_ie_opts* o, double* u_out,
                rfo_ie_info* info) {
  const int dim = m->dim, nv = nverts(m->n), nb = nblk(dim), N = 2 * nv;
  double* J = malloc(sizeof(double) * (size_t)nv * nb * 4);
  double* A = malloc(sizeof(double) * (size_t)nv * nb * 4);
  double* md = malloc(sizeof(double) * N);
  double* F = malloc(sizeof(double) * N);
  double* R = malloc(sizeof(double) * N);
  double* d = malloc(sizeof(double) * N);
  double* m0 = malloc(sizeof(double) * N);
  double* mk = malloc(sizeof(double) * N);
  double* uk = malloc(sizeof(double) * N);
  unsigned char* dm = calloc(nv, 1);
  if (m->dir) memcpy(dm, m->dir, nv);
  memcpy(u_out, u_old, sizeof(double) * N);
  rfo_storage(m, u_old, m0);
  int status = 1, newton = 0, linear = 0;
  double r0 = 0.0, r = 0.0;
  for (;;) {
    rfo_assemble(m, u_out, F, J, md);
    r = ie_residual(m, dm, u_out, m0, H, F, mk, R);
    if (newton == 0) r0 = r;
    if (r <= o->atol || r <= o->rtol * r0) { status = 0; break; }
    if (newton >= o->max_newton) break;
    rfo_make_A(nv, nb, J, md, 1.0 / H, A);
    rfo_gmg* g = rfo_gmg_create(dim, m->n, A, dm, o->nlevels, o->smoother, o->nu1, o->nu2, o->omega);
    int it = 0; double rr = 0.0;
    int st = rfo_bicgstab(dim, m->n, A, g, R, d, o->lin_rtol, o->lin_maxit, &it, &rr);
    rfo_gmg_free(g);
    linear += it;
    ++newton;
    if (st != 0) { status = st; break; }
    /* backtracking on the residual norm (max_ls halvings of the correction) */
    memcpy(uk, u_out, sizeof(double) * N);
    double lam = 1.0;
    for (int ls = 0;; ++ls) {
      for (int q = 0; q < N; ++q) u_out[q] = uk[q] + lam * d[q];
      if (o->max_ls <= 0) break;
      rfo_assemble(m, u_out, F, NULL, NULL);
      const double rt = ie_residual(m, dm, u_out, m0, H, F, mk, R);
      if (rt <= (1.0 - 1e-4 * lam) * r || ls >= o->max_ls) break;
      lam = 0.5 * lam;
    }
  }
  if (status != 0) memcpy(u_out, u_old, sizeof(double) * N);   /* a failed step keeps the state */
  if (info) { info->newton = newton; info->linear = linear; info->res0 = r0; info->res = r; }
  free(J); free(A); free(md); free(F); free(R); free(d); free(m0); free(mk); free(uk); free(dm);
  return status;
}
