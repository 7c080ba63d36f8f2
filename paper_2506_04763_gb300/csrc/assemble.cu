// assemble.cu — grid set-up (K0) and vertex-centred finite-volume assembly
// (K1: F, exact Jacobian J = F_u and lumped M; K1r: F only).
//
// Compiled with -fmad=false: every product and sum is rounded separately, in
// the order written.  The quantities on which a discrete decision rests — S_e
// (k_r clamps), p_c and p_n = p_w + p_c, the face gradients G, T_w and T_n
// (upwind directions), S_e at x_M and the S hat cap test — are in addition
// written with explicit round-to-nearest intrinsics (__dadd_rn, __dmul_rn, ...),
// so the decisions are taken on exactly the values that order defines.  The
// derivatives stay unfused too: several Jacobian entries are sums of nearly
// cancelling terms (e.g. the NAPL rows where k_rn ~ 0), whose rounding a fused
// multiply-add would change by far more than 1e-12 of the row.
//
// Method (arXiv 2506.04763):
//   Sec. 3.1, Eqs. (dsW),(dpN): dual-mesh control volumes b_i; storage lumped
//     at the vertex; one sub-control-volume face (SCVF) per element edge,
//     flux evaluated at the face midpoint x_M with face size A_f.
//   Sec. 3.2, Eqs. (up_krw),(up_krn): k_r taken from the upstream vertex by
//     the sign of v_alpha . n (v_alpha excludes the capillary-diffusion
//     part); T >= 0 picks the edge's lower vertex a.
//   Sec. 3.3, Eqs. (pdmin),(hSw),(krn_ip),(krw_ip): p_dmin per vertex and the
//     per-sub-control-volume saturation S hat, used in k_rn only.
//   Sec. 2, Eqs. (sW),(pN),(vW),(vN): the water flux splits into k_rw v_w and
//     the capillary-diffusion term, which is not upwinded.
// With p_w as primary pressure, p_n = p_w + p_c at vertices (p_c,i =
// p_dmin,i J(S_e,i)); per face of element e along axis k (edge a->b):
//   T_w = -K_e A_f (G(p_n) - rho_w g_k), T_n = -K_e A_f (G(p_n) - rho_n g_k),
//   T_c = -K_e A_f G(p_c),  G = d/dx_k of the element's Q1 interpolant at x_M,
//   F_w = rho_w (lam_w(S_up) T_w - lam_w(S(x_M)) T_c),
//   F_n = rho_n lam_n(S hat_up) T_n.
//
// K1 runs one thread per vertex: it visits the 2^d elements around its vertex
// and, in each, the d faces that touch it, and accumulates its own block row
// (27 or 9 2x2 blocks) in shared memory; no atomics, no second pass.  The row
// is written once with 1 KB-per-warp coalesced stores.
#include <cstdlib>

#include "rf_common.cuh"
#include "rf_kernels.h"

namespace rf {

struct Phys {
  double rho_w, rho_n, mu_w, mu_n, S_wr, S_nr, lam, den;
  double h[3], g[3];
  int scheme;   // SCHEME_* bits (0: the discretisation of Sec. 3)
};

// ---- constitutive laws (Brooks-Corey; J continued linearly outside [0.01, 1])
__device__ __forceinline__ void leverett_pow(double lam, double S, double& J, double& dJ) {
  if (lam == 2.0) {
    double r = __dsqrt_rn(S);
    J = __ddiv_rn(1.0, r);
    dJ = __ddiv_rn(-0.5, __dmul_rn(S, r));
  } else {
    J = pow(S, -1.0 / lam);
    dJ = (-1.0 / lam) * pow(S, -1.0 / lam - 1.0);
  }
}

// J(S_e) (decides nothing by itself but feeds p_c, p_n and T: exact rounding)
__device__ __forceinline__ void leverett(double lam, double Se, double& J, double& dJ) {
  if (Se < 0.01) {
    double j0, d0;
    leverett_pow(lam, 0.01, j0, d0);
    J = __dadd_rn(j0, __dmul_rn(d0, __dsub_rn(Se, 0.01)));
    dJ = d0;
  } else if (Se > 1.0) {
    const double sl = __ddiv_rn(-1.0, lam);
    J = __dadd_rn(1.0, __dmul_rn(sl, __dsub_rn(Se, 1.0)));
    dJ = sl;
  } else {
    leverett_pow(lam, Se, J, dJ);
  }
}

// k_rw, dk_rw/dS_e (k_r use S_e clamped to [0,1], derivative 0 outside)
__device__ __forceinline__ void krw_of(double lam, double Se, double& k, double& dk) {
  double Sc = fmin(fmax(Se, 0.0), 1.0);
  bool inside = Se > 0.0 && Se < 1.0;
  if (lam == 2.0) {
    double s2 = Sc * Sc;
    k = s2 * s2;
    dk = inside ? 4.0 * s2 * Sc : 0.0;
  } else {
    double ew = (2.0 + 3.0 * lam) / lam;
    k = pow(Sc, ew);
    dk = inside ? ew * pow(Sc, ew - 1.0) : 0.0;
  }
}

__device__ __forceinline__ void krn_of(double lam, double Se, double& k, double& dk) {
  double Sc = fmin(fmax(Se, 0.0), 1.0);
  bool inside = Se > 0.0 && Se < 1.0;
  double om = 1.0 - Sc;
  if (lam == 2.0) {
    double s2 = Sc * Sc;
    k = om * om * (1.0 - s2);
    dk = inside ? (-2.0 * om * (1.0 - s2) - 2.0 * Sc * om * om) : 0.0;
  } else {
    double en = (2.0 + lam) / lam, sa = pow(Sc, en);
    k = om * om * (1.0 - sa);
    dk = inside ? (-2.0 * om * (1.0 - sa) - en * om * om * pow(Sc, en - 1.0)) : 0.0;
  }
}

// Per-medium relative permeabilities (Sec. 6, Case 2: each medium has its own
// polynomial k_rw, k_rn).  law < 0 or a row of kind 0: the Brooks-Corey laws
// above.  Kind 1, row {1, a_w, n_w, a_n, b_n, c_n}: k_rw = a_w S^n_w, k_rn =
// a_n (1 - b_n S)^2 (1 - c_n S^2) while both factors are positive and 0 from
// the first of their roots on, S = S_e clamped to [0, 1], derivatives 0
// outside (0, 1).
__device__ __forceinline__ const double* law_row(const double* tab, int law) {
  return (law < 0 || tab[6 * law] == 0.0) ? nullptr : tab + 6 * law;
}

__device__ __forceinline__ void krw_law(double lam, const double* L, double Se, double& k, double& dk) {
  if (!L) { krw_of(lam, Se, k, dk); return; }
  const double aw = L[1];
  const int nw = (int)L[2];
  const double S = fmin(fmax(Se, 0.0), 1.0);
  double p = 1.0;                     // S^(n_w - 1)
  for (int t = 1; t < nw; ++t) p = p * S;
  k = aw * (p * S);
  dk = (Se > 0.0 && Se < 1.0) ? (aw * nw) * p : 0.0;
}

__device__ __forceinline__ void krn_law(double lam, const double* L, double Se, double& k, double& dk) {
  if (!L) { krn_of(lam, Se, k, dk); return; }
  const double an = L[3], bn = L[4], cn = L[5];
  const double S = fmin(fmax(Se, 0.0), 1.0);
  const double r = 1.0 - bn * S, q = 1.0 - cn * (S * S);
  if (r > 0.0 && q > 0.0) {
    k = an * (r * r) * q;
    dk = (Se > 0.0 && Se < 1.0) ? an * (-2.0 * bn * r * q - 2.0 * cn * S * (r * r)) : 0.0;
  } else {
    k = 0.0;
    dk = 0.0;
  }
}

// Eq. (hSw): S_e hat of vertex i inside an element of entry pressure pdc.
__device__ __forceinline__ void shat_of(double lam, double Se, double pdc, double pdmin, double& s, double& ds) {
  if (pdc == pdmin) { s = Se; ds = 1.0; return; }
  double r = __ddiv_rn(pdc, pdmin);
  double rl = (lam == 2.0) ? __dmul_rn(r, r) : pow(r, lam);
  double t = __dmul_rn(rl, Se);
  if (t >= 1.0) { s = 1.0; ds = 0.0; }
  else { s = t; ds = rl; }
}

// ---------------------------------------------------------------- K0
// p_dmin (Eq. pdmin) and lumped pore volume per vertex, parity-split order.
__global__ void k_vertex_setup(Dims d, const double* __restrict__ pd, const double* __restrict__ phi,
                               double vol, double* __restrict__ pdmin, double* __restrict__ phiv) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= d.nv) return;
  int i, j, k;
  pcoords(d, p, i, j, k);
  const int cx = d.nx - 1, cy = d.ny - 1, cz = d.dim == 3 ? d.nz - 1 : 1;
  const double frac = d.dim == 3 ? 0.125 : 0.25;
  double best = INFINITY, s = 0.0;
  for (int c = 0; c < (1 << d.dim); ++c) {
    int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = d.dim == 3 ? k - ((c >> 2) & 1) : 0;
    if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
    int64_t cell = ci + (int64_t)cx * (cj + (int64_t)cy * ck);
    best = fmin(best, pd[cell]);
    s += phi[cell] * vol * frac;
  }
  pdmin[p] = best;
  phiv[p] = s;
}

// natural <-> parity-split permutation of interleaved pairs / bytes
__global__ void k_perm_to_p(Dims d, const double2* __restrict__ nat, double2* __restrict__ out) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= d.nv) return;
  const uint32_t line = (uint32_t)v / (uint32_t)d.nx;   // nv < 2^31
  const int i = (int)((uint32_t)v - line * (uint32_t)d.nx);
  out[line * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1))] = nat[v];
}

__global__ void k_perm_from_p(Dims d, const double2* __restrict__ pl, double2* __restrict__ nat) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= d.nv) return;
  const uint32_t line = (uint32_t)v / (uint32_t)d.nx;   // nv < 2^31
  const int i = (int)((uint32_t)v - line * (uint32_t)d.nx);
  nat[v] = pl[line * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1))];
}

__global__ void k_perm_bytes_to_p(Dims d, const uint8_t* __restrict__ nat, uint8_t* __restrict__ out) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= d.nv) return;
  const uint32_t line = (uint32_t)v / (uint32_t)d.nx;   // nv < 2^31
  const int i = (int)((uint32_t)v - line * (uint32_t)d.nx);
  out[line * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1))] = nat ? nat[v] : 0;
}

__global__ void k_perm_scalar_to_p(Dims d, const double* __restrict__ nat, double* __restrict__ out) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= d.nv) return;
  const uint32_t line = (uint32_t)v / (uint32_t)d.nx;   // nv < 2^31
  const int i = (int)((uint32_t)v - line * (uint32_t)d.nx);
  out[line * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1))] = nat ? nat[v] : 0.0;
}

// ---------------------------------------------------------------- K1a
// Per-vertex quantities of the state (parity-split order): S_e, p_n = p_w +
// p_c, p_c, dp_c/dS_n, k_rw, dk_rw/dS_n.
__global__ void k_vertex_state(Dims d, Phys ph, const double2* __restrict__ u, const double* __restrict__ pdmin,
                               double* __restrict__ Se, double* __restrict__ pn, double* __restrict__ pc,
                               double* __restrict__ dpc, double* __restrict__ krw, double* __restrict__ dkrw) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= d.nv) return;
  double2 uv = u[p];
  double se = __ddiv_rn(__dsub_rn(__dsub_rn(1.0, uv.y), ph.S_wr), ph.den);
  double J, dJ, k, dk;
  leverett(ph.lam, se, J, dJ);
  krw_of(ph.lam, se, k, dk);
  double pdm = pdmin[p];
  double c = __dmul_rn(pdm, J);
  Se[p] = se;
  pc[p] = c;
  dpc[p] = -(pdm * dJ) / ph.den;
  pn[p] = __dadd_rn(uv.x, c);
  // the upwinded water mobility lambda_w = k_rw / mu_w and its S_n-derivative,
  // divided here once per vertex instead of once per face visit
  krw[p] = k / ph.mu_w;
  dkrw[p] = (-dk / ph.den) / ph.mu_w;
}

// ---------------------------------------------------------------- K1 / K1r
struct AsmIn {
  const double2* u;
  const double *Se, *pn, *pc, *dpc, *krw, *dkrw, *pdmin, *phiv;
  const double *K, *pd, *phi;     // per cell (natural cell order)
  double vol;                     // cell volume
  const uint8_t* dir;             // parity-split
  const double* pw_dir;           // parity-split
  const double2* q_in;            // parity-split (may be null)
  const uint8_t* law;             // per cell k_r law (natural cell order), or null
  const double* kr_tab;           // law table, 6 doubles per law
};

template <int DIM, bool WANT_J>
__global__ void __launch_bounds__(128) k_assemble(Dims d, Phys ph, AsmIn in, double2* __restrict__ F,
                                                  double* __restrict__ J, double2* __restrict__ mdiag) {
  extern __shared__ double acc[];  // [nb*4][blockDim]
  constexpr int NC = 1 << DIM, NE = 1 << (DIM - 1), NB = DIM == 3 ? 27 : 9;
  const int tid = threadIdx.x, BS = blockDim.x;
  int64_t p = blockIdx.x * (int64_t)BS + tid;
  const bool live = p < d.nv;
  if (WANT_J) {
#pragma unroll 4
    for (int t = 0; t < NB * 4; ++t) acc[t * BS + tid] = 0.0;
  }
  if (!live) return;
  int i, j, k;
  pcoords(d, p, i, j, k);
  const int cx = d.nx - 1, cy = d.ny - 1, cz = DIM == 3 ? d.nz - 1 : 1;
  double F0 = 0.0, F1 = 0.0;
  if (in.q_in) { double2 q = in.q_in[p]; F0 = q.x; F1 = q.y; }
  const double neg_inv_den = -1.0 / ph.den;
  const bool darcy = (ph.scheme & SCHEME_DARCY_UPWIND) != 0;
  // d G / d q_q = +-w / h_k takes one of DIM magnitudes per axis (w is a
  // product of DIM-1 factors 3/4 or 1/4): divide once per thread.  gtab[k][m]
  // = w / h_k with m = the number of 1/4 factors; IEEE division is correctly
  // rounded and sign-symmetric, so +-gtab equals the per-corner (+-w) / h_k.
  double gtab[DIM][DIM];
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk)
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      double w = 1.0;
#pragma unroll
      for (int t = 0; t < DIM - 1; ++t) w = w * (t < m ? 0.25 : 0.75);
      gtab[kk][m] = w / ph.h[kk];
    }

#pragma unroll
  for (int c = 0; c < NC; ++c) {
    // element whose corner c (bits: x,y,z offsets) is this vertex
    const int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = DIM == 3 ? k - ((c >> 2) & 1) : 0;
    if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
    const int64_t cell = ci + (int64_t)cx * (cj + (int64_t)cy * ck);
    const double Kc = in.K[cell], pdc = in.pd[cell];
    const double* law = in.law ? law_row(in.kr_tab, in.law[cell]) : nullptr;
    int64_t vq[NC];
    double se[NC], pnq[NC], pcq[NC], dpcq[NC], pwq[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      vq[q] = pidx(d, ci + (q & 1), cj + ((q >> 1) & 1), DIM == 3 ? ck + ((q >> 2) & 1) : 0);
      se[q] = in.Se[vq[q]];
      pnq[q] = in.pn[vq[q]];
      pcq[q] = in.pc[vq[q]];
      dpcq[q] = in.dpc[vq[q]];
      pwq[q] = darcy ? in.u[vq[q]].x : 0.0;
    }
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      // the face of this element along axis kk through this vertex's edge
      int oth[2], no = 0;
#pragma unroll
      for (int m = 0; m < DIM; ++m)
        if (m != kk) oth[no++] = m;
      double Af = 1.0;
#pragma unroll
      for (int t = 0; t < DIM - 1; ++t) Af = __dmul_rn(Af, __dmul_rn(ph.h[oth[t]], 0.5));
      const double KA = __dmul_rn(Kc, Af);
      int o[2] = {0, 0};
#pragma unroll
      for (int t = 0; t < DIM - 1; ++t) o[t] = (c >> oth[t]) & 1;
      const int a = c & ~(1 << kk), b = c | (1 << kk);
      const double sgn = ((c >> kk) & 1) ? 1.0 : -1.0;  // this vertex is b: +flux, a: -flux
      double gpn = 0.0, gpc = 0.0, gpw = 0.0;
#pragma unroll
      for (int e2 = 0; e2 < NE; ++e2) {
        int o2[2] = {e2 & 1, (e2 >> 1) & 1};
        double w = 1.0;
        int a2 = 0;
#pragma unroll
        for (int t = 0; t < DIM - 1; ++t) {
          w = w * (o2[t] == o[t] ? 0.75 : 0.25);
          a2 |= o2[t] << oth[t];
        }
        const int b2 = a2 | (1 << kk);
        gpn = __dadd_rn(gpn, __dmul_rn(w, __dsub_rn(pnq[b2], pnq[a2])));
        gpc = __dadd_rn(gpc, __dmul_rn(w, __dsub_rn(pcq[b2], pcq[a2])));
        if (darcy) gpw = __dadd_rn(gpw, __dmul_rn(w, __dsub_rn(pwq[b2], pwq[a2])));
      }
      gpn = __ddiv_rn(gpn, ph.h[kk]);
      gpc = __ddiv_rn(gpc, ph.h[kk]);
      gpw = __ddiv_rn(gpw, ph.h[kk]);
      double wM[NC], SeM = 0.0;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        double w = 0.5;
#pragma unroll
        for (int t = 0; t < DIM - 1; ++t) w = w * ((((q >> oth[t]) & 1) == o[t]) ? 0.75 : 0.25);
        wM[q] = w;
        SeM = __dadd_rn(SeM, __dmul_rn(w, se[q]));
      }
      const double Tw = __dmul_rn(-KA, __dsub_rn(gpn, __dmul_rn(ph.rho_w, ph.g[kk])));
      const double Tn = __dmul_rn(-KA, __dsub_rn(gpn, __dmul_rn(ph.rho_n, ph.g[kk])));
      const double Tc = __dmul_rn(-KA, gpc);
      // Darcy-velocity upwinding variant: the whole water flux by the sign of
      // T_pw = -K A_f (G(p_w) - rho_w g_k) (= T_w - T_c in exact arithmetic)
      const double Tpw = __dmul_rn(-KA, __dsub_rn(gpw, __dmul_rn(ph.rho_w, ph.g[kk])));
      const bool wa = darcy ? Tpw >= 0.0 : Tw >= 0.0, na = Tn >= 0.0;
      const int64_t vw = wa ? vq[a] : vq[b];
      const int64_t vn = na ? vq[a] : vq[b];
      double lw_up, dlw_up;   // k_rw / mu_w of the upwind vertex (with this element's law) and its S_n-derivative
      if (!law) {
        lw_up = in.krw[vw];
        dlw_up = in.dkrw[vw];
      } else {
        double k, dk;
        krw_law(ph.lam, law, in.Se[vw], k, dk);
        lw_up = k / ph.mu_w;
        dlw_up = (-dk / ph.den) / ph.mu_w;
      }
      double kM, dkM;
      krw_law(ph.lam, law, SeM, kM, dkM);
      const double lwM = kM / ph.mu_w;
      double sh, dsh, kn, dkn;
      shat_of(ph.lam, in.Se[vn], pdc, in.pdmin[vn], sh, dsh);
      krn_law(ph.lam, law, sh, kn, dkn);
      const double ln_up = kn / ph.mu_n;
      const double Fw = darcy ? ph.rho_w * (lw_up * Tpw) : ph.rho_w * (lw_up * Tw - lwM * Tc);
      const double Fn = ph.rho_n * (ln_up * Tn);
      F0 += sgn * Fw;
      F1 += sgn * Fn;
      if (WANT_J) {
        const double dlwM_dSeM = dkM / ph.mu_w;
        const double dln_up = dkn * dsh * neg_inv_den / ph.mu_n;
        const int qw = wa ? a : b, qn = na ? a : b;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          int nq = 0;   // number of 1/4 factors of this corner's weight
#pragma unroll
          for (int t = 0; t < DIM - 1; ++t) nq += (((q >> oth[t]) & 1) == o[t]) ? 0 : 1;
          const double gq = ((q >> kk) & 1) ? gtab[kk][nq] : -gtab[kk][nq];
          const double dT = -KA * gq;
          const double dlwM = wM[q] * dlwM_dSeM * neg_inv_den;
          const double d0 = ph.rho_w * lw_up * dT;
          const double d1 = darcy ? ph.rho_w * (q == qw ? dlw_up * Tpw : 0.0)
                                  : ph.rho_w * ((q == qw ? dlw_up * Tw : 0.0) + lw_up * dT * dpcq[q] - dlwM * Tc -
                                                lwM * dT * dpcq[q]);
          const double d2 = ph.rho_n * ln_up * dT;
          const double d3 = ph.rho_n * ((q == qn ? dln_up * Tn : 0.0) + ln_up * dT * dpcq[q]);
          const int dx = (q & 1) - (c & 1), dy = ((q >> 1) & 1) - ((c >> 1) & 1),
                    dz = DIM == 3 ? ((q >> 2) & 1) - ((c >> 2) & 1) : 0;
          const int bi = blk_of(DIM, dx, dy, dz);
          double* r = acc + (bi * 4) * BS + tid;
          r[0] += sgn * d0;
          r[BS] += sgn * d1;
          r[2 * BS] += sgn * d2;
          r[3 * BS] += sgn * d3;
        }
      }
    }
  }
  const bool dirv = in.dir[p] != 0;
  if (dirv) F0 = in.pw_dir[p] - in.u[p].x;
  F[p] = make_double2(F0, F1);
  if (WANT_J) {
    double pv = in.phiv[p];
    if (ph.scheme & SCHEME_SHAT_STORAGE) {
      // S hat storage: d m_n / d S_n = rho_n sum_j Phi_j |b_i^j| d S hat_e / d S_e
      const double frac = DIM == 3 ? 0.125 : 0.25, se = in.Se[p], pdm = in.pdmin[p];
      pv = 0.0;
      for (int c = 0; c < NC; ++c) {
        const int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = DIM == 3 ? k - ((c >> 2) & 1) : 0;
        if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
        const int64_t cell = ci + (int64_t)cx * (cj + (int64_t)cy * ck);
        double sh, dsh;
        shat_of(ph.lam, se, in.pd[cell], pdm, sh, dsh);
        pv += in.phi[cell] * in.vol * frac * dsh;
      }
    }
    mdiag[p] = make_double2(dirv ? 0.0 : -ph.rho_w * pv, ph.rho_n * pv);
    const int centre = DIM == 3 ? 13 : 4;
#pragma unroll 3
    for (int bi = 0; bi < NB; ++bi) {
      double e0 = acc[(bi * 4 + 0) * BS + tid], e1 = acc[(bi * 4 + 1) * BS + tid];
      double e2 = acc[(bi * 4 + 2) * BS + tid], e3 = acc[(bi * 4 + 3) * BS + tid];
      if (dirv) { e0 = (bi == centre) ? -1.0 : 0.0; e1 = 0.0; }
      double2* dst = reinterpret_cast<double2*>(J + ((int64_t)bi * d.nv + p) * 4);
      dst[0] = make_double2(e0, e1);
      dst[1] = make_double2(e2, e3);
    }
  }
}

// ---------------------------------------------------------------- K1, one thread per element
// Each SCV face is evaluated once, by the thread of its element, and its flux
// and derivatives go to both end vertices (a: -, b: +).  The one-thread-per-
// vertex kernel above evaluates every face twice, once from each end, and K1
// is FP64-pipe-bound on GB300, so this halves most of its FP64 work.
// Elements are processed in 2^DIM colours (parities of their lower corner):
// elements of one colour share no vertex, so each thread owns the rows of its
// corners for the launch and adds into them without atomics, face by face in
// a fixed order (deterministic).  J is zeroed before the first colour; the
// adds go straight to global memory (coalesced across the warp: neighbouring
// threads own neighbouring rows), which keeps the kernel free of shared
// memory and its occupancy at what its registers allow (K1 is FP64-latency-
// bound below ~8 warps per SM).  k_assemble_finish then adds the sources and
// applies the Dirichlet rows and M.  The face arithmetic is
// the vertex kernel's, expression by expression, so every upwind, cap and
// clamp decision and every flux and derivative value are bitwise the same;
// only the order in which a row's contributions are summed differs.
template <int DIM, bool WANT_J>
__global__ void __launch_bounds__(128) k_assemble_cells(Dims d, Phys ph, AsmIn in, int colour, int64_t ncol,
                                                        double2* __restrict__ F, double* __restrict__ J) {
  constexpr int NC = 1 << DIM, NE = 1 << (DIM - 1);
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ncol) return;
  const int cx = d.nx - 1, cy = d.ny - 1;
  const int px = colour & 1, py = (colour >> 1) & 1, pz = (colour >> 2) & 1;
  const int nxp = (cx - px + 1) / 2, nyp = (cy - py + 1) / 2;
  const uint32_t line = (uint32_t)t / (uint32_t)nxp, kl = line / (uint32_t)nyp;   // 32-bit: fewer than 2^31 cells
  const int ci = 2 * (int)((uint32_t)t - line * (uint32_t)nxp) + px;
  const int cj = 2 * (int)(line - kl * (uint32_t)nyp) + py;
  const int ck = DIM == 3 ? 2 * (int)kl + pz : 0;
  const int64_t cell = ci + (int64_t)cx * (cj + (int64_t)cy * ck);
  const double Kc = in.K[cell], pdc = in.pd[cell];
  const double* law = in.law ? law_row(in.kr_tab, in.law[cell]) : nullptr;
  const double neg_inv_den = -1.0 / ph.den;
  const bool darcy = (ph.scheme & SCHEME_DARCY_UPWIND) != 0;
  double gtab[DIM][DIM];   // +-w / h_k by the number of 1/4 factors (see k_assemble)
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk)
#pragma unroll
    for (int m = 0; m < DIM; ++m) {
      double w = 1.0;
#pragma unroll
      for (int tt = 0; tt < DIM - 1; ++tt) w = w * (tt < m ? 0.25 : 0.75);
      gtab[kk][m] = w / ph.h[kk];
    }
  int64_t vq[NC];
  double se[NC], pnq[NC], pcq[NC], dpcq[NC], pwq[NC], Fl[NC][2];
#pragma unroll
  for (int q = 0; q < NC; ++q) {
    vq[q] = pidx(d, ci + (q & 1), cj + ((q >> 1) & 1), DIM == 3 ? ck + ((q >> 2) & 1) : 0);
    se[q] = in.Se[vq[q]];
    pnq[q] = in.pn[vq[q]];
    pcq[q] = in.pc[vq[q]];
    dpcq[q] = in.dpc[vq[q]];
    pwq[q] = darcy ? in.u[vq[q]].x : 0.0;
    Fl[q][0] = 0.0;
    Fl[q][1] = 0.0;
  }
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk) {
    int oth[2], no = 0;
#pragma unroll
    for (int m = 0; m < DIM; ++m)
      if (m != kk) oth[no++] = m;
    double Af = 1.0;
#pragma unroll
    for (int tt = 0; tt < DIM - 1; ++tt) Af = __dmul_rn(Af, __dmul_rn(ph.h[oth[tt]], 0.5));
    const double KA = __dmul_rn(Kc, Af);
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      int o[2] = {0, 0};
#pragma unroll
      for (int tt = 0; tt < DIM - 1; ++tt) o[tt] = (e >> tt) & 1;
      int a = 0;
#pragma unroll
      for (int tt = 0; tt < DIM - 1; ++tt) a |= o[tt] << oth[tt];
      const int b = a | (1 << kk);
      double gpn = 0.0, gpc = 0.0, gpw = 0.0;
#pragma unroll
      for (int e2 = 0; e2 < NE; ++e2) {
        int o2[2] = {e2 & 1, (e2 >> 1) & 1};
        double w = 1.0;
        int a2 = 0;
#pragma unroll
        for (int tt = 0; tt < DIM - 1; ++tt) {
          w = w * (o2[tt] == o[tt] ? 0.75 : 0.25);
          a2 |= o2[tt] << oth[tt];
        }
        const int b2 = a2 | (1 << kk);
        gpn = __dadd_rn(gpn, __dmul_rn(w, __dsub_rn(pnq[b2], pnq[a2])));
        gpc = __dadd_rn(gpc, __dmul_rn(w, __dsub_rn(pcq[b2], pcq[a2])));
        if (darcy) gpw = __dadd_rn(gpw, __dmul_rn(w, __dsub_rn(pwq[b2], pwq[a2])));
      }
      gpn = __ddiv_rn(gpn, ph.h[kk]);
      gpc = __ddiv_rn(gpc, ph.h[kk]);
      gpw = __ddiv_rn(gpw, ph.h[kk]);
      double wM[NC], SeM = 0.0;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        double w = 0.5;
#pragma unroll
        for (int tt = 0; tt < DIM - 1; ++tt) w = w * ((((q >> oth[tt]) & 1) == o[tt]) ? 0.75 : 0.25);
        wM[q] = w;
        SeM = __dadd_rn(SeM, __dmul_rn(w, se[q]));
      }
      const double Tw = __dmul_rn(-KA, __dsub_rn(gpn, __dmul_rn(ph.rho_w, ph.g[kk])));
      const double Tn = __dmul_rn(-KA, __dsub_rn(gpn, __dmul_rn(ph.rho_n, ph.g[kk])));
      const double Tc = __dmul_rn(-KA, gpc);
      const double Tpw = __dmul_rn(-KA, __dsub_rn(gpw, __dmul_rn(ph.rho_w, ph.g[kk])));
      const bool wa = darcy ? Tpw >= 0.0 : Tw >= 0.0, na = Tn >= 0.0;
      const int qw = wa ? a : b, qn = na ? a : b;
      const int64_t vw = wa ? vq[a] : vq[b], vn = na ? vq[a] : vq[b];   // selects, not indexing
      double lw_up, dlw_up;   // k_rw / mu_w of the upwind vertex (with this element's law) and its S_n-derivative
      if (!law) {
        lw_up = in.krw[vw];
        dlw_up = in.dkrw[vw];
      } else {
        double k, dk;
        krw_law(ph.lam, law, wa ? se[a] : se[b], k, dk);
        lw_up = k / ph.mu_w;
        dlw_up = (-dk / ph.den) / ph.mu_w;
      }
      double kM, dkM;
      krw_law(ph.lam, law, SeM, kM, dkM);
      const double lwM = kM / ph.mu_w;
      double sh, dsh, kn, dkn;
      shat_of(ph.lam, na ? se[a] : se[b], pdc, in.pdmin[vn], sh, dsh);
      krn_law(ph.lam, law, sh, kn, dkn);
      const double ln_up = kn / ph.mu_n;
      const double Fw = darcy ? ph.rho_w * (lw_up * Tpw) : ph.rho_w * (lw_up * Tw - lwM * Tc);
      const double Fn = ph.rho_n * (ln_up * Tn);
      Fl[a][0] -= Fw;
      Fl[a][1] -= Fn;
      Fl[b][0] += Fw;
      Fl[b][1] += Fn;
      if (WANT_J) {
        const double dlwM_dSeM = dkM / ph.mu_w;
        const double dln_up = dkn * dsh * neg_inv_den / ph.mu_n;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
          int nq = 0;
#pragma unroll
          for (int tt = 0; tt < DIM - 1; ++tt) nq += (((q >> oth[tt]) & 1) == o[tt]) ? 0 : 1;
          const double gq = ((q >> kk) & 1) ? gtab[kk][nq] : -gtab[kk][nq];
          const double dT = -KA * gq;
          const double dlwM = wM[q] * dlwM_dSeM * neg_inv_den;
          const double d0 = ph.rho_w * lw_up * dT;
          const double d1 = darcy ? ph.rho_w * (q == qw ? dlw_up * Tpw : 0.0)
                                  : ph.rho_w * ((q == qw ? dlw_up * Tw : 0.0) + lw_up * dT * dpcq[q] - dlwM * Tc -
                                                lwM * dT * dpcq[q]);
          const double d2 = ph.rho_n * ln_up * dT;
          const double d3 = ph.rho_n * ((q == qn ? dln_up * Tn : 0.0) + ln_up * dT * dpcq[q]);
          const int bia = blk_of(DIM, (q & 1) - (a & 1), ((q >> 1) & 1) - ((a >> 1) & 1),
                                 DIM == 3 ? ((q >> 2) & 1) - ((a >> 2) & 1) : 0);
          const int bib = blk_of(DIM, (q & 1) - (b & 1), ((q >> 1) & 1) - ((b >> 1) & 1),
                                 DIM == 3 ? ((q >> 2) & 1) - ((b >> 2) & 1) : 0);
          double2* ja = reinterpret_cast<double2*>(J + ((int64_t)bia * d.nv + vq[a]) * 4);
          double2* jb = reinterpret_cast<double2*>(J + ((int64_t)bib * d.nv + vq[b]) * 4);
          double2 a0 = ja[0], a1 = ja[1], b0 = jb[0], b1 = jb[1];
          a0.x -= d0; a0.y -= d1; a1.x -= d2; a1.y -= d3;
          b0.x += d0; b0.y += d1; b1.x += d2; b1.y += d3;
          ja[0] = a0; ja[1] = a1;
          jb[0] = b0; jb[1] = b1;
        }
      }
    }
  }
  // add this element's residual contributions to its corners' rows
#pragma unroll
  for (int r = 0; r < NC; ++r) {
    double2 f = F[vq[r]];
    f.x += Fl[r][0];
    f.y += Fl[r][1];
    F[vq[r]] = f;
  }
}

// After all colours: sources, Dirichlet p_w rows (0 = p_dir - p_w: J row -e,
// M row 0) and the mass diagonal, per vertex.
template <int DIM, bool WANT_J>
__global__ void k_assemble_finish(Dims d, Phys ph, AsmIn in, double2* __restrict__ F, double* __restrict__ J,
                                  double2* __restrict__ mdiag) {
  constexpr int NC = 1 << DIM, NB = DIM == 3 ? 27 : 9;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= d.nv) return;
  double2 f = F[p];
  if (in.q_in) {
    const double2 q = in.q_in[p];
    f.x += q.x;
    f.y += q.y;
  }
  const bool dirv = in.dir[p] != 0;
  if (dirv) f.x = in.pw_dir[p] - in.u[p].x;
  F[p] = f;
  if (!WANT_J) return;
  double pv = in.phiv[p];
  if (ph.scheme & SCHEME_SHAT_STORAGE) {
    int i, j, k;
    pcoords(d, p, i, j, k);
    const int cx = d.nx - 1, cy = d.ny - 1, cz = DIM == 3 ? d.nz - 1 : 1;
    const double frac = DIM == 3 ? 0.125 : 0.25, se = in.Se[p], pdm = in.pdmin[p];
    pv = 0.0;
    for (int c = 0; c < NC; ++c) {
      const int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = DIM == 3 ? k - ((c >> 2) & 1) : 0;
      if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
      const int64_t cell = ci + (int64_t)cx * (cj + (int64_t)cy * ck);
      double sh, dsh;
      shat_of(ph.lam, se, in.pd[cell], pdm, sh, dsh);
      pv += in.phi[cell] * in.vol * frac * dsh;
    }
  }
  mdiag[p] = make_double2(dirv ? 0.0 : -ph.rho_w * pv, ph.rho_n * pv);
  if (dirv) {
    const int centre = DIM == 3 ? 13 : 4;
    for (int bi = 0; bi < NB; ++bi) {
      double2* dst = reinterpret_cast<double2*>(J + ((int64_t)bi * d.nv + p) * 4);
      dst[0] = make_double2(bi == centre ? -1.0 : 0.0, 0.0);
    }
  }
}

// ---------------------------------------------------------------- storage (S hat variant)
// sw[p] = sum over the sub-control volumes b_i^j of vertex p of Phi_j |b_i^j|
// S_w(b_i^j), with S_w = S_wr + S hat_e (1 - S_wr - S_nr) (Eq. (hSw)).
__global__ void k_storage_sw(Dims d, Phys ph, const double2* __restrict__ u, const double* __restrict__ pdmin,
                             const double* __restrict__ phi, const double* __restrict__ pd, double vol,
                             double* __restrict__ sw) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= d.nv) return;
  int i, j, k;
  pcoords(d, p, i, j, k);
  const int cx = d.nx - 1, cy = d.ny - 1, cz = d.dim == 3 ? d.nz - 1 : 1;
  const double frac = d.dim == 3 ? 0.125 : 0.25;
  const double se = __ddiv_rn(__dsub_rn(__dsub_rn(1.0, u[p].y), ph.S_wr), ph.den), pdm = pdmin[p];
  double s = 0.0;
  for (int c = 0; c < (1 << d.dim); ++c) {
    const int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = d.dim == 3 ? k - ((c >> 2) & 1) : 0;
    if (ci < 0 || ci >= cx || cj < 0 || cj >= cy || ck < 0 || ck >= cz) continue;
    const int64_t cell = ci + (int64_t)cx * (cj + (int64_t)cy * ck);
    double sh, dsh;
    shat_of(ph.lam, se, pd[cell], pdm, sh, dsh);
    s += phi[cell] * vol * frac * (ph.S_wr + sh * ph.den);
  }
  sw[p] = s;
}

// ---------------------------------------------------------------- launchers
void launch_vertex_setup(const Dims& d, const double* pd, const double* phi, double vol, double* pdmin,
                         double* phiv, void* s) {
  RF_LAUNCH(k_vertex_setup, (int)((d.nv + 255) / 256), 256, 0, s, d, pd, phi, vol, pdmin, phiv);
}

void launch_perm_to_p(const Dims& d, const double* nat, double* out, void* s) {
  RF_LAUNCH(k_perm_to_p, (int)((d.nv + 255) / 256), 256, 0, s, d, (const double2*)nat, (double2*)out);
}
void launch_perm_from_p(const Dims& d, const double* pl, double* nat, void* s) {
  RF_LAUNCH(k_perm_from_p, (int)((d.nv + 255) / 256), 256, 0, s, d, (const double2*)pl, (double2*)nat);
}
void launch_perm_bytes_to_p(const Dims& d, const uint8_t* nat, uint8_t* out, void* s) {
  RF_LAUNCH(k_perm_bytes_to_p, (int)((d.nv + 255) / 256), 256, 0, s, d, nat, out);
}
void launch_perm_scalar_to_p(const Dims& d, const double* nat, double* out, void* s) {
  RF_LAUNCH(k_perm_scalar_to_p, (int)((d.nv + 255) / 256), 256, 0, s, d, nat, out);
}

template <int DIM, bool WANT_J>
static void cells_t(const Dims& d, const Phys& ph, const AsmIn& in, const AsmArrays& a, void* s) {
  const int BS = 128;
  const int NC = 1 << DIM;
  const size_t smem = 0;
  if (WANT_J) cudaMemsetAsync(a.J, 0, sizeof(double) * 4 * (size_t)d.nb * d.nv, (cudaStream_t)s);
  cudaMemsetAsync(a.F, 0, sizeof(double) * 2 * (size_t)d.nv, (cudaStream_t)s);
  const int cx = d.nx - 1, cy = d.ny - 1, cz = DIM == 3 ? d.nz - 1 : 1;
  for (int c = 0; c < NC; ++c) {
    const int px = c & 1, py = (c >> 1) & 1, pz = (c >> 2) & 1;
    const int64_t ncol = (int64_t)((cx - px + 1) / 2) * ((cy - py + 1) / 2) * (DIM == 3 ? (cz - pz + 1) / 2 : 1);
    if (ncol <= 0) continue;
    RF_LAUNCH((k_assemble_cells<DIM, WANT_J>), (int)((ncol + BS - 1) / BS), BS, smem, s, d, ph, in, c, ncol,
              (double2*)a.F, a.J);
  }
  RF_LAUNCH((k_assemble_finish<DIM, WANT_J>), (int)((d.nv + 255) / 256), 256, 0, s, d, ph, in, (double2*)a.F, a.J,
            (double2*)a.mdiag);
}

static void launch_assemble_cells(const Dims& d, const Phys& ph, const AsmIn& in, const AsmArrays& a, bool want_j,
                                  void* s) {
  if (d.dim == 3) {
    if (want_j) cells_t<3, true>(d, ph, in, a, s);
    else cells_t<3, false>(d, ph, in, a, s);
  } else {
    if (want_j) cells_t<2, true>(d, ph, in, a, s);
    else cells_t<2, false>(d, ph, in, a, s);
  }
}

cudaError_t launch_assemble(const Dims& d, const PhysParams& pp, const AsmArrays& a, bool want_j, void* s) {
  Phys ph;
  ph.rho_w = pp.rho_w; ph.rho_n = pp.rho_n; ph.mu_w = pp.mu_w; ph.mu_n = pp.mu_n;
  ph.S_wr = pp.S_wr; ph.S_nr = pp.S_nr; ph.lam = pp.lambda;
  ph.den = 1.0 - pp.S_wr - pp.S_nr;
  ph.scheme = pp.scheme;
  for (int t = 0; t < 3; ++t) { ph.h[t] = pp.h[t]; ph.g[t] = pp.g[t]; }
  const int nblk = (int)((d.nv + 255) / 256);
  RF_LAUNCH(k_vertex_state, nblk, 256, 0, s, d, ph, (const double2*)a.u, a.pdmin, a.Se, a.pn, a.pc, a.dpc,
            a.krw, a.dkrw);
  AsmIn in;
  in.u = (const double2*)a.u; in.Se = a.Se; in.pn = a.pn; in.pc = a.pc; in.dpc = a.dpc; in.krw = a.krw;
  in.dkrw = a.dkrw; in.pdmin = a.pdmin; in.phiv = a.phiv; in.K = a.K; in.pd = a.pd; in.phi = a.phi;
  in.vol = a.vol; in.dir = a.dir;
  in.pw_dir = a.pw_dir; in.q_in = (const double2*)a.q_in;
  in.law = a.law; in.kr_tab = a.kr_tab;
  const char* pv = getenv("RF_ASM_VERTEX");   // read per assembly (an alternative kept for comparison)
  const bool per_vertex = pv && atoi(pv) != 0;
  if (!per_vertex) {
    launch_assemble_cells(d, ph, in, a, want_j, s);
    return cudaGetLastError();
  }
  const int BS = 128;
  const int grid = (int)((d.nv + BS - 1) / BS);
  const int nb = d.dim == 3 ? 27 : 9;
  size_t smem = want_j ? (size_t)nb * 4 * BS * sizeof(double) : 0;
  if (d.dim == 3) {
    if (want_j) {
      cudaFuncSetAttribute(k_assemble<3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      RF_LAUNCH((k_assemble<3, true>), grid, BS, smem, s, d, ph, in, (double2*)a.F, a.J, (double2*)a.mdiag);
    } else {
      RF_LAUNCH((k_assemble<3, false>), grid, BS, 0, s, d, ph, in, (double2*)a.F, a.J, (double2*)a.mdiag);
    }
  } else {
    if (want_j) {
      cudaFuncSetAttribute(k_assemble<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      RF_LAUNCH((k_assemble<2, true>), grid, BS, smem, s, d, ph, in, (double2*)a.F, a.J, (double2*)a.mdiag);
    } else {
      RF_LAUNCH((k_assemble<2, false>), grid, BS, 0, s, d, ph, in, (double2*)a.F, a.J, (double2*)a.mdiag);
    }
  }
  return cudaGetLastError();
}

void launch_storage_sw(const Dims& d, const PhysParams& pp, const double* u, const double* pdmin,
                       const double* phi, const double* pd, double vol, double* sw, void* s) {
  Phys ph;
  ph.rho_w = pp.rho_w; ph.rho_n = pp.rho_n; ph.mu_w = pp.mu_w; ph.mu_n = pp.mu_n;
  ph.S_wr = pp.S_wr; ph.S_nr = pp.S_nr; ph.lam = pp.lambda;
  ph.den = 1.0 - pp.S_wr - pp.S_nr;
  ph.scheme = pp.scheme;
  for (int t = 0; t < 3; ++t) { ph.h[t] = pp.h[t]; ph.g[t] = pp.g[t]; }
  RF_LAUNCH(k_storage_sw, (int)((d.nv + 255) / 256), 256, 0, s, d, ph, (const double2*)u, pdmin, phi, pd, vol, sw);
}

}  // namespace rf
