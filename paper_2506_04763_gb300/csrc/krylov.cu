// krylov.cu — the outer FP64 iteration of the stage solve and the LIMEX
// vector work.
//
// BiCGSTAB (van der Vorst), right-preconditioned by one multigrid V-cycle per
// application (the paper's Sec. 5 solver: "GMG preconditioned BiCGSTAB").
// One iteration is five fused FP64 vector kernels around the two V-cycles:
//   p = r + beta (p - omega v)        (+ cast of p to the preconditioner type)
//   v = A y, <r^, v>                  (outer operator A = shift M - J, FP64)
//   s = r - alpha v                   (+ cast of s)
//   t = A z, <t, s>, <t, t>
//   x += alpha y + omega z, r = s - omega t, |r|^2, <r^, r>
// Dot products are reduced deterministically: per-block partial sums (warp
// shuffles), then one single-block kernel adds the partials in block order and
// updates the scalars (alpha, omega, beta, rho) that stay in device memory.
// The preconditioned vectors y, z are the V-cycle outputs; in the FP32 modes
// they are FP32 and are read as such by the outer FP64 operator (exact
// conversion), halving their traffic.
#include "rf_common.cuh"
#include "rf_kernels.h"

namespace rf {

// scalar slots (double)
enum {
  S_RHO = 0, S_RHO_OLD, S_ALPHA, S_OMEGA, S_BETA, S_RR, S_BB, S_RHV, S_TS, S_TT,
  S_CONV, S_BAD, S_TRUE_RR, S_BREAK, S_RTOL, S_NSLOTS
};
static_assert(S_NSLOTS <= RF_SCAL_DONE, "the batch flag slot follows the scalars");
static constexpr int MAXB = 2048;   // max blocks of a reducing kernel
static constexpr int BS = 256;

int krylov_blocks(int64_t nv) {
  int64_t b = (nv + BS - 1) / BS;
  int64_t cap = (int64_t)num_sms() * 8;
  if (cap > MAXB) cap = MAXB;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* partial) {
  __shared__ double sh[NS][BS / 32];
#pragma unroll
  for (int q = 0; q < NS; ++q)
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_xor_sync(0xffffffffu, v[q], o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0)
#pragma unroll
    for (int q = 0; q < NS; ++q) sh[q][w] = v[q];
  __syncthreads();
  if (threadIdx.x < 32) {
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      double t = (l < BS / 32) ? sh[q][l] : 0.0;
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (l == 0) partial[q * MAXB + blockIdx.x] = t;
    }
  }
}

// sum partials of slots [0, ns) in fixed block order (one warp)
__device__ __forceinline__ double sum_partials(const double* partial, int slot, int nblk) {
  const int l = threadIdx.x & 31;
  double t = 0.0;
  for (int b = l; b < nblk; b += 32) t += partial[slot * MAXB + b];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  return t;
}

// ----------------------------------------------------------------- outer operator
template <typename XV, int NB>
__device__ __forceinline__ void spmv64_row(const Dims& d, const Nbr& nb, const double* __restrict__ J,
                                           const double2* __restrict__ md, double shift,
                                           const XV* __restrict__ x, int64_t p, double& y0, double& y1) {
  const int par = (int)((uint32_t)p % (uint32_t)d.nx) >= d.E;   // nv < 2^31
  double s0 = 0.0, s1 = 0.0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const double2* q = reinterpret_cast<const double2*>(J) + ((int64_t)b * d.nv + p) * 2;
    double2 a01 = __ldcs(q), a23 = __ldcs(q + 1);
    const XV xv = x[p + (par ? nb.off[1][b] : nb.off[0][b])];
    const double x0 = (double)xv.x, x1 = (double)xv.y;
    s0 = fma(a01.x, x0, s0);
    s0 = fma(a01.y, x1, s0);
    s1 = fma(a23.x, x0, s1);
    s1 = fma(a23.y, x1, s1);
  }
  const double2 m = md[p];
  const double xs = (double)x[p].y;
  y0 = shift * m.x * xs - s0;
  y1 = shift * m.y * xs - s1;
}

// Double-FP32 variant of the row product for an operand x that is exactly
// representable in FP32 (the FP32 preconditioner's output).  J is stored as
// FP32 pairs hi + lo with hi = fl32(a), lo = fl32(a - hi), |a - hi - lo| <=
// 2^-48 |a|.  hi*x is made exact with an FMA (p + e), lo*x is rounded (error
// <= 2^-48 |a x|), and the sum runs in a (sh, sl) pair with Knuth's two-sum.
// Every operation runs on the FP32 pipe; only the final combination is FP64.
__device__ __forceinline__ void df_acc(float& sh, float& sl, float hi, float lo, float x) {
  const float p = hi * x;
  const float e = fmaf(hi, x, -p);
  const float q = lo * x;
  const float s = sh + p;
  const float bp = s - sh;
  const float err = (sh - (s - bp)) + (p - bp);
  sh = s;
  sl += err + (e + q);
}

template <int NB>
__device__ __forceinline__ void spmvdf_row(const Dims& d, const Nbr& nb, const float4* __restrict__ Jdf,
                                           const double2* __restrict__ md, double shift,
                                           const float2* __restrict__ x, int64_t p, double& y0, double& y1) {
  const int par = (int)((uint32_t)p % (uint32_t)d.nx) >= d.E;   // nv < 2^31
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const float4* q = Jdf + ((int64_t)b * d.nv + p) * 2;
    const float4 hi = __ldcs(q), lo = __ldcs(q + 1);
    const float2 xv = x[p + (par ? nb.off[1][b] : nb.off[0][b])];
    df_acc(h0, l0, hi.x, lo.x, xv.x);
    df_acc(h0, l0, hi.y, lo.y, xv.y);
    df_acc(h1, l1, hi.z, lo.z, xv.x);
    df_acc(h1, l1, hi.w, lo.w, xv.y);
  }
  const double2 m = md[p];
  const double xs = (double)x[p].y;
  y0 = shift * m.x * xs - ((double)h0 + (double)l0);
  y1 = shift * m.y * xs - ((double)h1 + (double)l1);
}

template <int NB>
__global__ void __launch_bounds__(BS) k_bicg_v_df(Dims d, Nbr nb, const float4* __restrict__ Jdf,
                                                  const double2* __restrict__ md, double shift,
                                                  const float2* __restrict__ y, const double2* __restrict__ rh,
                                                  double2* __restrict__ v, double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[1] = {0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmvdf_row<NB>(d, nb, Jdf, md, shift, y, p, y0, y1);
    v[p] = make_double2(y0, y1);
    const double2 r = rh[p];
    acc[0] += r.x * y0 + r.y * y1;
  }
  block_reduce_store<1>(acc, partial + S_RHV * MAXB);
}

template <int NB>
__global__ void __launch_bounds__(BS) k_bicg_t_df(Dims d, Nbr nb, const float4* __restrict__ Jdf,
                                                  const double2* __restrict__ md, double shift,
                                                  const float2* __restrict__ z, const double2* __restrict__ s,
                                                  double2* __restrict__ t, double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[2] = {0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmvdf_row<NB>(d, nb, Jdf, md, shift, z, p, y0, y1);
    t[p] = make_double2(y0, y1);
    const double2 sv = s[p];
    acc[0] += y0 * sv.x + y1 * sv.y;
    acc[1] += y0 * y0 + y1 * y1;
  }
  block_reduce_store<2>(acc, partial + S_TS * MAXB);
}

// split J (FP64) into hi/lo FP32 pairs, layout [b][p][hi4, lo4]
__global__ void k_split_df(int64_t nblocks, const double4_16a* __restrict__ J, float4* __restrict__ Jdf) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nblocks; q += (int64_t)gridDim.x * blockDim.x) {
    const double4_16a a = J[q];
    const float h0 = (float)a.x, h1 = (float)a.y, h2 = (float)a.z, h3 = (float)a.w;
    Jdf[2 * q] = make_float4(h0, h1, h2, h3);
    Jdf[2 * q + 1] = make_float4((float)(a.x - (double)h0), (float)(a.y - (double)h1), (float)(a.z - (double)h2),
                                 (float)(a.w - (double)h3));
  }
}

template <typename XV, int NB>
__global__ void __launch_bounds__(BS) k_spmv64(Dims d, Nbr nb, const double* __restrict__ J,
                                               const double2* __restrict__ md, double shift,
                                               const XV* __restrict__ x, double2* __restrict__ y) {
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmv64_row<XV, NB>(d, nb, J, md, shift, x, p, y0, y1);
    y[p] = make_double2(y0, y1);
  }
}

// v = A y, partial <rh, v>
template <typename XV, int NB>
__global__ void __launch_bounds__(BS) k_bicg_v(Dims d, Nbr nb, const double* __restrict__ J,
                                               const double2* __restrict__ md, double shift,
                                               const XV* __restrict__ y, const double2* __restrict__ rh,
                                               double2* __restrict__ v, double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[1] = {0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmv64_row<XV, NB>(d, nb, J, md, shift, y, p, y0, y1);
    v[p] = make_double2(y0, y1);
    const double2 r = rh[p];
    acc[0] += r.x * y0 + r.y * y1;
  }
  block_reduce_store<1>(acc, partial + S_RHV * MAXB);
}

// t = A z, partials <t, s>, <t, t>
template <typename XV, int NB>
__global__ void __launch_bounds__(BS) k_bicg_t(Dims d, Nbr nb, const double* __restrict__ J,
                                               const double2* __restrict__ md, double shift,
                                               const XV* __restrict__ z, const double2* __restrict__ s,
                                               double2* __restrict__ t, double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[2] = {0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmv64_row<XV, NB>(d, nb, J, md, shift, z, p, y0, y1);
    t[p] = make_double2(y0, y1);
    const double2 sv = s[p];
    acc[0] += y0 * sv.x + y1 * sv.y;
    acc[1] += y0 * y0 + y1 * y1;
  }
  block_reduce_store<2>(acc, partial + S_TS * MAXB);
}

// true residual rt = b - A x (x FP64), |rt|^2 ; rt written into r
template <int NB>
__global__ void __launch_bounds__(BS) k_true_res(Dims d, Nbr nb, const double* __restrict__ J,
                                                 const double2* __restrict__ md, double shift,
                                                 const double2* __restrict__ x, const double2* __restrict__ b,
                                                 double2* __restrict__ r, double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[1] = {0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmv64_row<double2, NB>(d, nb, J, md, shift, x, p, y0, y1);
    const double2 bv = b[p];
    const double r0 = bv.x - y0, r1 = bv.y - y1;
    r[p] = make_double2(r0, r1);
    acc[0] += r0 * r0 + r1 * r1;
  }
  block_reduce_store<1>(acc, partial + S_TRUE_RR * MAXB);
}

// ----------------------------------------------------------------- vector kernels
template <typename LV>
__device__ __forceinline__ LV to_lo(double a, double b);
template <> __device__ __forceinline__ float2 to_lo<float2>(double a, double b) { return make_float2((float)a, (float)b); }
template <> __device__ __forceinline__ double2 to_lo<double2>(double a, double b) { return make_double2(a, b); }

// r = b, rh = b, x = 0, p = v = 0; partial |b|^2
__global__ void __launch_bounds__(BS) k_bicg_init(int64_t nv, const double2* __restrict__ b, double2* __restrict__ x,
                                                  double2* __restrict__ r, double2* __restrict__ rh,
                                                  double2* __restrict__ p, double2* __restrict__ v,
                                                  double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[1] = {0.0};
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 bv = b[q];
    r[q] = bv; rh[q] = bv;
    x[q] = make_double2(0.0, 0.0);
    p[q] = make_double2(0.0, 0.0);
    v[q] = make_double2(0.0, 0.0);
    acc[0] += bv.x * bv.x + bv.y * bv.y;
  }
  block_reduce_store<1>(acc, partial + S_BB * MAXB);
}

// restart from the true residual kept in r: rh = r, p = v = 0; partial |r|^2
__global__ void __launch_bounds__(BS) k_bicg_restart(int64_t nv, const double2* __restrict__ r,
                                                     double2* __restrict__ rh, double2* __restrict__ p,
                                                     double2* __restrict__ v, double* __restrict__ partial) {
  rf_pdl_begin();
  double acc[1] = {0.0};
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 rv = r[q];
    rh[q] = rv;
    p[q] = make_double2(0.0, 0.0);
    v[q] = make_double2(0.0, 0.0);
    acc[0] += rv.x * rv.x + rv.y * rv.y;
  }
  block_reduce_store<1>(acc, partial + S_RR * MAXB);
}

template <typename LV>
__global__ void __launch_bounds__(BS) k_bicg_p(int64_t nv, const double* __restrict__ scal,
                                               const double2* __restrict__ r, const double2* __restrict__ v,
                                               double2* __restrict__ p, LV* __restrict__ plo) {
  rf_pdl_begin();
  const double beta = scal[S_BETA], omega = scal[S_OMEGA];
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 rv = r[q], vv = v[q], pv = p[q];
    const double p0 = rv.x + beta * (pv.x - omega * vv.x);
    const double p1 = rv.y + beta * (pv.y - omega * vv.y);
    p[q] = make_double2(p0, p1);
    plo[q] = to_lo<LV>(p0, p1);
  }
}

template <typename LV>
__global__ void __launch_bounds__(BS) k_bicg_s(int64_t nv, const double* __restrict__ scal,
                                               const double2* __restrict__ r, const double2* __restrict__ v,
                                               double2* __restrict__ s, LV* __restrict__ slo) {
  rf_pdl_begin();
  const double alpha = scal[S_ALPHA];
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 rv = r[q], vv = v[q];
    const double s0 = rv.x - alpha * vv.x, s1 = rv.y - alpha * vv.y;
    s[q] = make_double2(s0, s1);
    slo[q] = to_lo<LV>(s0, s1);
  }
}

template <typename YV>
__global__ void __launch_bounds__(BS) k_bicg_xr(int64_t nv, const double* __restrict__ scal,
                                                const YV* __restrict__ y, const YV* __restrict__ z,
                                                const double2* __restrict__ s, const double2* __restrict__ t,
                                                const double2* __restrict__ rh, double2* __restrict__ x,
                                                double2* __restrict__ r, double* __restrict__ partial) {
  rf_pdl_begin();
  const double alpha = scal[S_ALPHA], omega = scal[S_OMEGA];
  double acc[2] = {0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const YV yv = y[q], zv = z[q];
    const double2 sv = s[q], tv = t[q], hv = rh[q];
    double2 xv = x[q];
    xv.x += alpha * (double)yv.x + omega * (double)zv.x;
    xv.y += alpha * (double)yv.y + omega * (double)zv.y;
    x[q] = xv;
    const double r0 = sv.x - omega * tv.x, r1 = sv.y - omega * tv.y;
    r[q] = make_double2(r0, r1);
    acc[0] += r0 * r0 + r1 * r1;
    acc[1] += hv.x * r0 + hv.y * r1;
  }
  block_reduce_store<2>(acc, partial + S_RR * MAXB);
}
static_assert(S_RR + 1 == S_BB, "slots");  // k_bicg_xr writes (rr, <rh,r>) into slots S_RR and S_RR+1

// ----------------------------------------------------------------- finalize
// stage: 0 init, 1 alpha, 2 omega, 3 x/r update, 4 true residual, 5 restart
__device__ __forceinline__ void finalize_body(int stage, int nblk, double* __restrict__ scal,
                                              const double* __restrict__ partial, double rtol) {
  if (threadIdx.x >= 32) return;
  if (stage == 0) {
    const double bb = sum_partials(partial, S_BB, nblk);
    if (threadIdx.x == 0) {
      scal[S_BB] = bb; scal[S_RR] = bb; scal[S_RHO] = bb; scal[S_RHO_OLD] = 1.0;
      scal[S_ALPHA] = 1.0; scal[S_OMEGA] = 1.0; scal[S_BETA] = 0.0;
      scal[S_CONV] = (bb == 0.0) ? 1.0 : 0.0; scal[S_BAD] = isfinite(bb) ? 0.0 : 1.0; scal[S_BREAK] = 0.0;
      scal[S_RTOL] = rtol;
      scal[RF_SCAL_DONE] = 0.0;
    }
  } else if (stage == 1) {
    const double rhv = sum_partials(partial, S_RHV, nblk);
    if (threadIdx.x == 0) {
      scal[S_RHV] = rhv;
      double a = scal[S_RHO] / rhv;
      // <r_hat, v> = 0: no BiCG half step.  alpha = 0 keeps x and r finite
      // (the iteration finishes as a minimal-residual step along z), and the
      // flag sends the host to the true-residual check and a restart.
      if (!isfinite(a)) { scal[S_BREAK] = 1.0; a = 0.0; }
      scal[S_ALPHA] = a;
    }
  } else if (stage == 2) {
    const double ts = sum_partials(partial, S_TS, nblk);
    const double tt = sum_partials(partial, S_TT, nblk);
    if (threadIdx.x == 0) {
      scal[S_TS] = ts; scal[S_TT] = tt;
      const double w = tt > 0.0 ? ts / tt : 0.0;
      scal[S_OMEGA] = w;
      if (!(w != 0.0) || !isfinite(w)) scal[S_BREAK] = 1.0;
    }
  } else if (stage == 3) {
    const double rr = sum_partials(partial, S_RR, nblk);
    const double rhr = sum_partials(partial, S_RR + 1, nblk);
    if (threadIdx.x == 0) {
      const double rho = scal[S_RHO];
      scal[S_RR] = rr;
      scal[S_BETA] = (rhr / rho) * (scal[S_ALPHA] / scal[S_OMEGA]);
      scal[S_RHO_OLD] = rho;
      scal[S_RHO] = rhr;
      scal[S_CONV] = (sqrt(rr) <= scal[S_RTOL] * sqrt(scal[S_BB])) ? 1.0 : 0.0;
      if (!isfinite(rr)) scal[S_BAD] = 1.0;
      if (!(rhr != 0.0) || !isfinite(scal[S_BETA])) scal[S_BREAK] = 1.0;
    }
  } else if (stage == 4) {
    const double rr = sum_partials(partial, S_TRUE_RR, nblk);
    if (threadIdx.x == 0) scal[S_TRUE_RR] = rr;
  } else if (stage == 5) {
    const double rr = sum_partials(partial, S_RR, nblk);
    if (threadIdx.x == 0) {
      scal[S_RR] = rr; scal[S_RHO] = rr; scal[S_RHO_OLD] = 1.0;
      scal[S_ALPHA] = 1.0; scal[S_OMEGA] = 1.0; scal[S_BETA] = 0.0;
      scal[S_CONV] = 0.0; scal[S_BREAK] = 0.0;
    }
  }
}

__global__ void k_finalize(int stage, int nblk, double* __restrict__ scal, const double* __restrict__ partial,
                           double rtol) {
  rf_pdl_begin();
  finalize_body(stage, nblk, scal, partial, rtol);
}

// ----------------------------------------------------------------- launchers
static inline void fin(int stage, int nblk, KrylovVecs& K, double rtol, void* s) {
  RF_LAUNCH_PDL(k_finalize, 1, 32, 0, s, stage, nblk, K.scal, K.partial, rtol);
}

void launch_spmv64(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                   const void* x, bool x_is_f32, double2* y, void* s) {
  const int g = krylov_blocks(d.nv);
  const double2* md = (const double2*)mdiag;
  if (d.nb == 27) {
    if (x_is_f32) RF_LAUNCH((k_spmv64<float2, 27>), g, BS, 0, s, d, nb, J, md, shift, (const float2*)x, y);
    else RF_LAUNCH((k_spmv64<double2, 27>), g, BS, 0, s, d, nb, J, md, shift, (const double2*)x, y);
  } else {
    if (x_is_f32) RF_LAUNCH((k_spmv64<float2, 9>), g, BS, 0, s, d, nb, J, md, shift, (const float2*)x, y);
    else RF_LAUNCH((k_spmv64<double2, 9>), g, BS, 0, s, d, nb, J, md, shift, (const double2*)x, y);
  }
}

void launch_bicg_init(int64_t nv, const double2* b, KrylovVecs& K, double rtol, void* s) {
  const int g = krylov_blocks(nv);
  RF_LAUNCH_PDL(k_bicg_init, g, BS, 0, s, nv, b, K.x, K.r, K.rh, K.p, K.v, K.partial);
  fin(0, g, K, rtol, s);
}

void launch_bicg_p(int64_t nv, KrylovVecs& K, bool lo_is_f32, bool /*first*/, void* s) {
  const int g = krylov_blocks(nv);
  if (lo_is_f32) RF_LAUNCH_PDL(k_bicg_p<float2>, g, BS, 0, s, nv, K.scal, K.r, K.v, K.p, (float2*)K.p_lo);
  else RF_LAUNCH_PDL(k_bicg_p<double2>, g, BS, 0, s, nv, K.scal, K.r, K.v, K.p, (double2*)K.p_lo);
}

// The operand is the FP64 copy y64 of the preconditioned vector: converting
// FP32 neighbours inside the row loop would cost one FP64-pipe instruction per
// use, as much as the FMA itself on this GPU.
void launch_bicg_v(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                   KrylovVecs& K, bool /*y_is_f32*/, void* s) {
  const int g = krylov_blocks(d.nv);
  const double2* md = (const double2*)mdiag;
  if (d.nb == 27) RF_LAUNCH_PDL((k_bicg_v<double2, 27>), g, BS, 0, s, d, nb, J, md, shift, (const double2*)K.y64, K.rh, K.v, K.partial);
  else RF_LAUNCH_PDL((k_bicg_v<double2, 9>), g, BS, 0, s, d, nb, J, md, shift, (const double2*)K.y64, K.rh, K.v, K.partial);
  fin(1, g, K, 0.0, s);
}

void launch_split_df(const Dims& d, const double* J, float* Jdf, void* s) {
  const int64_t nblocks = (int64_t)d.nb * d.nv;
  RF_LAUNCH(k_split_df, grid_for(nblocks, 256), 256, 0, s, nblocks, (const double4_16a*)J, (float4*)Jdf);
}

void launch_bicg_v_df(const Dims& d, const Nbr& nb, const float* Jdf, const double* mdiag, double shift,
                      KrylovVecs& K, void* s) {
  const int g = krylov_blocks(d.nv);
  const double2* md = (const double2*)mdiag;
  if (d.nb == 27) RF_LAUNCH_PDL(k_bicg_v_df<27>, g, BS, 0, s, d, nb, (const float4*)Jdf, md, shift, (const float2*)K.y, K.rh, K.v, K.partial);
  else RF_LAUNCH_PDL(k_bicg_v_df<9>, g, BS, 0, s, d, nb, (const float4*)Jdf, md, shift, (const float2*)K.y, K.rh, K.v, K.partial);
  fin(1, g, K, 0.0, s);
}

void launch_bicg_t_df(const Dims& d, const Nbr& nb, const float* Jdf, const double* mdiag, double shift,
                      KrylovVecs& K, void* s) {
  const int g = krylov_blocks(d.nv);
  const double2* md = (const double2*)mdiag;
  if (d.nb == 27) RF_LAUNCH_PDL(k_bicg_t_df<27>, g, BS, 0, s, d, nb, (const float4*)Jdf, md, shift, (const float2*)K.z, K.s, K.t, K.partial);
  else RF_LAUNCH_PDL(k_bicg_t_df<9>, g, BS, 0, s, d, nb, (const float4*)Jdf, md, shift, (const float2*)K.z, K.s, K.t, K.partial);
  fin(2, g, K, 0.0, s);
}

void launch_bicg_s(int64_t nv, KrylovVecs& K, bool lo_is_f32, void* s) {
  const int g = krylov_blocks(nv);
  if (lo_is_f32) RF_LAUNCH_PDL(k_bicg_s<float2>, g, BS, 0, s, nv, K.scal, K.r, K.v, K.s, (float2*)K.s_lo);
  else RF_LAUNCH_PDL(k_bicg_s<double2>, g, BS, 0, s, nv, K.scal, K.r, K.v, K.s, (double2*)K.s_lo);
}

void launch_bicg_t(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                   KrylovVecs& K, bool /*z_is_f32*/, void* s) {
  const int g = krylov_blocks(d.nv);
  const double2* md = (const double2*)mdiag;
  if (d.nb == 27) RF_LAUNCH_PDL((k_bicg_t<double2, 27>), g, BS, 0, s, d, nb, J, md, shift, (const double2*)K.z64, K.s, K.t, K.partial);
  else RF_LAUNCH_PDL((k_bicg_t<double2, 9>), g, BS, 0, s, d, nb, J, md, shift, (const double2*)K.z64, K.s, K.t, K.partial);
  fin(2, g, K, 0.0, s);
}

void launch_bicg_xr(int64_t nv, KrylovVecs& K, bool yz_is_f32, void* s) {
  const int g = krylov_blocks(nv);
  if (yz_is_f32)
    RF_LAUNCH_PDL(k_bicg_xr<float2>, g, BS, 0, s, nv, K.scal, (const float2*)K.y, (const float2*)K.z, K.s, K.t, K.rh, K.x, K.r, K.partial);
  else
    RF_LAUNCH_PDL(k_bicg_xr<double2>, g, BS, 0, s, nv, K.scal, (const double2*)K.y, (const double2*)K.z, K.s, K.t, K.rh, K.x, K.r, K.partial);
  fin(3, g, K, 0.0, s);
}

void launch_true_residual(const Dims& d, const Nbr& nb, const double* J, const double* mdiag, double shift,
                          const double2* b, KrylovVecs& K, void* s) {
  const int g = krylov_blocks(d.nv);
  const double2* md = (const double2*)mdiag;
  if (d.nb == 27) RF_LAUNCH_PDL(k_true_res<27>, g, BS, 0, s, d, nb, J, md, shift, K.x, b, K.r, K.partial);
  else RF_LAUNCH_PDL(k_true_res<9>, g, BS, 0, s, d, nb, J, md, shift, K.x, b, K.r, K.partial);
  fin(4, g, K, 0.0, s);
}

void launch_restart(int64_t nv, KrylovVecs& K, void* s) {
  const int g = krylov_blocks(nv);
  RF_LAUNCH_PDL(k_bicg_restart, g, BS, 0, s, nv, K.r, K.rh, K.p, K.v, K.partial);
  fin(5, g, K, 0.0, s);
}

__global__ void k_axpy_pairs(int64_t nv, double2* __restrict__ u, const double2* __restrict__ du) {
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    double2 a = u[q];
    const double2 b = du[q];
    a.x += b.x;
    a.y += b.y;
    u[q] = a;
  }
}
void launch_axpy_pairs(int64_t nv, double2* u, const double2* du, void* s) {
  RF_LAUNCH(k_axpy_pairs, krylov_blocks(nv), BS, 0, s, nv, u, du);
}

// ----------------------------------------------------------------- batched iteration
// The vector kernels and the outer operator of a BiCGSTAB iteration for the
// systems of a KBatch, one system per blockIdx.y (the finalisation: one block
// per system).  Each system runs the single-system kernel's loop over the same
// grid-x extent, so its values and its block partials, hence its reduced
// scalars, are bit for bit those of its own launches.  Finished systems
// (RF_SCAL_DONE) return at once.
__device__ __forceinline__ bool kdone(const SysKrylov& P) { return P.K.scal[RF_SCAL_DONE] != 0.0; }

template <typename LV>
__global__ void __launch_bounds__(BS) k_bicg_p_b(int64_t nv, const __grid_constant__ KBatch B) {
  rf_pdl_begin();
  const SysKrylov& P = B.s[blockIdx.y];
  if (kdone(P)) return;
  const double beta = P.K.scal[S_BETA], omega = P.K.scal[S_OMEGA];
  const double2* __restrict__ r = P.K.r;
  const double2* __restrict__ v = P.K.v;
  double2* __restrict__ pp = P.K.p;
  LV* __restrict__ plo = (LV*)P.K.p_lo;
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 rv = r[q], vv = v[q], pv = pp[q];
    const double p0 = rv.x + beta * (pv.x - omega * vv.x);
    const double p1 = rv.y + beta * (pv.y - omega * vv.y);
    pp[q] = make_double2(p0, p1);
    plo[q] = to_lo<LV>(p0, p1);
  }
}

template <typename LV>
__global__ void __launch_bounds__(BS) k_bicg_s_b(int64_t nv, const __grid_constant__ KBatch B) {
  rf_pdl_begin();
  const SysKrylov& P = B.s[blockIdx.y];
  if (kdone(P)) return;
  const double alpha = P.K.scal[S_ALPHA];
  const double2* __restrict__ r = P.K.r;
  const double2* __restrict__ v = P.K.v;
  double2* __restrict__ sv_out = P.K.s;
  LV* __restrict__ slo = (LV*)P.K.s_lo;
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 rv = r[q], vv = v[q];
    const double s0 = rv.x - alpha * vv.x, s1 = rv.y - alpha * vv.y;
    sv_out[q] = make_double2(s0, s1);
    slo[q] = to_lo<LV>(s0, s1);
  }
}

template <typename YV>
__global__ void __launch_bounds__(BS) k_bicg_xr_b(int64_t nv, const __grid_constant__ KBatch B) {
  rf_pdl_begin();
  const SysKrylov& P = B.s[blockIdx.y];
  if (kdone(P)) return;
  const double alpha = P.K.scal[S_ALPHA], omega = P.K.scal[S_OMEGA];
  const YV* __restrict__ y = (const YV*)P.K.y;
  const YV* __restrict__ z = (const YV*)P.K.z;
  const double2* __restrict__ s = P.K.s;
  const double2* __restrict__ t = P.K.t;
  const double2* __restrict__ rh = P.K.rh;
  double2* __restrict__ x = P.K.x;
  double2* __restrict__ r = P.K.r;
  double acc[2] = {0.0, 0.0};
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const YV yv = y[q], zv = z[q];
    const double2 sv = s[q], tv = t[q], hv = rh[q];
    double2 xv = x[q];
    xv.x += alpha * (double)yv.x + omega * (double)zv.x;
    xv.y += alpha * (double)yv.y + omega * (double)zv.y;
    x[q] = xv;
    const double r0 = sv.x - omega * tv.x, r1 = sv.y - omega * tv.y;
    r[q] = make_double2(r0, r1);
    acc[0] += r0 * r0 + r1 * r1;
    acc[1] += hv.x * r0 + hv.y * r1;
  }
  block_reduce_store<2>(acc, P.K.partial + S_RR * MAXB);
}

// v = A y with the fused <rh, v> (which = 0) or t = A z with <t, s>, <t, t> (which = 1)
template <int NB>
__global__ void __launch_bounds__(BS) k_bicg_op_b(Dims d, Nbr nb, const __grid_constant__ KBatch B, int which) {
  rf_pdl_begin();
  const SysKrylov& P = B.s[blockIdx.y];
  if (kdone(P)) return;
  const double2* md = (const double2*)P.mdiag;
  const double2* __restrict__ x = which ? P.K.z64 : P.K.y64;
  const double2* __restrict__ w = which ? P.K.s : P.K.rh;
  double2* __restrict__ out = which ? P.K.t : P.K.v;
  double acc[2] = {0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    double y0, y1;
    spmv64_row<double2, NB>(d, nb, P.J, md, P.shift, x, p, y0, y1);
    out[p] = make_double2(y0, y1);
    const double2 wv = w[p];
    if (which) {
      acc[0] += y0 * wv.x + y1 * wv.y;
      acc[1] += y0 * y0 + y1 * y1;
    } else {
      acc[0] += wv.x * y0 + wv.y * y1;
    }
  }
  if (which) block_reduce_store<2>(acc, P.K.partial + S_TS * MAXB);
  else {
    double a1[1] = {acc[0]};
    block_reduce_store<1>(a1, P.K.partial + S_RHV * MAXB);
  }
}

// The same for NS systems that share J (the LIMEX columns of one step): each
// block of J is loaded once per vertex and applied to every system's operand.
template <int NB, int NS>
__global__ void __launch_bounds__(BS) k_bicg_op_shared(Dims d, Nbr nb, const __grid_constant__ KBatch B, int which) {
  rf_pdl_begin();
  const SysKrylov* G = B.s + blockIdx.y * NS;   // this group's systems (one shared J)
  bool act[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) act[q] = !kdone(G[q]);
  const double* __restrict__ J = G[0].J;
  const double2* md = (const double2*)G[0].mdiag;
  double acc[NS][2];
#pragma unroll
  for (int q = 0; q < NS; ++q) { acc[q][0] = 0.0; acc[q][1] = 0.0; }
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    const int par = (int)((uint32_t)p % (uint32_t)d.nx) >= d.E;   // nv < 2^31
    double s0[NS], s1[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) { s0[q] = 0.0; s1[q] = 0.0; }
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const double2* qa = reinterpret_cast<const double2*>(J) + ((int64_t)b * d.nv + p) * 2;
      const double2 a01 = __ldcs(qa), a23 = __ldcs(qa + 1);
      const int off = par ? nb.off[1][b] : nb.off[0][b];
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        if (!act[q]) continue;
        const double2 xv = (which ? G[q].K.z64 : G[q].K.y64)[p + off];
        const double x0 = xv.x, x1 = xv.y;
        s0[q] = fma(a01.x, x0, s0[q]);
        s0[q] = fma(a01.y, x1, s0[q]);
        s1[q] = fma(a23.x, x0, s1[q]);
        s1[q] = fma(a23.y, x1, s1[q]);
      }
    }
    const double2 m = md[p];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      if (!act[q]) continue;
      const double xs = (which ? G[q].K.z64 : G[q].K.y64)[p].y;
      const double y0 = G[q].shift * m.x * xs - s0[q];
      const double y1 = G[q].shift * m.y * xs - s1[q];
      (which ? G[q].K.t : G[q].K.v)[p] = make_double2(y0, y1);
      const double2 wv = (which ? G[q].K.s : G[q].K.rh)[p];
      if (which) {
        acc[q][0] += y0 * wv.x + y1 * wv.y;
        acc[q][1] += y0 * y0 + y1 * y1;
      } else {
        acc[q][0] += wv.x * y0 + wv.y * y1;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    // every thread of the block takes part in each reduction (a barrier inside)
    if (which) {
      double a2[2] = {acc[q][0], acc[q][1]};
      block_reduce_store<2>(a2, G[q].K.partial + S_TS * MAXB);
    } else {
      double a1[1] = {acc[q][0]};
      block_reduce_store<1>(a1, G[q].K.partial + S_RHV * MAXB);
    }
    __syncthreads();   // the shared staging of block_reduce_store is reused by the next system
  }
}

__global__ void k_finalize_b(int stage, int nblk, const __grid_constant__ KBatch B) {
  rf_pdl_begin();
  const SysKrylov& P = B.s[blockIdx.x];
  if (kdone(P)) return;
  finalize_body(stage, nblk, P.K.scal, P.K.partial, 0.0);
}

__global__ void k_gather_scal(const __grid_constant__ KBatch B, double* __restrict__ out) {
  const int q = blockIdx.x, t = threadIdx.x;
  if (t < 16) out[16 * q + t] = B.s[q].K.scal[t];
}

static inline void fin_b(int stage, int nblk, const KBatch& B, void* s) {
  RF_LAUNCH_PDL(k_finalize_b, B.n, 32, 0, s, stage, nblk, B);
}

void launch_bicg_p_b(int64_t nv, const KBatch& B, bool lo_is_f32, void* s) {
  const dim3 g((unsigned)krylov_blocks(nv), (unsigned)B.n);
  if (lo_is_f32) RF_LAUNCH_PDL(k_bicg_p_b<float2>, g, BS, 0, s, nv, B);
  else RF_LAUNCH_PDL(k_bicg_p_b<double2>, g, BS, 0, s, nv, B);
}

void launch_bicg_s_b(int64_t nv, const KBatch& B, bool lo_is_f32, void* s) {
  const dim3 g((unsigned)krylov_blocks(nv), (unsigned)B.n);
  if (lo_is_f32) RF_LAUNCH_PDL(k_bicg_s_b<float2>, g, BS, 0, s, nv, B);
  else RF_LAUNCH_PDL(k_bicg_s_b<double2>, g, BS, 0, s, nv, B);
}

void launch_bicg_xr_b(int64_t nv, const KBatch& B, bool yz_is_f32, void* s) {
  const int gx = krylov_blocks(nv);
  const dim3 g((unsigned)gx, (unsigned)B.n);
  if (yz_is_f32) RF_LAUNCH_PDL(k_bicg_xr_b<float2>, g, BS, 0, s, nv, B);
  else RF_LAUNCH_PDL(k_bicg_xr_b<double2>, g, BS, 0, s, nv, B);
  fin_b(3, gx, B, s);
}

static void bicg_op_b(const Dims& d, const Nbr& nb, const KBatch& B, int share, int which, void* s) {
  const int gx = krylov_blocks(d.nv);
  if (share > 1) {
    const dim3 gg((unsigned)gx, (unsigned)(B.n / share));
#define RF_OPS(NBv, NSv) RF_LAUNCH_PDL((k_bicg_op_shared<NBv, NSv>), gg, BS, 0, s, d, nb, B, which)
    if (d.nb == 27) {
      switch (share) { case 1: RF_OPS(27, 1); break; case 2: RF_OPS(27, 2); break; case 3: RF_OPS(27, 3); break; default: RF_OPS(27, 4); }
    } else {
      switch (share) { case 1: RF_OPS(9, 1); break; case 2: RF_OPS(9, 2); break; case 3: RF_OPS(9, 3); break; default: RF_OPS(9, 4); }
    }
#undef RF_OPS
  } else {
    const dim3 g((unsigned)gx, (unsigned)B.n);
    if (d.nb == 27) RF_LAUNCH_PDL(k_bicg_op_b<27>, g, BS, 0, s, d, nb, B, which);
    else RF_LAUNCH_PDL(k_bicg_op_b<9>, g, BS, 0, s, d, nb, B, which);
  }
  fin_b(which ? 2 : 1, gx, B, s);
}

void launch_bicg_v_b(const Dims& d, const Nbr& nb, const KBatch& B, int share, void* s) {
  bicg_op_b(d, nb, B, share, 0, s);
}

void launch_bicg_t_b(const Dims& d, const Nbr& nb, const KBatch& B, int share, void* s) {
  bicg_op_b(d, nb, B, share, 1, s);
}

void launch_gather_scalars(const KBatch& B, double* out, void* s) {
  RF_LAUNCH(k_gather_scal, B.n, 32, 0, s, B, out);
}

// ----------------------------------------------------------------- implicit Euler
// Newton residual of one implicit Euler step: R = F(u) - (m(u) - m(u_old))/H.
// Linear storage: m(u) - m(u_old) = M (S_n - S_n,old) exactly (M = mdiag,
// zero in Dirichlet p_w rows).  S hat storage (sw, sw_old given): the water
// pore volume sums give dm_w = rho_w (sw - sw_old), dm_n = -rho_n (sw - sw_old),
// and Dirichlet p_w rows take no storage.  Also sums ||R||^2 (block partials).
__global__ void __launch_bounds__(BS) k_ie_residual(int64_t nv, const double2* __restrict__ F,
                                                    const double2* __restrict__ u, const double2* __restrict__ u_old,
                                                    const double2* __restrict__ mdiag, const double* __restrict__ sw,
                                                    const double* __restrict__ sw_old, const uint8_t* __restrict__ dir,
                                                    double rho_w, double rho_n, double inv_h, double2* __restrict__ R,
                                                    double* __restrict__ partial) {
  double acc[1] = {0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < nv; p += (int64_t)gridDim.x * BS) {
    const double2 f = F[p];
    double dw, dn;
    if (sw) {
      const double dsw = sw[p] - sw_old[p];
      dw = dir[p] ? 0.0 : rho_w * dsw;
      dn = -(rho_n * dsw);
    } else {
      const double2 m = mdiag[p];
      const double ds = u[p].y - u_old[p].y;
      dw = m.x * ds;
      dn = m.y * ds;
    }
    double2 r;
    r.x = f.x - dw * inv_h;
    r.y = f.y - dn * inv_h;
    R[p] = r;
    acc[0] += r.x * r.x + r.y * r.y;
  }
  block_reduce_store<1>(acc, partial);
}

// out = a + lam * d (pairs): a damped Newton update
__global__ void k_axpby_pairs(int64_t nv, double2* __restrict__ out, const double2* __restrict__ a,
                              const double2* __restrict__ d, double lam) {
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < nv; q += (int64_t)gridDim.x * BS) {
    const double2 x = a[q], y = d[q];
    out[q] = make_double2(x.x + lam * y.x, x.y + lam * y.y);
  }
}

void launch_axpby_pairs(int64_t nv, double* out, const double* a, const double2* d, double lam, void* s) {
  RF_LAUNCH(k_axpby_pairs, krylov_blocks(nv), BS, 0, s, nv, (double2*)out, (const double2*)a, d, lam);
}

__global__ void k_sum1(int nblk, const double* __restrict__ partial, double* __restrict__ out) {
  const double t = sum_partials(partial, 0, nblk);
  if (threadIdx.x == 0) out[0] = t;
}

void launch_ie_residual(int64_t nv, const double* F, const double* u, const double* u_old, const double* mdiag,
                        const double* sw, const double* sw_old, const uint8_t* dir, double rho_w, double rho_n,
                        double inv_h, double* R, double* out1, double* partial, void* s) {
  const int g = krylov_blocks(nv);
  RF_LAUNCH(k_ie_residual, g, BS, 0, s, nv, (const double2*)F, (const double2*)u, (const double2*)u_old,
            (const double2*)mdiag, sw, sw_old, dir, rho_w, rho_n, inv_h, (double2*)R, partial);
  RF_LAUNCH(k_sum1, 1, 32, 0, s, g, partial, out1);
}

// ----------------------------------------------------------------- LIMEX
// Aitken-Neville on the kappa column results T[j][q] (j = 0..kappa-1, n_j =
// j+1), element by element; T[0] <- T_kk, T[1] <- T_{k,k-1}.
__global__ void k_extrapolate(int64_t n2, int kappa, double* __restrict__ T) {
  for (int64_t q = blockIdx.x * (int64_t)BS + threadIdx.x; q < n2; q += (int64_t)gridDim.x * BS) {
    double row[4][4];
    for (int j = 0; j < kappa; ++j) {
      row[j][0] = T[(int64_t)j * n2 + q];
      for (int k = 1; k <= j; ++k) {
        const double f = (double)(j + 1) / (double)(j + 1 - k) - 1.0;
        row[j][k] = row[j][k - 1] + (row[j][k - 1] - row[j - 1][k - 1]) / f;
      }
    }
    T[q] = row[kappa - 1][kappa - 1];
    T[n2 + q] = row[kappa - 1][kappa > 1 ? kappa - 2 : 0];
  }
}
void launch_extrapolate(int64_t n2, int kappa, double* T, void* s) {
  RF_LAUNCH(k_extrapolate, krylov_blocks(n2 / 2), BS, 0, s, n2, kappa, T);
}

// Norms of the scaled error estimate, d = T_kk - T_{k,k-1}: slot 0 |grad p_w(T_kk)|^2, 1 |grad d_p|^2
// (Q1 H1-seminorm, 2-point Gauss per axis: exact for the bilinear/trilinear
// interpolant), 2 sum V_i S_n(T_kk)_i^2, 3 sum V_i d_S,i^2 (lumped L2).
// Thread per vertex: the element whose lowest corner is this vertex, and the
// vertex's own lumped term.
__global__ void __launch_bounds__(BS) k_error_norms(Dims d, double h0, double h1, double h2,
                                                    const double2* __restrict__ Tkk, const double2* __restrict__ Tkk1,
                                                    double* __restrict__ partial) {
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const double hh[3] = {h0, h1, h2};
  const double vol = h0 * h1 * (d.dim == 3 ? h2 : 1.0);
  const int nc = 1 << d.dim;
  const double g0 = 0.5 - 0.5 / sqrt(3.0), g1 = 0.5 + 0.5 / sqrt(3.0);
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < d.nv; p += (int64_t)gridDim.x * BS) {
    int i, j, k;
    pcoords(d, p, i, j, k);
    // lumped weight: number of elements around the vertex
    int cnt = 0;
    for (int c = 0; c < nc; ++c) {
      int ci = i - (c & 1), cj = j - ((c >> 1) & 1), ck = d.dim == 3 ? k - ((c >> 2) & 1) : 0;
      if (ci >= 0 && ci < d.nx - 1 && cj >= 0 && cj < d.ny - 1 && ck >= 0 && ck < (d.dim == 3 ? d.nz - 1 : 1)) ++cnt;
    }
    const double wv = cnt * vol / nc;
    const double2 tv = Tkk[p], t1 = Tkk1[p];
    const double2 dv = make_double2(tv.x - t1.x, tv.y - t1.y);
    acc[2] += wv * tv.y * tv.y;
    acc[3] += wv * dv.y * dv.y;
    if (i < d.nx - 1 && j < d.ny - 1 && (d.dim == 2 || k < d.nz - 1)) {
      double qa[8], qb[8];
      for (int c = 0; c < nc; ++c) {
        const int64_t pc = pidx(d, i + (c & 1), j + ((c >> 1) & 1), d.dim == 3 ? k + ((c >> 2) & 1) : 0);
        qa[c] = Tkk[pc].x;
        qb[c] = Tkk[pc].x - Tkk1[pc].x;
      }
      for (int gq = 0; gq < nc; ++gq) {
        const double xi[3] = {(gq & 1) ? g1 : g0, ((gq >> 1) & 1) ? g1 : g0, ((gq >> 2) & 1) ? g1 : g0};
        double ga = 0.0, gb = 0.0;
        for (int ax = 0; ax < d.dim; ++ax) {
          double da = 0.0, db = 0.0;
          for (int c = 0; c < nc; ++c) {
            double w = ((c >> ax) & 1) ? 1.0 : -1.0;
            for (int m = 0; m < d.dim; ++m)
              if (m != ax) w *= ((c >> m) & 1) ? xi[m] : 1.0 - xi[m];
            da += w * qa[c];
            db += w * qb[c];
          }
          da /= hh[ax];
          db /= hh[ax];
          ga += da * da;
          gb += db * db;
        }
        acc[0] += ga * vol / nc;
        acc[1] += gb * vol / nc;
      }
    }
  }
  block_reduce_store<4>(acc, partial);
}

// Phase masses of a state (lumped storage, Eq. dsW/dpN): sum_i rho_w (Phi V)_i
// (1 - S_n,i) and sum_i rho_n (Phi V)_i S_n,i; slots 0 and 1 of `partial`.
__global__ void __launch_bounds__(BS) k_phase_mass(int64_t nv, double rho_w, double rho_n,
                                                   const double* __restrict__ phiv, const double2* __restrict__ u,
                                                   const double* __restrict__ sw, double* __restrict__ partial) {
  double acc[2] = {0.0, 0.0};
  for (int64_t p = blockIdx.x * (int64_t)BS + threadIdx.x; p < nv; p += (int64_t)gridDim.x * BS) {
    const double pv = phiv[p];
    if (sw) {
      const double w = sw[p];
      acc[0] += rho_w * w;
      acc[1] += rho_n * (pv - w);
    } else {
      const double sn = u[p].y;
      acc[0] += rho_w * (pv * (1.0 - sn));
      acc[1] += rho_n * (pv * sn);
    }
  }
  block_reduce_store<2>(acc, partial);
}

__global__ void k_sum2(int nblk, const double* __restrict__ partial, double* __restrict__ out) {
  for (int q = 0; q < 2; ++q) {
    const double t = sum_partials(partial, q, nblk);
    if (threadIdx.x == 0) out[q] = t;
  }
}

void launch_phase_mass(int64_t nv, double rho_w, double rho_n, const double* phiv, const double* u, const double* sw,
                       double* out2, double* partial, void* s) {
  const int g = krylov_blocks(nv);
  RF_LAUNCH(k_phase_mass, g, BS, 0, s, nv, rho_w, rho_n, phiv, (const double2*)u, sw, partial);
  RF_LAUNCH(k_sum2, 1, 32, 0, s, g, partial, out2);
}

__global__ void k_sum4(int nblk, const double* __restrict__ partial, double* __restrict__ out) {
  for (int q = 0; q < 4; ++q) {
    const double t = sum_partials(partial, q, nblk);
    if (threadIdx.x == 0) out[q] = t;
  }
}

void launch_error_norms(const Dims& d, const double* h, const double* Tkk, const double* Tkk1, double* out4,
                        double* partial, void* s) {
  const int g = krylov_blocks(d.nv);
  RF_LAUNCH(k_error_norms, g, BS, 0, s, d, h[0], h[1], h[2], (const double2*)Tkk, (const double2*)Tkk1, partial);
  RF_LAUNCH(k_sum4, 1, 32, 0, s, g, partial, out4);
}

}  // namespace rf
