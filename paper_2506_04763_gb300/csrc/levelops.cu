// levelops.cu — geometric multigrid building blocks on the vertex-nested
// hierarchy (the preconditioner of the BiCGSTAB stage solve; the paper's
// Sec. 5 setup paragraph names BiCGSTAB + GMG without further detail):
//   - residual r = b - A x, damped point-block Jacobi, multicolour block
//     Gauss-Seidel (2^d colours by coordinate parity), all with the 2x2 block
//     stencil read as coalesced 16/32-byte loads in parity-split order;
//   - full-weighting restriction P^T and trilinear prolongation P (per
//     component; Dirichlet p_w unknowns excluded from the correction space);
//   - Galerkin coarse operators J_c = P^T J P, M_c = P^T M P in FP64;
//   - packing of A = shift*M - J into FP64 / FP32 / FP16-with-row-scales
//     storage and the 2x2 diagonal-block inverses;
//   - the coarsest level's dense LU (partial pivoting) and explicit inverse.
// All of these are HBM-bandwidth kernels except the set-up ones.
#include <cooperative_groups.h>

#include "rf_common.cuh"
#include "rf_kernels.h"

namespace cg = cooperative_groups;

namespace rf {

// ----------------------------------------------------------------- loads
template <int KIND> struct Ty;
template <> struct Ty<STORE_F64> { typedef double T; typedef double S; };
template <> struct Ty<STORE_F32> { typedef float T; typedef float S; };
template <> struct Ty<STORE_F16> { typedef float T; typedef __half S; };

// Streaming read of matrix data: read-only path, not kept in L1, and first in
// line for eviction from L2 (an L2 cache-hint policy), so that the x vector,
// which every colour launch gathers from its neighbours, keeps its place
// there.  -DRF_NO_L2_HINTS builds the loads without the L2 policies.
__device__ __forceinline__ uint64_t l2_policy_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_last() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
#ifdef RF_NO_L2_HINTS
__device__ __forceinline__ float4 ld_stream_f4(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ double2 ld_stream_d2(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint2 ld_stream_u2(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
template <typename V>
__device__ __forceinline__ V ld_keep(const V* p) { return *p; }
#else
__device__ __forceinline__ float4 ld_stream_f4(const float4* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p), "l"(l2_policy_first()));
  return v;
}
__device__ __forceinline__ double2 ld_stream_d2(const double2* p) {
  double2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
               : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(l2_policy_first()));
  return v;
}
__device__ __forceinline__ uint2 ld_stream_u2(const uint2* p) {
  uint2 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
               : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(l2_policy_first()));
  return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p), "l"(l2_policy_first()));
  return v;
}
// Neighbour values of x: kept in L1 (neighbouring threads share them) and
// last in line for eviction from L2.  Only values this launch does not write
// are read this way (GS reads other colours; residual / Jacobi read an input).
__device__ __forceinline__ float2 ld_keep(const float2* p) {
  float2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f32 {%0,%1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(l2_policy_last()));
  return v;
}
__device__ __forceinline__ double2 ld_keep(const double2* p) {
  double2 v;
  asm("ld.global.nc.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;" : "=d"(v.x), "=d"(v.y) : "l"(p), "l"(l2_policy_last()));
  return v;
}
#endif

// Stencil blocks that reach the other x-parity run of the vertex's own x-line
// (dx = -1, +1 with dy = dz = 0).  In a launch that sweeps a pair of colours
// differing only in x parity (k_gs_pair) these are the only neighbours of the
// second colour that the first one writes; the second colour reads them
// coherently at L2 (SAME = true), never through the read-only path.
template <int NB>
__host__ __device__ constexpr bool same_line_block(int b) {
  return NB == 27 ? (b == 12 || b == 14) : (b == 3 || b == 5);
}
template <bool SAME, int NB, typename V>
__device__ __forceinline__ V ld_xn(const V* p, int b) {
  if (SAME && same_line_block<NB>(b)) return __ldcg(p);
  return ld_keep(p);
}
template <bool SAME, int NB, typename V>
__device__ __forceinline__ V ld_xn_plain(const V* p, int b) {
  if (SAME && same_line_block<NB>(b)) return __ldcg(p);
  return *p;
}

// One stored 2x2 block as loaded (FP64: two double2; FP32: a float4; FP16:
// four halves), and its entries in the arithmetic type (FP16: times the row's
// per-entry FP32 scales).  Loading and unpacking are split so that a batch of
// loads can be issued before any of them is unpacked.
template <int KIND> struct RawBlock;
template <> struct RawBlock<STORE_F64> { double2 u, w; };
template <> struct RawBlock<STORE_F32> { float4 u; };
template <> struct RawBlock<STORE_F16> { uint2 u; };

template <int KIND>
__device__ __forceinline__ void load_raw(const void* A, int64_t nv, int b, int64_t p, RawBlock<KIND>& r) {
  const int64_t o = (int64_t)b * nv + p;
  if constexpr (KIND == STORE_F64) {
    const double2* q = reinterpret_cast<const double2*>(A) + o * 2;
    r.u = ld_stream_d2(q);
    r.w = ld_stream_d2(q + 1);
  } else if constexpr (KIND == STORE_F32) {
    r.u = ld_stream_f4(reinterpret_cast<const float4*>(A) + o);
  } else {
    r.u = ld_stream_u2(reinterpret_cast<const uint2*>(A) + o);
  }
}

template <int KIND>
__device__ __forceinline__ void unpack_block(const RawBlock<KIND>& r, const float4& sc, typename Ty<KIND>::T (&a)[4]) {
  if constexpr (KIND == STORE_F64) {
    a[0] = r.u.x; a[1] = r.u.y; a[2] = r.w.x; a[3] = r.w.y;
  } else if constexpr (KIND == STORE_F32) {
    a[0] = r.u.x; a[1] = r.u.y; a[2] = r.u.z; a[3] = r.u.w;
  } else {
    uint2 u = r.u;
    __half2 h01 = *reinterpret_cast<__half2*>(&u.x), h23 = *reinterpret_cast<__half2*>(&u.y);
    float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
    a[0] = f01.x * sc.x; a[1] = f01.y * sc.y; a[2] = f23.x * sc.z; a[3] = f23.y * sc.w;
  }
}

template <int KIND>
__device__ __forceinline__ void load_block(const void* A, int64_t nv, int b, int64_t p, const float4& sc,
                                           typename Ty<KIND>::T (&a)[4]) {
  RawBlock<KIND> r;
  load_raw<KIND>(A, nv, b, p, r);
  unpack_block<KIND>(r, sc, a);
}

// Row sum += (a_0 x_0 + a_1 x_1) for one block row: one explicit fused
// multiply-add and an explicit add, so that every kernel applying a block
// (per-block, batched, shared-matrix) rounds it identically, whatever the
// compiler would otherwise contract.
__device__ __forceinline__ float blk_acc(float s, float a0, float a1, float2 x) {
  return __fadd_rn(s, __fmaf_rn(a0, x.x, __fmul_rn(a1, x.y)));
}
__device__ __forceinline__ double blk_acc(double s, double a0, double a1, double2 x) {
  return __dadd_rn(s, __fma_rn(a0, x.x, __dmul_rn(a1, x.y)));
}

// FP16 storage holds the blocks of a row in pairs, one 16-byte load per pair
// (a warp reads 512 contiguous bytes per load, as with FP32 blocks): slot s
// of row p is half s % 2 of uint4 number (s / 2) * nv + p.  The two blocks of
// a pair have offsets of the same parity in every axis, so they reach
// vertices of the same colour: the first sweep from zero, which skips the
// blocks of colours not yet visited, skips whole pairs.  Slots (3D): the
// pairs dx = -1, +1 for each (dy, dz); then the dx = 0 pairs (dy = -1, +1 at
// dz = 0), (dz = -1, +1 at dy = 0), (dy = -1, +1 at dz = -1), (dy = -1, +1 at
// dz = +1); then the centre and an empty slot.  2D: dx = -1, +1 for each dy,
// then (dy = -1, +1 at dx = 0), then the centre and an empty slot.  A sweep
// that skips the centre reads none of the last pair.
__host__ __device__ constexpr int f16_block_of_slot(int nb, int s) {
  if (nb == 27) {
    if (s < 18) return ((s & 1) ? 2 : 0) + 3 * ((s >> 1) % 3) + 9 * ((s >> 1) / 3);
    switch (s) {
      case 18: return 10; case 19: return 16;   // (0, -1, 0), (0, +1, 0)
      case 20: return 4;  case 21: return 22;   // (0, 0, -1), (0, 0, +1)
      case 22: return 1;  case 23: return 7;    // (0, -1, -1), (0, +1, -1)
      case 24: return 19; case 25: return 25;   // (0, -1, +1), (0, +1, +1)
      case 26: return 13;                       // centre
      default: return -1;
    }
  }
  if (s < 6) return ((s & 1) ? 2 : 0) + 3 * (s >> 1);
  return s == 6 ? 1 : s == 7 ? 7 : s == 8 ? 4 : -1;
}
__host__ __device__ constexpr int f16_slot_of_block(int nb, int b) {
  int s = 0;
  while (s < nb && f16_block_of_slot(nb, s) != b) ++s;
  return s;
}

__device__ __forceinline__ void f16_half(const uint4& u, int h, const float4& sc, float (&a)[4]) {
  RawBlock<STORE_F16> r;
  r.u = h ? make_uint2(u.z, u.w) : make_uint2(u.x, u.y);
  unpack_block<STORE_F16>(r, sc, a);
}

// The FP16 stencil sum, slot by slot: CP pairs (2 CP blocks) and their x values
// loaded per memory round trip, then summed.  Per-block, batched and
// shared-matrix FP16 kernels all sum in this slot order with blk_acc.
template <int NB, int CP, bool SAME = false>
__device__ __forceinline__ void stencil_sum_f16(const LevelOp& L, int64_t p, int par,
                                                const float2* __restrict__ x, bool skip_centre, uint32_t skipmask,
                                                float& s0, float& s1) {
  constexpr int C = NB == 27 ? 13 : 4, NP = (NB + 1) / 2;
  const float4 sc = reinterpret_cast<const float4*>(L.scale)[p];
  const uint4* __restrict__ A = reinterpret_cast<const uint4*>(L.A);
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int q0 = 0; q0 < NP; q0 += CP) {
    uint4 raw[CP];
    float2 xv[CP][2];
    bool use[CP][2];
#pragma unroll
    for (int c = 0; c < CP; ++c) {
      const int q = q0 + c;
      if (q >= NP) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int b = f16_block_of_slot(NB, 2 * q + h);
        use[c][h] = b >= 0 && !(skip_centre && b == C) && !((skipmask >> (b >= 0 ? b : 0)) & 1u);
      }
      if (use[c][0] || use[c][1]) raw[c] = ld_stream_u4(A + (int64_t)q * L.d.nv + p);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int b = f16_block_of_slot(NB, 2 * q + h);
        if (use[c][h]) xv[c][h] = ld_xn<SAME, NB>(x + p + (par ? L.nb.off[1][b] : L.nb.off[0][b]), b);
      }
    }
#pragma unroll
    for (int c = 0; c < CP; ++c) {
      if (q0 + c >= NP) break;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!use[c][h]) continue;
        float a[4];
        f16_half(raw[c], h, sc, a);
        a0 = blk_acc(a0, a[0], a[1], xv[c][h]);
        a1 = blk_acc(a1, a[2], a[3], xv[c][h]);
      }
    }
  }
  s0 = a0; s1 = a1;
}

// sum over the stencil of blocks * x (centre optionally skipped)
template <int KIND, int NB, bool SAME = false>
__device__ __forceinline__ void stencil_sum(const LevelOp& L, int64_t p, int par,
                                            const typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                            bool skip_centre, uint32_t skipmask, typename Ty<KIND>::T& s0,
                                            typename Ty<KIND>::T& s1) {
  typedef typename Ty<KIND>::T T;
  constexpr int C = NB == 27 ? 13 : 4;
  float4 sc = make_float4(1.f, 1.f, 1.f, 1.f);
  if (KIND == STORE_F16) sc = reinterpret_cast<const float4*>(L.scale)[p];
  T a0 = 0, a1 = 0;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (skip_centre && b == C) continue;
    if ((skipmask >> b) & 1u) continue;   // neighbour known to be zero
    T a[4];
    load_block<KIND>(L.A, L.d.nv, b, p, sc, a);
    const int off = par ? L.nb.off[1][b] : L.nb.off[0][b];
    const typename V2<T>::t xv = ld_xn_plain<SAME, NB>(x + p + off, b);
    a0 = blk_acc(a0, a[0], a[1], xv);
    a1 = blk_acc(a1, a[2], a[3], xv);
  }
  s0 = a0; s1 = a1;
}

// stencil_sum with the loads of CH blocks (and their x values) issued before
// any is used: one memory round trip per CH blocks instead of one per block.
// The block loads are the `volatile` streaming loads of load_raw, which the
// compiler keeps in source order, so placing all CH of them ahead of the sums
// is what batches them (ordinary loads get sunk back next to their uses).
// The same blocks are summed in the same order with the same blk_acc, so the
// sums equal stencil_sum's bit for bit.
// This is what the small levels need, where a thread's chain of round trips,
// not bandwidth, sets the time.
// Stencil blocks (FP16: block pairs) whose loads a batched kernel issues per
// memory round trip; an unbatched FP16 kernel loads one pair per round trip.
__host__ __device__ constexpr int chunk_of(int kind) { return kind == STORE_F16 ? 2 : 9; }

template <int KIND, int NB, int CH, bool SAME = false>
__device__ __forceinline__ void stencil_sum_batched(const LevelOp& L, int64_t p, int par,
                                                    const typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                                    bool skip_centre, uint32_t skipmask, typename Ty<KIND>::T& s0,
                                                    typename Ty<KIND>::T& s1) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  constexpr int C = NB == 27 ? 13 : 4;
  float4 sc = make_float4(1.f, 1.f, 1.f, 1.f);
  if (KIND == STORE_F16) sc = reinterpret_cast<const float4*>(L.scale)[p];
  T a0 = 0, a1 = 0;
#pragma unroll
  for (int b0 = 0; b0 < NB; b0 += CH) {
    RawBlock<KIND> raw[CH];
    bool skip[CH];
    V xv[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      const int b = b0 + c;
      if (b >= NB) break;
      skip[c] = (skip_centre && b == C) || ((skipmask >> b) & 1u);
      if (!skip[c]) {
        load_raw<KIND>(L.A, L.d.nv, b, p, raw[c]);
        xv[c] = ld_xn<SAME, NB>(x + p + (par ? L.nb.off[1][b] : L.nb.off[0][b]), b);
      }
    }
    // unpacked only now: an FP16 block's scaling waits for its load, which
    // would otherwise hold back the loads issued after it
#pragma unroll
    for (int c = 0; c < CH; ++c) {
      if (b0 + c >= NB) break;
      if (skip[c]) continue;   // as in the per-block sum
      T a[4];
      unpack_block<KIND>(raw[c], sc, a);
      a0 = blk_acc(a0, a[0], a[1], xv[c]);
      a1 = blk_acc(a1, a[2], a[3], xv[c]);
    }
  }
  s0 = a0; s1 = a1;
}

template <int KIND, int NB, int CH, bool SAME = false>
__device__ __forceinline__ void stencil_sum_any(const LevelOp& L, int64_t p, int par,
                                                const typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                                bool skip_centre, uint32_t skipmask, typename Ty<KIND>::T& s0,
                                                typename Ty<KIND>::T& s1) {
  if constexpr (KIND == STORE_F16)
    stencil_sum_f16<NB, (CH > 0 ? CH : 1), SAME>(L, p, par, x, skip_centre, skipmask, s0, s1);
  else if constexpr (CH > 0)
    stencil_sum_batched<KIND, NB, CH, SAME>(L, p, par, x, skip_centre, skipmask, s0, s1);
  else
    stencil_sum<KIND, NB, SAME>(L, p, par, x, skip_centre, skipmask, s0, s1);
}

// (A x)_p, with A = shift*M - J on the fine level (blocks hold J)
template <int KIND, bool FINE, int NB, int CH = 0>
__device__ __forceinline__ void apply_row(const LevelOp& L, int64_t p, int par,
                                          const typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                          typename Ty<KIND>::T& s0, typename Ty<KIND>::T& s1) {
  typedef typename Ty<KIND>::T T;
  // batched: the mask is L.nomask (always zero) read at run time, which keeps
  // each block's load in its own conditional branch and so stops the compiler
  // from interleaving the batch's loads with the sums (it does that with a
  // constant zero mask, and the batch is lost)
  stencil_sum_any<KIND, NB, CH>(L, p, par, x, false, CH > 0 ? L.nomask : 0u, s0, s1);
  if (FINE) {
    const double2 m = reinterpret_cast<const double2*>(L.mdiag)[p];
    const T xs = x[p].y, sh = (T)L.shift;
    s0 = (T)(sh * (T)m.x) * xs - s0;
    s1 = (T)(sh * (T)m.y) * xs - s1;
  }
}

template <typename T>
__device__ __forceinline__ void dinv_apply(const T* Dinv, int64_t p, T r0, T r1, T& y0, T& y1) {
  const T* D = Dinv + p * 4;
  y0 = D[0] * r0 + D[1] * r1;
  y1 = D[2] * r0 + D[3] * r1;
}

// ----------------------------------------------------------------- residual
template <int KIND, bool FINE, int NB, int CH = 0>
__device__ __forceinline__ void residual_point(const LevelOp& L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                               const typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                               typename V2<typename Ty<KIND>::T>::t* __restrict__ r, int64_t p) {
  typedef typename Ty<KIND>::T T;
  const int par = (int)((uint32_t)p % (uint32_t)L.d.nx) >= L.d.E;   // nv < 2^31
  const typename V2<T>::t bv = b[p];
  T s0, s1;
  apply_row<KIND, FINE, NB, CH>(L, p, par, x, s0, s1);
  typename V2<T>::t o;
  o.x = bv.x - s0;
  o.y = bv.y - s1;
  r[p] = o;
}

template <int KIND, bool FINE, int NB, int CH>
__global__ void __launch_bounds__(CH > 0 ? 256 : 512) k_residual(LevelOp L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                                  const typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                                  typename V2<typename Ty<KIND>::T>::t* __restrict__ r) {
  rf_pdl_begin();
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= L.d.nv) return;
  residual_point<KIND, FINE, NB, CH>(L, b, x, r, p);
}

// ----------------------------------------------------------------- Jacobi
template <int KIND, bool FINE, int NB, int CH = 0>
__device__ __forceinline__ void jacobi_point(const LevelOp& L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                             const typename V2<typename Ty<KIND>::T>::t* __restrict__ xin,
                                             typename V2<typename Ty<KIND>::T>::t* __restrict__ xout, double omega,
                                             int zero_x, int64_t p) {
  typedef typename Ty<KIND>::T T;
  const typename V2<T>::t bv = b[p];
  T r0 = bv.x, r1 = bv.y, x0 = 0, x1 = 0;
  if (!zero_x) {
    const int par = (int)((uint32_t)p % (uint32_t)L.d.nx) >= L.d.E;   // nv < 2^31
    T s0, s1;
    apply_row<KIND, FINE, NB, CH>(L, p, par, xin, s0, s1);
    r0 -= s0;
    r1 -= s1;
    x0 = xin[p].x;
    x1 = xin[p].y;
  }
  T y0, y1;
  dinv_apply<T>(reinterpret_cast<const T*>(L.Dinv), p, r0, r1, y0, y1);
  typename V2<T>::t o;
  o.x = x0 + (T)omega * y0;
  o.y = x1 + (T)omega * y1;
  xout[p] = o;
}

template <int KIND, bool FINE, int NB, int CH>
__global__ void __launch_bounds__(CH > 0 ? 256 : 512) k_jacobi(LevelOp L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                                const typename V2<typename Ty<KIND>::T>::t* __restrict__ xin,
                                                typename V2<typename Ty<KIND>::T>::t* __restrict__ xout, double omega,
                                                int zero_x) {
  rf_pdl_begin();
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= L.d.nv) return;
  jacobi_point<KIND, FINE, NB, CH>(L, b, xin, xout, omega, zero_x, p);
}

// ----------------------------------------------------------------- multicolour GS
// One vertex p (x parity px) of a colour: x_p <- D_p^-1 (b_p - sum_{q != p} A_pq x_q).
template <int KIND, bool FINE, int NB, int CH = 0, bool SAME = false>
__device__ __forceinline__ void gs_vertex(const LevelOp& L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                          typename V2<typename Ty<KIND>::T>::t* __restrict__ x, int px, int64_t p,
                                          uint32_t skipmask) {
  typedef typename Ty<KIND>::T T;
  const typename V2<T>::t bv = b[p];
  T s0, s1;
  stencil_sum_any<KIND, NB, CH, SAME>(L, p, px, x, true, skipmask, s0, s1);
  // off-diagonal part of A: fine level A_pq = -J_pq (q != p), coarse A_pq
  const T r0 = FINE ? bv.x + s0 : bv.x - s0;
  const T r1 = FINE ? bv.y + s1 : bv.y - s1;
  T y0, y1;
  dinv_apply<T>(reinterpret_cast<const T*>(L.Dinv), p, r0, r1, y0, y1);
  typename V2<T>::t o;
  o.x = y0;
  o.y = y1;
  x[p] = o;
}

// One colour (px,py,pz) of the sweep.
// Work item t of the colour: t enumerates the colour's x-runs line by line.
template <int KIND, bool FINE, int NB, int CH = 0>
__device__ __forceinline__ void gs_point(const LevelOp& L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                         typename V2<typename Ty<KIND>::T>::t* __restrict__ x, int px, int py, int pz,
                                         int cnt_x, int lines_y, int64_t t, uint32_t skipmask) {
  typedef typename Ty<KIND>::T T;
  // 32-bit index arithmetic: a colour has fewer than 2^31 vertices
  const uint32_t tt = (uint32_t)t, line = tt / (uint32_t)cnt_x, kl = line / (uint32_t)lines_y;
  const int pos = (int)(tt - line * (uint32_t)cnt_x);
  const int jj = (int)(line - kl * (uint32_t)lines_y), kk = (int)kl;
  const int j = 2 * jj + py, k = 2 * kk + pz;
  const int64_t p = ((int64_t)j + (int64_t)L.d.ny * k) * L.d.nx + (px ? L.d.E : 0) + pos;
  gs_vertex<KIND, FINE, NB, CH>(L, b, x, px, p, skipmask);
}

template <int KIND, bool FINE, int NB, int CH>
__global__ void __launch_bounds__(CH > 0 ? 256 : 512) k_gs_colour(LevelOp L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                                   typename V2<typename Ty<KIND>::T>::t* __restrict__ x, int px, int py,
                                                   int pz, int cnt_x, int lines_y, int64_t count, uint32_t skipmask,
                                                   int reverse) {
  rf_pdl_begin();
  // reverse: blocks take the colour's vertices from the end (see gs_zigzag)
  const int64_t bx = reverse ? (int64_t)(gridDim.x - 1 - blockIdx.x) : (int64_t)blockIdx.x;
  int64_t t = bx * blockDim.x + threadIdx.x;
  if (t >= count) return;
  gs_point<KIND, FINE, NB, CH>(L, b, x, px, py, pz, cnt_x, lines_y, t, skipmask);
}

// Threads of a colour-pair block (k_gs_pair) at most.
constexpr int GS_PAIR_MAX_THREADS = 320;

// Vertex of item v of a pair block's run: line l0 + v / cnt of the pair's
// lines (enumerated y first), position v % cnt in the run of parity px.
__device__ __forceinline__ int64_t pair_vertex(const Dims& d, int l0, int v, int cnt, int px, int py, int pz,
                                               int lines_y) {
  const int li = v / cnt, pos = v - li * cnt;
  const int line = l0 + li, kl = line / lines_y;
  const int j = 2 * (line - kl * lines_y) + py, k = 2 * kl + pz;
  return ((int64_t)j + (int64_t)d.ny * k) * d.nx + (px ? d.E : 0) + pos;
}

// Two consecutive colours of a sweep that differ only in x parity,
// (first_px, py, pz) then (1 - first_px, py, pz), in one launch.  A vertex of
// either colour reaches the other one only on its own x-line (dx = -1, +1 with
// dy = dz = 0); all its other neighbours have colours that neither of the two
// writes.  So a block that owns whole x-lines updates the first colour's run
// of each of its lines, passes a block barrier, and then updates the second
// colour's runs, reading the just-written neighbours at L2: every vertex sees
// the values that the two separate colour launches give it, and the sums are
// the same operations in the same order.  One launch instead of two, and the
// other colours' x values are gathered once for both.  Block b owns lines
// [b * lpb, b * lpb + lpb) of the pair (reversed block order: see gs_zigzag).
template <int KIND, bool FINE, int NB, int CH, int FPX>
__global__ void __launch_bounds__(GS_PAIR_MAX_THREADS) k_gs_pair(LevelOp L, const typename V2<typename Ty<KIND>::T>::t* __restrict__ b,
                                                  typename V2<typename Ty<KIND>::T>::t* __restrict__ x,
                                                  int py, int pz, int lines_y, int nlines, int lpb,
                                                  uint32_t skip_first, uint32_t skip_second, int reverse) {
  rf_pdl_begin();
  const int bx = reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  const int l0 = bx * lpb;
  const int nl = min(lpb, nlines - l0);
  // one vertex per thread and run: the launch gives every block at least
  // lpb * (nx + 1) / 2 threads (a loop here would make the compiler hoist
  // the stencil's address arithmetic and double the registers)
  const int v = threadIdx.x;
  {
    const int cnt = FPX ? L.d.nx / 2 : (L.d.nx + 1) / 2;
    if (v < nl * cnt)
      gs_vertex<KIND, FINE, NB, CH, false>(L, b, x, FPX, pair_vertex(L.d, l0, v, cnt, FPX, py, pz, lines_y), skip_first);
  }
  __syncthreads();
  {
    const int cnt = FPX ? (L.d.nx + 1) / 2 : L.d.nx / 2;
    if (v < nl * cnt)
      gs_vertex<KIND, FINE, NB, CH, true>(L, b, x, 1 - FPX, pair_vertex(L.d, l0, v, cnt, 1 - FPX, py, pz, lines_y), skip_second);
  }
}

// ----------------------------------------------------------------- transfers
template <typename T>
__device__ __forceinline__ void restrict_point(const Dims& df, const Dims& dc, const uint8_t* __restrict__ dmf,
                                               const uint8_t* __restrict__ dmc, const typename V2<T>::t* __restrict__ rf,
                                               typename V2<T>::t* __restrict__ bc, int64_t pc) {
  typedef typename V2<T>::t V;
  int I, J, K;
  pcoords(dc, pc, I, J, K);
  const bool mc = dmc[pc] != 0;
  // all 3^d fine values and masks are loaded first (one memory round trip),
  // then summed in the fixed (dz, dy, dx) order
  V r[27];
  uint8_t m[27];
  bool in[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
    const int fi = 2 * I + dx, fj = 2 * J + dy, fk = df.dim == 3 ? 2 * K + dz : 0;
    in[q] = (df.dim == 3 || dz == 0) && fi >= 0 && fi < df.nx && fj >= 0 && fj < df.ny && fk >= 0 && fk < df.nz;
    if (in[q]) {
      const int64_t pf = pidx(df, fi, fj, fk);
      r[q] = rf[pf];
      m[q] = dmf[pf];
    } else {
      r[q].x = 0;
      r[q].y = 0;
      m[q] = 1;
    }
  }
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (!in[q]) continue;
    const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
    const T w = (T)((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
    if (!(mc || m[q])) s0 += w * r[q].x;
    s1 += w * r[q].y;
  }
  V o;
  o.x = s0;
  o.y = s1;
  bc[pc] = o;
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict(Dims df, Dims dc, const uint8_t* __restrict__ dmf,
                                                  const uint8_t* __restrict__ dmc,
                                                  const typename V2<T>::t* __restrict__ rf,
                                                  typename V2<T>::t* __restrict__ bc) {
  rf_pdl_begin();
  int64_t pc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pc >= dc.nv) return;
  restrict_point<T>(df, dc, dmf, dmc, rf, bc, pc);
}

template <typename T>
__device__ __forceinline__ void prolong_point(const Dims& df, const Dims& dc, const uint8_t* __restrict__ dmf,
                                              const uint8_t* __restrict__ dmc, const typename V2<T>::t* __restrict__ xc,
                                              typename V2<T>::t* __restrict__ xf, int64_t pf) {
  typedef typename V2<T>::t V;
  int fi, fj, fk;
  pcoords(df, pf, fi, fj, fk);
  const bool mf = dmf[pf] != 0;
  // the (up to) 2^d coarse parents, loaded first, summed in (K, J, I) order
  V c[8];
  uint8_t m[8];
  bool in[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int K = (fk >> 1) + ((q >> 2) & 1), J = (fj >> 1) + ((q >> 1) & 1), I = (fi >> 1) + (q & 1);
    in[q] = ((q & 1) == 0 || (fi & 1)) && (((q >> 1) & 1) == 0 || (fj & 1)) &&
            (((q >> 2) & 1) == 0 || (fk & 1)) && K < dc.nz && J < dc.ny && I < dc.nx;
    if (in[q]) {
      const int64_t pc = pidx(dc, I, J, K);
      c[q] = xc[pc];
      m[q] = dmc[pc];
    } else {
      c[q].x = 0;
      c[q].y = 0;
      m[q] = 1;
    }
  }
  const T wz = (df.dim == 3 && (fk & 1)) ? (T)0.5 : (T)1;
  const T wy = (fj & 1) ? (T)0.5 : (T)1;
  const T w = ((fi & 1) ? (T)0.5 : (T)1) * wy * wz;
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    if (!in[q]) continue;
    if (!(mf || m[q])) s0 += w * c[q].x;
    s1 += w * c[q].y;
  }
  V o = xf[pf];
  o.x += s0;
  o.y += s1;
  xf[pf] = o;
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong(Dims df, Dims dc, const uint8_t* __restrict__ dmf,
                                                 const uint8_t* __restrict__ dmc,
                                                 const typename V2<T>::t* __restrict__ xc,
                                                 typename V2<T>::t* __restrict__ xf) {
  rf_pdl_begin();
  int64_t pf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pf >= df.nv) return;
  prolong_point<T>(df, dc, dmf, dmc, xc, xf, pf);
}

// The same transfers, organised for memory-level parallelism.  The per-point
// kernels above put each gathered load behind its own bounds branch.  These
// issue every load before the first sum: a value outside the grid is read at
// an in-grid address and then skipped.  They also take the vertex from the
// launch shape (a plane per blockIdx.y, the position within it by one 32-bit
// division) and compute the gathered lines' offsets once per vertex, instead
// of pcoords and a 64-bit pidx per value.  Loads, masks, weights and the order
// of the sums are those of restrict_point / prolong_point, so the results are
// bitwise equal.  At 257^3 the transfers take 3.14 ms per solve against 4.14.
template <typename T>
__device__ __forceinline__ void restrict_planes_body(const Dims& df, const Dims& dc, const uint8_t* __restrict__ dmf,
                                                     const uint8_t* __restrict__ dmc,
                                                     const typename V2<T>::t* __restrict__ rf,
                                                     typename V2<T>::t* __restrict__ bc) {
  rf_pdl_begin();
  typedef typename V2<T>::t V;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= dc.nx * dc.ny) return;
  const int J = t / dc.nx, pos = t - J * dc.nx, K = blockIdx.y;
  const int I = pos < dc.E ? 2 * pos : 2 * (pos - dc.E) + 1;
  // 32-bit vertex indices: a grid has at most 2^31 vertices (rf_grid_create)
  const int pc = (J + dc.ny * K) * dc.nx + pos;
  const bool mc = dmc[pc] != 0;
  int xo[3];
  bool xin[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int fi = 2 * I + a - 1;
    xin[a] = fi >= 0 && fi < df.nx;
    xo[a] = (fi & 1) ? df.E + (fi >> 1) : (fi >> 1);
  }
  int lo[9];
  bool lin[9];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const int fj = 2 * J + b - 1, fk = df.dim == 3 ? 2 * K + c - 1 : 0;
      lin[3 * c + b] = (df.dim == 3 || c == 1) && fj >= 0 && fj < df.ny && fk >= 0 && fk < df.nz;
      lo[3 * c + b] = lin[3 * c + b] ? (fj + df.ny * fk) * df.nx : 0;   // (no overflow outside the grid)
    }
  // every load is issued, without a branch, before the first sum: a value
  // outside the grid is read at the vertex's own fine position (always
  // inside) and then skipped, so the 27 loads are one memory round trip
  const int pf0 = lo[4] + xo[1];
  V r[27];
  uint8_t m[27];
  bool in[27];
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int a = q % 3, bc3 = q / 3;   // bc3 = 3 * (dz + 1) + (dy + 1)
    in[q] = lin[bc3] && xin[a];
    const int pf = in[q] ? lo[bc3] + xo[a] : pf0;
    r[q] = rf[pf];
    m[q] = dmf[pf];
  }
  T s0 = 0, s1 = 0;
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    if (!in[q]) continue;
    const int dx = q % 3 - 1, dy = (q / 3) % 3 - 1, dz = q / 9 - 1;
    const T w = (T)((dx ? 0.5 : 1.0) * (dy ? 0.5 : 1.0) * (dz ? 0.5 : 1.0));
    if (!(mc || m[q])) s0 += w * r[q].x;
    s1 += w * r[q].y;
  }
  V o;
  o.x = s0;
  o.y = s1;
  bc[pc] = o;
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_planes(Dims df, Dims dc, const uint8_t* __restrict__ dmf,
                                                         const uint8_t* __restrict__ dmc,
                                                         const typename V2<T>::t* __restrict__ rf,
                                                         typename V2<T>::t* __restrict__ bc) {
  restrict_planes_body<T>(df, dc, dmf, dmc, rf, bc);
}

// Prolongation and correction x_f += P x_c, two fine vertices per thread:
// thread (I, fj, fk) updates fine vertex 2I (even half of the parity-split
// line) and 2I + 1 (odd half), whose coarse parents along x are I, and I and
// I + 1.  Their (up to 8) parents are loaded once, before the first sum (one
// memory round trip; a parent outside the coarse grid is read at coarse
// vertex 0 and skipped).  Each fine value then sums its parents in the
// (K, J, I) order of prolong_point with the same expressions, so the results
// are the per-point kernel's bit for bit.  The pairing halves the gathered
// loads and the index arithmetic per fine vertex (the one-vertex-per-thread
// form issued ~330 instructions per vertex and was issue-bound).
template <typename T>
__device__ __forceinline__ void prolong_pairs_body(const Dims& df, const Dims& dc, const uint8_t* __restrict__ dmf,
                                                   const uint8_t* __restrict__ dmc,
                                                   const typename V2<T>::t* __restrict__ xc,
                                                   typename V2<T>::t* __restrict__ xf) {
  rf_pdl_begin();
  typedef typename V2<T>::t V;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= dc.nx * df.ny) return;
  const int fj = t / dc.nx, I = t - fj * dc.nx, fk = blockIdx.y;
  const int J0 = fj >> 1, K0 = fk >> 1;
  const bool oy = (fj & 1) != 0, oz = df.dim == 3 && (fk & 1) != 0;
  const bool odd = 2 * I + 1 < df.nx;   // fine vertex 2I + 1 exists
  // 32-bit vertex indices: a grid has at most 2^31 vertices (rf_grid_create)
  const int fline = (fj + df.ny * fk) * df.nx;
  const int pe = fline + I, po = fline + df.E + I;
  const int xo[2] = {(I & 1) ? dc.E + (I >> 1) : (I >> 1), ((I + 1) & 1) ? dc.E + ((I + 1) >> 1) : ((I + 1) >> 1)};
  V c8[8];
  uint8_t m[8];
  bool in[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int ib = q & 1, jb = (q >> 1) & 1, kb = (q >> 2) & 1;
    in[q] = (!jb || oy) && (!kb || oz) && (!ib || odd) && K0 + kb < dc.nz && J0 + jb < dc.ny && I + ib < dc.nx;
    const int pc = in[q] ? ((J0 + jb) + dc.ny * (K0 + kb)) * dc.nx + xo[ib] : 0;
    c8[q] = xc[pc];
    m[q] = dmc[pc];
  }
  const V xe = xf[pe];
  const bool me = dmf[pe] != 0;
  V xo_v = xe;
  bool mo = false;
  if (odd) {
    xo_v = xf[po];
    mo = dmf[po] != 0;
  }
  const T wz = oz ? (T)0.5 : (T)1;
  const T wy = oy ? (T)0.5 : (T)1;
  {
    const T w = (T)1 * wy * wz;   // fine x even
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
      if (!in[q]) continue;
      if (!(me || m[q])) s0 += w * c8[q].x;
      s1 += w * c8[q].y;
    }
    V o = xe;
    o.x += s0;
    o.y += s1;
    xf[pe] = o;
  }
  if (odd) {
    const T w = (T)0.5 * wy * wz;   // fine x odd
    T s0 = 0, s1 = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (!in[q]) continue;
      if (!(mo || m[q])) s0 += w * c8[q].x;
      s1 += w * c8[q].y;
    }
    V o = xo_v;
    o.x += s0;
    o.y += s1;
    xf[po] = o;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_planes(Dims df, Dims dc, const uint8_t* __restrict__ dmf,
                                                        const uint8_t* __restrict__ dmc,
                                                        const typename V2<T>::t* __restrict__ xc,
                                                        typename V2<T>::t* __restrict__ xf) {
  prolong_pairs_body<T>(df, dc, dmf, dmc, xc, xf);
}

// ----------------------------------------------------------------- coarsest solve
// x = A^-1 b on the coarsest level: one warp per row of the explicit
// inverse, lanes over its columns (coalesced), FP64 sums.
template <typename T>
__device__ __forceinline__ void coarse_solve_body(int N, const double* __restrict__ Ainv, const T* __restrict__ b,
                                                  T* __restrict__ x) {
  rf_pdl_begin();
  extern __shared__ double sb[];
  for (int t = threadIdx.x; t < N; t += blockDim.x) sb[t] = (double)b[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= N) return;
  const double* row = Ainv + (int64_t)r * N;
  double s = 0.0;
  for (int c = lane; c < N; c += 32) s += row[c] * sb[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) x[r] = (T)s;
}

template <typename T>
__global__ void __launch_bounds__(256) k_coarse_solve(int N, const double* __restrict__ Ainv,
                                                      const T* __restrict__ b, T* __restrict__ x) {
  coarse_solve_body<T>(N, Ainv, b, x);
}

// ----------------------------------------------------------------- V-cycle tail
// Levels below a few 10^4 vertices cannot fill the GPU: launched one kernel per
// GS colour, each costs a launch gap.  Here one launch runs the whole V-cycle
// from level `first` down to the coarsest and back up, its phases separated by
// barriers (every thread reaches every barrier: all loop bounds below are
// uniform across the launch).  Two forms:
//   k_vcycle_tail: ONE thread-block cluster, hardware cluster barriers;
//   k_vcycle_coop: a cooperative launch of every co-resident block, grid
//     barriers in global memory whose waits give up after P.limit_ns (the
//     block then sets *P.status = 1 and leaves; the others see the flag in
//     their own waits and leave too, so the kernel always ends).

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier of a cooperative launch: bar[0] counts this generation's
// arrivals, bar[1] is the generation.  `gen` (held by thread 0) is the
// generation this block last passed.  The last block to arrive resets the
// count and then publishes gen + 1; the others wait for it, at most limit_ns.
// Returns false when the wait gave up or another block already had.
__device__ __forceinline__ bool grid_sync_bounded(unsigned* bar, unsigned expected, unsigned& gen,
                                                  double* status, long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned want = gen + 1;
    __threadfence();   // this block's phase results before its arrival
    if (atomicAdd(&bar[0], 1u) == expected - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicExch(&bar[1], want);
    } else {
      const unsigned long long t0 = global_ns();
      while (*(volatile unsigned*)&bar[1] != want) {
        if (*(volatile double*)status != 0.0 || (long long)(global_ns() - t0) > limit_ns) {
          *(volatile double*)status = 1.0;
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();   // the other blocks' results are read after the barrier
    gen = want;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Shared-memory rows of the tail (k_vcycle_tail_sm, FP32 levels).  A row's
// stencil sum takes its blocks from shared memory (sA: block b of local row
// lr at sA[b * rows + lr]) and gathers all its x values first, then sums the
// blocks in stencil order with blk_acc: the values of stencil_sum_batched.
// x is read with ordinary (coherent) loads: other CTAs of the cluster wrote it
// in earlier phases.
template <int NB>
__device__ __forceinline__ void sm_row_sum(const LevelOp& L, const float4* __restrict__ sA, int rows, int lr,
                                           int64_t p, int par, const float2* x, bool skip_centre,
                                           uint32_t skipmask, float& s0, float& s1) {
  constexpr int C = NB == 27 ? 13 : 4;
  float2 xv[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (!((skip_centre && b == C) || ((skipmask >> b) & 1u))) xv[b] = x[p + (par ? L.nb.off[1][b] : L.nb.off[0][b])];
  float a0 = 0.f, a1 = 0.f;
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if ((skip_centre && b == C) || ((skipmask >> b) & 1u)) continue;
    const float4 a = sA[b * rows + lr];
    a0 = blk_acc(a0, a.x, a.y, xv[b]);
    a1 = blk_acc(a1, a.z, a.w, xv[b]);
  }
  s0 = a0;
  s1 = a1;
}

// The line owned as item i by CTA `rank` of a cluster of cs CTAs.
__device__ __forceinline__ int sm_line(int rank, int cs, int i) { return rank + cs * i; }

// The V-cycle below level P.first; sync() separates phases and returns false
// when the launch must end (coop: a barrier gave up).  SM: the shared-memory
// form (FP32 levels, GS smoother; sm holds this CTA's rows, rank is its rank
// in the cluster), whose GS and residual phases update the vertices of the
// CTA's own x-lines.
template <int KIND, int NB, bool SM = false, typename Sync>
__device__ __forceinline__ void vcycle_tail_body(const TailParams& P, int64_t gt, int64_t nthr, Sync&& sync,
                                                 const float4* sm = nullptr, int rank = 0) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  // batched stencil loads (a thread's round trips set a phase's time); FP64
  // blocks three at a time, which keeps the whole V-cycle within the registers
  constexpr int CH = KIND == STORE_F64 ? 3 : chunk_of(KIND);
  const int ncol = 1 << P.L[P.first].op.d.dim;
  V* curs[RF_MAXL];
  auto gs_sweep_sm = [&](int l, const LevelOp& op, const V* b, V* x, bool forward, bool zero_start) {
    const int nx = op.d.nx, ny = op.d.ny, nlines = op.d.ny * (op.d.dim == 3 ? op.d.nz : 1);
    const int rows = P.sm_rows[l];
    const float4* sA = sm + P.sm_base[l];
    const float* sD = reinterpret_cast<const float*>(sA + NB * rows);
    // colour pairs (c, c ^ 1), as in k_gs_pair: the CTA owns whole x-lines,
    // so the pair's second colour waits only for a block barrier and reads
    // its same-line neighbours after it (plain loads); one cluster barrier
    // per pair
    for (int cc = 0; cc < ncol; cc += 2) {
      const int c1 = forward ? cc : ncol - 1 - cc;
#pragma unroll 1
      for (int h = 0; h < 2; ++h) {
        const int col = h ? (c1 ^ 1) : c1;
        const int px = col & 1, py = (col >> 1) & 1, pz = (col >> 2) & 1;
        const int cnt = px ? nx / 2 : (nx + 1) / 2;
        const uint32_t skip = (zero_start && forward) ? P.zmask[col] : 0u;
        const int items = P.sm_lines[l] * cnt;
        for (int t = threadIdx.x; t < items; t += blockDim.x) {
          const int i = t / cnt, pos = t - i * cnt;
          const int Ln = sm_line(rank, P.sm_cs, i);
          if (Ln >= nlines) continue;
          const int k = Ln / ny, j = Ln - k * ny;
          if ((j & 1) != py || (k & 1) != pz) continue;
          const int u = (px ? op.d.E : 0) + pos;
          const int64_t p = (int64_t)Ln * nx + u;
          const int lr = i * nx + u;
          const float2 bv = ((const float2*)b)[p];
          float s0, s1;
          sm_row_sum<NB>(op, sA, rows, lr, p, px, (const float2*)x, true, skip, s0, s1);
          const float r0 = bv.x - s0, r1 = bv.y - s1;   // coarse level: A_pq as stored
          float y0, y1;
          dinv_apply<float>(sD, lr, r0, r1, y0, y1);
          ((float2*)x)[p] = make_float2(y0, y1);
        }
        if (h == 0) __syncthreads();
      }
      if (!sync()) return false;
    }
    return true;
  };
  auto gs_sweep = [&](const LevelOp& op, const V* b, V* x, bool forward, bool zero_start) {
    for (int cc = 0; cc < ncol; ++cc) {
      const int col = forward ? cc : ncol - 1 - cc;
      const int px = col & 1, py = (col >> 1) & 1, pz = (col >> 2) & 1;
      const int cnt_x = px ? op.d.nx / 2 : (op.d.nx + 1) / 2;
      const int lines_y = (op.d.ny - py + 1) / 2;
      const int lines_z = op.d.dim == 3 ? (op.d.nz - pz + 1) / 2 : 1;
      const int64_t count = (int64_t)cnt_x * lines_y * lines_z;
      const uint32_t skip = (zero_start && forward) ? P.zmask[col] : 0u;
      for (int64_t t = gt; t < count; t += nthr) gs_point<KIND, false, NB, CH>(op, b, x, px, py, pz, cnt_x, lines_y, t, skip);
      if (!sync()) return false;
    }
    return true;
  };
  auto jacobi_sweep = [&](const LevelOp& op, const V* b, const V* xin, V* xout, bool zero_x) {
    for (int64_t p = gt; p < op.d.nv; p += nthr) jacobi_point<KIND, false, NB, CH>(op, b, xin, xout, P.omega, zero_x, p);
    return sync();
  };
  for (int l = P.first; l < P.coarsest; ++l) {
    const TailLevel& Lv = P.L[l];
    const TailLevel& Lc = P.L[l + 1];
    const V* b = (const V*)Lv.b;
    V* x = (V*)Lv.x;
    V* tmp = (V*)Lv.t;
    V* cur = x;
    if (P.smoother == 1) {
      for (int sw = 0; sw < P.nu1; ++sw) {
        if constexpr (SM) {
          if (!gs_sweep_sm(l, Lv.op, b, x, true, sw == 0)) return;
        } else {
          if (!gs_sweep(Lv.op, b, x, true, sw == 0)) return;
        }
      }
    } else {
      V* first = ((P.nu1 + P.nu2) & 1) ? x : tmp;
      if (!jacobi_sweep(Lv.op, b, nullptr, first, true)) return;
      cur = first;
      for (int sw = 1; sw < P.nu1; ++sw) {
        V* dst = (cur == x) ? tmp : x;
        if (!jacobi_sweep(Lv.op, b, cur, dst, false)) return;
        cur = dst;
      }
    }
    curs[l] = cur;
    if constexpr (SM) {
      const int nx = Lv.op.d.nx, nlines = Lv.op.d.ny * (Lv.op.d.dim == 3 ? Lv.op.d.nz : 1);
      const int rows = P.sm_rows[l];
      const float4* sA = sm + P.sm_base[l];
      for (int t = threadIdx.x; t < rows; t += blockDim.x) {
        const int i = t / nx, u = t - i * nx;
        const int Ln = sm_line(rank, P.sm_cs, i);
        if (Ln >= nlines) continue;
        const int64_t p = (int64_t)Ln * nx + u;
        const float2 bv = ((const float2*)b)[p];
        float s0, s1;
        sm_row_sum<NB>(Lv.op, sA, rows, t, p, u >= Lv.op.d.E, (const float2*)cur, false, 0u, s0, s1);
        ((float2*)Lv.r)[p] = make_float2(bv.x - s0, bv.y - s1);
      }
    } else {
      for (int64_t p = gt; p < Lv.op.d.nv; p += nthr) residual_point<KIND, false, NB, CH>(Lv.op, b, cur, (V*)Lv.r, p);
    }
    if (!sync()) return;
    for (int64_t p = gt; p < Lc.op.d.nv; p += nthr)
      restrict_point<T>(Lv.op.d, Lc.op.d, Lv.op.dmask, Lc.op.dmask, (const V*)Lv.r, (V*)Lc.b, p);
    if (!sync()) return;
  }
  {
    // x = A^-1 b on the coarsest level, one warp per row with lanes over the
    // columns and the xor-shuffle sum of coarse_solve_body: the same values
    // as the coarse-solve kernel, so the tail equals the V-cycle of
    // one launch per phase bit for bit
    const T* bc = (const T*)P.L[P.coarsest].b;
    T* xc = (T*)P.L[P.coarsest].x;
    const int lane = (int)(gt & 31);
    for (int64_t r = gt >> 5; r < P.N; r += nthr >> 5) {   // uniform per warp: nthr is a multiple of 32
      const double* row = P.Ainv + r * P.N;
      double s = 0.0;
      for (int c = lane; c < P.N; c += 32) s += row[c] * (double)bc[c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) xc[r] = (T)s;
    }
    if (!sync()) return;
  }
  for (int l = P.coarsest - 1; l >= P.first; --l) {
    const TailLevel& Lv = P.L[l];
    const TailLevel& Lc = P.L[l + 1];
    const V* b = (const V*)Lv.b;
    V* x = (V*)Lv.x;
    V* tmp = (V*)Lv.t;
    V* cur = curs[l];
    for (int64_t p = gt; p < Lv.op.d.nv; p += nthr)
      prolong_point<T>(Lv.op.d, Lc.op.d, Lv.op.dmask, Lc.op.dmask, (const V*)Lc.x, cur, p);
    if (!sync()) return;
    if (P.smoother == 1) {
      for (int sw = 0; sw < P.nu2; ++sw) {
        if constexpr (SM) {
          if (!gs_sweep_sm(l, Lv.op, b, x, false, false)) return;
        } else {
          if (!gs_sweep(Lv.op, b, x, false, false)) return;
        }
      }
    } else {
      for (int sw = 0; sw < P.nu2; ++sw) {
        V* dst = (cur == x) ? tmp : x;
        if (!jacobi_sweep(Lv.op, b, cur, dst, false)) return;
        cur = dst;
      }
    }
  }
}

template <int KIND, int NB>
__global__ void __launch_bounds__(TAIL_THREADS) k_vcycle_tail(const __grid_constant__ TailParams P) {
  cg::cluster_group cl = cg::this_cluster();
  const int64_t nthr = (int64_t)cl.num_blocks() * blockDim.x;
  const int64_t gt = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x;
  vcycle_tail_body<KIND, NB>(P, gt, nthr, [&]() {
    cl.sync();
    return true;
  });
}

// The tail with the levels' matrices in shared memory: each CTA of the
// cluster first copies the stencil blocks and D^-1 of its own x-lines
// (cp.async, 16 bytes per copy; the matrices are not written during the
// launch), then runs the V-cycle.  Its GS colour phases read no matrix data
// from L2 or HBM, only the x values around each vertex.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int NB>
__global__ void __launch_bounds__(TAIL_THREADS) k_vcycle_tail_sm(const __grid_constant__ TailParams P) {
  extern __shared__ float4 tail_sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  for (int l = P.first; l < P.coarsest; ++l) {
    const LevelOp& op = P.L[l].op;
    const int nx = op.d.nx, nlines = op.d.ny * (op.d.dim == 3 ? op.d.nz : 1);
    const int rows = P.sm_rows[l], items = (NB + 1) * rows;
    float4* dst = tail_sm + P.sm_base[l];
    const float4* A = reinterpret_cast<const float4*>(op.A);
    const float4* D = reinterpret_cast<const float4*>(op.Dinv);
    for (int t = threadIdx.x; t < items; t += blockDim.x) {
      const int b = t / rows, lr = t - b * rows;
      const int i = lr / nx, u = lr - i * nx;
      const int Ln = sm_line(rank, P.sm_cs, i);
      if (Ln >= nlines) continue;
      const int64_t p = (int64_t)Ln * nx + u;
      cp_async16(dst + t, b < NB ? A + (int64_t)b * op.d.nv + p : D + p);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int64_t nthr = (int64_t)cl.num_blocks() * blockDim.x;
  const int64_t gt = (int64_t)rank * blockDim.x + threadIdx.x;
  vcycle_tail_body<STORE_F32, NB, true>(
      P, gt, nthr,
      [&]() {
        cl.sync();
        return true;
      },
      tail_sm, rank);
}

template <int KIND, int NB>
__global__ void __launch_bounds__(TAIL_THREADS) k_vcycle_coop(const __grid_constant__ TailParams P) {
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned gen = 0;
  if (threadIdx.x == 0) gen = *(volatile unsigned*)&P.bar[1];   // cannot move before every block has read it
  vcycle_tail_body<KIND, NB>(P, gt, nthr, [&]() { return grid_sync_bounded(P.bar, gridDim.x, gen, P.status, P.limit_ns); });
}

// `rounds` bounded grid barriers expecting `gridDim.x + extra` arrivals (a
// check of the barrier: with extra > 0 every wait gives up after limit_ns).
__global__ void __launch_bounds__(256) k_barrier_check(unsigned* bar, int rounds, int extra, double* status,
                                                      long long limit_ns, unsigned* passed) {
  unsigned gen = 0;
  if (threadIdx.x == 0) gen = *(volatile unsigned*)&bar[1];
  for (int r = 0; r < rounds; ++r) {
    if (!grid_sync_bounded(bar, gridDim.x + (unsigned)extra, gen, status, limit_ns)) return;
    if (threadIdx.x == 0) atomicAdd(passed, 1u);
  }
}

template <typename K>
static int coop_blocks(K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * num_sms();
}

template <typename K, typename... A>
static cudaError_t coop_launch(K kernel, int blocks, int threads, void* s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = (cudaStream_t)s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launch();
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

int coop_tail_blocks(int kind, int nb) {
  if (nb == 27) {
    if (kind == STORE_F64) return coop_blocks(k_vcycle_coop<STORE_F64, 27>, TAIL_THREADS);
    if (kind == STORE_F32) return coop_blocks(k_vcycle_coop<STORE_F32, 27>, TAIL_THREADS);
    return coop_blocks(k_vcycle_coop<STORE_F16, 27>, TAIL_THREADS);
  }
  if (kind == STORE_F64) return coop_blocks(k_vcycle_coop<STORE_F64, 9>, TAIL_THREADS);
  if (kind == STORE_F32) return coop_blocks(k_vcycle_coop<STORE_F32, 9>, TAIL_THREADS);
  return coop_blocks(k_vcycle_coop<STORE_F16, 9>, TAIL_THREADS);
}

cudaError_t launch_vcycle_coop(const TailParams& P, int kind, int nb, int blocks, void* s) {
  if (nb == 27) {
    if (kind == STORE_F64) return coop_launch(k_vcycle_coop<STORE_F64, 27>, blocks, TAIL_THREADS, s, P);
    if (kind == STORE_F32) return coop_launch(k_vcycle_coop<STORE_F32, 27>, blocks, TAIL_THREADS, s, P);
    return coop_launch(k_vcycle_coop<STORE_F16, 27>, blocks, TAIL_THREADS, s, P);
  }
  if (kind == STORE_F64) return coop_launch(k_vcycle_coop<STORE_F64, 9>, blocks, TAIL_THREADS, s, P);
  if (kind == STORE_F32) return coop_launch(k_vcycle_coop<STORE_F32, 9>, blocks, TAIL_THREADS, s, P);
  return coop_launch(k_vcycle_coop<STORE_F16, 9>, blocks, TAIL_THREADS, s, P);
}

cudaError_t launch_barrier_check(unsigned* bar, int rounds, int extra, double* status, long long limit_ns,
                                 unsigned* passed, int* blocks_out, void* s) {
  const int blocks = coop_blocks(k_barrier_check, 256);
  if (blocks_out) *blocks_out = blocks;
  if (blocks < 1) return cudaErrorInvalidConfiguration;
  return coop_launch(k_barrier_check, blocks, 256, s, bar, rounds, extra, status, limit_ns, passed);
}

static uint32_t zero_start_mask(int dim, int col);

template <int KIND, int NB>
static cudaLaunchConfig_t tail_config(int csize, void* s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize, 1, 1);
  cfg.blockDim = dim3(TAIL_THREADS, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = (cudaStream_t)s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int KIND, int NB>
static cudaError_t tail_launch(const TailParams& P, int csize, void* s) {
  cudaError_t e = cudaFuncSetAttribute(k_vcycle_tail<KIND, NB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tail_config<KIND, NB>(csize, s, attr);
  count_launch();
  return cudaLaunchKernelEx(&cfg, k_vcycle_tail<KIND, NB>, P);
}

template <int KIND, int NB>
static int tail_size_t() {
  cudaFuncSetAttribute(k_vcycle_tail<KIND, NB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  const int sizes[2] = {16, 8};
  for (int q = 0; q < 2; ++q) {
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = tail_config<KIND, NB>(sizes[q], nullptr, attr);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_vcycle_tail<KIND, NB>, &cfg) == cudaSuccess && n >= 1) return sizes[q];
    cudaGetLastError();
  }
  return 0;
}

// largest cluster size (16, else 8) the device can co-schedule for the tail; 0: none
int tail_cluster_size(int kind, int nb) {
  if (nb == 27) return kind == STORE_F64 ? tail_size_t<STORE_F64, 27>() : kind == STORE_F32 ? tail_size_t<STORE_F32, 27>() : tail_size_t<STORE_F16, 27>();
  return kind == STORE_F64 ? tail_size_t<STORE_F64, 9>() : kind == STORE_F32 ? tail_size_t<STORE_F32, 9>() : tail_size_t<STORE_F16, 9>();
}

void fill_tail_masks(TailParams& P, int dim) {
  for (int c = 0; c < 8; ++c) P.zmask[c] = c < (1 << dim) ? zero_start_mask(dim, c) : 0u;
}

template <int NB>
static cudaLaunchConfig_t tail_sm_config(int csize, int bytes, void* s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = tail_config<STORE_F32, NB>(csize, s, attr);
  cfg.dynamicSmemBytes = (size_t)bytes;
  return cfg;
}

// The kernel's dynamic shared-memory cap is set to the device's opt-in
// maximum, not to this plan's size: grids of different sizes share the
// kernel, and each launch passes its own size.
template <int NB>
static bool tail_sm_fits(int csize, int bytes, int optin) {
  if (cudaFuncSetAttribute(k_vcycle_tail_sm<NB>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(k_vcycle_tail_sm<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tail_sm_config<NB>(csize, bytes, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_vcycle_tail_sm<NB>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

bool tail_sm_plan(TailParams& P, int nb, int csize) {
  P.sm_bytes = 0;
  P.sm_cs = 0;
  if (csize <= 0) return false;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  long long base = 0;
  for (int l = P.first; l < P.coarsest; ++l) {
    const Dims& d = P.L[l].op.d;
    const int nlines = d.ny * (d.dim == 3 ? d.nz : 1);
    P.sm_lines[l] = (nlines + csize - 1) / csize;
    P.sm_rows[l] = P.sm_lines[l] * d.nx;
    P.sm_base[l] = (int)base;
    base += (long long)(nb + 1) * P.sm_rows[l];
  }
  const long long bytes = 16 * base;
  if (bytes <= 0 || bytes > optin) return false;
  if (!(nb == 27 ? tail_sm_fits<27>(csize, (int)bytes, optin) : tail_sm_fits<9>(csize, (int)bytes, optin))) return false;
  P.sm_bytes = (int)bytes;
  P.sm_cs = csize;
  return true;
}

cudaError_t launch_vcycle_tail_sm(const TailParams& P, int nb, void* s) {
  cudaLaunchAttribute attr[1];
  count_launch();
  if (nb == 27) {
    cudaLaunchConfig_t cfg = tail_sm_config<27>(P.sm_cs, P.sm_bytes, s, attr);
    return cudaLaunchKernelEx(&cfg, k_vcycle_tail_sm<27>, P);
  }
  cudaLaunchConfig_t cfg = tail_sm_config<9>(P.sm_cs, P.sm_bytes, s, attr);
  return cudaLaunchKernelEx(&cfg, k_vcycle_tail_sm<9>, P);
}

cudaError_t launch_vcycle_tail(const TailParams& P, int kind, int nb, int csize, void* s) {
  if (nb == 27) {
    if (kind == STORE_F64) return tail_launch<STORE_F64, 27>(P, csize, s);
    if (kind == STORE_F32) return tail_launch<STORE_F32, 27>(P, csize, s);
    return tail_launch<STORE_F16, 27>(P, csize, s);
  }
  if (kind == STORE_F64) return tail_launch<STORE_F64, 9>(P, csize, s);
  if (kind == STORE_F32) return tail_launch<STORE_F32, 9>(P, csize, s);
  return tail_launch<STORE_F16, 9>(P, csize, s);
}

// Galerkin product one axis at a time.  Trilinear P is the tensor product
// P_z P_y P_x of 1D linear interpolations and the Dirichlet masks are diagonal,
// so P_m^T A P_m = D_c P^T (D_f A D_f) P D_c is computed as three 1D
// coarsenings (x, then y, then z): the output grid halves one axis, every
// block offset along that axis becomes a coarse offset, the other offsets stay.
// Output entry (I, D) along the axis = sum over fine rows 2I+a (weight w_a) and
// fine columns 2(I+D)+c (weight w_c), |2D+c-a| <= 1, w_0 = 1, w_+-1 = 1/2.
// The fine masks D_f are applied while reading the first stage, the coarse
// masks D_c (and the identity of coarse Dirichlet rows) when writing the last.
__global__ void __launch_bounds__(256) k_galerkin_axis(int axis, Dims din, const uint8_t* __restrict__ dmf,
                                                       const double* __restrict__ Jin, const double* __restrict__ Min,
                                                       const double2* __restrict__ mdiag, Dims dout,
                                                       const uint8_t* __restrict__ dmc, double* __restrict__ Jout,
                                                       double* __restrict__ Mout) {
  const int nb = dout.nb;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= dout.nv * nb) return;
  const int bo = (int)(t / dout.nv);
  const int64_t po = t - (int64_t)bo * dout.nv;
  int oc[3];
  pcoords(dout, po, oc[0], oc[1], oc[2]);
  int off[3] = {bo % 3 - 1, (bo / 3) % 3 - 1, dout.dim == 3 ? bo / 9 - 1 : 0};
  const int nin[3] = {din.nx, din.ny, din.nz}, nout[3] = {dout.nx, dout.ny, dout.nz};
  const int D = off[axis];
  double j0 = 0, j1 = 0, j2 = 0, j3 = 0, m0 = 0, m1 = 0;
  const int Ic = oc[axis];
  // the column vertex must exist on the output grid
  bool col_ok = Ic + D >= 0 && Ic + D < nout[axis];
  for (int q = 0; q < 3; ++q)
    if (q != axis && (oc[q] + off[q] < 0 || oc[q] + off[q] >= nout[q])) col_ok = false;
  if (col_ok) {
    for (int a = -1; a <= 1; ++a) {
      const int f = 2 * Ic + a;
      if (f < 0 || f >= nin[axis]) continue;
      int rc[3] = {oc[0], oc[1], oc[2]};
      rc[axis] = f;
      const int64_t pi = pidx(din, rc[0], rc[1], rc[2]);
      const double wa = a ? 0.5 : 1.0;
      const bool mrow = dmf && dmf[pi];
      for (int c = -1; c <= 1; ++c) {
        const int e = 2 * D + c - a;
        if (e < -1 || e > 1) continue;
        const int gcol = 2 * (Ic + D) + c;
        if (gcol < 0 || gcol >= nin[axis]) continue;
        const double w = wa * (c ? 0.5 : 1.0);
        int eo[3] = {off[0], off[1], off[2]};
        eo[axis] = e;
        const int bi = blk_of(din.dim, eo[0], eo[1], eo[2]);
        bool mcol = false;
        if (dmf) {
          int cc[3] = {rc[0] + eo[0], rc[1] + eo[1], rc[2] + eo[2]};
          mcol = dmf[pidx(din, cc[0], cc[1], cc[2])] != 0;
        }
        const double* A = Jin + ((int64_t)bi * din.nv + pi) * 4;
        const double a0 = mrow || mcol ? 0.0 : A[0], a1 = mrow ? 0.0 : A[1], a2 = mcol ? 0.0 : A[2], a3 = A[3];
        j0 += w * a0; j1 += w * a1; j2 += w * a2; j3 += w * a3;
        double s0, s1;
        if (Min) {
          const double* M = Min + ((int64_t)bi * din.nv + pi) * 2;
          s0 = M[0]; s1 = M[1];
        } else {
          const bool centre = eo[0] == 0 && eo[1] == 0 && eo[2] == 0;
          const double2 md = centre ? mdiag[pi] : make_double2(0.0, 0.0);
          s0 = md.x; s1 = md.y;
        }
        m0 += w * (mrow ? 0.0 : s0);
        m1 += w * s1;
      }
    }
    if (dmc) {
      const bool crow = dmc[po] != 0;
      const bool ccol = dmc[pidx(dout, oc[0] + off[0], oc[1] + off[1], oc[2] + off[2])] != 0;
      if (crow) { j0 = 0.0; j1 = 0.0; m0 = 0.0; }
      if (ccol) { j0 = 0.0; j2 = 0.0; }
      if (crow && bo == (dout.dim == 3 ? 13 : 4)) j0 = -1.0;   // Dirichlet row: A = +identity
    }
  }
  double* o = Jout + ((int64_t)bo * dout.nv + po) * 4;
  o[0] = j0; o[1] = j1; o[2] = j2; o[3] = j3;
  double* om = Mout + ((int64_t)bo * dout.nv + po) * 2;
  om[0] = m0; om[1] = m1;
}

void launch_galerkin_axis(int axis, const Dims& din, const uint8_t* dmf, const double* Jin, const double* Min,
                          const double* mdiag, const Dims& dout, const uint8_t* dmc, double* Jout, double* Mout,
                          void* s) {
  const int64_t n = dout.nv * dout.nb;
  RF_LAUNCH(k_galerkin_axis, (int)((n + 255) / 256), 256, 0, s, axis, din, dmf, Jin, Min, (const double2*)mdiag,
            dout, dmc, Jout, Mout);
}

__global__ void k_coarse_mask(Dims df, const uint8_t* __restrict__ dmf, Dims dc, uint8_t* __restrict__ dmc) {
  int64_t pc = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (pc >= dc.nv) return;
  int I, J, K;
  pcoords(dc, pc, I, J, K);
  dmc[pc] = dmf[pidx(df, 2 * I, 2 * J, df.dim == 3 ? 2 * K : 0)];
}

// ----------------------------------------------------------------- packing
// Per vertex: entries of A (coarse: shift*Mc - Jc; fine: J itself) into the
// storage kind, FP16 with one FP32 scale per entry position over the block
// row, and the inverse of the 2x2 diagonal block of A = shift*M - J.
template <int KIND>
__global__ void k_pack(Dims d, bool fine, const double* __restrict__ J, const double* __restrict__ M,
                       const double2* __restrict__ md, double shift, void* __restrict__ Aout,
                       float* __restrict__ scale, typename Ty<KIND>::T* __restrict__ Dinv) {
  typedef typename Ty<KIND>::T T;
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= d.nv) return;
  const int nb = d.nb, C = d.dim == 3 ? 13 : 4;
  if (Aout) {
    double mx[4] = {0, 0, 0, 0};
    for (int b = 0; b < nb; ++b) {
      const double* a = J + ((int64_t)b * d.nv + p) * 4;
      double e[4] = {a[0], a[1], a[2], a[3]};
      if (!fine) {
        const double* m = M + ((int64_t)b * d.nv + p) * 2;
        e[0] = -e[0]; e[1] = shift * m[0] - e[1]; e[2] = -e[2]; e[3] = shift * m[1] - e[3];
      }
      if (KIND == STORE_F16) {
        for (int q = 0; q < 4; ++q) mx[q] = fmax(mx[q], fabs(e[q]));
      } else {
        typename Ty<KIND>::S* o = reinterpret_cast<typename Ty<KIND>::S*>(Aout) + ((int64_t)b * d.nv + p) * 4;
        for (int q = 0; q < 4; ++q) o[q] = (typename Ty<KIND>::S)e[q];
      }
    }
    if (KIND == STORE_F16) {
      // A position whose largest magnitude is below the smallest normal float
      // holds only entries that FP32 arithmetic flushes anyway: scale 1, entries 0.
      float sc[4];
      for (int q = 0; q < 4; ++q) sc[q] = mx[q] >= 1.17549435e-38 ? (float)mx[q] : 1.0f;
      reinterpret_cast<float4*>(scale)[p] = make_float4(sc[0], sc[1], sc[2], sc[3]);
      for (int b = 0; b < nb; ++b) {
        const double* a = J + ((int64_t)b * d.nv + p) * 4;
        double e[4] = {a[0], a[1], a[2], a[3]};
        if (!fine) {
          const double* m = M + ((int64_t)b * d.nv + p) * 2;
          e[0] = -e[0]; e[1] = shift * m[0] - e[1]; e[2] = -e[2]; e[3] = shift * m[1] - e[3];
        }
        const int sl = f16_slot_of_block(nb, b);   // paired layout, see stencil_sum_f16
        __half* o = reinterpret_cast<__half*>(Aout) + (((int64_t)(sl >> 1) * d.nv + p) * 2 + (sl & 1)) * 4;
        for (int q = 0; q < 4; ++q) o[q] = __double2half(e[q] / (double)sc[q]);
      }
      if (nb & 1) {   // the empty slot
        __half* o = reinterpret_cast<__half*>(Aout) + (((int64_t)(nb >> 1) * d.nv + p) * 2 + 1) * 4;
        for (int q = 0; q < 4; ++q) o[q] = __float2half(0.f);
      }
    }
  }
  if (Dinv) {
    // diagonal block of A in FP64
    const double* a = J + ((int64_t)C * d.nv + p) * 4;
    double A00, A01, A10, A11;
    if (fine) {
      const double2 m = md[p];
      A00 = -a[0]; A01 = shift * m.x - a[1]; A10 = -a[2]; A11 = shift * m.y - a[3];
    } else {
      const double* m = M + ((int64_t)C * d.nv + p) * 2;
      A00 = -a[0]; A01 = shift * m[0] - a[1]; A10 = -a[2]; A11 = shift * m[1] - a[3];
    }
    const double det = A00 * A11 - A01 * A10;
    T* o = Dinv + p * 4;
    o[0] = (T)(A11 / det); o[1] = (T)(-A01 / det); o[2] = (T)(-A10 / det); o[3] = (T)(A00 / det);
  }
}

// dense coarsest matrix, rows/cols in parity-split unknown order 2p+alpha
__global__ void k_dense(Dims d, Nbr nb, const double* __restrict__ J, const double* __restrict__ M,
                        const double2* __restrict__ md, bool fine, double shift, double* __restrict__ D) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= d.nv * d.nb) return;
  const int b = (int)(t % d.nb);
  const int64_t p = t / d.nb;
  int i, j, k;
  pcoords(d, p, i, j, k);
  const int dx = b % 3 - 1, dy = (b / 3) % 3 - 1, dz = d.dim == 3 ? b / 9 - 1 : 0;
  const int ii = i + dx, jj = j + dy, kk = k + dz;
  if (ii < 0 || ii >= d.nx || jj < 0 || jj >= d.ny || kk < 0 || kk >= d.nz) return;
  const int64_t q = pidx(d, ii, jj, kk);
  const int64_t N = 2 * d.nv;
  const double* a = J + ((int64_t)b * d.nv + p) * 4;
  double e0 = -a[0], e1 = -a[1], e2 = -a[2], e3 = -a[3];
  const int C = d.dim == 3 ? 13 : 4;
  if (fine) {
    if (b == C) { e1 += shift * md[p].x; e3 += shift * md[p].y; }
  } else {
    const double* m = M + ((int64_t)b * d.nv + p) * 2;
    e1 += shift * m[0];
    e3 += shift * m[1];
  }
  D[(2 * p) * N + 2 * q] = e0;
  D[(2 * p) * N + 2 * q + 1] = e1;
  D[(2 * p + 1) * N + 2 * q] = e2;
  D[(2 * p + 1) * N + 2 * q + 1] = e3;
}

// LU with partial pivoting in one CTA (first maximal pivot on ties).  Per
// column: the pivot comes from candidates gathered while the previous column
// was applied; after the row swap the pivot row (from c on) and the column's
// multipliers go to shared memory, so the trailing update is a loop of
// independent loads and stores (warps over rows, lanes over columns) with no
// per-row dependency chain; the thread that updates column c+1 of a row
// records it as a candidate for the next pivot.  Four barriers per column.
// Dynamic shared memory: 2 N doubles.
__global__ void __launch_bounds__(1024) k_lu(int N, double* __restrict__ D, int* __restrict__ piv,
                                             int* __restrict__ status) {
  // one matrix per block: D, piv, status of matrix blockIdx.x
  D += (int64_t)blockIdx.x * N * N;
  piv += (int64_t)blockIdx.x * N;
  status += blockIdx.x;
  extern __shared__ double lu_sh[];
  double* prow = lu_sh;       // pivot row, columns c..N-1
  double* mult = lu_sh + N;   // multipliers of column c
  __shared__ double sval[32];
  __shared__ int sidx[32];
  __shared__ int sp;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  double best = -1.0;
  int bi = N;
  for (int r = tid; r < N; r += nt) {
    const double v = fabs(D[(int64_t)r * N]);
    if (v > best || (v == best && r < bi)) { best = v; bi = r; }
  }
  for (int c = 0; c < N; ++c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { sval[warp] = best; sidx[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bv = sval[0];
      int bidx = sidx[0];
      for (int w = 1; w < nw; ++w)
        if (sval[w] > bv || (sval[w] == bv && sidx[w] < bidx)) { bv = sval[w]; bidx = sidx[w]; }
      if (!(bv > 0.0) || !isfinite(bv)) { status[0] = 1; bidx = c; }
      sp = bidx;
      piv[c] = bidx;
    }
    __syncthreads();
    const int pr = sp;
    for (int t = tid; t < N; t += nt) {
      const double vc = D[(int64_t)c * N + t], vp = D[(int64_t)pr * N + t];
      if (pr != c) {
        D[(int64_t)c * N + t] = vp;
        D[(int64_t)pr * N + t] = vc;
      }
      if (t >= c) prow[t] = vp;
    }
    __syncthreads();
    const double dc = prow[c];
    for (int r = c + 1 + tid; r < N; r += nt) {
      const double l = (dc != 0.0) ? D[(int64_t)r * N + c] / dc : 0.0;
      // a NaN entry is never picked as pivot (fabs(NaN) > best is false) but
      // reaches the factors through its multiplier: report it
      if (!isfinite(l)) status[0] = 1;
      mult[r] = l;
      D[(int64_t)r * N + c] = l;
    }
    __syncthreads();
    best = -1.0;
    bi = N;
    for (int r = c + 1 + warp; r < N; r += nw) {
      double* Dr = D + (int64_t)r * N;
      const double l = mult[r];
      for (int t = c + 1 + lane; t < N; t += 32) {
        const double v = Dr[t] - l * prow[t];
        Dr[t] = v;
        if (t == c + 1) {
          const double av = fabs(v);
          if (av > best || (av == best && r < bi)) { best = av; bi = r; }
        }
      }
    }
    __syncthreads();
  }
}

// Columns of the inverse from the LU factors, one warp per column: x = P e_col,
// then L y = x and U z = y row by row, each row's dot product over the lanes
// with x kept in shared memory.
__global__ void __launch_bounds__(128) k_lu_inverse_cols(int N, const double* __restrict__ LU,
                                                         const int* __restrict__ piv, InvOut out) {
  // matrix blockIdx.y of the batch
  LU += (int64_t)blockIdx.y * N * N;
  piv += (int64_t)blockIdx.y * N;
  double* __restrict__ Ainv = out.Ainv[blockIdx.y];
  extern __shared__ double xs_all[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * (blockDim.x >> 5) + warp;
  if (col >= N) return;
  double* x = xs_all + (int64_t)warp * N;
  for (int r = lane; r < N; r += 32) x[r] = (r == col) ? 1.0 : 0.0;
  __syncwarp();
  if (lane == 0)
    for (int c = 0; c < N; ++c) {
      const int p = piv[c];
      if (p != c) { const double t = x[c]; x[c] = x[p]; x[p] = t; }
    }
  __syncwarp();
  for (int r = 1; r < N; ++r) {
    const double* Lr = LU + (int64_t)r * N;
    double s = 0.0;
    for (int c = lane; c < r; c += 32) s += Lr[c] * x[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] -= s;
    __syncwarp();
  }
  for (int r = N - 1; r >= 0; --r) {
    const double* Ur = LU + (int64_t)r * N;
    double s = 0.0;
    for (int c = r + 1 + lane; c < N; c += 32) s += Ur[c] * x[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) x[r] = (x[r] - s) / Ur[r];
    __syncwarp();
  }
  for (int r = lane; r < N; r += 32) Ainv[(int64_t)r * N + col] = x[r];
}

// natural-order FP64 export of a level operator
__global__ void k_export(Dims d, bool fine, const double* __restrict__ J, const double* __restrict__ M,
                         const double2* __restrict__ md, double shift, double* __restrict__ out) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= d.nv) return;
  const uint32_t line = (uint32_t)v / (uint32_t)d.nx;   // nv < 2^31
  const int i = (int)((uint32_t)v - line * (uint32_t)d.nx);
  const int64_t p = line * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1));
  const int C = d.dim == 3 ? 13 : 4;
  for (int b = 0; b < d.nb; ++b) {
    const double* a = J + ((int64_t)b * d.nv + p) * 4;
    double e[4] = {-a[0], -a[1], -a[2], -a[3]};
    if (fine) {
      if (b == C && md) { e[1] += shift * md[p].x; e[3] += shift * md[p].y; }
      if (!md) { e[0] = a[0]; e[1] = a[1]; e[2] = a[2]; e[3] = a[3]; }
    } else {
      const double* m = M + ((int64_t)b * d.nv + p) * 2;
      e[1] += shift * m[0];
      e[3] += shift * m[1];
    }
    double* o = out + (v * d.nb + b) * 4;
    o[0] = e[0]; o[1] = e[1]; o[2] = e[2]; o[3] = e[3];
  }
}

// gather the block rows and mass diagonals of listed natural vertices
__global__ void k_gather_rows(Dims d, const double* __restrict__ J, const double2* __restrict__ md,
                              const int64_t* __restrict__ verts, int count, double* __restrict__ Jout,
                              double2* __restrict__ mout) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count * d.nb) return;
  const int r = t / d.nb, b = t % d.nb;
  const int64_t v = verts[r];
  const uint32_t line = (uint32_t)v / (uint32_t)d.nx;   // nv < 2^31
  const int i = (int)((uint32_t)v - line * (uint32_t)d.nx);
  const int64_t p = line * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1));
  const double* a = J + ((int64_t)b * d.nv + p) * 4;
  double* o = Jout + ((int64_t)r * d.nb + b) * 4;
  o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; o[3] = a[3];
  if (b == 0) mout[r] = md[p];
}

void launch_gather_rows(const Dims& d, const double* J, const double* mdiag, const int64_t* verts, int count,
                        double* Jout, double* mout, void* s) {
  const int n = count * d.nb;
  RF_LAUNCH(k_gather_rows, (n + 127) / 128, 128, 0, s, d, J, (const double2*)mdiag, verts, count, Jout,
            (double2*)mout);
}

__global__ void k_cast_f64_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (float)in[t];
}
__global__ void k_cast_f32_f64(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  rf_pdl_begin();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}

// ----------------------------------------------------------------- batched
// Several systems of one level shape per launch (see SysBatch): blockIdx.y
// selects the system, whose operator pointers replace those of L; the point
// functions are the single-system ones, so every value is computed exactly as
// there.
__device__ __forceinline__ bool sys_done(const SysLevel& P) {
  return P.scal != nullptr && P.scal[RF_SCAL_DONE] != 0.0;
}

__device__ __forceinline__ LevelOp sys_op(const LevelOp& L, const SysLevel& P) {
  LevelOp o = L;
  o.A = P.A;
  o.scale = P.scale;
  o.Dinv = P.Dinv;
  o.mdiag = P.mdiag;
  o.shift = P.shift;
  o.dmask = P.dmask;
  return o;
}

template <int KIND, bool FINE, int NB, int CH>
__global__ void __launch_bounds__(CH > 0 ? 256 : 512) k_residual_b(const __grid_constant__ LevelOp L,
                                                                   const __grid_constant__ SysBatch B) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  rf_pdl_begin();
  const SysLevel& P = B.s[blockIdx.y];
  if (sys_done(P)) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= L.d.nv) return;
  residual_point<KIND, FINE, NB, CH>(sys_op(L, P), (const V*)P.in0, (const V*)P.in1, (V*)P.out, p);
}

template <int KIND, bool FINE, int NB, int CH>
__global__ void __launch_bounds__(CH > 0 ? 256 : 512) k_jacobi_b(const __grid_constant__ LevelOp L,
                                                                 const __grid_constant__ SysBatch B, double omega,
                                                                 int zero_x) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  rf_pdl_begin();
  const SysLevel& P = B.s[blockIdx.y];
  if (sys_done(P)) return;
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= L.d.nv) return;
  jacobi_point<KIND, FINE, NB, CH>(sys_op(L, P), (const V*)P.in0, (const V*)P.in1, (V*)P.out, omega, zero_x, p);
}

template <int KIND, bool FINE, int NB, int CH>
__global__ void __launch_bounds__(CH > 0 ? 256 : 512) k_gs_colour_b(const __grid_constant__ LevelOp L,
                                                                    const __grid_constant__ SysBatch B, int px,
                                                                    int py, int pz, int cnt_x, int lines_y,
                                                                    int64_t count, uint32_t skipmask, int reverse) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  rf_pdl_begin();
  const SysLevel& P = B.s[blockIdx.y];
  if (sys_done(P)) return;
  const int64_t bx = reverse ? (int64_t)(gridDim.x - 1 - blockIdx.x) : (int64_t)blockIdx.x;
  const int64_t t = bx * blockDim.x + threadIdx.x;
  if (t >= count) return;
  gs_point<KIND, FINE, NB, CH>(sys_op(L, P), (const V*)P.in0, (V*)P.out, px, py, pz, cnt_x, lines_y, t, skipmask);
}

// k_gs_pair for a batch of systems (blockIdx.y); a block of a converged
// system returns as a whole, before the barrier.
template <int KIND, bool FINE, int NB, int CH, int FPX>
__global__ void __launch_bounds__(GS_PAIR_MAX_THREADS) k_gs_pair_b(const __grid_constant__ LevelOp L,
                                                                    const __grid_constant__ SysBatch B, int py, int pz,
                                                                    int lines_y, int nlines, int lpb,
                                                                    uint32_t skip_first, uint32_t skip_second,
                                                                    int reverse) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  rf_pdl_begin();
  const SysLevel& P = B.s[blockIdx.y];
  if (sys_done(P)) return;
  const LevelOp Ls = sys_op(L, P);
  const V* b = (const V*)P.in0;
  V* x = (V*)P.out;
  const int bx = reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  const int l0 = bx * lpb;
  const int nl = min(lpb, nlines - l0);
  const int v = threadIdx.x;
  {
    const int cnt = FPX ? L.d.nx / 2 : (L.d.nx + 1) / 2;
    if (v < nl * cnt)
      gs_vertex<KIND, FINE, NB, CH, false>(Ls, b, x, FPX, pair_vertex(L.d, l0, v, cnt, FPX, py, pz, lines_y), skip_first);
  }
  __syncthreads();
  {
    const int cnt = FPX ? (L.d.nx + 1) / 2 : L.d.nx / 2;
    if (v < nl * cnt)
      gs_vertex<KIND, FINE, NB, CH, true>(Ls, b, x, 1 - FPX, pair_vertex(L.d, l0, v, cnt, 1 - FPX, py, pz, lines_y), skip_second);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_planes_b(Dims df, Dims dc, const __grid_constant__ SysBatch B) {
  const SysLevel& P = B.s[blockIdx.z];
  // (the single-system kernel, with the system's masks and vectors)
  if (sys_done(P)) {
    rf_pdl_begin();
    return;
  }
  restrict_planes_body<T>(df, dc, P.dmask, P.dmask_c, (const typename V2<T>::t*)P.in0, (typename V2<T>::t*)P.out);
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_planes_b(Dims df, Dims dc, const __grid_constant__ SysBatch B) {
  const SysLevel& P = B.s[blockIdx.z];
  if (sys_done(P)) {
    rf_pdl_begin();
    return;
  }
  prolong_pairs_body<T>(df, dc, P.dmask, P.dmask_c, (const typename V2<T>::t*)P.in0, (typename V2<T>::t*)P.out);
}

template <typename T>
__global__ void __launch_bounds__(256) k_coarse_solve_b(int N, const __grid_constant__ SysBatch B) {
  const SysLevel& P = B.s[blockIdx.y];
  if (sys_done(P)) {
    rf_pdl_begin();
    return;
  }
  coarse_solve_body<T>(N, (const double*)P.A, (const T*)P.in0, (T*)P.out);
}

__global__ void k_cast_f32_f64_b(int64_t n, const __grid_constant__ SysBatch B) {
  rf_pdl_begin();
  const SysLevel& P = B.s[blockIdx.y];
  if (sys_done(P)) return;
  const float* __restrict__ in = (const float*)P.in0;
  double* __restrict__ out = (double*)P.out;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (double)in[t];
}

// Finest level of systems that share J (the LIMEX columns of one step): one
// thread per vertex loads each stencil block once and applies it to the NS
// systems' vectors, each with its own shift (and D^-1).  Per system the sums
// run block by block in the order of stencil_sum with the same expressions,
// so the values equal the single-system kernels' bit for bit.
template <int KIND, int NB, int NS, bool SAME = false>
__device__ __forceinline__ void shared_row(const LevelOp& L, const SysLevel* G, int64_t p, int par, bool skip_centre,
                                           uint32_t skipmask, const bool (&act)[NS],
                                           typename Ty<KIND>::T (&s0)[NS], typename Ty<KIND>::T (&s1)[NS]) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  constexpr int C = NB == 27 ? 13 : 4;
  float4 sc = make_float4(1.f, 1.f, 1.f, 1.f);
  if (KIND == STORE_F16) sc = reinterpret_cast<const float4*>(G[0].scale)[p];
#pragma unroll
  for (int q = 0; q < NS; ++q) { s0[q] = 0; s1[q] = 0; }
  if constexpr (KIND == STORE_F16) {
    // pairs of slots, in the slot order of stencil_sum_f16
    const uint4* __restrict__ A = reinterpret_cast<const uint4*>(G[0].A);
#pragma unroll
    for (int qp = 0; qp < (NB + 1) / 2; ++qp) {
      bool use[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int b = f16_block_of_slot(NB, 2 * qp + h);
        use[h] = b >= 0 && !(skip_centre && b == C) && !((skipmask >> (b >= 0 ? b : 0)) & 1u);
      }
      if (!use[0] && !use[1]) continue;
      const uint4 raw = ld_stream_u4(A + (int64_t)qp * L.d.nv + p);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!use[h]) continue;
        const int b = f16_block_of_slot(NB, 2 * qp + h);
        float a[4];
        f16_half(raw, h, sc, a);
        const int off = par ? L.nb.off[1][b] : L.nb.off[0][b];
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          if (!act[q]) continue;
          const V xv = ld_xn_plain<SAME, NB>((const V*)G[q].in1 + p + off, b);
          s0[q] = blk_acc(s0[q], a[0], a[1], xv);
          s1[q] = blk_acc(s1[q], a[2], a[3], xv);
        }
      }
    }
    return;
  }
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (skip_centre && b == C) continue;
    if ((skipmask >> b) & 1u) continue;
    T a[4];
    load_block<KIND>(G[0].A, L.d.nv, b, p, sc, a);
    const int off = par ? L.nb.off[1][b] : L.nb.off[0][b];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      if (!act[q]) continue;
      const V xv = ld_xn_plain<SAME, NB>((const V*)G[q].in1 + p + off, b);
      s0[q] = blk_acc(s0[q], a[0], a[1], xv);
      s1[q] = blk_acc(s1[q], a[2], a[3], xv);
    }
  }
}

template <int KIND, int NB, int NS>
__global__ void __launch_bounds__(256) k_residual_shared(const __grid_constant__ LevelOp L,
                                                         const __grid_constant__ SysBatch B) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  rf_pdl_begin();
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= L.d.nv) return;
  const SysLevel* G = B.s + blockIdx.y * NS;   // this group's systems (one shared matrix)
  bool act[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) act[q] = !sys_done(G[q]);
  const int par = (int)((uint32_t)p % (uint32_t)L.d.nx) >= L.d.E;   // nv < 2^31
  T s0[NS], s1[NS];
  shared_row<KIND, NB, NS>(L, G, p, par, false, L.nomask, act, s0, s1);
  const double2 m = reinterpret_cast<const double2*>(G[0].mdiag)[p];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    if (!act[q]) continue;
    const V* x = (const V*)G[q].in1;
    const T xs = x[p].y, sh = (T)G[q].shift;
    const T a0 = (T)(sh * (T)m.x) * xs - s0[q];
    const T a1 = (T)(sh * (T)m.y) * xs - s1[q];
    const V bv = ((const V*)G[q].in0)[p];
    V o;
    o.x = bv.x - a0;
    o.y = bv.y - a1;
    ((V*)G[q].out)[p] = o;
  }
}

template <int KIND, int NB, int NS>
__global__ void __launch_bounds__(256) k_jacobi_shared(const __grid_constant__ LevelOp L,
                                                       const __grid_constant__ SysBatch B, double omega, int zero_x) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  rf_pdl_begin();
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= L.d.nv) return;
  const SysLevel* G = B.s + blockIdx.y * NS;   // this group's systems (one shared matrix)
  bool act[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) act[q] = !sys_done(G[q]);
  T s0[NS], s1[NS];
  if (!zero_x) {
    const int par = (int)((uint32_t)p % (uint32_t)L.d.nx) >= L.d.E;   // nv < 2^31
    shared_row<KIND, NB, NS>(L, G, p, par, false, L.nomask, act, s0, s1);
  }
  const double2 m = reinterpret_cast<const double2*>(G[0].mdiag)[p];
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    if (!act[q]) continue;
    const V bv = ((const V*)G[q].in0)[p];
    T r0 = bv.x, r1 = bv.y, x0 = 0, x1 = 0;
    if (!zero_x) {
      const V* x = (const V*)G[q].in1;
      const T xs = x[p].y, sh = (T)G[q].shift;
      const T a0 = (T)(sh * (T)m.x) * xs - s0[q];
      const T a1 = (T)(sh * (T)m.y) * xs - s1[q];
      r0 -= a0;
      r1 -= a1;
      x0 = x[p].x;
      x1 = x[p].y;
    }
    T y0, y1;
    dinv_apply<T>(reinterpret_cast<const T*>(G[q].Dinv), p, r0, r1, y0, y1);
    V o;
    o.x = x0 + (T)omega * y0;
    o.y = x1 + (T)omega * y1;
    ((V*)G[q].out)[p] = o;
  }
}

// One vertex p (x parity px) of a GS colour for a group of systems that share
// the finest level's matrix.
template <int KIND, int NB, int NS, bool SAME = false>
__device__ __forceinline__ void gs_shared_vertex(const LevelOp& L, const SysLevel* G, int64_t p, int px,
                                                 uint32_t skipmask, const bool (&act)[NS]) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  T s0[NS], s1[NS];
  shared_row<KIND, NB, NS, SAME>(L, G, p, px, true, skipmask, act, s0, s1);
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    if (!act[q]) continue;
    const V bv = ((const V*)G[q].in0)[p];
    const T r0 = bv.x + s0[q];   // fine level: A_pq = -J_pq off the diagonal
    const T r1 = bv.y + s1[q];
    T y0, y1;
    dinv_apply<T>(reinterpret_cast<const T*>(G[q].Dinv), p, r0, r1, y0, y1);
    V o;
    o.x = y0;
    o.y = y1;
    ((V*)G[q].out)[p] = o;
  }
}

template <int KIND, int NB, int NS>
__global__ void __launch_bounds__(256) k_gs_colour_shared(const __grid_constant__ LevelOp L,
                                                          const __grid_constant__ SysBatch B, int px, int py, int pz,
                                                          int cnt_x, int lines_y, int64_t count, uint32_t skipmask,
                                                          int reverse) {
  typedef typename Ty<KIND>::T T;
  typedef typename V2<T>::t V;
  rf_pdl_begin();
  const int64_t bx = reverse ? (int64_t)(gridDim.x - 1 - blockIdx.x) : (int64_t)blockIdx.x;
  const int64_t t = bx * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const SysLevel* G = B.s + blockIdx.y * NS;   // this group's systems (one shared matrix)
  bool act[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) act[q] = !sys_done(G[q]);
  // 32-bit index arithmetic: a colour has fewer than 2^31 vertices
  const uint32_t tt = (uint32_t)t, line = tt / (uint32_t)cnt_x, kl = line / (uint32_t)lines_y;
  const int pos = (int)(tt - line * (uint32_t)cnt_x);
  const int jj = (int)(line - kl * (uint32_t)lines_y), kk = (int)kl;
  const int j = 2 * jj + py, k = 2 * kk + pz;
  const int64_t p = ((int64_t)j + (int64_t)L.d.ny * k) * L.d.nx + (px ? L.d.E : 0) + pos;
  gs_shared_vertex<KIND, NB, NS>(L, G, p, px, skipmask, act);
}

// k_gs_pair for groups of NS systems that share one matrix (blockIdx.y: group).
template <int KIND, int NB, int NS, int FPX>
__global__ void __launch_bounds__(GS_PAIR_MAX_THREADS) k_gs_pair_shared(const __grid_constant__ LevelOp L,
                                                                         const __grid_constant__ SysBatch B, int py,
                                                                         int pz, int lines_y, int nlines, int lpb,
                                                                         uint32_t skip_first, uint32_t skip_second,
                                                                         int reverse) {
  rf_pdl_begin();
  const SysLevel* G = B.s + blockIdx.y * NS;
  bool act[NS];
#pragma unroll
  for (int q = 0; q < NS; ++q) act[q] = !sys_done(G[q]);
  const int bx = reverse ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
  const int l0 = bx * lpb;
  const int nl = min(lpb, nlines - l0);
  const int v = threadIdx.x;
  {
    const int cnt = FPX ? L.d.nx / 2 : (L.d.nx + 1) / 2;
    if (v < nl * cnt)
      gs_shared_vertex<KIND, NB, NS, false>(L, G, pair_vertex(L.d, l0, v, cnt, FPX, py, pz, lines_y), FPX, skip_first, act);
  }
  __syncthreads();
  {
    const int cnt = FPX ? (L.d.nx + 1) / 2 : L.d.nx / 2;
    if (v < nl * cnt)
      gs_shared_vertex<KIND, NB, NS, true>(L, G, pair_vertex(L.d, l0, v, cnt, 1 - FPX, py, pz, lines_y), 1 - FPX,
                                           skip_second, act);
  }
}

// ----------------------------------------------------------------- launchers
template <int KIND, bool FINE>
static void residual_t(const LevelOp& L, const void* b, const void* x, void* r, void* s) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  const int bs = L.block > 0 ? L.block : 256;
  const int g = (int)((L.d.nv + bs - 1) / bs);
  if (L.batched) {
    if (L.d.nb == 27)
      RF_LAUNCH_PDL((k_residual<KIND, FINE, 27, chunk_of(KIND)>), g, bs, 0, s, L, (const V*)b, (const V*)x, (V*)r);
    else
      RF_LAUNCH_PDL((k_residual<KIND, FINE, 9, chunk_of(KIND)>), g, bs, 0, s, L, (const V*)b, (const V*)x, (V*)r);
  } else if (L.d.nb == 27)
    RF_LAUNCH_PDL((k_residual<KIND, FINE, 27, 0>), g, bs, 0, s, L, (const V*)b, (const V*)x, (V*)r);
  else
    RF_LAUNCH_PDL((k_residual<KIND, FINE, 9, 0>), g, bs, 0, s, L, (const V*)b, (const V*)x, (V*)r);
}

template <int KIND, bool FINE>
static void jacobi_t(const LevelOp& L, const void* b, const void* xin, void* xout, double omega, bool zero_x,
                     void* s) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  const int bs = L.block > 0 ? L.block : 256;
  const int g = (int)((L.d.nv + bs - 1) / bs);
  if (L.batched) {
    if (L.d.nb == 27)
      RF_LAUNCH_PDL((k_jacobi<KIND, FINE, 27, chunk_of(KIND)>), g, bs, 0, s, L, (const V*)b, (const V*)xin, (V*)xout, omega, (int)zero_x);
    else
      RF_LAUNCH_PDL((k_jacobi<KIND, FINE, 9, chunk_of(KIND)>), g, bs, 0, s, L, (const V*)b, (const V*)xin, (V*)xout, omega, (int)zero_x);
  } else if (L.d.nb == 27)
    RF_LAUNCH_PDL((k_jacobi<KIND, FINE, 27, 0>), g, bs, 0, s, L, (const V*)b, (const V*)xin, (V*)xout, omega, (int)zero_x);
  else
    RF_LAUNCH_PDL((k_jacobi<KIND, FINE, 9, 0>), g, bs, 0, s, L, (const V*)b, (const V*)xin, (V*)xout, omega, (int)zero_x);
}

// First forward sweep from x = 0: the neighbours of colour c that have a
// higher colour are still zero, so their blocks are neither read nor applied.
static uint32_t zero_start_mask(int dim, int col) {
  uint32_t m = 0;
  const int nb = dim == 3 ? 27 : 9;
  for (int b = 0; b < nb; ++b) {
    const int dx = b % 3 - 1, dy = (b / 3) % 3 - 1, dz = dim == 3 ? b / 9 - 1 : 0;
    const int nc = ((col & 1) ^ (dx & 1)) | ((((col >> 1) & 1) ^ (dy & 1)) << 1) | ((((col >> 2) & 1) ^ (dz & 1)) << 2);
    if (nc > col) m |= 1u << b;
  }
  return m;
}

// Consecutive colour launches of a sweep walk the grid in alternating
// directions (blocks in order, then in reverse order): the vertices a launch
// starts with are the neighbours of those the previous launch ended with, whose
// x values are then still in L2.  The order within a colour changes nothing in
// the results.  `flip` starts a sweep reversed (after a launch that ended at
// the far end); RF_GS_ZIGZAG=0 keeps every launch in order.
static bool gs_zigzag() {
  const char* e = getenv("RF_GS_ZIGZAG");
  return !(e && atoi(e) == 0);
}

// The colour launches of one sweep: launch(px, py, pz, cnt_x, lines_y, count,
// skip, reverse) per colour, in sweep order.
template <typename F>
static void for_colours(const Dims& d, bool forward, bool zero_start, bool flip, F launch) {
  const int ncol = 1 << d.dim;
  const bool zigzag = gs_zigzag();
  int nl = 0;
  for (int cc = 0; cc < ncol; ++cc) {
    const int col = forward ? cc : ncol - 1 - cc;
    const uint32_t skip = (zero_start && forward) ? zero_start_mask(d.dim, col) : 0u;
    const int px = col & 1, py = (col >> 1) & 1, pz = (col >> 2) & 1;
    const int cnt_x = px ? d.nx / 2 : (d.nx + 1) / 2;
    const int lines_y = (d.ny - py + 1) / 2;
    const int lines_z = d.dim == 3 ? (d.nz - pz + 1) / 2 : 1;
    const int64_t count = (int64_t)cnt_x * lines_y * lines_z;
    if (count <= 0) continue;
    const int rev = zigzag ? ((nl + (flip ? 1 : 0)) & 1) : 0;
    ++nl;
    launch(px, py, pz, cnt_x, lines_y, count, skip, rev);
  }
}

// Colour pairs in one launch each (k_gs_pair) on FP32 and FP16 levels;
// RF_GS_PAIRS=0 launches every colour on its own.  Both give bitwise the same
// sweep.
static bool gs_pairs() {
  const char* e = getenv("RF_GS_PAIRS");
  return !(e && atoi(e) == 0);
}

// Lines per block and threads of a pair launch: enough whole warps for the
// longer run of all the block's lines at once (a thread updates one vertex
// of each run), at most GS_PAIR_MAX_THREADS; of these shapes, the one with
// the fewest idle threads over both runs.  Lines longer than
// 2 GS_PAIR_MAX_THREADS - 1 vertices have no shape: their colours are
// launched one by one.
static bool pair_shape(int nx, int& lpb, int& threads) {
  const int e = (nx + 1) / 2, o = nx / 2;
  if (e > GS_PAIR_MAX_THREADS) return false;
  lpb = 1;
  threads = ((e + 31) / 32) * 32;
  double best = -1.0;
  for (int l = 1; l * e <= GS_PAIR_MAX_THREADS; ++l) {
    const int t = ((l * e + 31) / 32) * 32;
    const double eff = (double)l * (e + o) / (2.0 * t);
    if (eff > best + 1e-9) {
      best = eff;
      lpb = l;
      threads = t;
    }
  }
  return true;
}

// The pair launches of one sweep: launch(first_px, py, pz, lines_y, nlines,
// skip_first, skip_second, reverse) per pair, in sweep order.  Colour c =
// px + 2 py + 4 pz, so the pairs are (0,1), (2,3), ... forward and (7,6),
// (5,4), ... backward: the sweep's colour order is unchanged.
template <typename F>
static void for_colour_pairs(const Dims& d, bool forward, bool zero_start, bool flip, F launch) {
  const int ncol = 1 << d.dim;
  const bool zigzag = gs_zigzag();
  int nl = 0;
  for (int cc = 0; cc < ncol; cc += 2) {
    const int c1 = forward ? cc : ncol - 1 - cc;
    const int c2 = c1 ^ 1;
    const uint32_t s1 = (zero_start && forward) ? zero_start_mask(d.dim, c1) : 0u;
    const uint32_t s2 = (zero_start && forward) ? zero_start_mask(d.dim, c2) : 0u;
    const int py = (c1 >> 1) & 1, pz = (c1 >> 2) & 1;
    const int lines_y = (d.ny - py + 1) / 2;
    const int lines_z = d.dim == 3 ? (d.nz - pz + 1) / 2 : 1;
    const int nlines = lines_y * lines_z;
    if (nlines <= 0 || d.nx <= 0) continue;
    const int rev = zigzag ? ((nl + (flip ? 1 : 0)) & 1) : 0;
    ++nl;
    launch(c1 & 1, py, pz, lines_y, nlines, s1, s2, rev);
  }
}

template <int KIND, bool FINE>
static void gs_t(const LevelOp& L, const void* b, void* x, bool forward, bool zero_start, bool flip, void* s) {
  typedef typename V2<typename Ty<KIND>::T>::t V;
  // FP64 levels keep one launch per colour: with pairs the all-FP64 solve
  // measured 3% slower (its fine smoother 6%), and the batched FP64 pair
  // kernel needs 129 registers, one 288-thread block per SM
  int lpb = 1, threads = 32;
  if (KIND != STORE_F64 && gs_pairs() && pair_shape(L.d.nx, lpb, threads)) {
    for_colour_pairs(L.d, forward, zero_start, flip,
                     [&](int fpx, int py, int pz, int lines_y, int nlines, uint32_t s1, uint32_t s2, int rev) {
      const int g = (nlines + lpb - 1) / lpb;
#define RF_PAIR(NBv, CHv, F)                                                                                     \
  RF_LAUNCH_PDL((k_gs_pair<KIND, FINE, NBv, CHv, F>), g, threads, 0, s, L, (const V*)b, (V*)x, py, pz, lines_y, \
                nlines, lpb, s1, s2, rev)
#define RF_PAIR_PX(NBv, CHv) \
  if (fpx) RF_PAIR(NBv, CHv, 1); else RF_PAIR(NBv, CHv, 0)
      if (L.batched) {
        if (L.d.nb == 27) { RF_PAIR_PX(27, chunk_of(KIND)); } else { RF_PAIR_PX(9, chunk_of(KIND)); }
      } else if (L.d.nb == 27) {
        RF_PAIR_PX(27, 0);
      } else {
        RF_PAIR_PX(9, 0);
      }
#undef RF_PAIR_PX
#undef RF_PAIR
    });
    return;
  }
  const int bs = L.block > 0 ? L.block : 256;
  for_colours(L.d, forward, zero_start, flip,
              [&](int px, int py, int pz, int cnt_x, int lines_y, int64_t count, uint32_t skip, int rev) {
    const int g = (int)((count + bs - 1) / bs);
    if (L.batched) {
      if (L.d.nb == 27)
        RF_LAUNCH_PDL((k_gs_colour<KIND, FINE, 27, chunk_of(KIND)>), g, bs, 0, s, L, (const V*)b, (V*)x, px, py, pz, cnt_x, lines_y, count, skip, rev);
      else
        RF_LAUNCH_PDL((k_gs_colour<KIND, FINE, 9, chunk_of(KIND)>), g, bs, 0, s, L, (const V*)b, (V*)x, px, py, pz, cnt_x, lines_y, count, skip, rev);
    } else if (L.d.nb == 27) {
      RF_LAUNCH_PDL((k_gs_colour<KIND, FINE, 27, 0>), g, bs, 0, s, L, (const V*)b, (V*)x, px, py, pz, cnt_x, lines_y, count, skip, rev);
    } else {
      RF_LAUNCH_PDL((k_gs_colour<KIND, FINE, 9, 0>), g, bs, 0, s, L, (const V*)b, (V*)x, px, py, pz, cnt_x, lines_y, count, skip, rev);
    }
  });
}

void launch_residual(const LevelOp& L, const void* b, const void* x, void* r, void* s) {
  switch (L.kind) {
    case STORE_F64: L.fine ? residual_t<STORE_F64, true>(L, b, x, r, s) : residual_t<STORE_F64, false>(L, b, x, r, s); break;
    case STORE_F32: L.fine ? residual_t<STORE_F32, true>(L, b, x, r, s) : residual_t<STORE_F32, false>(L, b, x, r, s); break;
    default: L.fine ? residual_t<STORE_F16, true>(L, b, x, r, s) : residual_t<STORE_F16, false>(L, b, x, r, s); break;
  }
}

void launch_jacobi(const LevelOp& L, const void* b, const void* xin, void* xout, double omega, bool zero_x, void* s) {
  switch (L.kind) {
    case STORE_F64: L.fine ? jacobi_t<STORE_F64, true>(L, b, xin, xout, omega, zero_x, s) : jacobi_t<STORE_F64, false>(L, b, xin, xout, omega, zero_x, s); break;
    case STORE_F32: L.fine ? jacobi_t<STORE_F32, true>(L, b, xin, xout, omega, zero_x, s) : jacobi_t<STORE_F32, false>(L, b, xin, xout, omega, zero_x, s); break;
    default: L.fine ? jacobi_t<STORE_F16, true>(L, b, xin, xout, omega, zero_x, s) : jacobi_t<STORE_F16, false>(L, b, xin, xout, omega, zero_x, s); break;
  }
}

void launch_gs_sweep(const LevelOp& L, const void* b, void* x, bool forward, bool zero_start, void* s, bool flip) {
  switch (L.kind) {
    case STORE_F64: L.fine ? gs_t<STORE_F64, true>(L, b, x, forward, zero_start, flip, s) : gs_t<STORE_F64, false>(L, b, x, forward, zero_start, flip, s); break;
    case STORE_F32: L.fine ? gs_t<STORE_F32, true>(L, b, x, forward, zero_start, flip, s) : gs_t<STORE_F32, false>(L, b, x, forward, zero_start, flip, s); break;
    default: L.fine ? gs_t<STORE_F16, true>(L, b, x, forward, zero_start, flip, s) : gs_t<STORE_F16, false>(L, b, x, forward, zero_start, flip, s); break;
  }
}

// one thread per vertex of the written level: x = its planes' vertices in
// blocks of 256, y = its planes (RF_TRANSFER_POINT=1 selects the per-point
// kernels with a flat grid; read at every launch, so a graph keeps the choice
// made when it was captured)
static bool transfer_point() {
  const char* e = getenv("RF_TRANSFER_POINT");
  return e && atoi(e) == 1;
}

void launch_restrict(const LevelOp& F, const LevelOp& C, const void* rf, void* bc, void* s) {
  if (transfer_point()) {
    const int g = (int)((C.d.nv + 255) / 256);
    if (F.kind == STORE_F64)
      RF_LAUNCH_PDL(k_restrict<double>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const double2*)rf, (double2*)bc);
    else
      RF_LAUNCH_PDL(k_restrict<float>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const float2*)rf, (float2*)bc);
    return;
  }
  const dim3 g((unsigned)((C.d.nx * C.d.ny + 255) / 256), (unsigned)C.d.nz);
  if (F.kind == STORE_F64)
    RF_LAUNCH_PDL(k_restrict_planes<double>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const double2*)rf, (double2*)bc);
  else
    RF_LAUNCH_PDL(k_restrict_planes<float>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const float2*)rf, (float2*)bc);
}

void launch_prolong(const LevelOp& F, const LevelOp& C, const void* xc, void* xf, void* s) {
  if (transfer_point()) {
    const int g = (int)((F.d.nv + 255) / 256);
    if (F.kind == STORE_F64)
      RF_LAUNCH_PDL(k_prolong<double>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const double2*)xc, (double2*)xf);
    else
      RF_LAUNCH_PDL(k_prolong<float>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const float2*)xc, (float2*)xf);
    return;
  }
  const dim3 g((unsigned)((C.d.nx * F.d.ny + 255) / 256), (unsigned)F.d.nz);   // two fine vertices per thread
  if (F.kind == STORE_F64)
    RF_LAUNCH_PDL(k_prolong_planes<double>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const double2*)xc, (double2*)xf);
  else
    RF_LAUNCH_PDL(k_prolong_planes<float>, g, 256, 0, s, F.d, C.d, F.dmask, C.dmask, (const float2*)xc, (float2*)xf);
}

void launch_coarse_solve(const LevelOp& C, const double* Ainv, const void* b, void* x, void* s) {
  const int N = (int)(2 * C.d.nv);
  const int g = (N + 7) / 8;   // 8 rows (warps) per 256-thread block
  const size_t smem = sizeof(double) * N;
  if (C.kind == STORE_F64)
    RF_LAUNCH_PDL(k_coarse_solve<double>, g, 256, smem, s, N, Ainv, (const double*)b, (double*)x);
  else
    RF_LAUNCH_PDL(k_coarse_solve<float>, g, 256, smem, s, N, Ainv, (const float*)b, (float*)x);
}


// ----------------------------------------------------------------- batched launchers
template <int KIND, bool FINE>
static void residual_bt(const LevelOp& L, const SysBatch& B, void* s) {
  const int bs = L.block > 0 ? L.block : 256;
  const dim3 g((unsigned)((L.d.nv + bs - 1) / bs), (unsigned)B.n);
  if (L.batched) {
    if (L.d.nb == 27) RF_LAUNCH_PDL((k_residual_b<KIND, FINE, 27, chunk_of(KIND)>), g, bs, 0, s, L, B);
    else RF_LAUNCH_PDL((k_residual_b<KIND, FINE, 9, chunk_of(KIND)>), g, bs, 0, s, L, B);
  } else if (L.d.nb == 27) {
    RF_LAUNCH_PDL((k_residual_b<KIND, FINE, 27, 0>), g, bs, 0, s, L, B);
  } else {
    RF_LAUNCH_PDL((k_residual_b<KIND, FINE, 9, 0>), g, bs, 0, s, L, B);
  }
}

template <int KIND, bool FINE>
static void jacobi_bt(const LevelOp& L, const SysBatch& B, double omega, bool zero_x, void* s) {
  const int bs = L.block > 0 ? L.block : 256;
  const dim3 g((unsigned)((L.d.nv + bs - 1) / bs), (unsigned)B.n);
  const int zx = zero_x ? 1 : 0;
  if (L.batched) {
    if (L.d.nb == 27) RF_LAUNCH_PDL((k_jacobi_b<KIND, FINE, 27, chunk_of(KIND)>), g, bs, 0, s, L, B, omega, zx);
    else RF_LAUNCH_PDL((k_jacobi_b<KIND, FINE, 9, chunk_of(KIND)>), g, bs, 0, s, L, B, omega, zx);
  } else if (L.d.nb == 27) {
    RF_LAUNCH_PDL((k_jacobi_b<KIND, FINE, 27, 0>), g, bs, 0, s, L, B, omega, zx);
  } else {
    RF_LAUNCH_PDL((k_jacobi_b<KIND, FINE, 9, 0>), g, bs, 0, s, L, B, omega, zx);
  }
}

template <int KIND, bool FINE>
static void gs_bt(const LevelOp& L, const SysBatch& B, bool forward, bool zero_start, bool flip, void* s) {
  int lpb = 1, threads = 32;
  if (KIND != STORE_F64 && gs_pairs() && pair_shape(L.d.nx, lpb, threads)) {   // as in gs_t
    for_colour_pairs(L.d, forward, zero_start, flip,
                     [&](int fpx, int py, int pz, int lines_y, int nlines, uint32_t s1, uint32_t s2, int rev) {
      const dim3 g((unsigned)((nlines + lpb - 1) / lpb), (unsigned)B.n);
#define RF_PAIR(NBv, CHv, F) \
  RF_LAUNCH_PDL((k_gs_pair_b<KIND, FINE, NBv, CHv, F>), g, threads, 0, s, L, B, py, pz, lines_y, nlines, lpb, s1, s2, rev)
#define RF_PAIR_PX(NBv, CHv) \
  if (fpx) RF_PAIR(NBv, CHv, 1); else RF_PAIR(NBv, CHv, 0)
      if (L.batched) {
        if (L.d.nb == 27) { RF_PAIR_PX(27, chunk_of(KIND)); } else { RF_PAIR_PX(9, chunk_of(KIND)); }
      } else if (L.d.nb == 27) {
        RF_PAIR_PX(27, 0);
      } else {
        RF_PAIR_PX(9, 0);
      }
#undef RF_PAIR_PX
#undef RF_PAIR
    });
    return;
  }
  const int bs = L.block > 0 ? L.block : 256;
  for_colours(L.d, forward, zero_start, flip,
              [&](int px, int py, int pz, int cnt_x, int lines_y, int64_t count, uint32_t skip, int rev) {
    const dim3 g((unsigned)((count + bs - 1) / bs), (unsigned)B.n);
    if (L.batched) {
      if (L.d.nb == 27)
        RF_LAUNCH_PDL((k_gs_colour_b<KIND, FINE, 27, chunk_of(KIND)>), g, bs, 0, s, L, B, px, py, pz, cnt_x, lines_y, count, skip, rev);
      else
        RF_LAUNCH_PDL((k_gs_colour_b<KIND, FINE, 9, chunk_of(KIND)>), g, bs, 0, s, L, B, px, py, pz, cnt_x, lines_y, count, skip, rev);
    } else if (L.d.nb == 27) {
      RF_LAUNCH_PDL((k_gs_colour_b<KIND, FINE, 27, 0>), g, bs, 0, s, L, B, px, py, pz, cnt_x, lines_y, count, skip, rev);
    } else {
      RF_LAUNCH_PDL((k_gs_colour_b<KIND, FINE, 9, 0>), g, bs, 0, s, L, B, px, py, pz, cnt_x, lines_y, count, skip, rev);
    }
  });
}

#define RF_KIND_FINE_SWITCH(L, CALL)                                                                  \
  switch ((L).kind) {                                                                                  \
    case STORE_F64: if ((L).fine) CALL(STORE_F64, true); else CALL(STORE_F64, false); break;         \
    case STORE_F32: if ((L).fine) CALL(STORE_F32, true); else CALL(STORE_F32, false); break;         \
    default: if ((L).fine) CALL(STORE_F16, true); else CALL(STORE_F16, false); break;                \
  }

void launch_residual_b(const LevelOp& L, const SysBatch& B, void* s) {
#define RF_CALL(K, F) residual_bt<K, F>(L, B, s)
  RF_KIND_FINE_SWITCH(L, RF_CALL)
#undef RF_CALL
}

void launch_jacobi_b(const LevelOp& L, const SysBatch& B, double omega, bool zero_x, void* s) {
#define RF_CALL(K, F) jacobi_bt<K, F>(L, B, omega, zero_x, s)
  RF_KIND_FINE_SWITCH(L, RF_CALL)
#undef RF_CALL
}

void launch_gs_sweep_b(const LevelOp& L, const SysBatch& B, bool forward, bool zero_start, void* s, bool flip) {
#define RF_CALL(K, F) gs_bt<K, F>(L, B, forward, zero_start, flip, s)
  RF_KIND_FINE_SWITCH(L, RF_CALL)
#undef RF_CALL
}

void launch_restrict_b(const LevelOp& F, const LevelOp& C, const SysBatch& B, void* s) {
  const dim3 g((unsigned)((C.d.nx * C.d.ny + 255) / 256), (unsigned)C.d.nz, (unsigned)B.n);
  if (F.kind == STORE_F64) RF_LAUNCH_PDL(k_restrict_planes_b<double>, g, 256, 0, s, F.d, C.d, B);
  else RF_LAUNCH_PDL(k_restrict_planes_b<float>, g, 256, 0, s, F.d, C.d, B);
}

void launch_prolong_b(const LevelOp& F, const LevelOp& C, const SysBatch& B, void* s) {
  const dim3 g((unsigned)((C.d.nx * F.d.ny + 255) / 256), (unsigned)F.d.nz, (unsigned)B.n);
  if (F.kind == STORE_F64) RF_LAUNCH_PDL(k_prolong_planes_b<double>, g, 256, 0, s, F.d, C.d, B);
  else RF_LAUNCH_PDL(k_prolong_planes_b<float>, g, 256, 0, s, F.d, C.d, B);
}

void launch_coarse_solve_b(const LevelOp& C, const SysBatch& B, void* s) {
  const int N = (int)(2 * C.d.nv);
  const dim3 g((unsigned)((N + 7) / 8), (unsigned)B.n);
  const size_t smem = sizeof(double) * N;
  if (C.kind == STORE_F64) RF_LAUNCH_PDL(k_coarse_solve_b<double>, g, 256, smem, s, N, B);
  else RF_LAUNCH_PDL(k_coarse_solve_b<float>, g, 256, smem, s, N, B);
}

void launch_cast_f32_to_f64_b(int64_t n, const SysBatch& B, void* s) {
  const dim3 g((unsigned)grid_for(n, 256), (unsigned)B.n);
  RF_LAUNCH_PDL(k_cast_f32_f64_b, g, 256, 0, s, n, B);
}

template <int KIND, int NS>
static void residual_sh(const LevelOp& L, const SysBatch& B, void* s) {
  const dim3 g((unsigned)((L.d.nv + 255) / 256), (unsigned)(B.n / NS));
  if (L.d.nb == 27) RF_LAUNCH_PDL((k_residual_shared<KIND, 27, NS>), g, 256, 0, s, L, B);
  else RF_LAUNCH_PDL((k_residual_shared<KIND, 9, NS>), g, 256, 0, s, L, B);
}
template <int KIND, int NS>
static void jacobi_sh(const LevelOp& L, const SysBatch& B, double omega, bool zero_x, void* s) {
  const dim3 g((unsigned)((L.d.nv + 255) / 256), (unsigned)(B.n / NS));
  if (L.d.nb == 27) RF_LAUNCH_PDL((k_jacobi_shared<KIND, 27, NS>), g, 256, 0, s, L, B, omega, zero_x ? 1 : 0);
  else RF_LAUNCH_PDL((k_jacobi_shared<KIND, 9, NS>), g, 256, 0, s, L, B, omega, zero_x ? 1 : 0);
}
template <int KIND, int NS>
static void gs_sh(const LevelOp& L, const SysBatch& B, bool forward, bool zero_start, bool flip, void* s) {
  int lpb = 1, threads = 32;
  if (KIND != STORE_F64 && gs_pairs() && pair_shape(L.d.nx, lpb, threads)) {   // as in gs_t
    for_colour_pairs(L.d, forward, zero_start, flip,
                     [&](int fpx, int py, int pz, int lines_y, int nlines, uint32_t s1, uint32_t s2, int rev) {
      const dim3 g((unsigned)((nlines + lpb - 1) / lpb), (unsigned)(B.n / NS));
#define RF_PAIR(NBv, F) \
  RF_LAUNCH_PDL((k_gs_pair_shared<KIND, NBv, NS, F>), g, threads, 0, s, L, B, py, pz, lines_y, nlines, lpb, s1, s2, rev)
      if (L.d.nb == 27) {
        if (fpx) RF_PAIR(27, 1); else RF_PAIR(27, 0);
      } else {
        if (fpx) RF_PAIR(9, 1); else RF_PAIR(9, 0);
      }
#undef RF_PAIR
    });
    return;
  }
  for_colours(L.d, forward, zero_start, flip,
              [&](int px, int py, int pz, int cnt_x, int lines_y, int64_t count, uint32_t skip, int rev) {
    const dim3 g((unsigned)((count + 255) / 256), (unsigned)(B.n / NS));
    if (L.d.nb == 27)
      RF_LAUNCH_PDL((k_gs_colour_shared<KIND, 27, NS>), g, 256, 0, s, L, B, px, py, pz, cnt_x, lines_y, count, skip, rev);
    else
      RF_LAUNCH_PDL((k_gs_colour_shared<KIND, 9, NS>), g, 256, 0, s, L, B, px, py, pz, cnt_x, lines_y, count, skip, rev);
  });
}

#define RF_KIND_NS_SWITCH(L, NSV, CALL)                                                                    \
  switch ((L).kind * 4 + (NSV) - 1) {                                                                      \
    case 0: CALL(STORE_F64, 1); break; case 1: CALL(STORE_F64, 2); break;                                  \
    case 2: CALL(STORE_F64, 3); break; case 3: CALL(STORE_F64, 4); break;                                  \
    case 4: CALL(STORE_F32, 1); break; case 5: CALL(STORE_F32, 2); break;                                  \
    case 6: CALL(STORE_F32, 3); break; case 7: CALL(STORE_F32, 4); break;                                  \
    case 8: CALL(STORE_F16, 1); break; case 9: CALL(STORE_F16, 2); break;                                  \
    case 10: CALL(STORE_F16, 3); break; default: CALL(STORE_F16, 4); break;                                \
  }

void launch_residual_shared(const LevelOp& L, const SysBatch& B, int share, void* s) {
#define RF_CALL(K, N) residual_sh<K, N>(L, B, s)
  RF_KIND_NS_SWITCH(L, share, RF_CALL)
#undef RF_CALL
}
void launch_jacobi_shared(const LevelOp& L, const SysBatch& B, int share, double omega, bool zero_x, void* s) {
#define RF_CALL(K, N) jacobi_sh<K, N>(L, B, omega, zero_x, s)
  RF_KIND_NS_SWITCH(L, share, RF_CALL)
#undef RF_CALL
}
void launch_gs_sweep_shared(const LevelOp& L, const SysBatch& B, int share, bool forward, bool zero_start, void* s,
                            bool flip) {
#define RF_CALL(K, N) gs_sh<K, N>(L, B, forward, zero_start, flip, s)
  RF_KIND_NS_SWITCH(L, share, RF_CALL)
#undef RF_CALL
}

void launch_coarse_mask(const Dims& df, const uint8_t* dmf, const Dims& dc, uint8_t* dmc, void* s) {
  RF_LAUNCH(k_coarse_mask, (int)((dc.nv + 255) / 256), 256, 0, s, df, dmf, dc, dmc);
}

void launch_pack_level(const Dims& d, bool fine, const double* J, const double* M, const double* mdiag,
                       double shift, int kind, void* A_out, float* scale_out, void* Dinv_out, void* s) {
  const int g = (int)((d.nv + 127) / 128);
  if (kind == STORE_F64)
    RF_LAUNCH(k_pack<STORE_F64>, g, 128, 0, s, d, fine, J, M, (const double2*)mdiag, shift, A_out, scale_out,
              (double*)Dinv_out);
  else if (kind == STORE_F32)
    RF_LAUNCH(k_pack<STORE_F32>, g, 128, 0, s, d, fine, J, M, (const double2*)mdiag, shift, A_out, scale_out,
              (float*)Dinv_out);
  else
    RF_LAUNCH(k_pack<STORE_F16>, g, 128, 0, s, d, fine, J, M, (const double2*)mdiag, shift, A_out, scale_out,
              (float*)Dinv_out);
}

void launch_dense_coarsest(const Dims& d, const Nbr& nb, const double* Jc, const double* Mc,
                           const double* mdiag, bool fine, double shift, double* D, void* s) {
  const int64_t n = d.nv * d.nb;
  RF_LAUNCH(k_dense, (int)((n + 127) / 128), 128, 0, s, d, nb, Jc, Mc, (const double2*)mdiag, fine, shift, D);
}

cudaError_t launch_dense_inverse_batched(int N, int nmat, double* D, double* const* Ainv, int* piv, int* status,
                                         void* s) {
  if (nmat < 1 || nmat > RF_MAXSHIFT) return cudaErrorInvalidValue;
  InvOut out;
  for (int j = 0; j < RF_MAXSHIFT; ++j) out.Ainv[j] = j < nmat ? Ainv[j] : nullptr;
  const size_t lsm = sizeof(double) * 2 * (size_t)N;   // 64 KB at N = 4096
  cudaFuncSetAttribute(k_lu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
  RF_LAUNCH(k_lu, nmat, 1024, lsm, s, N, D, piv, status);
  const size_t smem = sizeof(double) * 4 * (size_t)N;   // 4 warps per block, one x each (128 KB at N = 4096)
  cudaFuncSetAttribute(k_lu_inverse_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  RF_LAUNCH(k_lu_inverse_cols, dim3((N + 3) / 4, nmat), 128, smem, s, N, D, piv, out);
  return cudaGetLastError();
}

cudaError_t launch_dense_inverse(int N, double* D, double* Ainv, int* piv, double* work, int* status, void* s) {
  (void)work;
  return launch_dense_inverse_batched(N, 1, D, &Ainv, piv, status, s);
}

void launch_export_level(const Dims& d, bool fine, const double* J, const double* M, const double* mdiag,
                         double shift, double* A_nat, void* s) {
  RF_LAUNCH(k_export, (int)((d.nv + 127) / 128), 128, 0, s, d, fine, J, M, (const double2*)mdiag, shift, A_nat);
}

void launch_cast_f64_to_f32(const double* in, float* out, int64_t n, void* s) {
  RF_LAUNCH(k_cast_f64_f32, grid_for(n, 256), 256, 0, s, in, out, n);
}
void launch_cast_f32_to_f64(const float* in, double* out, int64_t n, void* s) {
  RF_LAUNCH_PDL(k_cast_f32_f64, grid_for(n, 256), 256, 0, s, in, out, n);
}

}  // namespace rf
