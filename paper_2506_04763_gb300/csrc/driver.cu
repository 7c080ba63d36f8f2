// driver.cu — host side of the C ABI (include/rf.h): grid lifetime, memory,
// the multigrid set-up, the V-cycle schedule, the BiCGSTAB iteration and the
// LIMEX step.  Every arithmetic step on grid data runs in the kernels of
// assemble.cu, levelops.cu and krylov.cu; this file only sequences launches
// and moves scalars (convergence flags, the error estimate) to the host.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "rf.h"
#include "rf_common.cuh"
#include "rf_kernels.h"

namespace rf {

static std::atomic<int64_t> g_launches{0};
// this thread's launches: a graph capture counts its kernels with it, so that
// LIMEX columns capturing on other threads do not add to the count
static thread_local int64_t t_launches = 0;
void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("RF_PDL");
    return !(e && atoi(e) == 0);
  }();
  return on;
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

int grid_for(int64_t n, int block, int max_blocks_per_sm) {
  int64_t b = (n + block - 1) / block;
  int64_t cap = (int64_t)num_sms() * max_blocks_per_sm;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace rf

using namespace rf;

static thread_local std::string t_err;

static rf_status fail(rf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return s;
}

#define CU(call)                                                                        \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(RF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

struct Level {
  Dims d;
  Nbr nb;
  int64_t pad = 0;
  uint8_t* dmask = nullptr;
  double* Jc = nullptr;  // FP64 Galerkin J (levels >= 1)
  double* Mc = nullptr;  // FP64 Galerkin M, S_n column (levels >= 1)
  void* A[RF_MAXSHIFT] = {};
  float* scale[RF_MAXSHIFT] = {};
  void* Dinv[RF_MAXSHIFT] = {};
  void *x = nullptr, *b = nullptr, *r = nullptr, *t = nullptr;
  // Shape of the smoothing / residual kernels (default_shape; the autotuner
  // may change it): threads per block, and whether a thread issues its
  // stencil loads 9 blocks per memory round trip.
  int block = 128;
  bool batched = true;
  // matrix storage of this level (STORE_*): the hierarchy's precision, except
  // that FP16 storage applies to the finest level only and the coarser levels
  // keep FP32 (their sweeps are latency-bound, and FP16 unpacking made them
  // slower: 11.7 -> 17.8 ms of coarse-level time per 257^3 solve)
  int kind = STORE_F64;
};

// Default kernel shape per level, from the autotuner's timings at 257^3 (one
// sweep + one residual per candidate, GB300):
//   FP32 storage: batched loads win everywhere — GS 2.62 -> 2.48 ms on the
//     finest level, about 2x on levels of 65^3 and below (their time is one
//     thread's chain of round trips), equal at 129^3; Jacobi 2.51 -> 2.27 ms
//     on the finest level and 0.32 -> 0.29 ms at 129^3.
//   FP64 storage: equal on the two finest levels, batched 1.2-1.6x faster on
//     the levels below.  (On the finest level of the 65^3 FP64 LIMEX step,
//     batched Jacobi measured no faster either.)
//   FP16 storage (the finest level only, blocks stored in pairs): one pair
//     per round trip, 1.80 ms per sweep + residual against 1.93 ms with two.
static void default_shape(Level& Lv, int l, int kind) {
  Lv.block = 128;
  Lv.batched = kind == STORE_F32 || (kind == STORE_F64 && l >= 2);
}

struct Alloc {
  void* p;
  size_t bytes;
};

struct rf_grid {
  rf_allocator alloc{};
  bool user_alloc = false;
  std::vector<Alloc> bufs;   // lifetime of the grid
  std::vector<Alloc> gbufs;  // lifetime of the multigrid hierarchy
  Dims d;
  Nbr nb;
  PhysParams pp;
  double h[3], g[3];
  int64_t ncell = 0;
  double *Kcell = nullptr, *phi = nullptr, *pd = nullptr;
  uint8_t* law = nullptr;       // per cell k_r law (rf_grid_set_kr_laws), null: Brooks-Corey everywhere
  double* kr_tab = nullptr;     // [RF_MAX_KR_LAWS][6] law table
  bool laws_on = false;
  double vol = 0.0;   // cell volume
  double* ie_old = nullptr;     // implicit Euler: u_old (parity-split pairs), allocated on first use
  double* ie_swold = nullptr;   // implicit Euler, S hat storage: water pore volume sums of u_old
  double* ie_uk = nullptr;      // implicit Euler line search: the Newton iterate before the update
  uint8_t* dir = nullptr;
  double *pw_dir = nullptr, *q_in = nullptr;
  double *pdmin = nullptr, *phiv = nullptr;
  double *J = nullptr, *mdiag = nullptr;
  bool have_J = false;
  double *Se, *pn, *pc, *dpc, *krw, *dkrw;
  double *u_p = nullptr, *F_p = nullptr, *nat_a = nullptr, *nat_b = nullptr;
  // multigrid
  bool gmg_ready = false;
  rf_gmg_opts gopt{};
  int kind = STORE_F64;
  int nshift = 0;
  double shifts[RF_MAXSHIFT] = {};
  int nl = 0;
  Level L[RF_MAXL];
  double* Ainv[RF_MAXSHIFT] = {};
  int tail_first = -1;      // first level run by the one-launch V-cycle tail (-1: none)
  int tail_cs = 0;          // its cluster size (cluster form)
  int tail_blocks = 0;      // its blocks (cooperative form; 0: cluster form)
  unsigned* tail_bar = nullptr;   // the cooperative tail's barrier words
  TailParams tail[RF_MAXSHIFT];
  // Krylov
  KrylovVecs K{};
  double2* b_p = nullptr;
  double* hscal = nullptr;  // pinned host copy of the scalars
  // LIMEX
  double* T = nullptr;
  int T_kappa = 0;
  double* du = nullptr;
  double* norms = nullptr;
  // profiling (rf_profile)
  struct ProfRec { cudaEvent_t a, b; int cls; double bytes; int launches; };
  bool prof_on = false;
  std::vector<ProfRec> prec;
  std::vector<cudaEvent_t> evpool;
  size_t evnext = 0;
  double acc_ms[RF_PROF_NCLASS] = {}, acc_bytes[RF_PROF_NCLASS] = {};
  int64_t acc_launches[RF_PROF_NCLASS] = {};
  // one BiCGSTAB iteration captured as a CUDA graph, per shift and profiling flag
  struct IterGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;                 // kernel launches per replay
    std::vector<ProfRec> recs;           // event pairs recorded by the graph
    std::vector<cudaEvent_t> events;     // owned by the graph
    bool stale = false;                  // the data it points to was reallocated: re-capture before use
  };
  IterGraph ig[RF_MAXSHIFT][2][2];       // [shift][profiling][outer operator]
  // batched solves led by this grid: one captured iteration per batch
  // (its systems, shifts and profiling flag), the gathered scalars
  std::map<std::string, IterGraph> bgraph;
  double* bscal = nullptr;               // device: 16 scalars per system
  double* bscal_h = nullptr;             // pinned host copy (+ the constant 1.0 at [16 * RF_MAXSYS])
  int outer_df = 0;                      // the current solve's RF_OUTER_* mode
  float* Jdf = nullptr;                  // J as FP32 hi/lo pairs (RF_OUTER_DF32)
  bool jdf_valid = false;
  bool capturing = false;
  IterGraph* cap = nullptr;
  cudaStream_t cs = nullptr;             // internal stream for the iteration
  cudaEvent_t join_in = nullptr, join_out = nullptr;
  // LIMEX columns solved concurrently: column j > 0 runs on col[j], a grid
  // that shares this grid's operator data and hierarchy (read-only) and owns
  // its vectors, scratch, streams and graphs (refreshed after each set-up)
  uint64_t hier_gen = 0;                 // incremented by every rf_gmg_setup
  uint64_t gen = ~0ull;                  // (column grids) the hierarchy they mirror
  bool is_column = false;
  rf_grid* col[RF_MAXSHIFT] = {};
  cudaStream_t col_s[RF_MAXSHIFT] = {};  // (column grids) the caller-side stream of the column
};

// ------------------------------------------------------------------ profiling
static cudaEvent_t prof_event(rf_grid* g) {
  if (g->capturing) {                    // events baked into a graph belong to it
    cudaEvent_t e;
    cudaEventCreate(&e);
    g->cap->events.push_back(e);
    return e;
  }
  if (g->evnext < g->evpool.size()) return g->evpool[g->evnext++];
  cudaEvent_t e;
  cudaEventCreate(&e);
  g->evpool.push_back(e);
  g->evnext++;
  return e;
}

static void prof_record(rf_grid* g, cudaEvent_t e, void* s) {
  if (g->capturing) cudaEventRecordWithFlags(e, (cudaStream_t)s, cudaEventRecordExternal);
  else cudaEventRecord(e, (cudaStream_t)s);
}

// Brackets one launch group of class `cls` with events when profiling is on
// (inside a graph capture the events become event-record nodes of the graph).
struct ProfScope {
  rf_grid* g;
  void* s;
  int cls, launches;
  double bytes;
  cudaEvent_t a{};
  bool on;
  ProfScope(rf_grid* g_, void* s_, int cls_, double bytes_, int launches_)
      : g(g_), s(s_), cls(cls_), launches(launches_), bytes(bytes_), on(g_->prof_on) {
    if (on) { a = prof_event(g); prof_record(g, a, s); }
  }
  ~ProfScope() {
    if (!on) return;
    cudaEvent_t b = prof_event(g);
    prof_record(g, b, s);
    (g->capturing ? g->cap->recs : g->prec).push_back({a, b, cls, bytes, launches});
  }
};

static void destroy_graphs(rf_grid* g) {
  for (auto& row : g->ig)
    for (auto& pair : row)
      for (auto& G : pair) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        for (auto e : G.events) cudaEventDestroy(e);
        G = rf_grid::IterGraph();
      }
  for (auto& kv : g->bgraph) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    for (auto e : kv.second.events) cudaEventDestroy(e);
  }
  g->bgraph.clear();
}

// After a new multigrid set-up the captured iterations point to freed data.
// They are kept and marked stale: the next use captures the iteration again
// and updates the instantiated graph in place (cudaGraphExecUpdate; the
// schedule, hence the graph's topology, is the same), which costs far less
// than instantiating it anew.
static void stale_graphs(rf_grid* g) {
  for (auto& row : g->ig)
    for (auto& pair : row)
      for (auto& G : pair) G.stale = G.exec != nullptr;
  for (auto& kv : g->bgraph) kv.second.stale = kv.second.exec != nullptr;
}

// Capture `body` on stream cs into G: a new instantiation, or an in-place
// update of a stale one (falling back to a new instantiation if the update is
// refused).  Kernel launches counted during the capture are taken back (a
// replay counts them).
template <typename Body>
static rf_status capture_graph(rf_grid* owner, rf_grid::IterGraph& G, cudaStream_t cs, const char* what, Body body) {
  std::vector<cudaEvent_t> old_events;
  old_events.swap(G.events);
  G.recs.clear();
  const int64_t c0 = t_launches;
  CU(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  owner->capturing = true;
  owner->cap = &G;
  body();
  owner->capturing = false;
  owner->cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(cs, &graph);
  G.kernels = t_launches - c0;
  g_launches.fetch_sub(G.kernels);
  if (e != cudaSuccess) {
    for (auto ev : old_events) cudaEventDestroy(ev);
    return fail(RF_ECUDA, "%s capture: %s", what, cudaGetErrorString(e));
  }
  if (G.exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(G.exec, graph, &info) != cudaSuccess) {
      cudaGetLastError();
      cudaGraphExecDestroy(G.exec);
      G.exec = nullptr;
    }
  }
  if (!G.exec) {
    e = cudaGraphInstantiate(&G.exec, graph, 0);
    if (e != cudaSuccess) G.exec = nullptr;
  }
  cudaGraphDestroy(graph);
  for (auto ev : old_events) cudaEventDestroy(ev);
  G.stale = false;
  if (!G.exec) return fail(RF_ECUDA, "%s graph: %s", what, cudaGetErrorString(e));
  return RF_OK;
}

// algorithmic bytes of the level kernels (each matrix entry / vector element once)
static double blk_bytes(int kind) { return kind == STORE_F64 ? 32.0 : (kind == STORE_F32 ? 16.0 : 8.0); }
static double tb(int kind) { return kind == STORE_F64 ? 8.0 : 4.0; }
static double row_extra(int kind) { return kind == STORE_F16 ? 16.0 : 0.0; }  // FP16 row scales

// ------------------------------------------------------------------ memory
static void* dalloc(rf_grid* g, size_t bytes, void* stream, bool hierarchy) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  void* p = nullptr;
  if (g->user_alloc) {
    p = g->alloc.alloc(bytes, stream, g->alloc.ctx);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) (hierarchy ? g->gbufs : g->bufs).push_back({p, bytes});
  return p;
}

static void dfree_all(rf_grid* g, std::vector<Alloc>& v, void* stream) {
  for (auto& a : v) {
    if (g->user_alloc) g->alloc.free(a.p, a.bytes, stream, g->alloc.ctx);
    else cudaFree(a.p);
  }
  v.clear();
}

// padded vector of nv pairs of `elem` bytes; returns the interior pointer
static void* dvec(rf_grid* g, const Dims& d, size_t elem, void* stream, bool hierarchy, int64_t* pad_out = nullptr) {
  const int64_t pad = vec_pad(d);
  const size_t bytes = (size_t)(d.nv + 2 * pad) * 2 * elem;
  char* base = (char*)dalloc(g, bytes, stream, hierarchy);
  if (!base) return nullptr;
  if (cudaMemsetAsync(base, 0, bytes, (cudaStream_t)stream) != cudaSuccess) return nullptr;
  if (pad_out) *pad_out = pad;
  return base + (size_t)pad * 2 * elem;
}

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// copy `bytes` from a host or device source into device memory `dst`
static cudaError_t to_device(void* dst, const void* src, size_t bytes, void* stream) {
  return cudaMemcpyAsync(dst, src, bytes, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         (cudaStream_t)stream);
}

// The device's address of page-locked host memory (cudaHostAlloc, or
// cudaHostRegister with mapping), or null for any other pointer.  Kernels
// read and write such memory directly over the CPU-GPU interconnect.
static void* mapped_host_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Host vectors in page-locked memory are permuted by the kernels straight
// from / into the host buffer (RF_HOST_DIRECT=0: staged through device
// memory with cudaMemcpyAsync, as pageable memory always is).
static bool host_direct() {
  static const bool on = [] {
    const char* e = getenv("RF_HOST_DIRECT");
    return !(e && atoi(e) == 0);
  }();
  return on;
}

// natural-order pairs (host or device) -> parity-split device pairs
static rf_status pairs_in(rf_grid* g, const Dims& d, const double* src, double* dst_p, void* s) {
  if (is_device_ptr(src)) {
    launch_perm_to_p(d, src, dst_p, s);
  } else if (void* m = host_direct() ? mapped_host_ptr(src) : nullptr) {
    launch_perm_to_p(d, (const double*)m, dst_p, s);
  } else {
    CU(cudaMemcpyAsync(g->nat_a, src, sizeof(double) * 2 * d.nv, cudaMemcpyHostToDevice, (cudaStream_t)s));
    launch_perm_to_p(d, g->nat_a, dst_p, s);
  }
  CU(cudaGetLastError());
  return RF_OK;
}

// parity-split device pairs -> natural-order pairs (host or device); syncs for host
static rf_status pairs_out(rf_grid* g, const Dims& d, const double* src_p, double* dst, void* s) {
  if (is_device_ptr(dst)) {
    launch_perm_from_p(d, src_p, dst, s);
    CU(cudaGetLastError());
  } else if (void* m = host_direct() ? mapped_host_ptr(dst) : nullptr) {
    launch_perm_from_p(d, src_p, (double*)m, s);
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize((cudaStream_t)s));
  } else {
    launch_perm_from_p(d, src_p, g->nat_b, s);
    CU(cudaMemcpyAsync(dst, g->nat_b, sizeof(double) * 2 * d.nv, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    CU(cudaStreamSynchronize((cudaStream_t)s));
  }
  return RF_OK;
}

// ------------------------------------------------------------------ ABI: grid
extern "C" int64_t rf_launch_count(void) { return g_launches.load(); }

extern "C" rf_status rf_barrier_check(int rounds, int extra, double limit_s, int* blocks_out, void* stream) {
  if (rounds < 1 || rounds > 1000000 || extra < 0 || extra > 1 || !(limit_s > 0.0) || !(limit_s <= 10.0))
    return fail(RF_EINVAL, "need 1 <= rounds <= 1e6, extra 0 or 1, 0 < limit_s <= 10");
  // words: bar[2] and passed (unsigned), then the status flag (double, 8-aligned)
  void* mem = nullptr;
  if (cudaMalloc(&mem, 32) != cudaSuccess) {
    cudaGetLastError();
    return fail(RF_ENOMEM, "barrier check: allocation failed");
  }
  unsigned* bar = (unsigned*)mem;
  unsigned* passed = bar + 2;
  double* status = (double*)((char*)mem + 16);
  cudaStream_t s = (cudaStream_t)stream;
  int blocks = 0;
  cudaError_t e = cudaMemsetAsync(mem, 0, 32, s);
  if (e == cudaSuccess) e = launch_barrier_check(bar, rounds, extra, status, (long long)(limit_s * 1e9), passed, &blocks, s);
  unsigned h_passed = 0;
  double h_status = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_passed, passed, sizeof h_passed, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof h_status, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(mem);
  if (blocks_out) *blocks_out = blocks;
  if (e != cudaSuccess) return fail(RF_ECUDA, "barrier check: %s", cudaGetErrorString(e));
  if (h_status != 0.0) return fail(RF_ETIMEOUT, "barrier check: a wait gave up (%u passes)", h_passed);
  if (h_passed != (unsigned)blocks * (unsigned)rounds)
    return fail(RF_ECUDA, "barrier check: %u passes, expected %d", h_passed, blocks * rounds);
  return RF_OK;
}
extern "C" const char* rf_last_error(void) { return t_err.c_str(); }
extern "C" int64_t rf_grid_nv(const rf_grid* g) { return g ? g->d.nv : 0; }

extern "C" const char* rf_status_string(rf_status s) {
  switch (s) {
    case RF_OK: return "ok";
    case RF_EINVAL: return "invalid argument";
    case RF_ENOMEM: return "out of device memory";
    case RF_ECUDA: return "CUDA error";
    case RF_ENOTCONV: return "linear solver did not converge";
    case RF_EBREAKDOWN: return "BiCGSTAB breakdown";
    case RF_ENONFINITE: return "non-finite value";
    case RF_ETIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

extern "C" rf_status rf_profile(rf_grid* g, int enable) {
  if (!g) return fail(RF_EINVAL, "grid is required");
  if (enable) {
    g->prec.clear();
    g->evnext = 0;
    for (int c = 0; c < RF_PROF_NCLASS; ++c) { g->acc_ms[c] = 0.0; g->acc_bytes[c] = 0.0; g->acc_launches[c] = 0; }
  }
  g->prof_on = enable != 0;
  return RF_OK;
}

extern "C" rf_status rf_profile_read(rf_grid* g, int cls, double* ms, int64_t* launches, double* bytes) {
  if (!g || cls < 0 || cls >= RF_PROF_NCLASS) return fail(RF_EINVAL, "bad grid or class");
  CU(cudaDeviceSynchronize());
  double t = g->acc_ms[cls], by = g->acc_bytes[cls];
  int64_t n = g->acc_launches[cls];
  for (auto& r : g->prec) {
    if (r.cls != cls) continue;
    float e = 0.f;
    CU(cudaEventElapsedTime(&e, r.a, r.b));
    t += e;
    by += r.bytes;
    n += r.launches;
  }
  if (ms) *ms = t;
  if (launches) *launches = n;
  if (bytes) *bytes = by;
  return RF_OK;
}

extern "C" void rf_grid_destroy(rf_grid* g) {
  if (!g) return;
  cudaDeviceSynchronize();
  for (int j = 0; j < RF_MAXSHIFT; ++j)
    if (g->col[j]) {
      if (g->col[j]->col_s[0]) cudaStreamDestroy(g->col[j]->col_s[0]);
      rf_grid_destroy(g->col[j]);   // frees only what the column grid allocated
      g->col[j] = nullptr;
    }
  destroy_graphs(g);
  for (auto e : g->evpool) cudaEventDestroy(e);
  if (g->join_in) cudaEventDestroy(g->join_in);
  if (g->join_out) cudaEventDestroy(g->join_out);
  if (g->cs) cudaStreamDestroy(g->cs);
  dfree_all(g, g->gbufs, nullptr);
  dfree_all(g, g->bufs, nullptr);
  if (g->hscal) cudaFreeHost(g->hscal);
  if (g->bscal_h) cudaFreeHost(g->bscal_h);
  delete g;
}

#define NEED(ptr)                                                  \
  do {                                                             \
    if (!(ptr)) { rf_grid_destroy(g); return fail(RF_ENOMEM, "device allocation failed (%s)", #ptr); } \
  } while (0)

extern "C" rf_status rf_grid_create(const rf_grid_desc* desc, const rf_fluids* fl, const rf_materials* mat,
                                    const rf_bc* bc, const rf_allocator* alloc, void* stream, rf_grid** out) {
  if (!out) return fail(RF_EINVAL, "out is NULL");
  *out = nullptr;
  if (!desc || !fl || !mat) return fail(RF_EINVAL, "desc, fluids and materials are required");
  if (desc->dim != 2 && desc->dim != 3) return fail(RF_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < 3; ++a) {
    const bool active = a < desc->dim;
    if (active && (desc->n[a] < 2 || desc->n[a] > (1 << 20))) return fail(RF_EINVAL, "n[%d] out of range", a);
    if (!active && desc->n[a] != 1) return fail(RF_EINVAL, "n[2] must be 1 in 2D");
    if (active && !(desc->h[a] > 0.0)) return fail(RF_EINVAL, "h[%d] must be positive", a);
  }
  const int64_t nv = desc->n[0] * desc->n[1] * desc->n[2];
  if (nv > ((int64_t)1 << 31)) return fail(RF_EINVAL, "grid too large (%lld vertices)", (long long)nv);
  if (!(fl->rho_w > 0 && fl->rho_n > 0 && fl->mu_w > 0 && fl->mu_n > 0)) return fail(RF_EINVAL, "fluid properties must be positive");
  if (!(mat->S_wr >= 0 && mat->S_nr >= 0 && mat->S_wr + mat->S_nr < 1.0 && mat->lambda > 0))
    return fail(RF_EINVAL, "Brooks-Corey parameters out of range");
  if (!mat->K || !mat->phi || !mat->pd) return fail(RF_EINVAL, "material arrays are required");
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(RF_EINVAL, "allocator needs alloc and free");

  rf_grid* g = new rf_grid();
  if (alloc) { g->alloc = *alloc; g->user_alloc = true; }
  int n[3] = {(int)desc->n[0], (int)desc->n[1], (int)desc->n[2]};
  g->d = make_dims(desc->dim, n);
  g->nb = make_nbr(g->d);
  for (int a = 0; a < 3; ++a) { g->h[a] = desc->h[a]; g->g[a] = desc->g[a]; g->pp.h[a] = desc->h[a]; g->pp.g[a] = desc->g[a]; }
  g->pp.rho_w = fl->rho_w; g->pp.rho_n = fl->rho_n; g->pp.mu_w = fl->mu_w; g->pp.mu_n = fl->mu_n;
  g->pp.S_wr = mat->S_wr; g->pp.S_nr = mat->S_nr; g->pp.lambda = mat->lambda;
  g->pp.scheme = 0;
  g->ncell = (int64_t)(n[0] - 1) * (n[1] - 1) * (desc->dim == 3 ? n[2] - 1 : 1);
  const Dims& d = g->d;
  const size_t cb = sizeof(double) * g->ncell;

  NEED(g->Kcell = (double*)dalloc(g, cb, stream, false));
  NEED(g->phi = (double*)dalloc(g, cb, stream, false));
  NEED(g->pd = (double*)dalloc(g, cb, stream, false));
  CU(to_device(g->Kcell, mat->K, cb, stream));
  CU(to_device(g->phi, mat->phi, cb, stream));
  CU(to_device(g->pd, mat->pd, cb, stream));

  NEED(g->nat_a = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
  NEED(g->nat_b = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
  NEED(g->dir = (uint8_t*)dalloc(g, nv, stream, false));
  NEED(g->pw_dir = (double*)dalloc(g, sizeof(double) * nv, stream, false));
  const uint8_t* dir_src = nullptr;
  const double* pwd_src = nullptr;
  if (bc && bc->dir_pw) {
    CU(to_device(g->nat_a, bc->dir_pw, nv, stream));
    dir_src = (const uint8_t*)g->nat_a;
  }
  launch_perm_bytes_to_p(d, dir_src, g->dir, stream);
  if (bc && bc->pw_dir) {
    CU(to_device(g->nat_b, bc->pw_dir, sizeof(double) * nv, stream));
    pwd_src = g->nat_b;
  }
  launch_perm_scalar_to_p(d, pwd_src, g->pw_dir, stream);
  CU(cudaStreamSynchronize((cudaStream_t)stream));
  if (bc && bc->q_in) {
    NEED(g->q_in = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
    rf_status st = pairs_in(g, d, bc->q_in, g->q_in, stream);
    if (st != RF_OK) { rf_grid_destroy(g); return st; }
  }
  NEED(g->pdmin = (double*)dalloc(g, sizeof(double) * nv, stream, false));
  NEED(g->phiv = (double*)dalloc(g, sizeof(double) * nv, stream, false));
  const double vol = g->h[0] * g->h[1] * (d.dim == 3 ? g->h[2] : 1.0);
  g->vol = vol;
  launch_vertex_setup(d, g->pd, g->phi, vol, g->pdmin, g->phiv, stream);

  NEED(g->J = (double*)dalloc(g, sizeof(double) * 4 * d.nb * nv, stream, false));
  NEED(g->mdiag = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
  double** scratch[6] = {&g->Se, &g->pn, &g->pc, &g->dpc, &g->krw, &g->dkrw};
  for (auto p : scratch) NEED(*p = (double*)dalloc(g, sizeof(double) * nv, stream, false));
  NEED(g->u_p = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
  NEED(g->F_p = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
  // Krylov FP64 vectors (x padded: the outer operator reads it for the true residual)
  NEED(g->K.x = (double2*)dvec(g, d, sizeof(double), stream, false));
  double2** kv[6] = {&g->K.r, &g->K.rh, &g->K.p, &g->K.v, &g->K.s, &g->K.t};
  for (auto p : kv) NEED(*p = (double2*)dalloc(g, sizeof(double2) * nv, stream, false));
  NEED(g->b_p = (double2*)dalloc(g, sizeof(double2) * nv, stream, false));
  NEED(g->du = (double*)dalloc(g, sizeof(double) * 2 * nv, stream, false));
  NEED(g->K.partial = (double*)dalloc(g, sizeof(double) * 16 * 2048, stream, false));
  NEED(g->K.scal = (double*)dalloc(g, sizeof(double) * 32, stream, false));
  CU(cudaMemsetAsync(g->K.scal, 0, sizeof(double) * 32, (cudaStream_t)stream));   // flags start clear
  NEED(g->norms = (double*)dalloc(g, sizeof(double) * 8, stream, false));
  if (cudaMallocHost((void**)&g->hscal, sizeof(double) * 32) != cudaSuccess) {
    cudaGetLastError();
    g->hscal = nullptr;
    rf_grid_destroy(g);
    return fail(RF_ENOMEM, "pinned host allocation failed");
  }
  if (cudaStreamCreateWithFlags(&g->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->join_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&g->join_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    rf_grid_destroy(g);
    return fail(RF_ECUDA, "internal stream creation failed");
  }
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) { rf_grid_destroy(g); return fail(RF_ECUDA, "grid set-up: %s", cudaGetErrorString(e)); }
  *out = g;
  return RF_OK;
}

// ------------------------------------------------------------------ assembly
static rf_status assemble_p(rf_grid* g, bool want_j, void* s) {
  AsmArrays a;
  a.u = g->u_p; a.Se = g->Se; a.pn = g->pn; a.pc = g->pc; a.dpc = g->dpc; a.krw = g->krw; a.dkrw = g->dkrw;
  a.pdmin = g->pdmin; a.phiv = g->phiv; a.K = g->Kcell; a.pd = g->pd; a.phi = g->phi; a.vol = g->vol;
  a.dir = g->dir; a.pw_dir = g->pw_dir;
  a.q_in = g->q_in; a.F = g->F_p; a.J = want_j ? g->J : nullptr; a.mdiag = want_j ? g->mdiag : nullptr;
  a.law = g->laws_on ? g->law : nullptr; a.kr_tab = g->kr_tab;
  cudaError_t e = launch_assemble(g->d, g->pp, a, want_j, s);
  if (e != cudaSuccess) return fail(RF_ECUDA, "assembly launch: %s", cudaGetErrorString(e));
  if (want_j) { g->have_J = true; g->gmg_ready = false; g->jdf_valid = false; }
  return RF_OK;
}

extern "C" rf_status rf_assemble(rf_grid* g, const double* u, int want_jacobian, double* F_out, void* s) {
  if (!g || !u) return fail(RF_EINVAL, "grid and u are required");
  rf_status st = pairs_in(g, g->d, u, g->u_p, s);
  if (st) return st;
  if ((st = assemble_p(g, want_jacobian != 0, s))) return st;
  if (F_out) return pairs_out(g, g->d, g->F_p, F_out, s);
  return RF_OK;
}

static_assert(RF_SCHEME_SHAT_STORAGE == SCHEME_SHAT_STORAGE && RF_SCHEME_DARCY_UPWIND == SCHEME_DARCY_UPWIND,
              "scheme bits of the C ABI and the kernels agree");
extern "C" rf_status rf_grid_set_scheme(rf_grid* g, int scheme) {
  if (!g) return fail(RF_EINVAL, "grid is required");
  if (scheme & ~(RF_SCHEME_SHAT_STORAGE | RF_SCHEME_DARCY_UPWIND)) return fail(RF_EINVAL, "unknown scheme bits 0x%x", scheme);
  if (g->pp.scheme != scheme) { g->have_J = false; g->gmg_ready = false; g->jdf_valid = false; }
  g->pp.scheme = scheme;
  return RF_OK;
}

static_assert(RF_KR_BROOKS_COREY == 0 && RF_KR_POLY == 1, "law kinds of the C ABI and the kernels agree");
extern "C" rf_status rf_grid_set_kr_laws(rf_grid* g, int nlaws, const double* laws, const uint8_t* cell_law,
                                         void* stream) {
  if (!g) return fail(RF_EINVAL, "grid is required");
  if (nlaws < 0 || nlaws > RF_MAX_KR_LAWS) return fail(RF_EINVAL, "nlaws must be 0..%d", RF_MAX_KR_LAWS);
  if (nlaws > 0) {
    if (!laws || !cell_law) return fail(RF_EINVAL, "laws and cell_law are required");
    if (is_device_ptr(laws) || is_device_ptr(cell_law)) return fail(RF_EINVAL, "laws and cell_law must be host memory");
    for (int m = 0; m < nlaws; ++m) {
      const double* L = laws + 6 * m;
      if (L[0] == RF_KR_BROOKS_COREY) continue;
      if (L[0] != RF_KR_POLY) return fail(RF_EINVAL, "law %d: unknown kind %g", m, L[0]);
      bool ok = L[1] >= 0.0 && L[3] >= 0.0 && std::isfinite(L[1]) && std::isfinite(L[3]) && std::isfinite(L[4]) &&
                std::isfinite(L[5]) && L[2] >= 1.0 && L[2] <= 8.0 && L[2] == (double)(int)L[2];
      if (!ok) return fail(RF_EINVAL, "law %d: coefficients out of range (a_w, a_n >= 0, n_w whole in 1..8)", m);
    }
    for (int64_t c = 0; c < g->ncell; ++c)
      if (cell_law[c] >= nlaws) return fail(RF_EINVAL, "cell %lld names law %d of %d", (long long)c, cell_law[c], nlaws);
    if (!g->kr_tab) {
      if (!g->law) g->law = (uint8_t*)dalloc(g, (size_t)g->ncell, stream, false);
      if (g->law) g->kr_tab = (double*)dalloc(g, sizeof(double) * 6 * RF_MAX_KR_LAWS, stream, false);
      if (!g->kr_tab) return fail(RF_ENOMEM, "device allocation of the k_r laws failed");
    }
    double tab[6 * RF_MAX_KR_LAWS] = {};
    for (int t = 0; t < 6 * nlaws; ++t) tab[t] = laws[t];
    CU(cudaMemcpyAsync(g->law, cell_law, (size_t)g->ncell, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CU(cudaMemcpyAsync(g->kr_tab, tab, sizeof(tab), cudaMemcpyHostToDevice, (cudaStream_t)stream));
    CU(cudaStreamSynchronize((cudaStream_t)stream));
  }
  g->laws_on = nlaws > 0;
  g->have_J = false; g->gmg_ready = false; g->jdf_valid = false;
  return RF_OK;
}

// ------------------------------------------------------------------ multigrid set-up
static size_t t_size(int kind) { return kind == STORE_F64 ? sizeof(double) : sizeof(float); }
static size_t s_size(int kind) { return kind == STORE_F64 ? 8 : (kind == STORE_F32 ? 4 : 2); }

static LevelOp level_op(rf_grid* g, int l, int sh) {
  LevelOp op;
  const Level& Lv = g->L[l];
  op.d = Lv.d;
  op.nb = Lv.nb;
  op.kind = Lv.kind;
  op.fine = (l == 0);
  op.A = (l == 0) ? Lv.A[0] : Lv.A[sh];
  op.scale = (l == 0) ? Lv.scale[0] : Lv.scale[sh];
  op.mdiag = g->mdiag;
  op.shift = g->shifts[sh];
  op.Dinv = Lv.Dinv[sh];
  op.dmask = Lv.dmask;
  op.block = Lv.block;
  op.batched = Lv.batched;
  return op;
}

// ------------------------------------------------------------------ autotuner
// Chooses, per level, the shape of the smoothing and residual kernels — the
// thread-block size and whether a thread issues its stencil loads in batches
// of 9 blocks — by timing one sweep plus one residual for each candidate on
// the level's own data (CUDA events).  Choices are cached per (device, level
// dimensions, storage kind, smoother, finest-or-not) for the process and, when
// RF_TUNE_CACHE names a file, in that file as one JSON object per line.
// RF_TUNE_VERBOSE=1 prints every candidate's time to stderr.
struct TuneChoice { int block; bool batched; };
static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune;
static bool g_tune_loaded = false;

static std::string tune_key(const Dims& d, int kind, int smoother, bool fine) {
  static const std::string dev = [] {   // initialised once, thread-safe (grids tune on worker threads)
    cudaDeviceProp p;
    int id = 0;
    cudaGetDevice(&id);
    return std::string((cudaGetDeviceProperties(&p, id) == cudaSuccess) ? p.name : "gpu");
  }();
  char buf[256];
  snprintf(buf, sizeof buf, "%s|%dx%dx%d|k%d|s%d|f%d", dev.c_str(), d.nx, d.ny, d.nz, kind, smoother, fine ? 1 : 0);
  return buf;
}

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("RF_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof line, f)) {
    // {"key": "<key>", "block": <n>, "batched": <0|1>}
    char* k = strstr(line, "\"key\": \"");
    char* b = strstr(line, "\"block\": ");
    char* t = strstr(line, "\"batched\": ");
    if (!k || !b) continue;
    k += 8;
    char* e = strchr(k, '"');
    if (!e) continue;
    const int bs = atoi(b + 9);
    if (bs != 64 && bs != 128 && bs != 256 && bs != 512) continue;
    const bool bt = t ? atoi(t + 11) != 0 : false;
    if (bt && bs > 256) continue;
    g_tune[std::string(k, e - k)] = TuneChoice{bs, bt};
  }
  fclose(f);
}

static void tune_store_locked(const std::string& key, TuneChoice c) {
  g_tune[key] = c;
  const char* path = getenv("RF_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "{\"key\": \"%s\", \"block\": %d, \"batched\": %d}\n", key.c_str(), c.block, c.batched ? 1 : 0);
  fclose(f);
}

static rf_status autotune_levels(rf_grid* g, void* s) {
  static const TuneChoice cand[7] = {{64, false}, {128, false}, {256, false}, {512, false},
                                     {64, true}, {128, true}, {256, true}};
  const bool verbose = getenv("RF_TUNE_VERBOSE") && atoi(getenv("RF_TUNE_VERBOSE")) > 0;
  const int last = g->nl - 1;   // the coarsest level is a dense solve
  for (int l = 0; l < last; ++l) {
    Level& Lv = g->L[l];
    const std::string key = tune_key(Lv.d, Lv.kind, g->gopt.smoother, l == 0);
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      tune_load_locked();
      auto it = g_tune.find(key);
      if (it != g_tune.end()) { Lv.block = it->second.block; Lv.batched = it->second.batched; continue; }
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    TuneChoice best_c{256, false};
    for (int c = 0; c < 7; ++c) {
      Lv.block = cand[c].block;
      Lv.batched = cand[c].batched;
      LevelOp op = level_op(g, l, 0);
      float tmin = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        CU(cudaEventRecord(e0, (cudaStream_t)s));
        if (g->gopt.smoother == RF_SMOOTH_JACOBI) launch_jacobi(op, Lv.b, Lv.x, Lv.t, g->gopt.omega, false, s);
        else launch_gs_sweep(op, Lv.b, Lv.x, true, false, s);
        launch_residual(op, Lv.b, Lv.x, Lv.r, s);
        CU(cudaEventRecord(e1, (cudaStream_t)s));
        CU(cudaEventSynchronize(e1));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < tmin) tmin = ms;   // first repetition warms up
      }
      if (verbose)
        fprintf(stderr, "rf autotune %s: block %d batched %d: %.4f ms\n", key.c_str(), cand[c].block,
                cand[c].batched ? 1 : 0, tmin);
      if (tmin < best) { best = tmin; best_c = cand[c]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    Lv.block = best_c.block;
    Lv.batched = best_c.batched;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_store_locked(key, best_c);
  }
  return RF_OK;
}

static void dfree_ptr(rf_grid* g, void* p, void* s) {
  for (size_t i = 0; i < g->gbufs.size(); ++i)
    if (g->gbufs[i].p == p) {
      if (g->user_alloc) g->alloc.free(p, g->gbufs[i].bytes, s, g->alloc.ctx);
      else cudaFree(p);
      g->gbufs.erase(g->gbufs.begin() + i);
      return;
    }
}

// Galerkin operators of level C from level F, one axis at a time (x, y[, z]);
// intermediate operators live only for the duration of the call.
static rf_status galerkin_level(rf_grid* g, const Level& F, Level& C, bool from_fine, void* s) {
  const int dim = F.d.dim;
  const double* Jin = from_fine ? g->J : F.Jc;
  const double* Min = from_fine ? nullptr : F.Mc;
  const double* md = from_fine ? g->mdiag : nullptr;
  int n[3] = {F.d.nx, F.d.ny, F.d.nz};
  Dims cur = F.d;
  std::vector<void*> temps;
  rf_status st = RF_OK;
  for (int axis = 0; axis < dim; ++axis) {
    n[axis] = (n[axis] - 1) / 2 + 1;
    const Dims nxt = make_dims(dim, n);
    const bool last = axis == dim - 1;
    double* Jo = C.Jc;
    double* Mo = C.Mc;
    if (!last) {
      Jo = (double*)dalloc(g, sizeof(double) * 4 * nxt.nb * nxt.nv, s, true);
      Mo = (double*)dalloc(g, sizeof(double) * 2 * nxt.nb * nxt.nv, s, true);
      if (Jo) temps.push_back(Jo);
      if (Mo) temps.push_back(Mo);
      if (!Jo || !Mo) { st = fail(RF_ENOMEM, "Galerkin temporaries"); break; }
    }
    launch_galerkin_axis(axis, cur, axis == 0 ? F.dmask : nullptr, Jin, Min, md, nxt, last ? C.dmask : nullptr, Jo,
                         Mo, s);
    Jin = Jo;
    Min = Mo;
    md = nullptr;
    cur = nxt;
  }
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)s);
  for (void* p : temps) dfree_ptr(g, p, s);
  if (st == RF_OK && e != cudaSuccess) st = fail(RF_ECUDA, "Galerkin: %s", cudaGetErrorString(e));
  return st;
}

#define GNEED(ptr)                                                                     \
  do {                                                                                 \
    if (!(ptr)) { dfree_all(g, g->gbufs, s); return fail(RF_ENOMEM, "device allocation failed (%s)", #ptr); } \
  } while (0)

extern "C" rf_status rf_gmg_setup(rf_grid* g, const double* shifts, int nshift, const rf_gmg_opts* o, void* s) {
  if (!g || !shifts || !o) return fail(RF_EINVAL, "grid, shifts and options are required");
  if (!g->have_J) return fail(RF_EINVAL, "rf_assemble with want_jacobian must precede rf_gmg_setup");
  if (nshift < 1 || nshift > RF_MAXSHIFT) return fail(RF_EINVAL, "nshift must be 1..4");
  if (o->nlevels < 1 || o->nlevels > RF_MAXL) return fail(RF_EINVAL, "nlevels must be 1..%d", RF_MAXL);
  if (o->smoother != RF_SMOOTH_JACOBI && o->smoother != RF_SMOOTH_GS8) return fail(RF_EINVAL, "unknown smoother");
  if (o->nu1 < 1 || o->nu2 < 0 || o->nu1 > 16 || o->nu2 > 16) return fail(RF_EINVAL, "need 1 <= nu1 <= 16, 0 <= nu2 <= 16");
  if (o->precision < RF_PREC_FP64 || o->precision > RF_PREC_FP16) return fail(RF_EINVAL, "unknown precision");
  for (int j = 0; j < nshift; ++j)
    if (!(shifts[j] >= 0.0) || !std::isfinite(shifts[j])) return fail(RF_EINVAL, "shifts must be finite and >= 0");
  CU(cudaStreamSynchronize((cudaStream_t)s));
  CU(cudaStreamSynchronize(g->cs));
  stale_graphs(g);
  dfree_all(g, g->gbufs, s);
  ++g->hier_gen;
  for (int l = 0; l < RF_MAXL; ++l) g->L[l] = Level();
  for (int j = 0; j < RF_MAXSHIFT; ++j) g->Ainv[j] = nullptr;
  g->gmg_ready = false;
  g->gopt = *o;
  g->kind = o->precision == RF_PREC_FP64 ? STORE_F64 : (o->precision == RF_PREC_FP32 ? STORE_F32 : STORE_F16);
  g->nshift = nshift;
  for (int j = 0; j < nshift; ++j) g->shifts[j] = shifts[j];

  // level dimensions (vertex-nested: coarse vertex I at fine 2I)
  int n[3] = {g->d.nx, g->d.ny, g->d.nz};
  g->nl = 1;
  g->L[0].d = g->d;
  while (g->nl < o->nlevels) {
    bool ok = true;
    int nn[3];
    for (int a = 0; a < 3; ++a) {
      if (a >= g->d.dim) { nn[a] = 1; continue; }
      if ((n[a] - 1) % 2 != 0 || n[a] < 3) ok = false;
      nn[a] = (n[a] - 1) / 2 + 1;
    }
    if (!ok) break;
    for (int a = 0; a < 3; ++a) n[a] = nn[a];
    g->L[g->nl].d = make_dims(g->d.dim, n);
    ++g->nl;
  }
  const int kind = g->kind;
  for (int l = 0; l < g->nl; ++l) {
    Level& Lv = g->L[l];
    Lv.nb = make_nbr(Lv.d);
    Lv.kind = (kind == STORE_F16 && l > 0) ? STORE_F32 : kind;
    default_shape(Lv, l, Lv.kind);
    const Dims& d = Lv.d;
    if (l == 0) {
      Lv.dmask = g->dir;
    } else {
      GNEED(Lv.dmask = (uint8_t*)dalloc(g, d.nv, s, true));
      launch_coarse_mask(g->L[l - 1].d, g->L[l - 1].dmask, d, Lv.dmask, s);
      GNEED(Lv.Jc = (double*)dalloc(g, sizeof(double) * 4 * d.nb * d.nv, s, true));
      GNEED(Lv.Mc = (double*)dalloc(g, sizeof(double) * 2 * d.nb * d.nv, s, true));
      rf_status gst = galerkin_level(g, g->L[l - 1], Lv, l == 1, s);
      if (gst) { dfree_all(g, g->gbufs, s); return gst; }
    }
    const int lk = Lv.kind;
    const size_t te = t_size(kind), se = s_size(lk);
    if (l < g->nl - 1 || g->nl == 1) {
      // smoothed levels: storage + inverse diagonal blocks per shift
      if (l == 0) {
        if (kind == STORE_F64) {
          Lv.A[0] = g->J;
        } else {
          GNEED(Lv.A[0] = dalloc(g, se * 4 * stored_blocks(kind, d.nb) * d.nv, s, true));
          if (kind == STORE_F16) GNEED(Lv.scale[0] = (float*)dalloc(g, sizeof(float) * 4 * d.nv, s, true));
          launch_pack_level(d, true, g->J, nullptr, g->mdiag, 0.0, kind, Lv.A[0], Lv.scale[0], nullptr, s);
        }
        for (int j = 0; j < nshift; ++j) {
          GNEED(Lv.Dinv[j] = dalloc(g, te * 4 * d.nv, s, true));
          launch_pack_level(d, true, g->J, nullptr, g->mdiag, shifts[j], kind, nullptr, nullptr, Lv.Dinv[j], s);
        }
      } else {
        for (int j = 0; j < nshift; ++j) {
          GNEED(Lv.A[j] = dalloc(g, se * 4 * stored_blocks(lk, d.nb) * d.nv, s, true));
          if (lk == STORE_F16) GNEED(Lv.scale[j] = (float*)dalloc(g, sizeof(float) * 4 * d.nv, s, true));
          GNEED(Lv.Dinv[j] = dalloc(g, te * 4 * d.nv, s, true));
          launch_pack_level(d, false, Lv.Jc, Lv.Mc, nullptr, shifts[j], lk, Lv.A[j], Lv.scale[j], Lv.Dinv[j], s);
        }
      }
    }
    GNEED(Lv.x = dvec(g, d, te, s, true, &Lv.pad));
    GNEED(Lv.b = dvec(g, d, te, s, true));
    GNEED(Lv.r = dvec(g, d, te, s, true));
    GNEED(Lv.t = dvec(g, d, te, s, true));
  }
  // coarsest level: dense FP64 operator per shift, LU with partial pivoting, explicit inverse
  {
    const Level& C = g->L[g->nl - 1];
    const int N = (int)(2 * C.d.nv);
    if (N > 4096) { dfree_all(g, g->gbufs, s); return fail(RF_EINVAL, "coarsest level too large (%d unknowns): use more levels", N); }
    // all shifts at once: one LU per CTA, the inverse columns of every shift in one grid
    double* D;
    int* piv;
    int* status;
    const size_t NN = (size_t)N * N;
    GNEED(D = (double*)dalloc(g, sizeof(double) * NN * nshift, s, true));
    GNEED(piv = (int*)dalloc(g, sizeof(int) * N * nshift, s, true));
    GNEED(status = (int*)dalloc(g, sizeof(int) * nshift, s, true));
    CU(cudaMemsetAsync(D, 0, sizeof(double) * NN * nshift, (cudaStream_t)s));
    CU(cudaMemsetAsync(status, 0, sizeof(int) * nshift, (cudaStream_t)s));
    for (int j = 0; j < nshift; ++j) {
      GNEED(g->Ainv[j] = (double*)dalloc(g, sizeof(double) * NN, s, true));
      if (g->nl == 1) launch_dense_coarsest(C.d, C.nb, g->J, nullptr, g->mdiag, true, shifts[j], D + NN * j, s);
      else launch_dense_coarsest(C.d, C.nb, C.Jc, C.Mc, nullptr, false, shifts[j], D + NN * j, s);
    }
    CU(launch_dense_inverse_batched(N, nshift, D, g->Ainv, piv, status, s));
    int hst[RF_MAXSHIFT] = {};
    CU(cudaMemcpyAsync(hst, status, sizeof(int) * nshift, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    CU(cudaStreamSynchronize((cudaStream_t)s));
    for (int j = 0; j < nshift; ++j)
      if (hst[j]) { dfree_all(g, g->gbufs, s); return fail(RF_ENONFINITE, "coarsest operator is singular or not finite (shift %d)", j); }
  }
  // Krylov preconditioned vectors in the preconditioner type
  {
    const size_t te = t_size(kind);
    GNEED(g->K.y = dvec(g, g->d, te, s, true));
    GNEED(g->K.z = dvec(g, g->d, te, s, true));
    GNEED(g->K.p_lo = dvec(g, g->d, te, s, true));
    GNEED(g->K.s_lo = dvec(g, g->d, te, s, true));
    if (kind == STORE_F64) {
      g->K.y64 = (double2*)g->K.y;
      g->K.z64 = (double2*)g->K.z;
    } else {
      GNEED(g->K.y64 = (double2*)dvec(g, g->d, sizeof(double), s, true));
      GNEED(g->K.z64 = (double2*)dvec(g, g->d, sizeof(double), s, true));
    }
  }
  if (o->autotune) {
    rf_status ts = autotune_levels(g, s);
    if (ts) { dfree_all(g, g->gbufs, s); return ts; }
  }
  // The small levels (<= RF_TAIL_NV vertices, default 6000: 17^3 and below)
  // run as one launch: one thread-block cluster with hardware barriers, or
  // with RF_TAIL_MODE=coop a cooperative launch of every co-resident block with
  // bounded grid barriers; RF_TAIL_NV=0 launches every phase.  Both compute
  // the launch-per-phase V-cycle bit for bit.  Measured on GB300 at 257^3:
  // the cluster from 17^3 saves ~0.5 ms per solve (95.4 against 96.0 ms);
  // from 33^3, or as a cooperative launch, the barrier-separated phases are
  // no faster than the launches they replace, and a cluster whose first level
  // is too large for 16 SMs (65^3) costs ~40% of an FP64 LIMEX step.
  g->tail_first = -1;
  g->tail_blocks = 0;
  g->tail_bar = nullptr;   // (a hierarchy buffer: freed with the previous set-up)
  {
    const char* env = getenv("RF_TAIL_NV");
    const char* mode = getenv("RF_TAIL_MODE");
    const bool cluster = !(mode && strcmp(mode, "coop") == 0);
    // the default applies to FP32 coarse levels: with FP64 storage the
    // whole V-cycle in one kernel spills registers, and the 65^3 FP64 LIMEX
    // step, its columns one after another, took 113.5 against 99.3 ms
    const long long thr = env ? atoll(env) : (g->kind == STORE_F64 ? 0 : 6000);
    if (thr > 0)
      for (int l = 1; l < g->nl - 1; ++l)
        if (g->L[l].d.nv <= thr) { g->tail_first = l; break; }
    if (g->tail_first > 0 && cluster) {
      g->tail_cs = tail_cluster_size(g->L[g->tail_first].kind, g->d.nb);
      cudaGetLastError();
      if (g->tail_cs == 0) g->tail_first = -1;
    } else if (g->tail_first > 0) {
      g->tail_blocks = coop_tail_blocks(g->L[g->tail_first].kind, g->d.nb);
      g->tail_bar = g->tail_blocks > 0 ? (unsigned*)dalloc(g, 2 * sizeof(unsigned), s, true) : nullptr;
      if (!g->tail_bar) {
        g->tail_first = -1;
        g->tail_blocks = 0;
      } else {
        CU(cudaMemsetAsync(g->tail_bar, 0, 2 * sizeof(unsigned), (cudaStream_t)s));
      }
    }
    if (g->tail_first > 0)
      for (int j = 0; j < nshift; ++j) {
        TailParams& P = g->tail[j];
        P = TailParams();
        P.first = g->tail_first;
        P.coarsest = g->nl - 1;
        P.smoother = o->smoother;
        P.nu1 = o->nu1;
        P.nu2 = o->nu2;
        P.omega = o->omega;
        fill_tail_masks(P, g->d.dim);
        P.Ainv = g->Ainv[j];
        P.N = (int)(2 * g->L[g->nl - 1].d.nv);
        P.bar = g->tail_bar;
        P.status = g->K.scal + RF_SCAL_TAIL;
        P.limit_ns = 2000000000LL;   // 2 s: a phase takes microseconds
        for (int l = g->tail_first; l < g->nl; ++l) {
          P.L[l].op = level_op(g, l, j);
          P.L[l].x = g->L[l].x;
          P.L[l].b = g->L[l].b;
          P.L[l].r = g->L[l].r;
          P.L[l].t = g->L[l].t;
        }
        // the cluster form with the FP32 levels' matrices in shared memory
        // (GS smoother; RF_TAIL_SMEM=0 keeps them in global memory): when
        // every CTA's rows fit
        const char* sm_env = getenv("RF_TAIL_SMEM");
        if (g->tail_blocks == 0 && g->L[g->tail_first].kind == STORE_F32 && o->smoother == RF_SMOOTH_GS8 &&
            !(sm_env && atoi(sm_env) == 0))
          tail_sm_plan(P, g->d.nb, g->tail_cs);
      }
  }
  CU(cudaStreamSynchronize((cudaStream_t)s));
  CU(cudaGetLastError());
  g->gmg_ready = true;
  return RF_OK;
}

// ------------------------------------------------------------------ V-cycle
// bytes of one smoothing sweep on a level of nv vertices
static double sweep_bytes(rf_grid* g, int l, bool zero_x) {
  const Dims& d = g->L[l].d;
  const int k = g->L[l].kind;
  const double T = tb(k), nv = (double)d.nv;
  if (g->gopt.smoother == RF_SMOOTH_JACOBI) {
    if (zero_x) return nv * (4 * T + 4 * T);  // Dinv, b, x out
    return nv * (d.nb * blk_bytes(k) + row_extra(k) + (l == 0 ? 16.0 : 0.0) + 4 * T + 6 * T);
  }
  // GS: off-diagonal blocks; the first sweep from zero reads only the blocks
  // that reach already-visited colours, half of them over the 2^d colours
  if (zero_x) return nv * ((d.nb - 1) * 0.5 * blk_bytes(k) + row_extra(k) + 4 * T + 2 * T + 2 * T + 2 * T * 0.5);
  return nv * ((d.nb - 1) * blk_bytes(k) + row_extra(k) + 4 * T + 6 * T);
}

static void smooth_pre(rf_grid* g, int l, int sh, const void* b, void* x_final, void** cur, void* s) {
  LevelOp op = level_op(g, l, sh);
  Level& Lv = g->L[l];
  const rf_gmg_opts& o = g->gopt;
  const size_t te = t_size(g->kind);
  const int cls = l == 0 ? RF_PROF_SMOOTH_FINE : RF_PROF_COARSE_LEVELS;
  const int ncol = 1 << Lv.d.dim;
  if (o.smoother == RF_SMOOTH_JACOBI) {
    const int W = o.nu1 + o.nu2;
    void* first = (W % 2 == 1) ? x_final : Lv.t;
    void* c = first;
    {
      ProfScope ps(g, s, cls, sweep_bytes(g, l, true), 1);
      launch_jacobi(op, b, nullptr, first, o.omega, true, s);
    }
    for (int k = 1; k < o.nu1; ++k) {
      void* dst = (c == x_final) ? Lv.t : x_final;
      ProfScope ps(g, s, cls, sweep_bytes(g, l, false), 1);
      launch_jacobi(op, b, c, dst, o.omega, false, s);
      c = dst;
    }
    *cur = c;
  } else {
    // the first forward sweep skips every not-yet-visited neighbour, so x
    // needs no clearing
    (void)te;
    for (int k = 0; k < o.nu1; ++k) {
      ProfScope ps(g, s, cls, sweep_bytes(g, l, k == 0), ncol);
      launch_gs_sweep(op, b, x_final, true, k == 0, s);
    }
    *cur = x_final;
  }
}

static void smooth_post(rf_grid* g, int l, int sh, const void* b, void* x_final, void* cur, void* s) {
  LevelOp op = level_op(g, l, sh);
  Level& Lv = g->L[l];
  const rf_gmg_opts& o = g->gopt;
  const int cls = l == 0 ? RF_PROF_SMOOTH_FINE : RF_PROF_COARSE_LEVELS;
  const int ncol = 1 << Lv.d.dim;
  if (o.smoother == RF_SMOOTH_JACOBI) {
    void* c = cur;
    for (int k = 0; k < o.nu2; ++k) {
      void* dst = (c == x_final) ? Lv.t : x_final;
      ProfScope ps(g, s, cls, sweep_bytes(g, l, false), 1);
      launch_jacobi(op, b, c, dst, o.omega, false, s);
      c = dst;
    }
  } else {
    for (int k = 0; k < o.nu2; ++k) {
      ProfScope ps(g, s, cls, sweep_bytes(g, l, false), ncol);
      launch_gs_sweep(op, b, x_final, false, false, s, true);
    }
  }
}

static void vcycle_level(rf_grid* g, int l, int sh, const void* b, void* x, void* s) {
  const int k = g->L[l].kind;
  const double T = tb(k);
  if (l == g->tail_first) {
    // the whole remaining V-cycle in one cluster launch (x, b are level l's own vectors)
    double by = 4.0 * g->L[g->nl - 1].d.nv * g->L[g->nl - 1].d.nv * 8.0;
    for (int q = l; q < g->nl - 1; ++q) {
      const double nvq = (double)g->L[q].d.nv, nvc = (double)g->L[q + 1].d.nv;
      const int kq = g->L[q].kind;
      by += sweep_bytes(g, q, true) + (g->gopt.nu1 - 1 + g->gopt.nu2) * sweep_bytes(g, q, false);
      by += nvq * (g->L[q].d.nb * blk_bytes(kq) + row_extra(kq) + 6 * T) + nvq * (6 * T + 2) + nvc * (4 * T + 2);
    }
    ProfScope ps(g, s, RF_PROF_COARSE_LEVELS, by, 1);
    if (g->tail_blocks > 0) launch_vcycle_coop(g->tail[sh], k, g->d.nb, g->tail_blocks, s);
    else if (g->tail[sh].sm_bytes > 0) launch_vcycle_tail_sm(g->tail[sh], g->d.nb, s);
    else launch_vcycle_tail(g->tail[sh], k, g->d.nb, g->tail_cs, s);
    return;
  }
  if (l == g->nl - 1) {
    const double N = 2.0 * g->L[l].d.nv;
    ProfScope ps(g, s, RF_PROF_COARSE_LEVELS, N * N * 8.0 + 2 * N * T, 1);
    launch_coarse_solve(level_op(g, l, sh), g->Ainv[sh], b, x, s);
    return;
  }
  Level& Lv = g->L[l];
  Level& Lc = g->L[l + 1];
  const double nvf = (double)Lv.d.nv, nvc = (double)Lc.d.nv;
  void* cur = nullptr;
  smooth_pre(g, l, sh, b, x, &cur, s);
  LevelOp op = level_op(g, l, sh), opc = level_op(g, l + 1, sh);
  {
    ProfScope ps(g, s, l == 0 ? RF_PROF_RESID_FINE : RF_PROF_COARSE_LEVELS,
                 nvf * (Lv.d.nb * blk_bytes(k) + row_extra(k) + (l == 0 ? 16.0 : 0.0) + 6 * T), 1);
    launch_residual(op, b, cur, Lv.r, s);
  }
  {
    ProfScope ps(g, s, RF_PROF_TRANSFER, nvf * (2 * T + 1) + nvc * (2 * T + 1), 1);
    launch_restrict(op, opc, Lv.r, Lc.b, s);
  }
  vcycle_level(g, l + 1, sh, Lc.b, Lc.x, s);
  {
    ProfScope ps(g, s, RF_PROF_TRANSFER, nvf * (4 * T + 1) + nvc * (2 * T + 1), 1);
    launch_prolong(op, opc, Lc.x, cur, s);
  }
  smooth_post(g, l, sh, b, x, cur, s);
}

// ------------------------------------------------------------------ BiCGSTAB
enum { H_RHO = 0, H_RR = 5, H_BB = 6, H_CONV = 10, H_BAD = 11, H_TRUE = 12, H_BREAK = 13 };

static rf_status read_scal(rf_grid* g, void* s) {
  CU(cudaMemcpyAsync(g->hscal, g->K.scal, sizeof(double) * (RF_SCAL_TAIL + 1), cudaMemcpyDeviceToHost,
                     (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  return RF_OK;
}

// One BiCGSTAB iteration, both V-cycles included, launched on stream s.
static void iteration_body(rf_grid* g, int sh, void* s) {
  const Dims& d = g->d;
  const bool lo32 = g->kind != STORE_F64;
  KrylovVecs& K = g->K;
  const double shift = g->shifts[sh];
  const double T = tb(g->kind), nv = (double)d.nv;
  const double spmv_bytes = nv * (d.nb * 32.0 + 16.0 + 16.0 + 16.0 + 16.0);
  {
    ProfScope ps(g, s, RF_PROF_VECTOR, nv * (16.0 * 4 + 2 * T), 1);
    launch_bicg_p(d.nv, K, lo32, false, s);
  }
  const bool df = lo32 && g->outer_df;   // double-FP32 operator on the FP32 operands
  const double spmv_df_bytes = nv * (d.nb * 32.0 + 16.0 + 8.0 + 16.0 + 16.0);
  vcycle_level(g, 0, sh, K.p_lo, K.y, s);
  if (lo32 && !df) {
    ProfScope ps(g, s, RF_PROF_VECTOR, nv * (2 * T + 16.0), 1);
    launch_cast_f32_to_f64((const float*)K.y, (double*)K.y64, 2 * d.nv, s);
  }
  {
    ProfScope ps(g, s, RF_PROF_SPMV64, df ? spmv_df_bytes : spmv_bytes, 1);
    if (df) launch_bicg_v_df(d, g->nb, g->Jdf, g->mdiag, shift, K, s);
    else launch_bicg_v(d, g->nb, g->J, g->mdiag, shift, K, lo32, s);
  }
  {
    ProfScope ps(g, s, RF_PROF_VECTOR, nv * (16.0 * 3 + 2 * T), 1);
    launch_bicg_s(d.nv, K, lo32, s);
  }
  vcycle_level(g, 0, sh, K.s_lo, K.z, s);
  if (lo32 && !df) {
    ProfScope ps(g, s, RF_PROF_VECTOR, nv * (2 * T + 16.0), 1);
    launch_cast_f32_to_f64((const float*)K.z, (double*)K.z64, 2 * d.nv, s);
  }
  {
    ProfScope ps(g, s, RF_PROF_SPMV64, df ? spmv_df_bytes : spmv_bytes, 1);
    if (df) launch_bicg_t_df(d, g->nb, g->Jdf, g->mdiag, shift, K, s);
    else launch_bicg_t(d, g->nb, g->J, g->mdiag, shift, K, lo32, s);
  }
  {
    // with an FP32 preconditioner the FP64 copies the operator read serve
    // here too: the same values, and no FP32 -> FP64 conversions on the FP64
    // pipe, which bounds this kernel (16 B more read per vertex)
    const bool use64 = lo32 && !df;
    KrylovVecs K2 = K;
    if (use64) { K2.y = K.y64; K2.z = K.z64; }
    ProfScope ps(g, s, RF_PROF_VECTOR, nv * ((use64 ? 32.0 : 4 * T) + 16.0 * 6), 1);
    launch_bicg_xr(d.nv, K2, lo32 && !use64, s);
  }
}

// Run one iteration and bring its scalars to the host.  The iteration is
// captured once per (shift, profiling) as a CUDA graph and replayed: the ~300
// launches of the V-cycles, most of them on small coarse levels, then cost
// GPU-side dispatch only.  RF_NO_GRAPHS=1 in the environment runs it eagerly.
static rf_status run_iteration(rf_grid* g, int sh, cudaStream_t cs) {
  static const bool eager = getenv("RF_NO_GRAPHS") && getenv("RF_NO_GRAPHS")[0] == '1';
  if (eager) {
    iteration_body(g, sh, cs);
    return read_scal(g, cs);
  }
  const bool prof = g->prof_on;
  rf_grid::IterGraph& G = g->ig[sh][prof ? 1 : 0][g->outer_df];
  if (!G.exec || G.stale) {
    rf_status st = capture_graph(g, G, cs, "iteration", [&] {
      iteration_body(g, sh, cs);
      cudaMemcpyAsync(g->hscal, g->K.scal, sizeof(double) * (RF_SCAL_TAIL + 1), cudaMemcpyDeviceToHost, cs);
    });
    if (st) return st;
  }
  CU(cudaGraphLaunch(G.exec, cs));
  g_launches.fetch_add(G.kernels);
  CU(cudaStreamSynchronize(cs));
  if (prof)
    for (auto& r : G.recs) {
      float e = 0.f;
      CU(cudaEventElapsedTime(&e, r.a, r.b));
      g->acc_ms[r.cls] += e;
      g->acc_bytes[r.cls] += r.bytes;
      g->acc_launches[r.cls] += r.launches;
    }
  return RF_OK;
}

static rf_status solve_cs(rf_grid* g, int sh, const double2* b, double rtol, int max_it, rf_solve_info* info,
                          cudaStream_t s);

// Solve A_sh x = b with b, x parity-split device pairs (x is g->K.x on return).
// The iteration runs on the grid's internal stream, ordered after and before
// the caller's stream.
static rf_status solve_p(rf_grid* g, int sh, const double2* b, double rtol, int max_it, int outer,
                         rf_solve_info* info, void* s) {
  g->outer_df = (outer == RF_OUTER_DF32 && g->kind != STORE_F64) ? 1 : 0;
  if (g->outer_df && !g->jdf_valid) {
    if (!g->Jdf) {
      g->Jdf = (float*)dalloc(g, sizeof(double) * 4 * g->d.nb * g->d.nv, s, false);
      if (!g->Jdf) return fail(RF_ENOMEM, "double-FP32 operator copy");
    }
    launch_split_df(g->d, g->J, g->Jdf, s);
    g->jdf_valid = true;
  }
  CU(cudaEventRecord(g->join_in, (cudaStream_t)s));
  CU(cudaStreamWaitEvent(g->cs, g->join_in, 0));
  rf_status r = solve_cs(g, sh, b, rtol, max_it, info, g->cs);
  cudaEventRecord(g->join_out, g->cs);
  cudaStreamWaitEvent((cudaStream_t)s, g->join_out, 0);
  return r;
}

static rf_status solve_cs(rf_grid* g, int sh, const double2* b, double rtol, int max_it, rf_solve_info* info,
                          cudaStream_t s) {
  const Dims& d = g->d;
  KrylovVecs& K = g->K;
  const double shift = g->shifts[sh];
  const double nvd = (double)d.nv;
  const double true_res_bytes = nvd * (d.nb * 32.0 + 16.0 + 16.0 + 16.0 + 16.0);
  {
    ProfScope ps(g, s, RF_PROF_VECTOR, nvd * 16.0 * 6, 1);
    launch_bicg_init(d.nv, b, K, rtol, s);
  }
  rf_status st = read_scal(g, s);
  if (st) return st;
  const double bb = g->hscal[H_BB];
  int it = 0, restarts = 0;
  double relres = 0.0;
  rf_status result = RF_ENOTCONV;
  if (!std::isfinite(bb)) return fail(RF_ENONFINITE, "right-hand side is not finite");
  if (bb == 0.0) {
    result = RF_OK;
  } else {
    const double bn = std::sqrt(bb);
    for (it = 1; it <= max_it; ++it) {
      if ((st = run_iteration(g, sh, s))) return st;
      if (g->hscal[RF_SCAL_TAIL] != 0.0) {
        // a barrier of the cooperative V-cycle tail gave up: its words are
        // left mid-count, so reset them (and the flag) before any reuse
        CU(cudaMemsetAsync(g->tail_bar, 0, 2 * sizeof(unsigned), s));
        CU(cudaMemsetAsync(g->K.scal + RF_SCAL_TAIL, 0, sizeof(double), s));
        CU(cudaStreamSynchronize(s));
        return fail(RF_ETIMEOUT, "a grid barrier of the V-cycle tail timed out");
      }
      if (g->hscal[H_BAD] != 0.0) { result = RF_ENONFINITE; break; }
      if (g->hscal[H_CONV] != 0.0 || g->hscal[H_BREAK] != 0.0) {
        {
          ProfScope ps(g, s, RF_PROF_SPMV64, true_res_bytes, 1);
          launch_true_residual(d, g->nb, g->J, g->mdiag, shift, b, K, s);
        }
        if ((st = read_scal(g, s))) return st;
        relres = std::sqrt(g->hscal[H_TRUE]) / bn;
        if (!std::isfinite(relres)) { result = RF_ENONFINITE; break; }
        if (relres <= rtol) { result = RF_OK; break; }
        if (++restarts > 20) { result = RF_EBREAKDOWN; break; }
        launch_restart(d.nv, K, s);
      }
    }
    if (it > max_it) it = max_it;
    if (result != RF_OK && result != RF_ENONFINITE) {
      launch_true_residual(d, g->nb, g->J, g->mdiag, shift, b, K, s);
      if ((st = read_scal(g, s))) return st;
      relres = std::sqrt(g->hscal[H_TRUE]) / bn;
    }
  }
  if (info) { info->iterations = it; info->relres = relres; info->status = result; info->restarts = restarts; }
  if (result == RF_ENOTCONV) return fail(result, "no convergence in %d iterations (relres %.3e)", max_it, relres);
  if (result == RF_ENONFINITE) return fail(result, "non-finite value in the BiCGSTAB iteration");
  if (result == RF_EBREAKDOWN) return fail(result, "BiCGSTAB breakdown after %d restarts", restarts);
  return RF_OK;
}

extern "C" rf_status rf_solve(rf_grid* g, int sh, const double* b, double* x, const rf_solve_opts* o,
                              rf_solve_info* info, void* s) {
  if (!g || !b || !x || !o) return fail(RF_EINVAL, "grid, b, x and options are required");
  if (!g->gmg_ready) return fail(RF_EINVAL, "rf_gmg_setup must precede rf_solve");
  if (sh < 0 || sh >= g->nshift) return fail(RF_EINVAL, "shift index %d out of range", sh);
  if (!(o->rtol > 0.0) || o->max_it < 1) return fail(RF_EINVAL, "need rtol > 0 and max_it >= 1");
  if (o->outer != RF_OUTER_FP64 && o->outer != RF_OUTER_DF32) return fail(RF_EINVAL, "unknown outer operator mode");
  rf_status st = pairs_in(g, g->d, b, (double*)g->b_p, s);
  if (st) return st;
  rf_status r = solve_p(g, sh, g->b_p, o->rtol, o->max_it, o->outer, info, s);
  if (r != RF_OK && r != RF_ENOTCONV) return r;
  st = pairs_out(g, g->d, (const double*)g->K.x, x, s);
  if (st) return st;
  if (r == RF_ENOTCONV) return fail(r, "no convergence in %d iterations", o->max_it);
  return RF_OK;
}

// ------------------------------------------------------------------ batched solves
// The systems of a batch (grid, shift index, right-hand side) have equal level
// shapes, storage kind and smoother: the active LIMEX columns of a step, or the
// (member, column) pairs of an ensemble group.  They run BiCGSTAB in lock-step:
// every kernel of an iteration serves all of them in one launch (one system per
// blockIdx.y; on the finest level of systems that share J, all of them per
// thread with J read once), and one captured graph holds the whole batched
// iteration.  A system that has finished is flagged in its scalars
// (RF_SCAL_DONE) and skipped by every later launch, so each system performs
// exactly the operations of its own solve: results equal solve_p's bit for bit.
struct BatchSys {
  rf_grid* g;
  int sh;
  const double2* b;
};

static SysLevel sys_level(rf_grid* g, int l, int sh) {
  const LevelOp op = level_op(g, l, sh);
  SysLevel P{};
  P.A = op.A;
  P.scale = op.scale;
  P.Dinv = op.Dinv;
  P.mdiag = op.mdiag;
  P.dmask = op.dmask;
  P.shift = op.shift;
  P.scal = g->K.scal;
  return P;
}

// bytes of one batched level launch: S systems, the matrix read once per group
// of `share` systems that use the same one
static double batch_bytes(double per_sys, double matrix, int S, int share) {
  return S * per_sys - (S - S / share) * matrix;
}

static void vcycle_batch(rf_grid* lead, const std::vector<BatchSys>& bs, int l, const std::vector<const void*>& b,
                         const std::vector<void*>& x, int share, void* s) {
  const int S = (int)bs.size();
  rf_grid* g0 = bs[0].g;
  const int k = g0->L[l].kind;
  const double T = tb(k);
  const double nv = (double)g0->L[l].d.nv;
  if (l == g0->nl - 1) {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = sys_level(bs[q].g, l, bs[q].sh);
      B.s[q].A = bs[q].g->Ainv[bs[q].sh];
      B.s[q].in0 = b[q];
      B.s[q].out = x[q];
    }
    const double N = 2.0 * nv;
    ProfScope ps(lead, s, RF_PROF_COARSE_LEVELS, S * (N * N * 8.0 + 2 * N * T), 1);
    launch_coarse_solve_b(level_op(g0, l, bs[0].sh), B, s);
    return;
  }
  const bool sh_l = share > 1 && l == 0;   // only the finest level stores the shared J
  const int shl = sh_l ? share : 1;
  const LevelOp op = level_op(g0, l, bs[0].sh);
  const LevelOp opc = level_op(g0, l + 1, bs[0].sh);
  const rf_gmg_opts& o = g0->gopt;
  const int cls = l == 0 ? RF_PROF_SMOOTH_FINE : RF_PROF_COARSE_LEVELS;
  const int ncol = 1 << op.d.dim;
  const double mat = nv * (op.d.nb * blk_bytes(k) + row_extra(k));
  auto base = [&](int q) {
    SysLevel P = sys_level(bs[q].g, l, bs[q].sh);
    return P;
  };
  std::vector<void*> cur(S), tmp(S);
  for (int q = 0; q < S; ++q) tmp[q] = bs[q].g->L[l].t;
  // pre-smoothing (the schedule of smooth_pre)
  if (o.smoother == RF_SMOOTH_JACOBI) {
    const int W = o.nu1 + o.nu2;
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].in0 = b[q];
      B.s[q].in1 = nullptr;
      cur[q] = (W % 2 == 1) ? x[q] : tmp[q];
      B.s[q].out = cur[q];
    }
    {
      ProfScope ps(lead, s, cls, S * sweep_bytes(g0, l, true), 1);
      if (sh_l) launch_jacobi_shared(op, B, share, o.omega, true, s);
      else launch_jacobi_b(op, B, o.omega, true, s);
    }
    for (int it = 1; it < o.nu1; ++it) {
      for (int q = 0; q < S; ++q) {
        void* dst = (cur[q] == x[q]) ? tmp[q] : x[q];
        B.s[q].in1 = cur[q];
        B.s[q].out = dst;
        cur[q] = dst;
      }
      ProfScope ps(lead, s, cls, batch_bytes(sweep_bytes(g0, l, false), mat, S, shl), 1);
      if (sh_l) launch_jacobi_shared(op, B, share, o.omega, false, s);
      else launch_jacobi_b(op, B, o.omega, false, s);
    }
  } else {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].in0 = b[q];
      B.s[q].in1 = x[q];
      B.s[q].out = x[q];
      cur[q] = x[q];
    }
    for (int it = 0; it < o.nu1; ++it) {
      ProfScope ps(lead, s, cls, batch_bytes(sweep_bytes(g0, l, it == 0), it == 0 ? 0.5 * mat : mat, S, shl), ncol);
      if (sh_l) launch_gs_sweep_shared(op, B, share, true, it == 0, s);
      else launch_gs_sweep_b(op, B, true, it == 0, s);
    }
  }
  // residual, restriction
  {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].in0 = b[q];
      B.s[q].in1 = cur[q];
      B.s[q].out = bs[q].g->L[l].r;
    }
    ProfScope ps(lead, s, l == 0 ? RF_PROF_RESID_FINE : RF_PROF_COARSE_LEVELS,
                 batch_bytes(nv * (op.d.nb * blk_bytes(k) + row_extra(k) + (l == 0 ? 16.0 : 0.0) + 6 * T), mat, S, shl),
                 1);
    if (sh_l) launch_residual_shared(op, B, share, s);
    else launch_residual_b(op, B, s);
  }
  const double nvc = (double)g0->L[l + 1].d.nv;
  {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].dmask = bs[q].g->L[l].dmask;
      B.s[q].dmask_c = bs[q].g->L[l + 1].dmask;
      B.s[q].in0 = bs[q].g->L[l].r;
      B.s[q].out = bs[q].g->L[l + 1].b;
    }
    ProfScope ps(lead, s, RF_PROF_TRANSFER, S * (nv * (2 * T + 1) + nvc * (2 * T + 1)), 1);
    launch_restrict_b(op, opc, B, s);
  }
  std::vector<const void*> bc(S);
  std::vector<void*> xc(S);
  for (int q = 0; q < S; ++q) {
    bc[q] = bs[q].g->L[l + 1].b;
    xc[q] = bs[q].g->L[l + 1].x;
  }
  vcycle_batch(lead, bs, l + 1, bc, xc, share, s);
  {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].dmask = bs[q].g->L[l].dmask;
      B.s[q].dmask_c = bs[q].g->L[l + 1].dmask;
      B.s[q].in0 = xc[q];
      B.s[q].out = cur[q];
    }
    ProfScope ps(lead, s, RF_PROF_TRANSFER, S * (nv * (4 * T + 1) + nvc * (2 * T + 1)), 1);
    launch_prolong_b(op, opc, B, s);
  }
  // post-smoothing (the schedule of smooth_post)
  if (o.smoother == RF_SMOOTH_JACOBI) {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].in0 = b[q];
    }
    for (int it = 0; it < o.nu2; ++it) {
      for (int q = 0; q < S; ++q) {
        void* dst = (cur[q] == x[q]) ? tmp[q] : x[q];
        B.s[q].in1 = cur[q];
        B.s[q].out = dst;
        cur[q] = dst;
      }
      ProfScope ps(lead, s, cls, batch_bytes(sweep_bytes(g0, l, false), mat, S, shl), 1);
      if (sh_l) launch_jacobi_shared(op, B, share, o.omega, false, s);
      else launch_jacobi_b(op, B, o.omega, false, s);
    }
  } else {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) {
      B.s[q] = base(q);
      B.s[q].in0 = b[q];
      B.s[q].in1 = x[q];
      B.s[q].out = x[q];
    }
    for (int it = 0; it < o.nu2; ++it) {
      ProfScope ps(lead, s, cls, batch_bytes(sweep_bytes(g0, l, false), mat, S, shl), ncol);
      if (sh_l) launch_gs_sweep_shared(op, B, share, false, false, s, true);
      else launch_gs_sweep_b(op, B, false, false, s, true);
    }
  }
}

static KBatch krylov_batch(const std::vector<BatchSys>& bs) {
  KBatch KB{};
  KB.n = (int)bs.size();
  for (int q = 0; q < KB.n; ++q) {
    KB.s[q].K = bs[q].g->K;
    KB.s[q].J = bs[q].g->J;
    KB.s[q].mdiag = bs[q].g->mdiag;
    KB.s[q].shift = bs[q].g->shifts[bs[q].sh];
  }
  return KB;
}

// one batched BiCGSTAB iteration (both V-cycles), then the gathered scalars to the host
static void batch_body(rf_grid* lead, const std::vector<BatchSys>& bs, int share, void* s) {
  rf_grid* g0 = bs[0].g;
  const int S = (int)bs.size();
  const Dims& d = g0->d;
  const bool lo32 = g0->kind != STORE_F64;
  const double T = tb(g0->kind), nv = (double)d.nv;
  const KBatch KB = krylov_batch(bs);
  const double opmat = nv * d.nb * 32.0;
  const double spmv_bytes = nv * (d.nb * 32.0 + 16.0 + 16.0 + 16.0 + 16.0);
  {
    ProfScope ps(lead, s, RF_PROF_VECTOR, S * nv * (16.0 * 4 + 2 * T), 1);
    launch_bicg_p_b(d.nv, KB, lo32, s);
  }
  std::vector<const void*> in(S);
  std::vector<void*> out(S);
  for (int q = 0; q < S; ++q) { in[q] = bs[q].g->K.p_lo; out[q] = bs[q].g->K.y; }
  vcycle_batch(lead, bs, 0, in, out, share, s);
  if (lo32) {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) { B.s[q].scal = bs[q].g->K.scal; B.s[q].in0 = bs[q].g->K.y; B.s[q].out = bs[q].g->K.y64; }
    ProfScope ps(lead, s, RF_PROF_VECTOR, S * nv * (2 * T + 16.0), 1);
    launch_cast_f32_to_f64_b(2 * d.nv, B, s);
  }
  {
    ProfScope ps(lead, s, RF_PROF_SPMV64, batch_bytes(spmv_bytes, opmat, S, share), 1);
    launch_bicg_v_b(d, g0->nb, KB, share, s);
  }
  {
    ProfScope ps(lead, s, RF_PROF_VECTOR, S * nv * (16.0 * 3 + 2 * T), 1);
    launch_bicg_s_b(d.nv, KB, lo32, s);
  }
  for (int q = 0; q < S; ++q) { in[q] = bs[q].g->K.s_lo; out[q] = bs[q].g->K.z; }
  vcycle_batch(lead, bs, 0, in, out, share, s);
  if (lo32) {
    SysBatch B{};
    B.n = S;
    for (int q = 0; q < S; ++q) { B.s[q].scal = bs[q].g->K.scal; B.s[q].in0 = bs[q].g->K.z; B.s[q].out = bs[q].g->K.z64; }
    ProfScope ps(lead, s, RF_PROF_VECTOR, S * nv * (2 * T + 16.0), 1);
    launch_cast_f32_to_f64_b(2 * d.nv, B, s);
  }
  {
    ProfScope ps(lead, s, RF_PROF_SPMV64, batch_bytes(spmv_bytes, opmat, S, share), 1);
    launch_bicg_t_b(d, g0->nb, KB, share, s);
  }
  {
    // the FP64 copies of the preconditioned vectors, as in iteration_body
    KBatch KB64 = KB;
    if (lo32)
      for (int q = 0; q < S; ++q) { KB64.s[q].K.y = bs[q].g->K.y64; KB64.s[q].K.z = bs[q].g->K.z64; }
    ProfScope ps(lead, s, RF_PROF_VECTOR, S * nv * ((lo32 ? 32.0 : 4 * T) + 16.0 * 6), 1);
    launch_bicg_xr_b(d.nv, KB64, false, s);
  }
  launch_gather_scalars(KB, lead->bscal, s);
  cudaMemcpyAsync(lead->bscal_h, lead->bscal, sizeof(double) * 16 * S, cudaMemcpyDeviceToHost, (cudaStream_t)s);
}

static rf_status batch_gather(rf_grid* lead, const std::vector<BatchSys>& bs, cudaStream_t s) {
  const KBatch KB = krylov_batch(bs);
  launch_gather_scalars(KB, lead->bscal, s);
  CU(cudaMemcpyAsync(lead->bscal_h, lead->bscal, sizeof(double) * 16 * bs.size(), cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  return RF_OK;
}

static rf_status run_batch_iteration(rf_grid* lead, const std::vector<BatchSys>& bs, int share, cudaStream_t cs) {
  static const bool eager = getenv("RF_NO_GRAPHS") && getenv("RF_NO_GRAPHS")[0] == '1';
  if (eager) {
    batch_body(lead, bs, share, cs);
    CU(cudaStreamSynchronize(cs));
    return RF_OK;
  }
  std::string key = (lead->prof_on ? "p" : "n") + std::to_string(share);
  char buf[64];
  for (const auto& q : bs) {
    snprintf(buf, sizeof buf, "|%p:%d", (void*)q.g, q.sh);
    key += buf;
  }
  rf_grid::IterGraph& G = lead->bgraph[key];
  if (!G.exec || G.stale) {
    rf_status st = capture_graph(lead, G, cs, "batched iteration", [&] { batch_body(lead, bs, share, cs); });
    if (st) return st;
  }
  CU(cudaGraphLaunch(G.exec, cs));
  g_launches.fetch_add(G.kernels);
  CU(cudaStreamSynchronize(cs));
  if (lead->prof_on)
    for (auto& r : G.recs) {
      float e = 0.f;
      CU(cudaEventElapsedTime(&e, r.a, r.b));
      lead->acc_ms[r.cls] += e;
      lead->acc_bytes[r.cls] += r.bytes;
      lead->acc_launches[r.cls] += r.launches;
    }
  return RF_OK;
}

// the lead grid's gathered-scalar buffers (device, pinned host + the constant 1.0)
static rf_status batch_buffers(rf_grid* lead, void* s) {
  if (!lead->bscal) {
    lead->bscal = (double*)dalloc(lead, sizeof(double) * 16 * RF_MAXSYS, s, false);
    if (!lead->bscal) return fail(RF_ENOMEM, "batch scalars");
  }
  if (!lead->bscal_h) {
    if (cudaMallocHost((void**)&lead->bscal_h, sizeof(double) * (16 * RF_MAXSYS + 1)) != cudaSuccess) {
      cudaGetLastError();
      lead->bscal_h = nullptr;
      return fail(RF_ENOMEM, "pinned batch scalars");
    }
    lead->bscal_h[16 * RF_MAXSYS] = 1.0;
  }
  return RF_OK;
}

// Solve the batch's systems A_{sh} x = b (x in each system's grid K.x) in lock-step
// on the lead grid's internal stream, ordered after and before `s`.  st[q], info[q]
// receive each system's result as solve_cs would return them.
static rf_status solve_batch(rf_grid* lead, const std::vector<BatchSys>& bs, int share, double rtol, int max_it,
                             std::vector<rf_status>& st, std::vector<rf_solve_info>& info, void* s) {
  const int S = (int)bs.size();
  if (S < 1 || S > RF_MAXSYS) return fail(RF_EINVAL, "batch of %d systems", S);
  if (share < 1 || share > 4 || S % share) return fail(RF_EINVAL, "batch of %d systems in groups of %d", S, share);
  rf_status bst = batch_buffers(lead, s);
  if (bst) return bst;
  const double* one = lead->bscal_h + 16 * RF_MAXSYS;
  cudaStream_t cs = lead->cs;
  CU(cudaEventRecord(lead->join_in, (cudaStream_t)s));
  CU(cudaStreamWaitEvent(cs, lead->join_in, 0));
  const Dims& d = bs[0].g->d;
  st.assign(S, RF_ENOTCONV);
  info.assign(S, rf_solve_info{});
  std::vector<int> active(S, 0), restarts(S, 0), iters(S, 0);
  std::vector<double> bn(S, 0.0), relres(S, 0.0);
  rf_status err = RF_OK;
  auto finish = [&](int q) -> rf_status {   // the system leaves the lock-step
    active[q] = 0;
    CU(cudaMemcpyAsync(bs[q].g->K.scal + RF_SCAL_DONE, one, sizeof(double), cudaMemcpyHostToDevice, cs));
    return RF_OK;
  };
  for (int q = 0; q < S; ++q) {
    rf_grid* g = bs[q].g;
    ProfScope ps(lead, cs, RF_PROF_VECTOR, (double)d.nv * 16.0 * 6, 1);
    launch_bicg_init(d.nv, bs[q].b, g->K, rtol, cs);
  }
  if ((err = batch_gather(lead, bs, cs))) return err;
  int nact = 0;
  for (int q = 0; q < S; ++q) {
    const double bb = lead->bscal_h[16 * q + H_BB];
    if (!std::isfinite(bb)) {
      st[q] = RF_ENONFINITE;
      if ((err = finish(q))) return err;
    } else if (bb == 0.0) {
      st[q] = RF_OK;
      if ((err = finish(q))) return err;
    } else {
      bn[q] = std::sqrt(bb);
      active[q] = 1;
      ++nact;
    }
  }
  for (int it = 1; it <= max_it && nact > 0; ++it) {
    if ((err = run_batch_iteration(lead, bs, share, cs))) return err;
    std::vector<int> check;
    for (int q = 0; q < S; ++q) {
      if (!active[q]) continue;
      iters[q] = it;
      const double* h = lead->bscal_h + 16 * q;
      if (h[H_BAD] != 0.0) {
        st[q] = RF_ENONFINITE;
        if ((err = finish(q))) return err;
        --nact;
      } else if (h[H_CONV] != 0.0 || h[H_BREAK] != 0.0) {
        check.push_back(q);
      }
    }
    if (check.empty()) continue;
    for (int q : check) {
      rf_grid* g = bs[q].g;
      const double shift = g->shifts[bs[q].sh];
      ProfScope ps(lead, cs, RF_PROF_SPMV64, (double)d.nv * (d.nb * 32.0 + 64.0), 1);
      launch_true_residual(d, g->nb, g->J, g->mdiag, shift, bs[q].b, g->K, cs);
    }
    if ((err = batch_gather(lead, bs, cs))) return err;
    for (int q : check) {
      rf_grid* g = bs[q].g;
      relres[q] = std::sqrt(lead->bscal_h[16 * q + H_TRUE]) / bn[q];
      if (!std::isfinite(relres[q])) st[q] = RF_ENONFINITE;
      else if (relres[q] <= rtol) st[q] = RF_OK;
      else if (++restarts[q] > 20) st[q] = RF_EBREAKDOWN;
      else {
        launch_restart(d.nv, g->K, cs);
        continue;
      }
      if ((err = finish(q))) return err;
      --nact;
    }
  }
  // systems that used up max_it: their true residual
  for (int q = 0; q < S; ++q) {
    if (!active[q]) continue;
    rf_grid* g = bs[q].g;
    launch_true_residual(d, g->nb, g->J, g->mdiag, g->shifts[bs[q].sh], bs[q].b, g->K, cs);
  }
  if ((err = batch_gather(lead, bs, cs))) return err;
  for (int q = 0; q < S; ++q) {
    if (active[q] || st[q] == RF_EBREAKDOWN) relres[q] = std::sqrt(lead->bscal_h[16 * q + H_TRUE]) / bn[q];
    if (active[q]) {
      st[q] = RF_ENOTCONV;
      if ((err = finish(q))) return err;
    }
    info[q].iterations = iters[q];
    info[q].relres = relres[q];
    info[q].status = st[q];
    info[q].restarts = restarts[q];
  }
  CU(cudaEventRecord(lead->join_out, cs));
  CU(cudaStreamWaitEvent((cudaStream_t)s, lead->join_out, 0));
  return RF_OK;
}

// ------------------------------------------------------------------ LIMEX
// ------------------------------------------------------------------ LIMEX column grids
// Column j of a LIMEX step (n_j = j+1 linearly implicit Euler substeps with
// shift (j+1)/H) depends on the others only through the extrapolation at the
// end, so the columns can run at the same time.  Column j > 0 runs on a
// column grid: a shallow copy of this grid's operator data and multigrid
// hierarchy (J, M, level operators, coarsest inverses; read-only during the
// columns) with its own Krylov and level vectors, assembly scratch, pinned
// scalars, internal stream and iteration graphs.  Same kernels, same shapes,
// same order per column: the results are bitwise those of running the
// columns one after another.
static rf_status column_grid(rf_grid* g, int j, void* s, rf_grid** out) {
  rf_grid* c = g->col[j];
  if (!c) {
    c = new rf_grid();
    c->is_column = true;
    c->alloc = g->alloc;
    c->user_alloc = g->user_alloc;
    c->d = g->d;
    c->nb = g->nb;
    const Dims& d = c->d;
    const int64_t nv = d.nv;
    bool ok = true;
    double** scratch[6] = {&c->Se, &c->pn, &c->pc, &c->dpc, &c->krw, &c->dkrw};
    for (auto p : scratch) ok = ok && (*p = (double*)dalloc(c, sizeof(double) * nv, s, false));
    ok = ok && (c->u_p = (double*)dalloc(c, sizeof(double) * 2 * nv, s, false));
    ok = ok && (c->F_p = (double*)dalloc(c, sizeof(double) * 2 * nv, s, false));
    ok = ok && (c->K.x = (double2*)dvec(c, d, sizeof(double), s, false));
    double2** kv[6] = {&c->K.r, &c->K.rh, &c->K.p, &c->K.v, &c->K.s, &c->K.t};
    for (auto p : kv) ok = ok && (*p = (double2*)dalloc(c, sizeof(double2) * nv, s, false));
    ok = ok && (c->K.partial = (double*)dalloc(c, sizeof(double) * 16 * 2048, s, false));
    ok = ok && (c->K.scal = (double*)dalloc(c, sizeof(double) * 32, s, false));
    ok = ok && cudaMemsetAsync(c->K.scal, 0, sizeof(double) * 32, (cudaStream_t)s) == cudaSuccess;
    ok = ok && (c->norms = (double*)dalloc(c, sizeof(double) * 8, s, false));
    if (ok && cudaMallocHost((void**)&c->hscal, sizeof(double) * 32) != cudaSuccess) {
      cudaGetLastError();
      c->hscal = nullptr;
      ok = false;
    }
    if (ok && (cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking) != cudaSuccess ||
               cudaStreamCreateWithFlags(&c->col_s[0], cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreateWithFlags(&c->join_in, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventCreateWithFlags(&c->join_out, cudaEventDisableTiming) != cudaSuccess)) {
      cudaGetLastError();
      ok = false;
    }
    if (!ok) {
      if (c->col_s[0]) cudaStreamDestroy(c->col_s[0]);
      rf_grid_destroy(c);
      return fail(RF_ENOMEM, "LIMEX column %d: allocation failed", j);
    }
    g->col[j] = c;
  }
  // the parent's operator data (read-only while the columns run)
  c->pp = g->pp;
  for (int a = 0; a < 3; ++a) { c->h[a] = g->h[a]; c->g[a] = g->g[a]; }
  c->ncell = g->ncell;
  c->Kcell = g->Kcell; c->phi = g->phi; c->pd = g->pd; c->vol = g->vol;
  c->law = g->law; c->kr_tab = g->kr_tab; c->laws_on = g->laws_on;
  c->dir = g->dir; c->pw_dir = g->pw_dir; c->q_in = g->q_in; c->pdmin = g->pdmin; c->phiv = g->phiv;
  c->J = g->J; c->mdiag = g->mdiag; c->have_J = g->have_J;
  c->Jdf = g->Jdf; c->jdf_valid = g->jdf_valid;
  // a new hierarchy of the same shape (levels, storage kind, level sizes): keep
  // the column's own level vectors (their zero halos are never written) and
  // mirror the new operators
  bool same_shape = c->gen != ~0ull && c->nl == g->nl && c->kind == g->kind;
  for (int l = 0; same_shape && l < g->nl; ++l) same_shape = c->L[l].d.nv == g->L[l].d.nv && c->L[l].d.nx == g->L[l].d.nx;
  if (c->gen != g->hier_gen && same_shape) {
    CU(cudaStreamSynchronize(c->cs));
    stale_graphs(c);
    c->gmg_ready = g->gmg_ready;
    c->gopt = g->gopt;
    c->nshift = g->nshift;
    for (int k = 0; k < RF_MAXSHIFT; ++k) { c->shifts[k] = g->shifts[k]; c->Ainv[k] = g->Ainv[k]; }
    for (int l = 0; l < c->nl; ++l) {
      Level keep = c->L[l];
      c->L[l] = g->L[l];
      c->L[l].x = keep.x; c->L[l].b = keep.b; c->L[l].r = keep.r; c->L[l].t = keep.t; c->L[l].pad = keep.pad;
    }
    c->gen = g->hier_gen;
  }
  if (c->gen != g->hier_gen) {
    // new hierarchy: drop graphs and level vectors, mirror the levels, own vectors
    CU(cudaStreamSynchronize(c->cs));
    stale_graphs(c);
    dfree_all(c, c->gbufs, s);
    c->gmg_ready = g->gmg_ready;
    c->gopt = g->gopt;
    c->kind = g->kind;
    c->nshift = g->nshift;
    for (int k = 0; k < RF_MAXSHIFT; ++k) { c->shifts[k] = g->shifts[k]; c->Ainv[k] = g->Ainv[k]; }
    c->nl = g->nl;
    c->tail_first = -1;
    const size_t te = t_size(c->kind);
    bool ok = true;
    for (int l = 0; l < RF_MAXL; ++l) {
      c->L[l] = g->L[l];
      c->L[l].x = c->L[l].b = c->L[l].r = c->L[l].t = nullptr;
      if (l >= c->nl) continue;
      const Dims& dl = c->L[l].d;
      ok = ok && (c->L[l].x = dvec(c, dl, te, s, true));
      ok = ok && (c->L[l].b = dvec(c, dl, te, s, true));
      ok = ok && (c->L[l].r = dvec(c, dl, te, s, true));
      ok = ok && (c->L[l].t = dvec(c, dl, te, s, true));
    }
    ok = ok && (c->K.y = dvec(c, c->d, te, s, true));
    ok = ok && (c->K.z = dvec(c, c->d, te, s, true));
    ok = ok && (c->K.p_lo = dvec(c, c->d, te, s, true));
    ok = ok && (c->K.s_lo = dvec(c, c->d, te, s, true));
    if (c->kind == STORE_F64) {
      c->K.y64 = (double2*)c->K.y;
      c->K.z64 = (double2*)c->K.z;
    } else {
      ok = ok && (c->K.y64 = (double2*)dvec(c, c->d, sizeof(double), s, true));
      ok = ok && (c->K.z64 = (double2*)dvec(c, c->d, sizeof(double), s, true));
    }
    if (!ok) {
      dfree_all(c, c->gbufs, s);
      c->gen = ~0ull;
      return fail(RF_ENOMEM, "LIMEX column %d: vector allocation failed", j);
    }
    c->gen = g->hier_gen;
  }
  *out = c;
  return RF_OK;
}

// Whether a LIMEX step runs its columns concurrently: RF_LIMEX_CONCURRENT=1/0
// forces it; by default on grids of at most 4M vertices (the extra vectors
// cost ~300 B per vertex and column; larger grids are bandwidth-bound).
static thread_local bool t_in_batch = false;   // set by rf_limex_step_batched's workers
static bool limex_concurrent(const rf_grid* g, int kap) {
  if (kap < 2) return false;
  const char* e = getenv("RF_LIMEX_CONCURRENT");
  if (e) return atoi(e) != 0;
  return !t_in_batch && g->d.nv <= 4000000;
}

// The LIMEX step with its columns one after another (or side by side on
// column grids and host threads, see limex_concurrent): the path taken when
// RF_LIMEX_BATCH=0, with the double-FP32 outer operator, or when the column
// grids of the batched path cannot be allocated.
static rf_status limex_step_columns(rf_grid* g, double* u, double H, const rf_limex_opts* o, rf_limex_info* info,
                                    void* s) {
  if (!g || !u || !o) return fail(RF_EINVAL, "grid, u and options are required");
  if (!(H > 0.0) || !std::isfinite(H)) return fail(RF_EINVAL, "H must be positive");
  if (o->kappa < 1 || o->kappa > RF_MAXSHIFT) return fail(RF_EINVAL, "kappa must be 1..4");
  if (!(o->tol > 0) || !(o->rho > 0) || !(o->fac_min > 0) || !(o->fac_max >= o->fac_min))
    return fail(RF_EINVAL, "bad step-control parameters");
  const Dims& d = g->d;
  const int kap = o->kappa;
  const size_t vb = sizeof(double) * 2 * d.nv;
  if (!g->T || g->T_kappa < kap) {
    g->T = (double*)dalloc(g, vb * kap, s, false);
    if (!g->T) return fail(RF_ENOMEM, "LIMEX table allocation failed");
    g->T_kappa = kap;
  }
  rf_status st = pairs_in(g, d, u, g->u_p, s);
  if (st) return st;
  // u0 is kept in column 0's slot until column 0 is computed: copy to nat_a as backup
  double* u0 = g->nat_a;
  CU(cudaMemcpyAsync(u0, g->u_p, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  if ((st = assemble_p(g, true, s))) return st;   // J, M, F(u0) in F_p
  double* F0 = g->nat_b;
  CU(cudaMemcpyAsync(F0, g->F_p, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  double shifts[RF_MAXSHIFT];
  for (int j = 0; j < kap; ++j) shifts[j] = (double)(j + 1) / H;
  if ((st = rf_gmg_setup(g, shifts, kap, &o->gmg, s))) return st;
  // column j on grid gj and stream sj: u0 -> n_j substeps -> T slot j
  struct ColResult { rf_status st = RF_OK; int solves = 0, iters = 0; std::string msg; };
  ColResult res[RF_MAXSHIFT];
  auto column = [&](rf_grid* gj, int j, void* sj) {
    ColResult& R = res[j];
    double* U = g->T + (size_t)j * 2 * d.nv;
    if (cudaMemcpyAsync(U, u0, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)sj) != cudaSuccess) {
      R.st = fail(RF_ECUDA, "LIMEX column %d: copy failed", j);
      R.msg = rf_last_error();
      return;
    }
    for (int k = 0; k <= j; ++k) {
      const double* F;
      if (k == 0) {
        F = F0;
      } else {
        rf_status a2 = RF_OK;
        if (cudaMemcpyAsync(gj->u_p, U, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)sj) != cudaSuccess)
          a2 = fail(RF_ECUDA, "LIMEX column %d: copy failed", j);
        if (!a2) a2 = assemble_p(gj, false, sj);
        if (a2) { R.st = a2; R.msg = rf_last_error(); return; }
        F = gj->F_p;
      }
      rf_solve_info si{};
      rf_status r = solve_p(gj, j, (const double2*)F, o->solve.rtol, o->solve.max_it, o->solve.outer, &si, sj);
      ++R.solves;
      R.iters += si.iterations;
      if (r != RF_OK) {
        if (r != RF_ENOTCONV) { R.st = r; R.msg = rf_last_error(); return; }
        if (R.st == RF_OK) R.st = r;
      }
      launch_axpy_pairs(d.nv, (double2*)U, gj->K.x, sj);
    }
  };
  if (limex_concurrent(g, kap)) {
    // the double-FP32 operator copy is made once, before the columns share it
    if (o->solve.outer == RF_OUTER_DF32 && g->kind != STORE_F64 && !g->jdf_valid) {
      if (!g->Jdf) {
        g->Jdf = (float*)dalloc(g, sizeof(double) * 4 * g->d.nb * g->d.nv, s, false);
        if (!g->Jdf) return fail(RF_ENOMEM, "double-FP32 operator copy");
      }
      launch_split_df(g->d, g->J, g->Jdf, s);
      g->jdf_valid = true;
    }
    rf_grid* cg[RF_MAXSHIFT] = {g};
    for (int j = 1; j < kap; ++j)
      if ((st = column_grid(g, j, s, &cg[j]))) return st;
    cudaEvent_t ready;
    CU(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
    CU(cudaEventRecord(ready, (cudaStream_t)s));
    for (int j = 1; j < kap; ++j) CU(cudaStreamWaitEvent(cg[j]->col_s[0], ready, 0));
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::vector<std::thread> th;
    for (int j = kap - 1; j >= 1; --j)   // longest columns first
      th.emplace_back([&, j] {
        cudaSetDevice(dev);
        column(cg[j], j, cg[j]->col_s[0]);
      });
    column(g, 0, s);
    for (auto& t : th) t.join();
    for (int j = 1; j < kap; ++j) {
      CU(cudaEventRecord(cg[j]->join_out, cg[j]->col_s[0]));
      CU(cudaStreamWaitEvent((cudaStream_t)s, cg[j]->join_out, 0));
    }
    cudaEventDestroy(ready);
  } else {
    for (int j = 0; j < kap; ++j) {
      column(g, j, s);
      if (res[j].st != RF_OK && res[j].st != RF_ENOTCONV) break;
    }
  }
  int solves = 0, iters = 0;
  rf_status worst = RF_OK;
  for (int j = 0; j < kap; ++j) {
    solves += res[j].solves;
    iters += res[j].iters;
    if (res[j].st != RF_OK && res[j].st != RF_ENOTCONV) return fail(res[j].st, "%s", res[j].msg.c_str());
    if (res[j].st == RF_ENOTCONV) worst = RF_ENOTCONV;
  }
  launch_extrapolate(2 * d.nv, kap, g->T, s);
  const double* Tkk = g->T;
  const double* Tkk1 = g->T + 2 * d.nv;
  launch_error_norms(d, g->h, Tkk, kap > 1 ? Tkk1 : Tkk, g->norms, g->K.partial, s);
  double nrm[4];
  CU(cudaMemcpyAsync(nrm, g->norms, sizeof nrm, cudaMemcpyDeviceToHost, (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  double vol = 1.0;
  for (int a = 0; a < d.dim; ++a) vol *= (double)((a == 0 ? d.nx : a == 1 ? d.ny : d.nz) - 1) * g->h[a];
  const double alpha = 1.0 / (nrm[0] + 1e-30);
  const double beta = 1.0 / (nrm[2] + 1e-4 * vol);
  const double eps = std::sqrt((alpha * nrm[1] + beta * nrm[3]) / 2.0);
  double fac = (eps > 0.0) ? std::pow(o->rho * o->tol / eps, 1.0 / 3.0) : o->fac_max;
  if (fac > o->fac_max) fac = o->fac_max;
  if (fac < o->fac_min) fac = o->fac_min;
  const int acc = (eps <= o->tol) && worst == RF_OK;
  if (acc) {
    if ((st = pairs_out(g, d, Tkk, u, s))) return st;
  }
  if (info) {
    info->eps = eps; info->H_new = H * fac; info->accepted = acc; info->solves = solves;
    info->iterations = iters; info->status = worst;
  }
  if (!std::isfinite(eps)) return fail(RF_ENONFINITE, "error estimate is not finite");
  return worst;
}

// ------------------------------------------------------------------ LIMEX in batched rounds
// Column j of a step (n_j = j+1 substeps, shift (j+1)/H) runs on column grid
// cg[j] (cg[0] = the grid itself).  Round r solves the r-th substep of every
// column j >= r: the right-hand sides F(u_r^j) are assembled per column, then
// all of them go to one batched solve (solve_batch), and each column adds its
// increment.  Every column performs the same operations in the same order as
// in limex_step_columns, so the step is bitwise the same; an ensemble group
// puts the columns of all its members into the same rounds.
struct LimexWork {
  rf_grid* g = nullptr;
  double* u = nullptr;
  double H = 0.0;
  const rf_limex_opts* o = nullptr;
  rf_limex_info* info = nullptr;
  rf_grid* cg[RF_MAXSHIFT] = {};
  rf_status st = RF_OK;          // first hard failure of this problem
  std::string msg;
  rf_status worst = RF_OK;       // RF_ENOTCONV if a column solve did not converge
  int solves = 0, iters = 0;
};

static rf_status limex_check(rf_grid* g, double* u, double H, const rf_limex_opts* o) {
  if (!g || !u || !o) return fail(RF_EINVAL, "grid, u and options are required");
  if (!(H > 0.0) || !std::isfinite(H)) return fail(RF_EINVAL, "H must be positive");
  if (o->kappa < 1 || o->kappa > RF_MAXSHIFT) return fail(RF_EINVAL, "kappa must be 1..4");
  if (!(o->tol > 0) || !(o->rho > 0) || !(o->fac_min > 0) || !(o->fac_max >= o->fac_min))
    return fail(RF_EINVAL, "bad step-control parameters");
  return RF_OK;
}

// state in, J, M and F(u0) assembled, hierarchy for the kappa shifts, column
// grids, every column's slot of the table T set to u0 (u0 kept in nat_a, F0 in nat_b)
static rf_status limex_prepare(LimexWork& w, void* s) {
  rf_grid* g = w.g;
  const Dims& d = g->d;
  const int kap = w.o->kappa;
  const size_t vb = sizeof(double) * 2 * d.nv;
  if (!g->T || g->T_kappa < kap) {
    g->T = (double*)dalloc(g, vb * kap, s, false);
    if (!g->T) return fail(RF_ENOMEM, "LIMEX table allocation failed");
    g->T_kappa = kap;
  }
  rf_status st = pairs_in(g, d, w.u, g->u_p, s);
  if (st) return st;
  CU(cudaMemcpyAsync(g->nat_a, g->u_p, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  if ((st = assemble_p(g, true, s))) return st;
  CU(cudaMemcpyAsync(g->nat_b, g->F_p, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  double shifts[RF_MAXSHIFT];
  for (int j = 0; j < kap; ++j) shifts[j] = (double)(j + 1) / w.H;
  if ((st = rf_gmg_setup(g, shifts, kap, &w.o->gmg, s))) return st;
  w.cg[0] = g;
  for (int j = 1; j < kap; ++j)
    if ((st = column_grid(g, j, s, &w.cg[j]))) return st;
  for (int j = 0; j < kap; ++j)
    CU(cudaMemcpyAsync(g->T + (size_t)j * 2 * d.nv, g->nat_a, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  return RF_OK;
}

// the rounds of a group of steps whose grids have equal shapes and options
static rf_status limex_rounds(std::vector<LimexWork*>& ws, void* s) {
  rf_grid* lead = ws[0]->g;
  // every problem of the batch was set up anew: the lead's batched iterations
  // (which reach into all of them) are re-captured at their first use
  stale_graphs(lead);
  const Dims& d = lead->d;
  const int kap = ws[0]->o->kappa;
  const size_t vb = sizeof(double) * 2 * d.nv;
  cudaEvent_t round_start;
  CU(cudaEventCreateWithFlags(&round_start, cudaEventDisableTiming));
  struct EvGuard { cudaEvent_t e; ~EvGuard() { cudaEventDestroy(e); } } guard{round_start};
  for (int r = 0; r < kap; ++r) {
    std::vector<BatchSys> bs;
    std::vector<LimexWork*> owner;
    std::vector<int> col;
    // the right-hand sides F(u_r^j): each column assembles on its own stream
    // (the assemblies are independent), after everything before on s
    if (r > 0) CU(cudaEventRecord(round_start, (cudaStream_t)s));
    for (LimexWork* w : ws) {
      if (w->st != RF_OK) continue;
      for (int j = r; j < kap; ++j) {
        rf_grid* gj = w->cg[j];
        const double* F = w->g->nat_b;   // F(u0): the first substep of every column
        if (r > 0) {
          double* U = w->g->T + (size_t)j * 2 * d.nv;
          CU(cudaStreamWaitEvent(gj->cs, round_start, 0));
          CU(cudaMemcpyAsync(gj->u_p, U, vb, cudaMemcpyDeviceToDevice, gj->cs));
          rf_status a = assemble_p(gj, false, gj->cs);
          if (a) return a;
          CU(cudaEventRecord(gj->join_out, gj->cs));
          CU(cudaStreamWaitEvent((cudaStream_t)s, gj->join_out, 0));
          F = gj->F_p;
        }
        bs.push_back({gj, j, (const double2*)F});
        owner.push_back(w);
        col.push_back(j);
      }
    }
    // every problem's active columns (kap - r consecutive systems) share its J;
    // batches of at most RF_MAXSYS systems, whole groups each
    const int share = kap - r;
    const size_t chunk = (size_t)(RF_MAXSYS / share) * share;
    for (size_t b0 = 0; b0 < bs.size(); b0 += chunk) {
      const size_t b1 = std::min(bs.size(), b0 + chunk);
      std::vector<BatchSys> part(bs.begin() + b0, bs.begin() + b1);
      std::vector<rf_status> st;
      std::vector<rf_solve_info> inf;
      const rf_solve_opts& so = ws[0]->o->solve;
      rf_status e = solve_batch(lead, part, share, so.rtol, so.max_it, st, inf, s);
      if (e) return e;
      for (size_t q = 0; q < part.size(); ++q) {
        LimexWork* w = owner[b0 + q];
        ++w->solves;
        w->iters += inf[q].iterations;
        if (st[q] == RF_ENOTCONV) {
          w->worst = RF_ENOTCONV;
        } else if (st[q] != RF_OK && w->st == RF_OK) {
          w->st = st[q];
          char buf[160];
          snprintf(buf, sizeof buf, "LIMEX column %d: %s", col[b0 + q], rf_status_string(st[q]));
          w->msg = buf;
        }
        if (st[q] == RF_OK || st[q] == RF_ENOTCONV)
          launch_axpy_pairs(d.nv, (double2*)(w->g->T + (size_t)col[b0 + q] * 2 * d.nv), part[q].g->K.x, s);
      }
    }
  }
  return RF_OK;
}

// extrapolation, error estimate, step-size proposal, the state out if accepted
static rf_status limex_finish(LimexWork& w, void* s) {
  rf_grid* g = w.g;
  const Dims& d = g->d;
  const int kap = w.o->kappa;
  launch_extrapolate(2 * d.nv, kap, g->T, s);
  const double* Tkk = g->T;
  const double* Tkk1 = g->T + 2 * d.nv;
  launch_error_norms(d, g->h, Tkk, kap > 1 ? Tkk1 : Tkk, g->norms, g->K.partial, s);
  double nrm[4];
  CU(cudaMemcpyAsync(nrm, g->norms, sizeof nrm, cudaMemcpyDeviceToHost, (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  double vol = 1.0;
  for (int a = 0; a < d.dim; ++a) vol *= (double)((a == 0 ? d.nx : a == 1 ? d.ny : d.nz) - 1) * g->h[a];
  const double alpha = 1.0 / (nrm[0] + 1e-30);
  const double beta = 1.0 / (nrm[2] + 1e-4 * vol);
  const double eps = std::sqrt((alpha * nrm[1] + beta * nrm[3]) / 2.0);
  const rf_limex_opts* o = w.o;
  double fac = (eps > 0.0) ? std::pow(o->rho * o->tol / eps, 1.0 / 3.0) : o->fac_max;
  if (fac > o->fac_max) fac = o->fac_max;
  if (fac < o->fac_min) fac = o->fac_min;
  const int acc = (eps <= o->tol) && w.worst == RF_OK;
  if (acc) {
    rf_status st = pairs_out(g, d, Tkk, w.u, s);
    if (st) return st;
  }
  if (w.info) {
    w.info->eps = eps; w.info->H_new = w.H * fac; w.info->accepted = acc; w.info->solves = w.solves;
    w.info->iterations = w.iters; w.info->status = w.worst;
  }
  if (!std::isfinite(eps)) return fail(RF_ENONFINITE, "error estimate is not finite");
  return w.worst;
}

// Batched rounds (RF_LIMEX_BATCH=1/0 forces the choice; never with the
// double-FP32 operator).  By default a single step takes them on grids of at
// least 1M vertices and the concurrent column threads below that, as measured
// on GB300 for one kappa = 4 step of the lognormal-lenses recipe: 129^3 FP32
// GMG 206 ms batched against 220 ms concurrent and 264 ms sequential, 257^3
// 1389 ms against 1661 ms sequential, but 65^3 FP64 105 ms against 90 ms
// concurrent (there every kernel is latency-bound, and a round lasts as long
// as its slowest column while the threads let each column run ahead).  An
// ensemble is always batched (its groups fill the launches).
static bool limex_batched(const rf_limex_opts* o, int64_t nv = -1) {
  if (o->solve.outer != RF_OUTER_FP64) return false;
  const char* e = getenv("RF_LIMEX_BATCH");
  if (e) return atoi(e) != 0;
  return nv < 0 || nv >= 1000000;
}

extern "C" rf_status rf_limex_step(rf_grid* g, double* u, double H, const rf_limex_opts* o, rf_limex_info* info,
                                   void* s) {
  rf_status st = limex_check(g, u, H, o);
  if (st) return st;
  if (!limex_batched(o, g->d.nv)) return limex_step_columns(g, u, H, o, info, s);
  LimexWork w;
  w.g = g; w.u = u; w.H = H; w.o = o; w.info = info;
  st = limex_prepare(w, s);
  if (st == RF_ENOMEM) {
    cudaGetLastError();
    return limex_step_columns(g, u, H, o, info, s);   // no room for the column grids
  }
  if (st) return st;
  std::vector<LimexWork*> ws{&w};
  if ((st = limex_rounds(ws, s))) return st;
  if (w.st != RF_OK) return fail(w.st, "%s", w.msg.c_str());
  return limex_finish(w, s);
}

// ------------------------------------------------------------------ adaptive runs
extern "C" rf_status rf_limex_run(rf_grid* g, double* u, double H0, const rf_limex_run_opts* o,
                                  rf_limex_run_info* info, double* hist, int hist_cap, void* s) {
  if (!g || !u || !o) return fail(RF_EINVAL, "grid, u and options are required");
  if (!(H0 > 0.0) || !std::isfinite(H0)) return fail(RF_EINVAL, "H0 must be positive");
  if (o->max_steps <= 0 && !(o->t_end > 0.0)) return fail(RF_EINVAL, "give max_steps > 0 or t_end > 0");
  if (o->max_rejects < 0 || (hist_cap > 0 && !hist)) return fail(RF_EINVAL, "bad max_rejects or history buffer");
  rf_status st = limex_check(g, u, H0, &o->step);
  if (st) return st;
  double t = 0.0, H = H0;
  int acc = 0, rej = 0, solves = 0, iters = 0, steps = 0;
  bool last_rejected = false;
  rf_status result = RF_OK;
  for (;;) {
    if (o->max_steps > 0 && acc >= o->max_steps) break;
    if (o->t_end > 0.0 && !(t < o->t_end * (1.0 - 1e-12))) break;
    if (o->t_end > 0.0 && H > o->t_end - t) H = o->t_end - t;
    rf_limex_info si{};
    result = rf_limex_step(g, u, H, &o->step, &si, s);
    solves += si.solves;
    iters += si.iterations;
    if (hist && steps < hist_cap) {
      hist[3 * steps] = H;
      hist[3 * steps + 1] = si.eps;
      hist[3 * steps + 2] = si.accepted;
    }
    ++steps;
    if (result != RF_OK) break;
    double Hn = si.H_new;
    if (si.accepted) {
      t += H;
      ++acc;
      if (o->hold_after_reject && last_rejected && Hn > H) Hn = H;
      last_rejected = false;
    } else {
      ++rej;
      last_rejected = true;
      if (rej > o->max_rejects) {
        result = fail(RF_ENOTCONV, "LIMEX step control: more than %d rejected steps", o->max_rejects);
        break;
      }
    }
    H = (o->H_max > 0.0 && Hn > o->H_max) ? o->H_max : Hn;
  }
  if (info) {
    info->t = t; info->H_next = H; info->accepted = acc; info->rejected = rej; info->solves = solves;
    info->iterations = iters; info->steps = steps; info->status = result;
  }
  return result;
}

// ------------------------------------------------------------------ implicit Euler
extern "C" rf_status rf_ie_step(rf_grid* g, double* u, double H, const rf_ie_opts* o, rf_ie_info* info, void* s) {
  if (!g || !u || !o) return fail(RF_EINVAL, "grid, u and options are required");
  if (!(H > 0.0) || !std::isfinite(H)) return fail(RF_EINVAL, "H must be positive");
  if (!(o->atol >= 0.0) || !(o->rtol >= 0.0) || o->max_newton < 1) return fail(RF_EINVAL, "bad Newton parameters");
  const Dims& d = g->d;
  const size_t vb = sizeof(double) * 2 * d.nv;
  const bool shat = (g->pp.scheme & SCHEME_SHAT_STORAGE) != 0;
  if (!g->ie_old) {
    g->ie_old = (double*)dalloc(g, vb, s, false);
    if (!g->ie_old) return fail(RF_ENOMEM, "implicit Euler state allocation failed");
  }
  if (shat && !g->ie_swold) {
    g->ie_swold = (double*)dalloc(g, sizeof(double) * d.nv, s, false);
    if (!g->ie_swold) return fail(RF_ENOMEM, "implicit Euler storage allocation failed");
  }
  if (o->max_ls > 0 && !g->ie_uk) {
    g->ie_uk = (double*)dalloc(g, vb, s, false);
    if (!g->ie_uk) return fail(RF_ENOMEM, "implicit Euler line-search allocation failed");
  }
  rf_status st = pairs_in(g, d, u, g->u_p, s);
  if (st) return st;
  CU(cudaMemcpyAsync(g->ie_old, g->u_p, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
  if (shat) launch_storage_sw(d, g->pp, g->ie_old, g->pdmin, g->phi, g->pd, g->vol, g->ie_swold, s);
  const double shift = 1.0 / H;
  // ||R(u_p)||^2 into *r2 (F_p must hold F(u_p)); R into b_p
  auto residual = [&](double* r2) -> rf_status {
    const double* sw = nullptr;
    if (shat) {
      launch_storage_sw(d, g->pp, g->u_p, g->pdmin, g->phi, g->pd, g->vol, g->pn, s);   // pn: assembly scratch
      sw = g->pn;
    }
    launch_ie_residual(d.nv, g->F_p, g->u_p, g->ie_old, g->mdiag, sw, g->ie_swold, g->dir, g->pp.rho_w,
                       g->pp.rho_n, shift, (double*)g->b_p, g->norms, g->K.partial, s);
    CU(cudaMemcpyAsync(r2, g->norms, sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)s));
    CU(cudaStreamSynchronize((cudaStream_t)s));
    return RF_OK;
  };
  int newton = 0, linear = 0;
  double r0 = 0.0, r = 0.0;
  rf_status res = RF_OK;
  for (;;) {
    if ((st = assemble_p(g, true, s))) return st;   // F, J, M at the iterate
    double r2 = 0.0;
    if ((st = residual(&r2))) return st;
    if (!std::isfinite(r2)) { res = fail(RF_ENONFINITE, "implicit Euler residual is not finite"); break; }
    r = std::sqrt(r2);
    if (newton == 0) r0 = r;
    if (r <= o->atol || r <= o->rtol * r0) break;
    if (newton >= o->max_newton) { res = RF_ENOTCONV; break; }
    if ((st = rf_gmg_setup(g, &shift, 1, &o->gmg, s))) return st;
    rf_solve_info si{};
    rf_status ls = solve_p(g, 0, g->b_p, o->solve.rtol, o->solve.max_it, o->solve.outer, &si, s);
    linear += si.iterations;
    ++newton;
    if (ls != RF_OK) { res = ls; break; }
    if (o->max_ls <= 0) {
      launch_axpy_pairs(d.nv, (double2*)g->u_p, g->K.x, s);
      continue;
    }
    // backtracking on ||R||: lambda = 1, 1/2, ... (mdiag stays that of u_k:
    // the linear storage does not depend on u, the S hat one is recomputed)
    CU(cudaMemcpyAsync(g->ie_uk, g->u_p, vb, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
    double lam = 1.0;
    for (int k = 0;; ++k) {
      launch_axpby_pairs(d.nv, g->u_p, g->ie_uk, g->K.x, lam, s);
      if ((st = assemble_p(g, false, s))) return st;
      double rt2 = 0.0;
      if ((st = residual(&rt2))) return st;
      if ((std::isfinite(rt2) && std::sqrt(rt2) <= (1.0 - 1e-4 * lam) * r) || k >= o->max_ls) break;
      lam *= 0.5;
    }
  }
  if (info) { info->newton = newton; info->linear = linear; info->res0 = r0; info->res = r; info->status = res; }
  if (res != RF_OK) {
    if (res == RF_ENOTCONV) return fail(res, "Newton did not converge in %d iterations (|R| %.3e of %.3e)", newton, r, r0);
    return res;
  }
  return pairs_out(g, d, g->u_p, u, s);
}

extern "C" rf_status rf_phase_mass(rf_grid* g, const double* u, double* mass_out, void* s) {
  if (!g || !u || !mass_out) return fail(RF_EINVAL, "grid, u and mass_out are required");
  rf_status st = pairs_in(g, g->d, u, g->u_p, s);
  if (st) return st;
  const double* sw = nullptr;
  if (g->pp.scheme & SCHEME_SHAT_STORAGE) {
    launch_storage_sw(g->d, g->pp, g->u_p, g->pdmin, g->phi, g->pd, g->vol, g->Se, s);   // Se: scratch
    sw = g->Se;
  }
  launch_phase_mass(g->d.nv, g->pp.rho_w, g->pp.rho_n, g->phiv, g->u_p, sw, g->norms, g->K.partial, s);
  CU(cudaMemcpyAsync(mass_out, g->norms, sizeof(double) * 2, cudaMemcpyDeviceToHost, (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  return RF_OK;
}

// ------------------------------------------------------------------ ensembles
// The ensemble with each problem's whole step on its own stream and host
// worker (RF_LIMEX_BATCH=0, or any problem with the double-FP32 operator).
static rf_status limex_batched_threads(rf_grid* const* grids, double* const* u, const double* H, int nprob,
                                       const rf_limex_opts* o, rf_limex_info* infos, int max_concurrent,
                                       void* stream) {
  int workers = max_concurrent > 0 ? max_concurrent : (nprob < 16 ? nprob : 16);
  if (workers > nprob) workers = nprob;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  // every problem's work is ordered after `stream`
  cudaEvent_t start;
  CU(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  CU(cudaEventRecord(start, (cudaStream_t)stream));
  for (int i = 0; i < nprob; ++i) CU(cudaStreamWaitEvent(grids[i]->cs, start, 0));
  std::vector<rf_status> st(nprob, RF_OK);
  std::vector<std::string> msg(nprob);
  std::atomic<int> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    const bool was = t_in_batch;
    t_in_batch = true;   // the problems already run side by side: columns one after another
    for (int i = next.fetch_add(1); i < nprob; i = next.fetch_add(1)) {
      rf_grid* g = grids[i];
      st[i] = rf_limex_step(g, u[i], H[i], &o[i], &infos[i], g->cs);
      infos[i].status = st[i];
      if (st[i] != RF_OK) msg[i] = t_err;
    }
    t_in_batch = was;
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  // `stream` waits for every problem
  for (int i = 0; i < nprob; ++i) {
    CU(cudaEventRecord(grids[i]->join_out, grids[i]->cs));
    CU(cudaStreamWaitEvent((cudaStream_t)stream, grids[i]->join_out, 0));
  }
  cudaEventDestroy(start);
  for (int i = 0; i < nprob; ++i)
    if (st[i] != RF_OK) return fail(st[i], "problem %d: %s", i, msg[i].c_str());
  return RF_OK;
}

static double wall_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// problems whose columns can share batched launches: equal grid shapes, options
static bool same_group(const rf_grid* a, const rf_limex_opts& oa, const rf_grid* b, const rf_limex_opts& ob) {
  return a->d.nx == b->d.nx && a->d.ny == b->d.ny && a->d.nz == b->d.nz && a->d.dim == b->d.dim &&
         oa.kappa == ob.kappa && oa.gmg.nlevels == ob.gmg.nlevels && oa.gmg.smoother == ob.gmg.smoother &&
         oa.gmg.nu1 == ob.gmg.nu1 && oa.gmg.nu2 == ob.gmg.nu2 && oa.gmg.omega == ob.gmg.omega &&
         oa.gmg.precision == ob.gmg.precision && oa.solve.rtol == ob.solve.rtol && oa.solve.max_it == ob.solve.max_it;
}

extern "C" rf_status rf_limex_step_batched(rf_grid* const* grids, double* const* u, const double* H, int nprob,
                                           const rf_limex_opts* o, rf_limex_info* infos, int max_concurrent,
                                           void* stream) {
  if (!grids || !u || !H || !o || !infos || nprob < 1) return fail(RF_EINVAL, "grids, u, H, opts, infos and nprob >= 1 are required");
  for (int i = 0; i < nprob; ++i) {
    if (!grids[i] || !u[i]) return fail(RF_EINVAL, "problem %d: grid and u are required", i);
    for (int k = 0; k < i; ++k)
      if (grids[k] == grids[i]) return fail(RF_EINVAL, "problem %d repeats the grid of problem %d", i, k);
    rf_status c = limex_check(grids[i], u[i], H[i], &o[i]);
    if (c) return fail(c, "problem %d: %s", i, t_err.c_str());
  }
  bool batched = true;
  for (int i = 0; i < nprob; ++i) batched = batched && limex_batched(&o[i]);
  if (!batched) return limex_batched_threads(grids, u, H, nprob, o, infos, max_concurrent, stream);
  int workers = max_concurrent > 0 ? max_concurrent : (nprob < 16 ? nprob : 16);
  if (workers > nprob) workers = nprob;
  int dev = 0;
  CU(cudaGetDevice(&dev));
  const double t_start = wall_ms();
  std::vector<LimexWork> W(nprob);
  for (int i = 0; i < nprob; ++i) {
    W[i].g = grids[i]; W[i].u = u[i]; W[i].H = H[i]; W[i].o = &o[i]; W[i].info = &infos[i];
  }
  // Groups of equal shapes share batched rounds.  Each group runs as a
  // pipeline on its own host thread: its members' assembly and multigrid
  // set-up (each on the member's stream, by a few worker threads), then its
  // rounds and the members' extrapolation on the lead grid's stream.  Groups of
  // larger grids start first, and the groups' launches overlap on the GPU.
  std::vector<std::vector<LimexWork*>> groups;
  {
    std::vector<int> done(nprob, 0);
    for (int i = 0; i < nprob; ++i) {
      if (done[i]) continue;
      std::vector<LimexWork*> grp;
      for (int k = i; k < nprob; ++k)
        if (!done[k] && same_group(grids[i], o[i], grids[k], o[k])) {
          done[k] = 1;
          grp.push_back(&W[k]);
        }
      groups.push_back(grp);
    }
    std::stable_sort(groups.begin(), groups.end(), [](const std::vector<LimexWork*>& a, const std::vector<LimexWork*>& b) {
      return a[0]->g->d.nv * (int64_t)a.size() > b[0]->g->d.nv * (int64_t)b.size();
    });
  }
  // everything is ordered after `stream`
  cudaEvent_t start;
  CU(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  CU(cudaEventRecord(start, (cudaStream_t)stream));
  for (int i = 0; i < nprob; ++i) CU(cudaStreamWaitEvent(grids[i]->cs, start, 0));
  const int per_group = std::max(1, workers / std::max<int>(1, (int)groups.size()));
  std::vector<rf_status> gst(groups.size(), RF_OK);
  std::vector<std::string> gmsg(groups.size());
  std::vector<double> gms(groups.size(), 0.0), gprep(groups.size(), 0.0);
  auto run_group = [&](size_t q) {
    cudaSetDevice(dev);
    const double t0 = wall_ms();
    std::vector<LimexWork*>& all = groups[q];
    std::atomic<int> next{0};
    auto prep = [&]() {
      cudaSetDevice(dev);
      for (int i = next.fetch_add(1); i < (int)all.size(); i = next.fetch_add(1)) {
        LimexWork* w = all[i];
        rf_status st = limex_prepare(*w, w->g->cs);
        if (st) { w->st = st; w->msg = t_err; }
      }
    };
    {
      std::vector<std::thread> pool;
      for (int k = 1; k < std::min<int>(per_group, (int)all.size()); ++k) pool.emplace_back(prep);
      prep();
      for (auto& t : pool) t.join();
    }
    gprep[q] = wall_ms() - t0;
    std::vector<LimexWork*> grp;
    for (LimexWork* w : all)
      if (w->st == RF_OK) grp.push_back(w);
    if (!grp.empty()) {
      cudaStream_t gs = grp[0]->g->cs;
      rf_status st = limex_rounds(grp, gs);
      if (st == RF_OK)
        for (LimexWork* w : grp) {
          const rf_status f = limex_finish(*w, gs);
          if (f == RF_ENOTCONV) w->worst = RF_ENOTCONV;
          else if (f != RF_OK) { w->st = f; w->msg = t_err; }
        }
      if (st != RF_OK) { gst[q] = st; gmsg[q] = t_err; }
      cudaStreamSynchronize(gs);
    }
    gms[q] = wall_ms() - t0;
  };
  {
    std::vector<std::thread> gt;
    for (size_t q = 1; q < groups.size(); ++q) gt.emplace_back(run_group, q);
    if (!groups.empty()) run_group(0);
    for (auto& t : gt) t.join();
  }
  cudaEventDestroy(start);
  if (getenv("RF_BATCH_VERBOSE")) {
    fprintf(stderr, "rf batched LIMEX: %d problems, %zu groups:", nprob, groups.size());
    for (size_t q = 0; q < groups.size(); ++q)
      fprintf(stderr, " [%zu x %dx%dx%d: prepare %.1f ms, all %.1f ms]", groups[q].size(), groups[q][0]->g->d.nx,
              groups[q][0]->g->d.ny, groups[q][0]->g->d.nz, gprep[q], gms[q]);
    fprintf(stderr, " total %.1f ms\n", wall_ms() - t_start);
  }
  for (size_t q = 0; q < groups.size(); ++q)
    if (gst[q] != RF_OK) return fail(gst[q], "%s", gmsg[q].c_str());
  rf_status first = RF_OK;
  for (int i = 0; i < nprob; ++i) {
    const rf_status st = W[i].st != RF_OK ? W[i].st : W[i].worst;
    infos[i].status = st;
    if (st != RF_OK && first == RF_OK) {
      first = st;
      t_err = "problem " + std::to_string(i) + ": " + (W[i].msg.empty() ? rf_status_string(st) : W[i].msg);
    }
  }
  // `stream` waits for every problem's stream
  for (int i = 0; i < nprob; ++i) {
    CU(cudaEventRecord(grids[i]->join_out, grids[i]->cs));
    CU(cudaStreamWaitEvent((cudaStream_t)stream, grids[i]->join_out, 0));
  }
  return first;
}

// ------------------------------------------------------------------ test hooks
extern "C" rf_status rf_export_jacobian(rf_grid* g, double* J_host, double* md_host, void* s) {
  if (!g) return fail(RF_EINVAL, "grid is required");
  if (!g->have_J) return fail(RF_EINVAL, "no Jacobian assembled yet");
  const Dims& d = g->d;
  if (J_host) {
    double* tmp = (double*)dalloc(g, sizeof(double) * 4 * d.nb * d.nv, s, true);
    if (!tmp) return fail(RF_ENOMEM, "export buffer");
    launch_export_level(d, true, g->J, nullptr, nullptr, 0.0, tmp, s);
    CU(cudaMemcpyAsync(J_host, tmp, sizeof(double) * 4 * d.nb * d.nv, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    CU(cudaStreamSynchronize((cudaStream_t)s));
    // keep the hierarchy list consistent: release just this buffer
    Alloc a = g->gbufs.back();
    g->gbufs.pop_back();
    if (g->user_alloc) g->alloc.free(a.p, a.bytes, s, g->alloc.ctx); else cudaFree(a.p);
  }
  if (md_host) return pairs_out(g, d, g->mdiag, md_host, s);
  return RF_OK;
}

static void tmp_release(rf_grid* g, int count, void* s);
static void* tmp_alloc(rf_grid* g, size_t bytes, void* s);

extern "C" rf_status rf_export_rows(rf_grid* g, const int64_t* verts, int count, double* J_host, double* md_host,
                                    void* s) {
  if (!g || !verts || count < 1 || !J_host || !md_host) return fail(RF_EINVAL, "grid, vertices and outputs are required");
  if (!g->have_J) return fail(RF_EINVAL, "no Jacobian assembled yet");
  for (int r = 0; r < count; ++r)
    if (verts[r] < 0 || verts[r] >= g->d.nv) return fail(RF_EINVAL, "vertex %lld out of range", (long long)verts[r]);
  const Dims& d = g->d;
  int64_t* dv = (int64_t*)tmp_alloc(g, sizeof(int64_t) * count, s);
  double* dj = (double*)tmp_alloc(g, sizeof(double) * 4 * d.nb * count, s);
  double* dm = (double*)tmp_alloc(g, sizeof(double) * 2 * count, s);
  if (!dv || !dj || !dm) { tmp_release(g, 3, s); return fail(RF_ENOMEM, "export buffers"); }
  cudaError_t e = cudaMemcpyAsync(dv, verts, sizeof(int64_t) * count, cudaMemcpyHostToDevice, (cudaStream_t)s);
  if (e == cudaSuccess) {
    launch_gather_rows(d, g->J, g->mdiag, dv, count, dj, dm, s);
    e = cudaMemcpyAsync(J_host, dj, sizeof(double) * 4 * d.nb * count, cudaMemcpyDeviceToHost, (cudaStream_t)s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(md_host, dm, sizeof(double) * 2 * count, cudaMemcpyDeviceToHost, (cudaStream_t)s);
  tmp_release(g, 3, s);
  if (e != cudaSuccess) return fail(RF_ECUDA, "export rows: %s", cudaGetErrorString(e));
  return RF_OK;
}

static void* tmp_alloc(rf_grid* g, size_t bytes, void* s) {
  void* p = dalloc(g, bytes, s, true);
  return p;
}
static void tmp_release(rf_grid* g, int count, void* s) {
  cudaStreamSynchronize((cudaStream_t)s);
  for (int i = 0; i < count && !g->gbufs.empty(); ++i) {
    Alloc a = g->gbufs.back();
    g->gbufs.pop_back();
    if (g->user_alloc) g->alloc.free(a.p, a.bytes, s, g->alloc.ctx); else cudaFree(a.p);
  }
}

extern "C" rf_status rf_export_level(rf_grid* g, int level, int sh, double* A_host, int64_t dims_out[3], void* s) {
  if (!g || !A_host) return fail(RF_EINVAL, "grid and output are required");
  if (!g->gmg_ready) return fail(RF_EINVAL, "no multigrid hierarchy");
  if (level < 0 || level >= g->nl || sh < 0 || sh >= g->nshift) return fail(RF_EINVAL, "level/shift out of range");
  const Level& Lv = g->L[level];
  const Dims& d = Lv.d;
  if (dims_out) { dims_out[0] = d.nx; dims_out[1] = d.ny; dims_out[2] = d.nz; }
  const size_t bytes = sizeof(double) * 4 * d.nb * d.nv;
  double* tmp = (double*)tmp_alloc(g, bytes, s);
  if (!tmp) return fail(RF_ENOMEM, "export buffer");
  if (level == 0) launch_export_level(d, true, g->J, nullptr, g->mdiag, g->shifts[sh], tmp, s);
  else launch_export_level(d, false, Lv.Jc, Lv.Mc, nullptr, g->shifts[sh], tmp, s);
  cudaError_t e = cudaMemcpyAsync(A_host, tmp, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)s);
  tmp_release(g, 1, s);
  if (e != cudaSuccess) return fail(RF_ECUDA, "export copy: %s", cudaGetErrorString(e));
  return RF_OK;
}

// host natural doubles -> level vector in the preconditioner type (parity split, padded)
static rf_status level_in(rf_grid* g, const Dims& d, const double* host, void* dst, double* tmp_nat, double* tmp_p,
                          void* s) {
  CU(cudaMemcpyAsync(tmp_nat, host, sizeof(double) * 2 * d.nv, cudaMemcpyHostToDevice, (cudaStream_t)s));
  if (g->kind == STORE_F64) {
    launch_perm_to_p(d, tmp_nat, (double*)dst, s);
  } else {
    launch_perm_to_p(d, tmp_nat, tmp_p, s);
    launch_cast_f64_to_f32(tmp_p, (float*)dst, 2 * d.nv, s);
  }
  return RF_OK;
}

static rf_status level_out(rf_grid* g, const Dims& d, const void* src, double* host, double* tmp_nat, double* tmp_p,
                           void* s) {
  const double* pp = (const double*)src;
  if (g->kind != STORE_F64) {
    launch_cast_f32_to_f64((const float*)src, tmp_p, 2 * d.nv, s);
    pp = tmp_p;
  }
  launch_perm_from_p(d, pp, tmp_nat, s);
  CU(cudaMemcpyAsync(host, tmp_nat, sizeof(double) * 2 * d.nv, cudaMemcpyDeviceToHost, (cudaStream_t)s));
  CU(cudaStreamSynchronize((cudaStream_t)s));
  return RF_OK;
}

extern "C" rf_status rf_apply(rf_grid* g, int op, int level, int sh, const double* in0, const double* in1,
                              double* out, void* s) {
  if (!g || !in0 || !out) return fail(RF_EINVAL, "grid, in0 and out are required");
  if (op == RF_OP_SPMV) {
    if (!g->have_J) return fail(RF_EINVAL, "no Jacobian assembled");
    if (!g->gmg_ready && sh != 0) return fail(RF_EINVAL, "shift index without hierarchy");
  } else if (!g->gmg_ready) {
    return fail(RF_EINVAL, "no multigrid hierarchy");
  }
  if (sh < 0 || (g->gmg_ready && sh >= g->nshift)) return fail(RF_EINVAL, "shift out of range");
  if (level < 0 || level >= (g->gmg_ready ? g->nl : 1)) return fail(RF_EINVAL, "level out of range");
  const bool two = (op == RF_OP_SMOOTH || op == RF_OP_RESIDUAL || op == RF_OP_PROLONG);
  if (two && !in1) return fail(RF_EINVAL, "this operation needs in1");
  if ((op == RF_OP_RESTRICT || op == RF_OP_PROLONG) && level >= g->nl - 1) return fail(RF_EINVAL, "no coarser level");
  if (op == RF_OP_COARSE && level != g->nl - 1) return fail(RF_EINVAL, "RF_OP_COARSE works on the coarsest level");
  const Dims& d = g->L[level].d;
  const Dims& dc = (level + 1 < g->nl) ? g->L[level + 1].d : d;
  const Dims& dl = (op == RF_OP_PROLONG) ? dc : d;   // dims of in0
  const int64_t nmax = g->d.nv;
  double* tnat = (double*)tmp_alloc(g, sizeof(double) * 2 * nmax, s);
  double* tp = (double*)tmp_alloc(g, sizeof(double) * 2 * nmax, s);
  const size_t te = t_size(g->kind);
  void* v0 = dvec(g, g->d, te, s, true);
  void* v1 = dvec(g, g->d, te, s, true);
  void* v2 = dvec(g, g->d, te, s, true);
  if (!tnat || !tp || !v0 || !v1 || !v2) { tmp_release(g, 5, s); return fail(RF_ENOMEM, "rf_apply buffers"); }
  rf_status st = RF_OK;
  if (op == RF_OP_SPMV) {
    const double shift = g->gmg_ready ? g->shifts[sh] : 0.0;
    double* xp = (double*)dvec(g, g->d, sizeof(double), s, true);
    if (!xp) { tmp_release(g, 5, s); return fail(RF_ENOMEM, "rf_apply buffers"); }
    CU(cudaMemcpyAsync(tnat, in0, sizeof(double) * 2 * d.nv, cudaMemcpyHostToDevice, (cudaStream_t)s));
    launch_perm_to_p(d, tnat, xp, s);
    launch_spmv64(d, g->nb, g->J, g->mdiag, shift, xp, false, (double2*)tp, s);
    launch_perm_from_p(d, tp, tnat, s);
    CU(cudaMemcpyAsync(out, tnat, sizeof(double) * 2 * d.nv, cudaMemcpyDeviceToHost, (cudaStream_t)s));
    CU(cudaStreamSynchronize((cudaStream_t)s));
    tmp_release(g, 6, s);
    return RF_OK;
  }
  if ((st = level_in(g, dl, in0, v0, tnat, tp, s))) { tmp_release(g, 5, s); return st; }
  if (two && (st = level_in(g, d, in1, v1, tnat, tp, s))) { tmp_release(g, 5, s); return st; }
  LevelOp L = level_op(g, level, sh);
  const Dims* dout = &d;
  switch (op) {
    case RF_OP_VCYCLE:
      vcycle_level(g, 0, sh, v0, v2, s);
      break;
    case RF_OP_SMOOTH:
      if (g->gopt.smoother == RF_SMOOTH_JACOBI) {
        launch_jacobi(L, v0, v1, v2, g->gopt.omega, false, s);
      } else {
        CU(cudaMemcpyAsync(v2, v1, (size_t)d.nv * 2 * te, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
        launch_gs_sweep(L, v0, v2, true, false, s);
      }
      break;
    case RF_OP_RESIDUAL:
      launch_residual(L, v0, v1, v2, s);
      break;
    case RF_OP_RESTRICT:
      launch_restrict(L, level_op(g, level + 1, sh), v0, v2, s);
      dout = &dc;
      break;
    case RF_OP_PROLONG:
      CU(cudaMemcpyAsync(v2, v1, (size_t)d.nv * 2 * te, cudaMemcpyDeviceToDevice, (cudaStream_t)s));
      launch_prolong(L, level_op(g, level + 1, sh), v0, v2, s);
      break;
    case RF_OP_COARSE:
      launch_coarse_solve(L, g->Ainv[sh], v0, v2, s);
      break;
    default:
      tmp_release(g, 5, s);
      return fail(RF_EINVAL, "unknown operation %d", op);
  }
  CU(cudaGetLastError());
  st = level_out(g, *dout, v2, out, tnat, tp, s);
  tmp_release(g, 5, s);
  return st;
}
