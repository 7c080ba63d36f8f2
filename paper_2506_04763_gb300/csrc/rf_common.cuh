// rf_common.cuh — shared device/host definitions of the sm_103a kernels.
//
// Data layout in HBM ("parity-split" order, used by every internal array):
// within each x-line (fixed j,k) the even-x vertices come first, then the
// odd-x vertices:  p(i,j,k) = (j + ny*k)*nx + (i odd ? E + i/2 : i/2),
// E = (nx+1)/2.  One colour of the multicolour smoother (fixed parity in x,
// y, z) is then a set of contiguous runs, so its sweep reads the matrix with
// fully coalesced 16-byte loads.  A neighbour at offset (dx,dy,dz) lives at
// p + xoff(parity of i, dx) + dy*nx + dz*nx*ny with xoff(even) = {E-1, 0, E}
// and xoff(odd) = {-E, 0, 1-E}.
//
// Matrices are stored block-major ("structure of arrays" over vertices):
// block b of vertex p occupies entries [(b*nv + p)*4 .. +3], b = (dx+1) +
// 3(dy+1) [+ 9(dz+1)], entries (w,p_w),(w,S_n),(n,p_w),(n,S_n).  A warp that
// handles 32 consecutive vertices reads 512 B (FP32) or 1 KB (FP64)
// contiguous bytes per block.  Blocks that reach outside the grid hold zeros.
//
// Vectors are interleaved (p_w, S_n) pairs (double2 / float2) with a zero
// halo of `pad` pairs on both sides, so neighbour loads never leave the
// allocation; a neighbour outside the grid is multiplied by a zero block.
#pragma once
#include <utility>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#define RF_MAXL 12
#define RF_MAXSHIFT 4

namespace rf {

template <typename T> struct V2;
template <> struct V2<float> { typedef float2 t; };
template <> struct V2<double> { typedef double2 t; };

// Neighbour offsets of one level (by x-parity of the centre vertex).
struct Nbr {
  int off[2][27];
};

struct Dims {
  int nx, ny, nz, dim, nb, E;
  int64_t nv;
};

__host__ __device__ inline int64_t pidx(const Dims& d, int i, int j, int k) {
  return ((int64_t)j + (int64_t)d.ny * k) * d.nx + ((i & 1) ? d.E + (i >> 1) : (i >> 1));
}

// (i,j,k) of a parity-split index
__host__ __device__ inline void pcoords(const Dims& d, int64_t p, int& i, int& j, int& k) {
  int64_t line = p / d.nx;
  int pos = (int)(p - line * d.nx);
  i = (pos < d.E) ? 2 * pos : 2 * (pos - d.E) + 1;
  j = (int)(line % d.ny);
  k = (int)(line / d.ny);
}

__host__ __device__ inline int blk_of(int dim, int dx, int dy, int dz) {
  return dim == 3 ? (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1) : (dx + 1) + 3 * (dy + 1);
}

inline Dims make_dims(int dim, const int n[3]) {
  Dims d;
  d.dim = dim; d.nx = n[0]; d.ny = n[1]; d.nz = n[2];
  d.nb = dim == 3 ? 27 : 9;
  d.E = (n[0] + 1) / 2;
  d.nv = (int64_t)n[0] * n[1] * n[2];
  return d;
}

inline Nbr make_nbr(const Dims& d) {
  Nbr r;
  for (int par = 0; par < 2; ++par)
    for (int b = 0; b < 27; ++b) {
      int dx = b % 3 - 1, dy = (b / 3) % 3 - 1, dz = b / 9 - 1;
      if (d.dim == 2 && b >= 9) { r.off[par][b] = 0; continue; }
      int xo = dx == 0 ? 0 : (par == 0 ? (dx < 0 ? d.E - 1 : d.E) : (dx < 0 ? -d.E : 1 - d.E));
      r.off[par][b] = xo + dy * d.nx + (d.dim == 3 ? dz * d.nx * d.ny : 0);
    }
  return r;
}

// halo of a padded vector (in pairs), rounded for alignment
inline int64_t vec_pad(const Dims& d) {
  int64_t p = (int64_t)d.nx * d.ny + 2 * (int64_t)d.nx + 2;
  return (p + 63) / 64 * 64;
}

// Kernel launch accounting (every launch in this library goes through it).
void count_launch();
int grid_for(int64_t n, int block, int max_blocks_per_sm = 8);
int num_sms();
// Programmatic dependent launch for the solve-path kernels (RF_PDL=0 turns it off).
bool pdl_enabled();

// Every kernel launched through RF_LAUNCH_PDL starts with rf_pdl_begin(): it
// waits until the preceding kernel in the stream has completed and its writes
// are visible (griddepcontrol.wait; a no-op without a programmatic
// dependency), then lets the next kernel be launched early
// (griddepcontrol.launch_dependents takes effect once every block of this grid
// has issued it, i.e. when its last wave is resident, so the next grid's blocks
// only fill SMs that this grid no longer needs, and they wait in turn).
__device__ __forceinline__ void rf_pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launch with the programmatic-stream-serialisation attribute (the kernel
// must begin with rf_pdl_begin())
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
  count_launch();
  if (!pdl_enabled()) {
    kernel<<<grid, block, smem, stream>>>(std::forward<Args>(args)...);
    return;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace rf

#define RF_LAUNCH(kernel, grid, block, smem, stream, ...)                 \
  do {                                                                    \
    ::rf::count_launch();                                                 \
    kernel<<<(grid), (block), (smem), (cudaStream_t)(stream)>>>(__VA_ARGS__); \
  } while (0)

#define RF_LAUNCH_PDL(kernel, grid, block, smem, stream, ...) \
  ::rf::launch_pdl(kernel, dim3(grid), dim3(block), (size_t)(smem), (cudaStream_t)(stream), __VA_ARGS__)
