// noalloc.cu — rf_dense_inverse_noalloc: the library's one entry point that
// allocates no memory at all.
//
// Everything else in this library takes device memory from the grid's
// allocator.  Some callers cannot call cudaMalloc: applications whose device
// memory is owned entirely by another allocator (a framework's caching pool
// or a fixed per-process budget) and code on latency-critical paths that must
// not pay for cudaMalloc/cudaFree, which may synchronise the device.  For them
// this entry point inverts a dense FP64 matrix (the operation the multigrid
// set-up applies to the coarsest-level operator) with its working storage in
// a file-scope device array that the library reserves when it is loaded.
//
// The array holds the LU factors, the pivots and a status word for matrices up
// to RF_NOALLOC_MAX_N x RF_NOALLOC_MAX_N (the inverse's per-column vectors live
// in the kernel's shared memory).  Every GPU that loads the library keeps it
// (about 2 MiB) until the process exits.
// All calls on a device share it: two calls whose work overlaps on the GPU
// (different streams, or different host threads) race on it and must be
// serialised by the caller.  The status word is cleared by every call; the
// rest is overwritten before it is read.
#include <mutex>

#include "rf.h"
#include "rf_common.cuh"
#include "rf_kernels.h"

namespace {

constexpr int kMaxN = RF_NOALLOC_MAX_N;
constexpr size_t kMat = (size_t)kMaxN * kMaxN;          // doubles per N x N matrix
// layout in doubles: [LU: kMat][pivots: kMaxN ints][status: 1 int], padded
constexpr size_t kWords = kMat + kMaxN / 2 + 64;

static __device__ __align__(256) double g_noalloc_scratch[kWords];

std::mutex g_mu;
constexpr int kMaxDevices = 256;
void* g_scratch_addr[kMaxDevices] = {};   // device address of the array, per device

// The device address of the scratch array on the current device; looked up once
// per device (the array's host-side name is not a device address).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// Whether p is memory the kernels of the CURRENT device may use: device memory
// of that device, or managed memory.  Memory of another GPU is refused: the
// copy into the scratch array would cross devices and the kernel would write
// Ainv through a peer mapping that may not exist.
bool on_this_device(const void* p) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" rf_status rf_dense_inverse_noalloc(int N, const double* A, double* Ainv, void* stream) {
  if (N < 1 || N > kMaxN) return RF_EINVAL;   // beyond the reserved scratch
  if (!A || !Ainv) return RF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
    cudaGetLastError();
    return RF_EINVAL;
  }
  if (cap != cudaStreamCaptureStatusNone) return RF_EINVAL;   // the read-back below cannot be captured
  if (!on_this_device(A) || !on_this_device(Ainv)) return RF_EINVAL;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return RF_ECUDA;
  double* LU = static_cast<double*>(base);
  int* piv = reinterpret_cast<int*>(LU + kMat);
  int* status = piv + kMaxN;
  if (cudaMemcpyAsync(LU, A, sizeof(double) * (size_t)N * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return RF_ECUDA;
  if (cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) return RF_ECUDA;
  if (rf::launch_dense_inverse(N, LU, Ainv, piv, nullptr, status, stream) != cudaSuccess) return RF_ECUDA;
  int h = 0;
  if (cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return RF_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return RF_ECUDA;
  return h ? RF_ENONFINITE : RF_OK;
}
