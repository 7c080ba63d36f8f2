// probe.cu — inspection hook rf_fp64_fma_rate: the FP64 fused multiply-add
// throughput of the current GPU, measured in the calling process.
//
// GB300's FP64 units are far slower than its FP32 units, so the FP64 kernels
// of the solve path (the outer operator, the BiCGSTAB vector updates, the
// assembly) can be bound by the FP64 pipe rather than by HBM.  Their
// roofline needs this peak next to the measured copy bandwidth.  The kernel
// runs 8 independent FMA chains per thread (enough to cover the pipe's
// latency), on 8 blocks of 256 threads per SM, and is timed with CUDA events
// on the caller's stream after one untimed launch.
#include "rf.h"
#include "rf_common.cuh"
#include "rf_kernels.h"

namespace {

// written only when the chains reach a value they never reach; keeps the
// compiler from removing the loop (no allocation needed)
__device__ double g_fma_sink;

__global__ void __launch_bounds__(256) k_fma64(int iters, double a, double c) {
  const double t = 1e-9 * (double)(blockIdx.x * blockDim.x + threadIdx.x);
  double x0 = t, x1 = t + 0.1, x2 = t + 0.2, x3 = t + 0.3, x4 = t + 0.4, x5 = t + 0.5, x6 = t + 0.6, x7 = t + 0.7;
  for (int i = 0; i < iters; ++i) {
    x0 = fma(x0, a, c); x1 = fma(x1, a, c); x2 = fma(x2, a, c); x3 = fma(x3, a, c);
    x4 = fma(x4, a, c); x5 = fma(x5, a, c); x6 = fma(x6, a, c); x7 = fma(x7, a, c);
  }
  const double s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  if (s == -1.0) g_fma_sink = s;   // never true: x stays positive
}

}  // namespace

extern "C" rf_status rf_fp64_fma_rate(void* stream, double* fma_per_s) {
  if (!fma_per_s) return RF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int blocks = rf::num_sms() * 8, threads = 256, iters = 1 << 14;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RF_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return RF_ECUDA; }
  rf_status st = RF_OK;
  float best = 1e30f;
  for (int rep = 0; rep < 4 && st == RF_OK; ++rep) {
    cudaEventRecord(e0, s);
    k_fma64<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7);
    rf::count_launch();
    cudaEventRecord(e1, s);
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = RF_ECUDA;
    else if (rep > 0 && ms < best) best = ms;   // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != RF_OK) return st;
  *fma_per_s = (double)blocks * threads * iters * 8.0 / (best * 1e-3);
  return RF_OK;
}
