// hz_measure_fp64_rate: the FP64 FMA throughput of the current device, measured.
//
// The Krylov kernels of the solver are bound by GB300's FP64 pipe rather than by HBM, so their
// roofline needs the pipe's rate on this GPU at its present clocks. The probe runs independent
// DFMA chains in full warps on every SM (enough warps and chains per warp to hide the pipe's
// latency) and times them with CUDA events on the caller's stream.
#include <cuda_runtime.h>

#include "hz_internal.h"

namespace hz {
namespace {

constexpr int PROBE_THREADS = 256;

__device__ double g_probe_sink;

template <int CHAINS>
__global__ void __launch_bounds__(PROBE_THREADS) dfma_probe_kernel(int iters, double a, double b) {
  double acc[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c] = fma(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += acc[c];
  // a store the compiler cannot drop, taken only for a value the chains never reach
  if (s == -1.0) g_probe_sink = s;
}

// One timed launch of CHAINS-chain threads, `per_sm` blocks per SM; FMAs per ms, or < 0 on error.
template <int CHAINS>
double probe_rate(int sms, int per_sm, int iters, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
  const dim3 grid(sms * per_sm);
  // a = 1 - 2^-30 and b small keep the chains finite and away from subnormals
  const double a = 1.0 - 9.313225746154785e-10, b = 1e-9;
  dfma_probe_kernel<CHAINS><<<grid, PROBE_THREADS, 0, s>>>(iters / 8 + 1, a, b);  // warm-up
  cudaEventRecord(e0, s);
  dfma_probe_kernel<CHAINS><<<grid, PROBE_THREADS, 0, s>>>(iters, a, b);
  cudaEventRecord(e1, s);
  float t = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&t, e0, e1) != cudaSuccess || !(t > 0.f))
    return -1.0;
  return (double)grid.x * PROBE_THREADS * CHAINS * (double)iters / t;
}

}  // namespace
}  // namespace hz

extern "C" hz_status hz_measure_fp64_rate(int iters, void* stream, double* tflops, double* ms) {
  if (!tflops || iters < 1 || iters > (1 << 24)) return HZ_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return HZ_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return HZ_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HZ_ECUDA;
  }
  // the best of a few shapes: 4 or 8 blocks of 256 threads per SM, 8 or 16 independent chains
  double best = -1.0, best_ms = 0.0;
  bool failed = false;
  for (int per_sm : {4, 8}) {
    for (int chains : {8, 16}) {
      const double r = chains == 8 ? hz::probe_rate<8>(sms, per_sm, iters, s, e0, e1)
                                   : hz::probe_rate<16>(sms, per_sm, iters, s, e0, e1);
      if (r < 0) {
        failed = true;
        break;
      }
      if (r > best) {
        best = r;
        best_ms = (double)sms * per_sm * hz::PROBE_THREADS * chains * (double)iters / r;
      }
    }
    if (failed) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (failed || !(best > 0)) return HZ_ECUDA;
  *tflops = 2.0 * best * 1e3 / 1e12;
  if (ms) *ms = best_ms;
  return HZ_OK;
}
