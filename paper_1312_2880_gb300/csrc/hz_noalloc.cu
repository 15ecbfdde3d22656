// hz_apply_dot_noalloc: v = A u with dot = <w, v> in one pass, allocating nothing.
//
// Some callers cannot allocate device memory when they call into this library: hosts that own
// every byte of the device through their own pool (a framework's caching allocator, a memory
// budget enforced by a serving runtime), where a stray cudaMalloc fragments or oversubscribes
// the pool, and latency-critical loops, where cudaMalloc and cudaFree may synchronise the
// device. This entry point needs no problem object and no arena: the caller passes the inputs
// and the outputs, and the only scratch (per-block partial sums and a completion counter) is a
// fixed, file-scope __device__ array that every device holding this library keeps until the
// process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "hz_common.cuh"
#include "hz_internal.h"

namespace hz {
namespace {

constexpr int NB = 256;                 // threads per block
constexpr int MAX_BLOCKS = 2048;        // partial sums the scratch holds (two doubles per block)
constexpr int MAX_DEVICES = 64;
constexpr size_t SCRATCH_BYTES = 256 + sizeof(double) * 2 * MAX_BLOCKS;  // counter slot + partials

// Scratch shared by every call on a device: bytes [0, 4) hold the block counter, bytes [256, ...)
// the per-block partial sums. In host code this name is only a host-side stand-in; the device
// address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

std::mutex g_mutex;
void* g_scratch_ptr[MAX_DEVICES] = {};

__global__ void __launch_bounds__(NB) apply_dot_static_kernel(double2* __restrict__ v, double2* __restrict__ dot,
                                                               const double2* __restrict__ u,
                                                               const double2* __restrict__ w,
                                                               const double* __restrict__ kh, int n, double beta,
                                                               double out_scale, unsigned char* __restrict__ scratch) {
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + 256);
  const int wdt = n + 1;
  const int N = wdt * wdt;
  double re = 0.0, im = 0.0;
  for (int e = blockIdx.x * NB + threadIdx.x; e < N; e += gridDim.x * NB) {
    const int j = e / wdt, i = e - j * wdt;
    Nbr b = neighbours(i, j, n);
    double2 nb = cadd<double>(cadd<double>(u[j * wdt + b.iw], u[j * wdt + b.ie]),
                              cadd<double>(u[b.js * wdt + i], u[b.jn * wdt + i]));
    double2 a = cadd<double>(cmul<double>(row_diag<double>(kh[e], b.sides, beta), u[e]), nb);
    a = make_double2(a.x * out_scale, a.y * out_scale);
    v[e] = a;
    double2 ww = w[e];
    re = fma(ww.x, a.x, fma(ww.y, a.y, re));
    im = fma(ww.x, a.y, fma(-ww.y, a.x, im));
  }
  // fixed-order block sum, then the last block adds the partials in block order
  __shared__ double s_re[NB / 32], s_im[NB / 32];
  __shared__ int is_last;
  for (int off = 16; off; off >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, off);
    im += __shfl_down_sync(0xffffffffu, im, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { s_re[warp] = re; s_im[warp] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double br = 0.0, bi = 0.0;
    for (int q = 0; q < NB / 32; ++q) { br += s_re[q]; bi += s_im[q]; }
    partials[2 * blockIdx.x] = br;
    partials[2 * blockIdx.x + 1] = bi;
    __threadfence();
    is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return;
  if (threadIdx.x == 0) {
    __threadfence();
    double tr = 0.0, ti = 0.0;
    for (int q = 0; q < (int)gridDim.x; ++q) {
      tr += __ldcg(&partials[2 * q]);
      ti += __ldcg(&partials[2 * q + 1]);
    }
    *dot = make_double2(tr, ti);
    *ticket = 0;
  }
}

// Device address of the scratch on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// True when the byte ranges [a, a + na) and [b, b + nb) share a byte.
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
  return pa < pb + nb && pb < pa + na;
}

}  // namespace
}  // namespace hz

extern "C" hz_status hz_apply_dot_noalloc(int n, const double* kh, double beta, const double* u, const double* w,
                                          double* v, double* dot, void* stream) {
  if (n < 2 || n > HZ_NOALLOC_MAX_N || !kh || !u || !w || !v || !dot) return HZ_EINVAL;
  {
    // v and dot are written while u, w and kh are still being read (by other blocks): no output
    // may share a byte with an input or with the other output.
    const size_t N = (size_t)(n + 1) * (size_t)(n + 1);
    const size_t cb = sizeof(double2) * N, rb = sizeof(double) * N, db = sizeof(double2);
    if (hz::overlaps(v, cb, u, cb) || hz::overlaps(v, cb, w, cb) || hz::overlaps(v, cb, kh, rb) ||
        hz::overlaps(dot, db, v, cb) || hz::overlaps(dot, db, u, cb) || hz::overlaps(dot, db, w, cb) ||
        hz::overlaps(dot, db, kh, rb))
      return HZ_EINVAL;
  }
  void* scratch = nullptr;
  if (hz::scratch_address(&scratch) != cudaSuccess) return HZ_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the counter must start at zero; partials are overwritten before they are read
  if (cudaMemsetAsync(scratch, 0, sizeof(unsigned int), s) != cudaSuccess) return HZ_ECUDA;
  long long N = (long long)(n + 1) * (n + 1);
  int G = (int)((N + hz::NB - 1) / hz::NB);
  if (G > hz::MAX_BLOCKS) G = hz::MAX_BLOCKS;
  double out_scale = (double)n * (double)n;
  hz::apply_dot_static_kernel<<<G, hz::NB, 0, s>>>((double2*)v, (double2*)dot, (const double2*)u, (const double2*)w,
                                                    kh, n, beta, out_scale, (unsigned char*)scratch);
  return cudaGetLastError() == cudaSuccess ? HZ_OK : HZ_ECUDA;
}
