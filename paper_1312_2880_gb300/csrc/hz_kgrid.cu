// Kaczmarz level (Sec. 4-5: Gauss-Seidel on the normal equations, 4 sweeps before and after the
// coarse-grid correction) held in global memory and relaxed by ONE persistent launch per pass.
//
// A colour phase is a set of independent row actions (rows of one colour have disjoint supports),
// so a pass is 5 nu phases that need ordering only between neighbouring rows: a row action reads
// and writes its 5-point support, rows j - 1 .. j + 1. Every block of the cooperative launch owns
// a band of whole grid rows (at least one) and runs the colour's rows in it; after a phase it
// publishes its progress, and before the next one it waits until the bands above and below have
// finished the same phase. The level (u, f~, k H: 20 bytes a node in FP32) stays in L2, and no
// block waits for the whole grid. Pre pass: zero guess, nu sweeps (colours 0..4), residual with
// the (B) operator and full weighting. Post pass: bilinear correction, nu sweeps (colours 4..0).
// The row action and the transfers are the per-launch kernels' (hz_gnode.cuh), in the same order,
// so this form gives the colour launches' bits.
//
// Why neighbours suffice (bands of at least three rows): phase k + 1 in band b reads and writes
// rows j0 - 1 .. j1; the writes of phase k to those rows come from row actions in rows
// j0 - 2 .. j1 + 1, all in bands b - 1, b, b + 1, which have finished it; and two rows of one
// colour never share a node, so bands running the same phase side by side never touch the same
// node. The restriction of coarse row J (fine row 2J in the band) reads u in rows 2J - 2 .. 2J + 2,
// whose last values come from row actions in rows j0 - 3 .. j1 + 2: again bands b - 1 .. b + 1.
//
// Progress counters live in device memory (BandSync), one per block, and advance by one per
// phase; comparisons use wrap-safe differences. A wait polls a bounded number of times; when it
// runs out (or finds the error word set) it sets the error word and every later wait of every
// block returns at once, so the launch always ends; the host reads the error word after the solve
// and reports HZ_ETIMEOUT.
#include <cuda_runtime.h>

#include <mutex>

#include "hz_common.cuh"
#include "hz_gnode.cuh"
#include "hz_internal.h"

namespace hz {

namespace {

constexpr int GT = 512;                        // threads per block
constexpr unsigned int SYNC_POLLS = 1u << 20;  // at most about 1 s of polls (L2 round trips) per wait

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Rows [j0, j1) of band b out of nb over the n + 1 grid rows (nb <= (n + 1) / 3: three rows or more).
struct Band {
  int j0, j1;
  __device__ Band(int b, int nb, int n) : j0((int)((long long)b * (n + 1) / nb)), j1((int)((long long)(b + 1) * (n + 1) / nb)) {}
};

// End of phase `done` (1-based count of phases this launch has finished): publish it, then wait
// until the neighbouring bands have published it too. Returns false once any wait has run out.
__device__ bool band_step(BandSync bs, unsigned int base, unsigned int done, int* s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = ld_acquire(bs.err) == 0u;
    if (ok) {
      const int b = blockIdx.x, nb = gridDim.x;
      const unsigned int target = base + done;
      // the band's writes, ordered before this thread by the barrier above, are released with
      // the progress (release at GPU scope is cumulative); the acquiring loads below order the
      // neighbours' writes before the block's next phase (through the barrier at the end)
      st_release(&bs.ctr[b], target);
      for (int side = 0; side < 2 && ok; ++side) {
        const int q = side ? b + 1 : b - 1;
        if (q < 0 || q >= nb) continue;
        unsigned int polls = 0;
        while ((int)(ld_acquire(&bs.ctr[q]) - target) < 0) {
          if (ld_acquire(bs.err) != 0u || ++polls > SYNC_POLLS) {
            atomicExch(bs.err, 1u);
            ok = false;
            break;
          }
        }
      }
    }
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return *s_ok != 0;
}

// One colour phase on the band's rows.
template <class T, class F2>
__device__ __forceinline__ void colour_phase(const Band& bd, c2<T>* u, int pu, const F2* f, int pf, const T* kh, int pk,
                                             int n, int colour, T beta) {
  const int w5 = (n + 5) / 5;
  const int slots = (bd.j1 - bd.j0) * w5;
  for (int s = threadIdx.x; s < slots; s += GT) {
    const int r = s / w5, m = s - r * w5, j = bd.j0 + r;
    const int i = ((colour - 2 * j) % 5 + 5) % 5 + 5 * m;
    if (i <= n) gnode::kacz_row<T, F2>(u, pu, f, pf, kh, pk, n, i, j, beta);
  }
}

template <class T, class F2>
__global__ void __launch_bounds__(GT) kacz_grid_pre_kernel(c2<T>* __restrict__ u, int pu, c2<T>* __restrict__ fc,
                                                           int pc, const F2* __restrict__ f, int pf,
                                                           const T* __restrict__ kh, int pk, int n, T bA, T bB,
                                                           int nu, const int* __restrict__ stop, BandSync bs) {
  pdl_enter();
  if (stop && stop[0]) return;
  __shared__ unsigned int s_base;
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_base = ld_acquire(&bs.ctr[blockIdx.x]);
  const Band bd(blockIdx.x, gridDim.x, n);
  const int w = n + 1;
  for (int q = threadIdx.x; q < (bd.j1 - bd.j0) * w; q += GT) {
    const int r = q / w, i = q - r * w;
    u[(long long)(bd.j0 + r) * pu + i] = c2<T>{0, 0};
  }
  __syncthreads();
  const unsigned int base = s_base;
  unsigned int done = 0;
  if (!band_step(bs, base, ++done, &s_ok)) return;
  for (int sweep = 0; sweep < nu; ++sweep)
    for (int ph = 0; ph < 5; ++ph) {
      colour_phase<T, F2>(bd, u, pu, f, pf, kh, pk, n, ph, bA);
      if (!band_step(bs, base, ++done, &s_ok)) return;
    }
  // coarse rows J whose fine row 2J lies in the band
  const int nc = n / 2, wc = nc + 1, J0 = (bd.j0 + 1) / 2, J1 = (bd.j1 + 1) / 2;
  for (int q = threadIdx.x; q < (J1 - J0) * wc; q += GT) {
    const int r = q / wc, I = q - r * wc, J = J0 + r;
    fc[(long long)J * pc + I] = gnode::restrict_node<T, F2>(u, pu, f, pf, kh, pk, n, bB, I, J);
  }
}

template <class T, class F2>
__global__ void __launch_bounds__(GT) kacz_grid_post_kernel(c2<T>* __restrict__ u, int pu,
                                                            const c2<T>* __restrict__ ec, int pc,
                                                            const F2* __restrict__ f, int pf,
                                                            const T* __restrict__ kh, int pk, int n, T bA, int nu,
                                                            const int* __restrict__ stop, BandSync bs) {
  pdl_enter();
  if (stop && stop[0]) return;
  __shared__ unsigned int s_base;
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_base = ld_acquire(&bs.ctr[blockIdx.x]);
  const Band bd(blockIdx.x, gridDim.x, n);
  const int w = n + 1;
  for (int q = threadIdx.x; q < (bd.j1 - bd.j0) * w; q += GT) {
    const int r = q / w, i = q - r * w;
    gnode::prolong_add_node<T>(u, pu, ec, pc, i, bd.j0 + r);
  }
  __syncthreads();
  const unsigned int base = s_base;
  unsigned int done = 0;
  for (int sweep = 0; sweep < nu; ++sweep)
    for (int ph = 0; ph < 5; ++ph) {
      if (!band_step(bs, base, ++done, &s_ok)) return;
      colour_phase<T, F2>(bd, u, pu, f, pf, kh, pk, n, 4 - ph, bA);
    }
  // the launch boundary orders the last phase before the next kernel; every band has published
  // the same number of phases, so the counters stay in step for the next launch
}

// Blocks of a level's cooperative launches: one band of at least three rows each, no more than
// both kernels of the precision can keep resident at once, nor than KGRID_MAX_BLOCKS. The pre and
// post launches of a level use the same count: they share the level's counters.
template <class KPre, class KPost>
int grid_blocks(KPre pre, KPost post, int n, int* cap_cache) {
  if (*cap_cache == 0) {
    int dev = 0, sms = 0, a = 0, b = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, pre, GT, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, post, GT, 0) != cudaSuccess || a < 1 || b < 1)
      return -1;
    const int cap = sms * (a < b ? a : b);
    *cap_cache = cap < KGRID_MAX_BLOCKS ? cap : KGRID_MAX_BLOCKS;
  }
  const int bands = (n + 1) / 3 > 0 ? (n + 1) / 3 : 1;
  return bands < *cap_cache ? bands : *cap_cache;
}

template <class K, class... Args>
cudaError_t coop_launch(K kernel, int blocks, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks, 1, 1);
  cfg.blockDim = dim3(GT, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__global__ void coop_probe_kernel(int* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *out = 1;
}

}  // namespace

bool kacz_grid_available() {
  static std::once_flag once;
  static bool ok = false;
  std::call_once(once, [] {
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
        !coop)
      return;
    // a cooperative launch captured into a graph, instantiated and run once
    cudaStream_t s = nullptr;
    int* d = nullptr;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    bool good = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
                cudaMalloc(&d, sizeof(int)) == cudaSuccess && cudaMemsetAsync(d, 0, sizeof(int), s) == cudaSuccess &&
                cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (good) {
      const bool launched = coop_launch(coop_probe_kernel, 2, s, d) == cudaSuccess;
      good = cudaStreamEndCapture(s, &g) == cudaSuccess && launched;
    }
    good = good && cudaGraphInstantiate(&ge, g, 0) == cudaSuccess && cudaGraphLaunch(ge, s) == cudaSuccess &&
           cudaStreamSynchronize(s) == cudaSuccess;
    int v = 0;
    good = good && cudaMemcpy(&v, d, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && v == 1;
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
    if (d) cudaFree(d);
    if (s) cudaStreamDestroy(s);
    cudaGetLastError();  // a refused capture leaves no error behind
    ok = good;
  });
  return ok;
}

int kgrid_blocks(bool fp32, int n) {
  static int cap32 = 0, cap64 = 0;
  return fp32 ? grid_blocks(kacz_grid_pre_kernel<float, float2>, kacz_grid_post_kernel<float, float2>, n, &cap32)
              : grid_blocks(kacz_grid_pre_kernel<double, double2>, kacz_grid_post_kernel<double, double2>, n, &cap64);
}

cudaError_t launch_kacz_grid_pre(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                 int pk, int n, double bA, double bB, int nu, const int* stop, BandSync bs,
                                 cudaStream_t s) {
  const int b = kgrid_blocks(fp32, n);
  if (b < 1) return cudaErrorInvalidConfiguration;
  if (fp32)
    return coop_launch(kacz_grid_pre_kernel<float, float2>, b, s, (float2*)u, pu, (float2*)fc, pc, (const float2*)f,
                       pf, (const float*)kh, pk, n, (float)bA, (float)bB, nu, stop, bs);
  return coop_launch(kacz_grid_pre_kernel<double, double2>, b, s, (double2*)u, pu, (double2*)fc, pc,
                     (const double2*)f, pf, (const double*)kh, pk, n, bA, bB, nu, stop, bs);
}

cudaError_t launch_kacz_grid_post(bool fp32, void* u, int pu, const void* ec, int pc, const void* f, int pf,
                                  const void* kh, int pk, int n, double bA, int nu, const int* stop, BandSync bs,
                                  cudaStream_t s) {
  const int b = kgrid_blocks(fp32, n);
  if (b < 1) return cudaErrorInvalidConfiguration;
  if (fp32)
    return coop_launch(kacz_grid_post_kernel<float, float2>, b, s, (float2*)u, pu, (const float2*)ec, pc,
                       (const float2*)f, pf, (const float*)kh, pk, n, (float)bA, nu, stop, bs);
  return coop_launch(kacz_grid_post_kernel<double, double2>, b, s, (double2*)u, pu, (const double2*)ec, pc,
                     (const double2*)f, pf, (const double*)kh, pk, n, bA, nu, stop, bs);
}

}  // namespace hz
