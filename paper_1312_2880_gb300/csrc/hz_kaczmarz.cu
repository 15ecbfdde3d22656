// Kaczmarz relaxation of the kH ~ 1.25 level (Sec. 4-5: Gauss-Seidel on the normal equations,
// 4 sweeps before and after the coarse-grid correction) without one launch per colour.
//
// A row action on row p of A u = f~ reads u over p's 5-point support and adds
// conj(a_pq) (f~_p - a_p u) / |a_p|^2 to it; rows of one colour (i + 2j) mod 5 have disjoint
// supports, so a colour is a set of independent updates equal to the sequential sweep over it.
//
// kacz_level_*: the whole level lives in one block's shared memory (small levels), with each row's
//   diagonal and 1/|a_p|^2 computed once per launch (operations in hz_level.cuh). Pre mode: zero guess, nu sweeps (colours
//   0..4), then the residual with the (B) operator and full weighting onto the coarse level. Post
//   mode: u_pre + P e_c, then nu sweeps (colours 4..0).
// kacz_sweep_tile: one full sweep (all five colours) per launch over tiles with a 10-node halo:
//   a colour phase moves information two nodes (a row reads and writes its neighbours), so after
//   five phases the tile interior holds exactly the sequential sweep's values. Out of place.
#include <cuda_runtime.h>

#include "hz_common.cuh"
#include "hz_internal.h"
#include "hz_level.cuh"

namespace hz {

namespace {

constexpr int LB = 1024;  // threads of the whole-level kernel
constexpr int TB = 256;   // threads of the tile kernel
constexpr int KT = 32;    // tile edge
constexpr int KH = 10;    // halo: 2 nodes per colour phase
constexpr int KR = KT + 2 * KH;

// Row action on row (i, j) of a level whose values sit in shared arrays of row pitch w with
// origin (gx, gy): all indices are grid indices, translated to shared positions.
template <class T>
__device__ __forceinline__ void row_action(c2<T>* su, const c2<T>* sf, const T* sk, int w, int gx, int gy, int i,
                                           int j, int n, T beta) {
  Nbr b = neighbours(i, j, n);
  const int c = i - gx, r = j - gy;
  const int p = r * w + c;
  const int qw = r * w + (b.iw - gx), qe = r * w + (b.ie - gx), qs = (b.js - gy) * w + c, qn = (b.jn - gy) * w + c;
  c2<T> d = row_diag<T>(sk[p], b.sides, beta);
  c2<T> up = su[p];
  c2<T> au = cadd<T>(cmul<T>(d, up), cadd<T>(cadd<T>(su[qw], su[qe]), cadd<T>(su[qs], su[qn])));
  c2<T> res = csub<T>(sf[p], au);
  T cx = (i == 0 || i == n) ? (T)4 : (T)2;
  T cy = (j == 0 || j == n) ? (T)4 : (T)2;
  c2<T> delta = cscale<T>(res, rcp(cabs2<T>(d) + cx + cy));
  su[p] = cadd<T>(up, cmulc<T>(d, delta));
  su[qw] = cadd<T>(su[qw], delta);
  su[qe] = cadd<T>(su[qe], delta);
  su[qs] = cadd<T>(su[qs], delta);
  su[qn] = cadd<T>(su[qn], delta);
}

// The same row action for a node strictly inside the square: neighbours at p +- 1, p +- w, no
// boundary term, |a_p|^2 = |d|^2 + 4.
template <class T>
__device__ __forceinline__ void row_action_inner(c2<T>* su, const c2<T>* sf, const T* sk, int w, int p, T beta) {
  const T k = sk[p], k2 = k * k;
  const c2<T> d = mk<T>(k2 - (T)4, beta * k2);
  const c2<T> up = su[p];
  c2<T> au = cadd<T>(cmul<T>(d, up), cadd<T>(cadd<T>(su[p - 1], su[p + 1]), cadd<T>(su[p - w], su[p + w])));
  c2<T> delta = cscale<T>(csub<T>(sf[p], au), rcp(cabs2<T>(d) + (T)4));
  su[p] = cadd<T>(up, cmulc<T>(d, delta));
  su[p - 1] = cadd<T>(su[p - 1], delta);
  su[p + 1] = cadd<T>(su[p + 1], delta);
  su[p - w] = cadd<T>(su[p - w], delta);
  su[p + w] = cadd<T>(su[p + w], delta);
}

__device__ __forceinline__ int mod5(int x) { return ((x % 5) + 5) % 5; }

// ------------------------------------------------------------------ whole level in one block
// Shared layout of the whole-level kernels: u, f~, d (complex) and 1/|a|^2 (real) per node.
template <class T>
struct LevelSmem {
  c2<T>* su;
  c2<T>* sf;
  c2<T>* sd;
  T* sinv;
  __device__ LevelSmem(unsigned char* smem, int N) {
    su = reinterpret_cast<c2<T>*>(smem);
    sf = su + N;
    sd = sf + N;
    sinv = reinterpret_cast<T*>(sd + N);
  }
};

template <class T>
__global__ void __launch_bounds__(LB) kacz_level_pre_kernel(c2<T>* __restrict__ u, int pu, c2<T>* __restrict__ fc,
                                                             int pc, const c2<T>* __restrict__ f, int pf,
                                                             const T* __restrict__ kh, int pk, int n, T bA, T bB,
                                                             int nu, const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  fc += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = n + 1, N = w * w;
  LevelSmem<T> S(smem, N);
  for (int q = threadIdx.x; q < N; q += LB) {
    const int j = q / w, i = q - j * w;
    S.su[q] = mk<T>(0, 0);
    S.sf[q] = f[(long long)j * pf + i];
    lvl::row_consts<T>(kh[(long long)j * pk + i], i, j, n, bA, &S.sd[q], &S.sinv[q]);
  }
  __syncthreads();
  lvl::kacz_sweeps<T>(S.su, S.sf, S.sd, S.sinv, n, nu, false);
  for (int q = threadIdx.x; q < N; q += LB) u[(long long)(q / w) * pu + q % w] = S.su[q];
  lvl::residual<T>(S.sd, S.su, S.sf, kh, pk, n, bB);  // the residual replaces the diagonals
  __syncthreads();
  lvl::restrict_fw<T>(fc, pc, S.sd, n);
}

template <class T>
__global__ void __launch_bounds__(LB) kacz_level_post_kernel(c2<T>* __restrict__ u, int pu,
                                                              const c2<T>* __restrict__ ec, int pc,
                                                              const c2<T>* __restrict__ f, int pf,
                                                              const T* __restrict__ kh, int pk, int n, T bA, int nu,
                                                              const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  ec += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = n + 1, N = w * w;
  LevelSmem<T> S(smem, N);
  for (int q = threadIdx.x; q < N; q += LB) {
    const int j = q / w, i = q - j * w;
    const c2<T>* e0 = ec + (long long)(j >> 1) * pc;
    S.su[q] = xr::cadd<T>(u[(long long)j * pu + i], xr::bilinear<T>(e0, e0 + pc, i >> 1, i & 1, j & 1));
    S.sf[q] = f[(long long)j * pf + i];
    lvl::row_consts<T>(kh[(long long)j * pk + i], i, j, n, bA, &S.sd[q], &S.sinv[q]);
  }
  __syncthreads();
  lvl::kacz_sweeps<T>(S.su, S.sf, S.sd, S.sinv, n, nu, true);
  for (int q = threadIdx.x; q < N; q += LB) u[(long long)(q / w) * pu + q % w] = S.su[q];
}

template <class T, class F2>
__global__ void __launch_bounds__(TB) kacz_sweep_tile_kernel(c2<T>* __restrict__ uout, int po,
                                                              const c2<T>* __restrict__ uin, int pu,
                                                              const F2* __restrict__ f, int pf,
                                                              const T* __restrict__ kh, int pk, int n, T bA, int post,
                                                              const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  uout += blockIdx.z * bi.su;
  if (uin) uin += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  extern __shared__ __align__(16) unsigned char smem[];
  c2<T>* su = reinterpret_cast<c2<T>*>(smem);
  c2<T>* sf = su + KR * KR;
  T* sk = reinterpret_cast<T*>(sf + KR * KR);
  const int x0 = blockIdx.x * KT, y0 = blockIdx.y * KT;
  const int gx = x0 - KH, gy = y0 - KH;
  for (int q = threadIdx.x; q < KR * KR; q += TB) {
    int r = q / KR, c = q - r * KR, i = gx + c, j = gy + r;
    if ((unsigned)i <= (unsigned)n && (unsigned)j <= (unsigned)n) {
      su[q] = uin ? uin[(long long)j * pu + i] : mk<T>(0, 0);
      sf[q] = ldc<T>(f, (long long)j * pf + i);
      sk[q] = kh[(long long)j * pk + i];
    }
  }
  __syncthreads();
  constexpr int PER_ROW = (KR + 4) / 5;
  if (gx >= 1 && gy >= 1 && gx + KR <= n && gy + KR <= n) {
    // region strictly inside the square: no mirrors, no boundary terms
    __shared__ int c0tab[KR];
    for (int ph = 0; ph < 5; ++ph) {
      const int colour = post ? 4 - ph : ph;
      if (threadIdx.x < KR) c0tab[threadIdx.x] = mod5(colour - 2 * (gy + (int)threadIdx.x) - gx);
      __syncthreads();
      for (int q = threadIdx.x; q < KR * PER_ROW; q += TB) {
        const int r = q / PER_ROW, m = q - r * PER_ROW;
        const int c = c0tab[r] + 5 * m;
        if (r < 1 || r > KR - 2 || c < 1 || c > KR - 2) continue;
        row_action_inner<T>(su, sf, sk, KR, r * KR + c, bA);
      }
      __syncthreads();
    }
  } else
  for (int ph = 0; ph < 5; ++ph) {
    const int colour = post ? 4 - ph : ph;
    for (int q = threadIdx.x; q < KR * PER_ROW; q += TB) {
      int r = q / PER_ROW, m = q - r * PER_ROW;
      int j = gy + r;
      int c = ((colour - 2 * j - gx) % 5 + 5) % 5 + 5 * m;
      int i = gx + c;
      if (c >= KR || (unsigned)i > (unsigned)n || (unsigned)j > (unsigned)n) continue;
      // the row's whole support (mirror neighbours included) must lie in the tile region
      Nbr b = neighbours(i, j, n);
      if (b.iw < gx || b.ie >= gx + KR || b.js < gy || b.jn >= gy + KR) continue;
      row_action<T>(su, sf, sk, KR, gx, gy, i, j, n, bA);
    }
    __syncthreads();
  }
  for (int q = threadIdx.x; q < KR * KR; q += TB) {
    int r = q / KR, c = q - r * KR, i = gx + c, j = gy + r;
    if (r >= KH && r < KH + KT && c >= KH && c < KH + KT && (unsigned)i <= (unsigned)n && (unsigned)j <= (unsigned)n)
      uout[(long long)j * po + i] = su[q];
  }
}

template <class T>
size_t level_smem(int n) {
  return (size_t)(n + 1) * (n + 1) * (3 * sizeof(c2<T>) + sizeof(T));
}

template <class T>
cudaError_t set_level_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kacz_level_pre_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       KACZ_LEVEL_MAX_SMEM);
  if (e) return e;
  e = cudaFuncSetAttribute(kacz_level_post_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, KACZ_LEVEL_MAX_SMEM);
  if (!e) done = true;
  return e;
}

}  // namespace

bool kacz_level_fits(bool fp32, int n) {
  return (fp32 ? level_smem<float>(n) : level_smem<double>(n)) <= (size_t)KACZ_LEVEL_MAX_SMEM;
}

cudaError_t launch_kacz_level_pre(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh,
                                  int pk, int n, double bA, double bB, int nu, const int* stop, cudaStream_t s, const Inst& bi) {
  if (!kacz_level_fits(fp32, n)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (fp32) {
    if ((e = set_level_attr<float>())) return e;
    pdl_launch(kacz_level_pre_kernel<float>, dim3(1, 1, bi.count), LB, level_smem<float>(n), s, (float2*)u, pu, (float2*)fc, pc, (const float2*)f,
                                                                     pf, (const float*)kh, pk, n, (float)bA, (float)bB,
                                                                     nu, stop, bi);
  } else {
    if ((e = set_level_attr<double>())) return e;
    pdl_launch(kacz_level_pre_kernel<double>, dim3(1, 1, bi.count), LB, level_smem<double>(n), s, (double2*)u, pu, (double2*)fc, pc,
                                                                       (const double2*)f, pf, (const double*)kh, pk, n,
                                                                       bA, bB, nu, stop, bi);
  }
  return cudaGetLastError();
}

cudaError_t launch_kacz_level_post(bool fp32, void* u, int pu, const void* ec, int pc, const void* f, int pf,
                                   const void* kh, int pk, int n, double bA, int nu, const int* stop, cudaStream_t s, const Inst& bi) {
  if (!kacz_level_fits(fp32, n)) return cudaErrorInvalidValue;
  cudaError_t e;
  if (fp32) {
    if ((e = set_level_attr<float>())) return e;
    pdl_launch(kacz_level_post_kernel<float>, dim3(1, 1, bi.count), LB, level_smem<float>(n), s, (float2*)u, pu, (const float2*)ec, pc,
                                                                      (const float2*)f, pf, (const float*)kh, pk, n,
                                                                      (float)bA, nu, stop, bi);
  } else {
    if ((e = set_level_attr<double>())) return e;
    pdl_launch(kacz_level_post_kernel<double>, dim3(1, 1, bi.count), LB, level_smem<double>(n), s, (double2*)u, pu, (const double2*)ec, pc,
                                                                        (const double2*)f, pf, (const double*)kh, pk, n,
                                                                        bA, nu, stop, bi);
  }
  return cudaGetLastError();
}

template <class T, class F2>
cudaError_t tile_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(kacz_sweep_tile_kernel<T, F2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)(KR * KR * (2 * sizeof(c2<T>) + sizeof(T))));
  if (!e) done = true;
  return e;
}

cudaError_t launch_kacz_sweep_tile(bool fp32, void* uout, int po, const void* uin, int pu, const void* f, int pf,
                                   bool f64_src, const void* kh, int pk, int n, double bA, bool post, const int* stop,
                                   cudaStream_t s, const Inst& bi) {
  dim3 grid((n + KT) / KT, (n + KT) / KT, bi.count);
  cudaError_t e;
  const size_t sm64 = KR * KR * (2 * sizeof(double2) + sizeof(double)), sm32 = KR * KR * (2 * sizeof(float2) + sizeof(float));
  if (!fp32) {
    if ((e = tile_attr<double, double2>())) return e;
  } else if (f64_src) {
    if ((e = tile_attr<float, double2>())) return e;
  } else if ((e = tile_attr<float, float2>())) {
    return e;
  }
  if (!fp32)
    pdl_launch(kacz_sweep_tile_kernel<double, double2>, grid, TB, sm64, s, (double2*)uout, po, (const double2*)uin, pu,
                                                                (const double2*)f, pf, (const double*)kh, pk, n, bA,
                                                                post, stop, bi);
  else if (f64_src)
    pdl_launch(kacz_sweep_tile_kernel<float, double2>, grid, TB, sm32, s, (float2*)uout, po, (const float2*)uin, pu,
                                                               (const double2*)f, pf, (const float*)kh, pk, n,
                                                               (float)bA, post, stop, bi);
  else
    pdl_launch(kacz_sweep_tile_kernel<float, float2>, grid, TB, sm32, s, (float2*)uout, po, (const float2*)uin, pu,
                                                              (const float2*)f, pf, (const float*)kh, pk, n, (float)bA,
                                                              post, stop, bi);
  return cudaGetLastError();
}

}  // namespace hz
