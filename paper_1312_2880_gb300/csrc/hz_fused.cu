// Fused V-cycle passes for Gauss-Seidel levels with one pre- and one post-sweep (Sec. 5), each a
// single pass over the level's arrays through shared-memory tiles.
//
// smooth_restrict: red-black sweep from a zero guess (red nodes become f~/d, then black nodes
//   solve their rows against them), the residual f~ - B u with the level's (B) operator, and
//   full weighting of that residual onto the coarse grid. A block owns a 2W x 2H' fine tile
//   whose even nodes are its coarse outputs; it computes red nodes on the tile plus a 3-node
//   halo, black nodes on a 2-node halo, residuals on a 1-node halo, so every value it writes
//   equals the unfused sequence's. Reads f and k H once, writes u and the coarse f.
// prolong_smooth: u = u_pre + P e_c (bilinear), then the post-sweep black first and red second,
//   on the tile plus a 2-node halo (black on 1, red on 0); writes the result out of place (into
//   the FP64 Krylov vector on the finest grid).
// Nodes outside the square never enter a stencil: boundary rows use mirror neighbours (ghost
// elimination), which lie inside the tile's halo.
#include <cuda_runtime.h>

#include "hz_common.cuh"
#include "hz_internal.h"

namespace hz {

namespace {

constexpr int FT = 256;  // threads per block

// Owned fine nodes of a tile (W x H). FP64 tiles are small: the FP64 passes are bound by each
// SM's FP64 pipe, so spreading a level over more blocks (and SMs) pays for the larger share of
// halo nodes. Measured FP64 solves of the n = 512 wedge: 117.5 ms with 64 x 16 tiles everywhere,
// 112.4 ms with 32 x 8 everywhere (116.9 and 121.6 ms with 32 x 8 only below n_l = 256 or 512).
template <class T>
struct TileShape;
template <>
struct TileShape<float> {
  static constexpr int W = 64, H = 32;
};
template <>
struct TileShape<double> {
  static constexpr int W = 32, H = 8;
};

__device__ __forceinline__ bool in_grid(int i, int j, int n) { return (unsigned)i <= (unsigned)n && (unsigned)j <= (unsigned)n; }

template <class T>
__device__ __forceinline__ c2<T> nb_sum(const c2<T>* s, int rw, int c, int r, int i, int j, int n, int gx, int gy) {
  Nbr b = neighbours(i, j, n);
  return xr::nb4<T>(s[r * rw + (b.iw - gx)], s[r * rw + (b.ie - gx)], s[(b.js - gy) * rw + c],
                    s[(b.jn - gy) * rw + c]);
}

// ---------------------------------------------------------------- interior tiles
// Tiles whose region lies strictly inside the square (no boundary rows, no mirrors, every node
// present) run these paths in FP32: a 32 x 8 thread layout walks rows and columns with fixed
// strides, so there is no index division and no per-node bounds or boundary logic. Their rows do
// not fill whole warps (a region row of 69 nodes takes a full warp pass plus one of 2-5 lanes).
// GB300 issues an FP64 warp instruction at the same cost however few lanes are active, so FP64
// tiles take the general path below, whose flat index walk keeps warps full (measured: the FP64
// solve of the n = 512 wedge 138 -> 117 ms, the same bits).
template <class T>
__host__ __device__ constexpr bool interior_path() { return sizeof(T) == 4; }

constexpr int TXN = 32, TYN = 8;

template <class T, class F2>
__device__ __forceinline__ void smooth_restrict_inner(c2<T>* __restrict__ u, int pu, c2<T>* __restrict__ fc, int pc,
                                                      const F2* __restrict__ f, int pf, const T* __restrict__ kh,
                                                      int pk, T bA, T bB, c2<T>* su, c2<T>* sf, T* sk, int gx,
                                                      int gy) {
  constexpr int W = TileShape<T>::W, HH = TileShape<T>::H;
  constexpr int RW = W + 5, RH = HH + 5;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < RH; r += TYN) {
    const F2* fr = f + (long long)(gy + r) * pf + gx;
    const T* kr = kh + (long long)(gy + r) * pk + gx;
    for (int c = tx; c < RW; c += TXN) {
      sf[r * RW + c] = ldc<T>(fr, c);
      sk[r * RW + c] = kr[c];
    }
  }
  __syncthreads();
  // red nodes everywhere: u = f~ / d (zero guess)
  for (int r = ty; r < RH; r += TYN) {
    const int par = (0 - gx - gy - r) & 1;
    for (int c = 2 * tx + par; c < RW; c += 2 * TXN) {
      const int q = r * RW + c;
      su[q] = xr::cdiv<T>(sf[q], xr::diag<T>(sk[q], 0, bA));
    }
  }
  __syncthreads();
  // black nodes one in from the edge
  for (int r = 1 + ty; r < RH - 1; r += TYN) {
    const int par = (1 - gx - gy - r) & 1;
    for (int c = 2 * tx + par; c < RW - 1; c += 2 * TXN) {
      if (c < 1) continue;
      const int q = r * RW + c;
      const c2<T> nb = xr::nb4<T>(su[q - 1], su[q + 1], su[q - RW], su[q + RW]);
      su[q] = xr::gs<T>(sf[q], nb, xr::diag<T>(sk[q], 0, bA));
    }
  }
  __syncthreads();
  // owned nodes out; residual f~ - B u two in from the edge, into sf
  for (int r = 3 + ty; r < 3 + HH; r += TYN) {
    c2<T>* ur = u + (long long)(gy + r) * pu + gx;
    for (int c = 3 + tx; c < 3 + W; c += TXN) ur[c] = su[r * RW + c];
  }
  for (int r = 2 + ty; r < RH - 2; r += TYN) {
    for (int c = 2 + tx; c < RW - 2; c += TXN) {
      const int q = r * RW + c;
      const c2<T> nb = xr::nb4<T>(su[q - 1], su[q + 1], su[q - RW], su[q + RW]);
      sf[q] = xr::resid<T>(sf[q], su[q], nb, xr::diag<T>(sk[q], 0, bB));
    }
  }
  __syncthreads();
  // full weighting: one coarse node per (tx, row step)
  const int I0 = (gx + 3) / 2, J0 = (gy + 3) / 2;
  for (int Jl = ty; Jl < HH / 2; Jl += TYN) {
    for (int Il = tx; Il < W / 2; Il += TXN) {
      const int q = (2 * Jl + 3) * RW + (2 * Il + 3);
      const c2<T> top = xr::fw3<T>(sf[q - RW - 1], sf[q - RW], sf[q - RW + 1]);
      const c2<T> mid = xr::fw3<T>(sf[q - 1], sf[q], sf[q + 1]);
      const c2<T> bot = xr::fw3<T>(sf[q + RW - 1], sf[q + RW], sf[q + RW + 1]);
      fc[(long long)(J0 + Jl) * pc + I0 + Il] = xr::cscale<T>(xr::fw3<T>(top, mid, bot), (T)0.25);
    }
  }
}

template <class T, class F2, class O2>
__device__ __forceinline__ void prolong_smooth_inner(O2* __restrict__ out, int po, const c2<T>* __restrict__ upre,
                                                     int pu, const c2<T>* __restrict__ ec, int pc,
                                                     const F2* __restrict__ f, int pf, const T* __restrict__ kh,
                                                     int pk, T bA, c2<T>* su, c2<T>* sf, T* sk, int gx, int gy) {
  constexpr int W = TileShape<T>::W, HH = TileShape<T>::H;
  constexpr int RW = W + 4, RH = HH + 4;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int r = ty; r < RH; r += TYN) {
    const int j = gy + r, J = j >> 1, oj = j & 1;
    const F2* fr = f + (long long)j * pf + gx;
    const T* kr = kh + (long long)j * pk + gx;
    const c2<T>* ur = upre + (long long)j * pu + gx;
    const c2<T>* e0 = ec + (long long)J * pc;
    const c2<T>* e1 = e0 + pc;
    for (int c = tx; c < RW; c += TXN) {
      const int i = gx + c, I = i >> 1, oi = i & 1;
      su[r * RW + c] = xr::cadd<T>(ur[c], xr::bilinear<T>(e0, e1, I, oi, oj));
      sf[r * RW + c] = ldc<T>(fr, c);
      sk[r * RW + c] = kr[c];
    }
  }
  __syncthreads();
  for (int r = 1 + ty; r < RH - 1; r += TYN) {  // black, one in from the edge
    const int par = (1 - gx - gy - r) & 1;
    for (int c = 2 * tx + par; c < RW - 1; c += 2 * TXN) {
      if (c < 1) continue;
      const int q = r * RW + c;
      const c2<T> nb = xr::nb4<T>(su[q - 1], su[q + 1], su[q - RW], su[q + RW]);
      su[q] = xr::gs<T>(sf[q], nb, xr::diag<T>(sk[q], 0, bA));
    }
  }
  __syncthreads();
  for (int r = 2 + ty; r < 2 + HH; r += TYN) {  // red on the owned tile
    const int par = (0 - gx - gy - r) & 1;
    for (int c = 2 * tx + par; c < 2 + W; c += 2 * TXN) {
      if (c < 2) continue;
      const int q = r * RW + c;
      const c2<T> nb = xr::nb4<T>(su[q - 1], su[q + 1], su[q - RW], su[q + RW]);
      su[q] = xr::gs<T>(sf[q], nb, xr::diag<T>(sk[q], 0, bA));
    }
  }
  __syncthreads();
  for (int r = 2 + ty; r < 2 + HH; r += TYN) {
    O2* orow = out + (long long)(gy + r) * po + gx;
    for (int c = 2 + tx; c < 2 + W; c += TXN) stc<T>(orow, c, su[r * RW + c]);
  }
}

template <class T, class F2>
__global__ void __launch_bounds__(FT) smooth_restrict_kernel(c2<T>* __restrict__ u, int pu, c2<T>* __restrict__ fc,
                                                              int pc, const F2* __restrict__ f, int pf,
                                                              const T* __restrict__ kh, int pk, int n, T bA, T bB,
                                                              const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  fc += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  constexpr int W = TileShape<T>::W, HH = TileShape<T>::H;
  constexpr int RW = W + 5, RH = HH + 5, RN = RW * RH, HW = (RW + 1) / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  c2<T>* su = reinterpret_cast<c2<T>*>(smem);
  c2<T>* sf = su + RN;
  T* sk = reinterpret_cast<T*>(sf + RN);
  const int x0 = blockIdx.x * W, y0 = blockIdx.y * HH;
  const int gx = x0 - 3, gy = y0 - 3;
  if (interior_path<T>() && gx >= 1 && gy >= 1 && gx + RW <= n && gy + RH <= n) {
    smooth_restrict_inner<T, F2>(u, pu, fc, pc, f, pf, kh, pk, bA, bB, su, sf, sk, gx, gy);
    return;
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int q = tid; q < RN; q += FT) {
    int r = q / RW, c = q - r * RW, i = gx + c, j = gy + r;
    if (in_grid(i, j, n)) {
      sf[q] = ldc<T>(f, (long long)j * pf + i);
      sk[q] = kh[(long long)j * pk + i];
    }
  }
  __syncthreads();
  // red nodes of the whole region: zero neighbours, u = f~ / d
  for (int q = tid; q < RH * HW; q += FT) {
    int r = q / HW, m = q - r * HW;
    int j = gy + r;
    int c = 2 * m + ((0 - gx - j) & 1);
    int i = gx + c;
    if (c < RW && in_grid(i, j, n)) {
      int sides = (i == 0) + (i == n) + (j == 0) + (j == n);
      su[r * RW + c] = xr::cdiv<T>(sf[r * RW + c], xr::diag<T>(sk[r * RW + c], sides, bA));
    }
  }
  __syncthreads();
  // black nodes one in from the region edge
  for (int q = tid; q < RH * HW; q += FT) {
    int r = q / HW, m = q - r * HW;
    int j = gy + r;
    int c = 2 * m + ((1 - gx - j) & 1);
    int i = gx + c;
    if (r >= 1 && r <= RH - 2 && c >= 1 && c <= RW - 2 && in_grid(i, j, n)) {
      Nbr b = neighbours(i, j, n);
      c2<T> s = nb_sum<T>(su, RW, c, r, i, j, n, gx, gy);
      su[r * RW + c] = xr::gs<T>(sf[r * RW + c], s, xr::diag<T>(sk[r * RW + c], b.sides, bA));
    }
  }
  __syncthreads();
  // write the owned nodes; residual f~ - B u two in from the edge (into sf)
  for (int q = tid; q < RN; q += FT) {
    int r = q / RW, c = q - r * RW, i = gx + c, j = gy + r;
    if (!in_grid(i, j, n)) continue;
    if (r >= 3 && r < 3 + HH && c >= 3 && c < 3 + W) u[(long long)j * pu + i] = su[q];
  }
  __syncthreads();
  for (int q = tid; q < RN; q += FT) {
    int r = q / RW, c = q - r * RW, i = gx + c, j = gy + r;
    if (r >= 2 && r <= RH - 3 && c >= 2 && c <= RW - 3 && in_grid(i, j, n)) {
      Nbr b = neighbours(i, j, n);
      c2<T> s = nb_sum<T>(su, RW, c, r, i, j, n, gx, gy);
      sf[q] = xr::resid<T>(sf[q], su[q], s, xr::diag<T>(sk[q], b.sides, bB));
    }
  }
  __syncthreads();
  // full weighting onto the owned coarse nodes
  const int nc = n / 2;
  for (int q = tid; q < (W / 2) * (HH / 2); q += FT) {
    int J = y0 / 2 + q / (W / 2), I = x0 / 2 + q % (W / 2);
    if (I > nc || J > nc) continue;
    fc[(long long)J * pc + I] = xr::fw_node<T>(sf - gy * RW - gx, RW, n, I, J);
  }
}

template <class T, class F2, class O2>
__global__ void __launch_bounds__(FT) prolong_smooth_kernel(O2* __restrict__ out, int po, const c2<T>* __restrict__ upre,
                                                             int pu, const c2<T>* __restrict__ ec, int pc,
                                                             const F2* __restrict__ f, int pf,
                                                             const T* __restrict__ kh, int pk, int n, T bA,
                                                             const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  out += blockIdx.z * bi.so;
  upre += blockIdx.z * bi.su;
  ec += blockIdx.z * bi.sc;
  f += blockIdx.z * bi.sf;
  constexpr int W = TileShape<T>::W, HH = TileShape<T>::H;
  constexpr int RW = W + 4, RH = HH + 4, RN = RW * RH, HW = RW / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  c2<T>* su = reinterpret_cast<c2<T>*>(smem);
  c2<T>* sf = su + RN;
  T* sk = reinterpret_cast<T*>(sf + RN);
  const int x0 = blockIdx.x * W, y0 = blockIdx.y * HH;
  const int gx = x0 - 2, gy = y0 - 2;
  if (interior_path<T>() && gx >= 1 && gy >= 1 && gx + RW <= n && gy + RH <= n) {
    prolong_smooth_inner<T, F2, O2>(out, po, upre, pu, ec, pc, f, pf, kh, pk, bA, su, sf, sk, gx, gy);
    return;
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  for (int q = tid; q < RN; q += FT) {
    int r = q / RW, c = q - r * RW, i = gx + c, j = gy + r;
    if (in_grid(i, j, n)) {
      sf[q] = ldc<T>(f, (long long)j * pf + i);
      sk[q] = kh[(long long)j * pk + i];
    }
  }
  // u_pre + P e, one parity class (i mod 2, j mod 2) after the other (gx and gy are even), so that
  // a warp takes one interpolation case: a warp mixing the four cases would issue all of them
  constexpr int CE = (RW + 1) / 2, CO = RW / 2, RE = (RH + 1) / 2, RO = RH / 2;
  for (int q = tid; q < RN; q += FT) {
    int oi, oj, t;
    if (q < CE * RE) { oi = 0; oj = 0; t = q; }
    else if (q < CE * RE + CO * RE) { oi = 1; oj = 0; t = q - CE * RE; }
    else if (q < CE * RE + CO * RE + CE * RO) { oi = 0; oj = 1; t = q - CE * RE - CO * RE; }
    else { oi = 1; oj = 1; t = q - CE * RE - CO * RE - CE * RO; }
    const int wcls = oi ? CO : CE, mr = t / wcls, mc = t - mr * wcls;
    const int r = 2 * mr + oj, c = 2 * mc + oi, i = gx + c, j = gy + r;
    if (in_grid(i, j, n)) {
      const c2<T>* e0 = ec + (long long)(j >> 1) * pc;
      su[r * RW + c] = xr::cadd<T>(upre[(long long)j * pu + i], xr::bilinear<T>(e0, e0 + pc, i >> 1, oi, oj));
    }
  }
  __syncthreads();
  // black nodes one in from the region edge
  for (int q = tid; q < RH * HW; q += FT) {
    int r = q / HW, m = q - r * HW;
    int j = gy + r;
    int c = 2 * m + ((1 - gx - j) & 1);
    int i = gx + c;
    if (r >= 1 && r <= RH - 2 && c >= 1 && c <= RW - 2 && in_grid(i, j, n)) {
      Nbr b = neighbours(i, j, n);
      c2<T> s = nb_sum<T>(su, RW, c, r, i, j, n, gx, gy);
      su[r * RW + c] = xr::gs<T>(sf[r * RW + c], s, xr::diag<T>(sk[r * RW + c], b.sides, bA));
    }
  }
  __syncthreads();
  // red nodes of the owned tile
  for (int q = tid; q < RH * HW; q += FT) {
    int r = q / HW, m = q - r * HW;
    int j = gy + r;
    int c = 2 * m + ((0 - gx - j) & 1);
    int i = gx + c;
    if (r >= 2 && r < 2 + HH && c >= 2 && c < 2 + W && in_grid(i, j, n)) {
      Nbr b = neighbours(i, j, n);
      c2<T> s = nb_sum<T>(su, RW, c, r, i, j, n, gx, gy);
      su[r * RW + c] = xr::gs<T>(sf[r * RW + c], s, xr::diag<T>(sk[r * RW + c], b.sides, bA));
    }
  }
  __syncthreads();
  for (int q = tid; q < RN; q += FT) {
    int r = q / RW, c = q - r * RW, i = gx + c, j = gy + r;
    if (r >= 2 && r < 2 + HH && c >= 2 && c < 2 + W && in_grid(i, j, n)) stc<T>(out, (long long)j * po + i, su[q]);
  }
}

template <class T>
constexpr size_t sr_smem() {
  return (size_t)(TileShape<T>::W + 5) * (TileShape<T>::H + 5) * (2 * sizeof(c2<T>) + sizeof(T));
}
template <class T>
constexpr size_t ps_smem() {
  return (size_t)(TileShape<T>::W + 4) * (TileShape<T>::H + 4) * (2 * sizeof(c2<T>) + sizeof(T));
}

template <class T, class F2>
cudaError_t sr_t(void* u, int pu, void* fc, int pc, const void* f, int pf, const void* kh, int pk, int n, double bA,
                 double bB, const int* stop, cudaStream_t s, const Inst& bi) {
  constexpr size_t sm = sr_smem<T>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(smooth_restrict_kernel<T, F2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    attr = true;
  }
  constexpr int CW = TileShape<T>::W / 2, CH = TileShape<T>::H / 2;
  int nc = n / 2;
  dim3 grid((nc + CW) / CW, (nc + CH) / CH, bi.count);
  pdl_launch(smooth_restrict_kernel<T, F2>, grid, dim3(TXN, TYN), sm, s, (c2<T>*)u, pu, (c2<T>*)fc, pc, (const F2*)f, pf,
                                                                (const T*)kh, pk, n, (T)bA, (T)bB, stop, bi);
  return cudaGetLastError();
}

template <class T, class F2, class O2>
cudaError_t ps_t(void* out, int po, const void* upre, int pu, const void* ec, int pc, const void* f, int pf,
                 const void* kh, int pk, int n, double bA, const int* stop, cudaStream_t s, const Inst& bi) {
  constexpr size_t sm = ps_smem<T>();
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(prolong_smooth_kernel<T, F2, O2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e) return e;
    attr = true;
  }
  constexpr int W = TileShape<T>::W, HH = TileShape<T>::H;
  dim3 grid((n + W) / W, (n + HH) / HH, bi.count);
  pdl_launch(prolong_smooth_kernel<T, F2, O2>, grid, dim3(TXN, TYN), sm, s, (O2*)out, po, (const c2<T>*)upre, pu,
                                                                    (const c2<T>*)ec, pc, (const F2*)f, pf,
                                                                    (const T*)kh, pk, n, (T)bA, stop, bi);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_smooth_restrict(bool fp32, void* u, int pu, void* fc, int pc, const void* f, int pf, bool f64_src,
                                   const void* kh, int pk, int n, double bA, double bB, const int* stop,
                                   cudaStream_t s, const Inst& bi, int variant) {
  if (fp32 && f64_src) return cudaErrorInvalidValue;  // the FP32 form's inputs are FP32
  if (variant >= 1 && variant < FUSED_VARIANTS)
    return launch_smooth_restrict_stream(fp32, u, pu, fc, pc, f, pf, kh, pk, n, bA, bB, stream_rows(variant), stop, s,
                                         bi);
  if (!fp32) return sr_t<double, double2>(u, pu, fc, pc, f, pf, kh, pk, n, bA, bB, stop, s, bi);
  return sr_t<float, float2>(u, pu, fc, pc, f, pf, kh, pk, n, bA, bB, stop, s, bi);
}

cudaError_t launch_prolong_smooth(bool fp32, void* out, int po, bool out_f64, const void* upre, int pu, const void* ec,
                                  int pc, const void* f, int pf, bool f64_src, const void* kh, int pk, int n, double bA,
                                  const int* stop, cudaStream_t s, const Inst& bi, int variant) {
  if (fp32 && (f64_src || out_f64)) return cudaErrorInvalidValue;  // the FP32 form's inputs and outputs are FP32
  if (variant >= 1 && variant < FUSED_VARIANTS)
    return launch_prolong_smooth_stream(fp32, out, po, upre, pu, ec, pc, f, pf, kh, pk, n, bA, stream_rows(variant),
                                        stop, s, bi);
  if (!fp32) return ps_t<double, double2, double2>(out, po, upre, pu, ec, pc, f, pf, kh, pk, n, bA, stop, s, bi);
  return ps_t<float, float2, float2>(out, po, upre, pu, ec, pc, f, pf, kh, pk, n, bA, stop, s, bi);
}

}  // namespace hz
