// V-cycle kernels (Sec. 5): red-black Gauss-Seidel and 5-colour Kaczmarz sweeps, residual with
// full-weighting restriction, bilinear correction, the coarsest-grid dense solve, and set-up.
//
// All kernels work on one level's (n+1)^2 grid in the h^2-scaled form described in
// hz_common.cuh, in precision T (double or float). Arrays are row-major with a pitch in
// elements. Sweeps run in place: nodes of one colour never read each other (red-black), and
// rows of one Kaczmarz colour (i + 2j) mod 5 have disjoint 5-point supports, so a colour is a
// set of independent updates and equals the sequential sweep over it.
#include <cuda_runtime.h>

#include "hz_common.cuh"
#include "hz_internal.h"
#include "hz_gnode.cuh"
#include "hz_level.cuh"

namespace hz {

namespace {

constexpr int BX = 32, BY = 8;

inline dim3 grid2(int nx, int ny) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY); }

// ---------------------------------------------------------------- Gauss-Seidel (Sec. 4)

// One colour of a red-black sweep: every node with (i + j) % 2 == colour solves its own row
// with its neighbours (all of the other colour) held fixed: u_p = (f~_p - sum_nb u_q) / d_p.
// omega != 1: over-relaxed (SOR), u_p <- (1 - omega) u_p + omega (f~_p - sum_nb u_q) / d_p.
template <class T, class F2>
__global__ void gs_colour_kernel(c2<T>* __restrict__ u, int pu, const F2* __restrict__ f, int pf,
                                 const T* __restrict__ kh, int pk, int n, int colour, T beta, T omega,
                                 const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j > n) return;
  int i = 2 * m + ((colour ^ j) & 1);
  if (i > n) return;
  Nbr b = neighbours(i, j, n);
  c2<T> nb = cadd<T>(cadd<T>(u[(long long)j * pu + b.iw], u[(long long)j * pu + b.ie]),
                     cadd<T>(u[(long long)b.js * pu + i], u[(long long)b.jn * pu + i]));
  c2<T> d = row_diag<T>(kh[(long long)j * pk + i], b.sides, beta);
  c2<T> fv = ldc<T>(f, (long long)j * pf + i);
  c2<T> g = cdiv<T>(csub<T>(fv, nb), d);
  if (omega != (T)1) g = xr::cadd<T>(xr::cscale<T>(u[(long long)j * pu + i], (T)1 - omega), xr::cscale<T>(g, omega));
  u[(long long)j * pu + i] = g;
}

// First half-sweep from a zero guess: nodes of `colour` get f~/d (their neighbours are zero;
// omega f~/d for SOR), nodes of the other colour are set to zero. Replaces zero-fill + first colour.
template <class T, class F2>
__global__ void gs_first_kernel(c2<T>* __restrict__ u, int pu, const F2* __restrict__ f, int pf,
                                const T* __restrict__ kh, int pk, int n, int colour, T beta, T omega,
                                const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n || j > n) return;
  c2<T> out = mk<T>(0, 0);
  if (((i + j) & 1) == colour) {
    int sides = (i == 0) + (i == n) + (j == 0) + (j == n);
    out = cdiv<T>(ldc<T>(f, (long long)j * pf + i), row_diag<T>(kh[(long long)j * pk + i], sides, beta));
    if (omega != (T)1) out = xr::cscale<T>(out, omega);
  }
  u[(long long)j * pu + i] = out;
}

// ---------------------------------------------------------------- damped Jacobi (Sec. 4, remark)

// One damped Jacobi sweep, every node at once, out of place: out = in + omega (f~ - A in) / d;
// from a zero guess (in == nullptr) out = omega f~ / d.
template <class T, class F2>
__global__ void jacobi_kernel(c2<T>* __restrict__ out, int po, const c2<T>* __restrict__ in, int pu,
                              const F2* __restrict__ f, int pf, const T* __restrict__ kh, int pk, int n, T beta,
                              T omega, const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  out += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n || j > n) return;
  const c2<T> d = xr::diag<T>(kh[(long long)j * pk + i], lvl::sides_at(i, j, n), beta);
  const c2<T> fv = ldc<T>(f, (long long)j * pf + i);
  c2<T> v;
  if (!in) {
    v = xr::cscale<T>(xr::cdiv<T>(fv, d), omega);
  } else {
    in += blockIdx.z * bi.su;
    const Nbr b = neighbours(i, j, n);
    const c2<T>* row = in + (long long)j * pu;
    const c2<T> up = row[i];
    const c2<T> r = xr::resid<T>(fv, up, xr::nb4<T>(row[b.iw], row[b.ie], in[(long long)b.js * pu + i],
                                                   in[(long long)b.jn * pu + i]), d);
    v = xr::cadd<T>(up, xr::cscale<T>(xr::cdiv<T>(r, d), omega));
  }
  out[(long long)j * po + i] = v;
}

// ---------------------------------------------------------------- Kaczmarz (Sec. 4-5)

// One colour of a row-action Kaczmarz sweep on A u = f (Gauss-Seidel on A A^H y = f with
// u = A^H y): for each row p of colour (i + 2j) % 5, delta = (f~_p - (A u)_p) / |a_p|^2 and
// u_q += conj(a_pq) delta over the row's support (lvl::act_nodes, the row action of every
// Kaczmarz form). A mirror neighbour at the boundary carries coefficient 2 and receives 2 delta.
template <class T, class F2>
__global__ void kacz_colour_kernel(c2<T>* __restrict__ u, int pu, const F2* __restrict__ f, int pf,
                                   const T* __restrict__ kh, int pk, int n, int colour, T beta,
                                   const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j > n) return;
  int i = ((colour - 2 * j) % 5 + 5) % 5 + 5 * m;
  if (i > n) return;
  gnode::kacz_row<T, F2>(u, pu, f, pf, kh, pk, n, i, j, beta);
}

// ---------------------------------------------------------------- transfers (Sec. 5)

// f~_c(I, J) = 4 * FW(f~ - B u): full weighting 1/16 [1 2 1; 2 4 2; 1 2 1] of the fine
// residual around fine node (2I, 2J), fine nodes outside the square mirrored inside. The
// factor 4 = (2H)^2 / H^2 moves the residual to the coarse level's scaling.
template <class T, class F2>
__global__ void restrict_residual_kernel(c2<T>* __restrict__ fc, int pc, const c2<T>* __restrict__ u, int pu,
                                         const F2* __restrict__ f, int pf, const T* __restrict__ kh, int pk, int n,
                                         T beta, const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  fc += blockIdx.z * bi.sc;
  u += blockIdx.z * bi.su;
  f += blockIdx.z * bi.sf;
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  int nc = n / 2;
  if (I > nc || J > nc) return;
  fc[(long long)J * pc + I] = gnode::restrict_node<T, F2>(u, pu, f, pf, kh, pk, n, beta, I, J);
}

// u += P e_c, bilinear interpolation from the (n/2+1)^2 grid.
template <class T>
__global__ void prolong_add_kernel(c2<T>* __restrict__ u, int pu, const c2<T>* __restrict__ ec, int pc, int n,
                                   const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  ec += blockIdx.z * bi.sc;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n || j > n) return;
  gnode::prolong_add_node<T>(u, pu, ec, pc, i, j);
}

// ---------------------------------------------------------------- coarsest grid

// u = A_c^{-1} f~ with the dense inverse stored transposed (column c contiguous), one block.
template <class T>
__global__ void coarse_solve_kernel(c2<T>* __restrict__ u, int pu, const c2<T>* __restrict__ f, int pf,
                                    const c2<T>* __restrict__ ainvT, int nc, const int* __restrict__ stop, Inst bi) {
  pdl_enter();
  if (stop && stop[blockIdx.z * bi.stop_stride]) return;
  u += blockIdx.z * bi.su;
  f += blockIdx.z * bi.su;
  extern __shared__ unsigned char smem_raw[];
  c2<T>* fs = reinterpret_cast<c2<T>*>(smem_raw);
  int w = nc + 1, m = w * w;
  for (int q = threadIdx.x; q < m; q += blockDim.x) fs[q] = f[(long long)(q / w) * pf + q % w];
  __syncthreads();
  for (int r = threadIdx.x; r < m; r += blockDim.x) u[(long long)(r / w) * pu + r % w] = lvl::coarse_row<T>(ainvT, fs, m, r);
}

// Dense scaled operator of the coarsest level (row-major, m x m) next to the identity, then
// Gauss-Jordan elimination with partial pivoting (largest modulus, lowest row on ties) in one
// block; writes the inverse transposed in precision T.
template <class T>
__global__ void coarse_setup_kernel(c2<T>* __restrict__ ainvT, double2* __restrict__ work, const T* __restrict__ kh,
                                    int pk, int nc, double beta, int* __restrict__ status) {
  pdl_enter();
  int w = nc + 1, m = w * w;
  double2* A = work;
  double2* B = work + (long long)m * m;
  __shared__ double2 fac[1089];
  __shared__ double bestv[1024];
  __shared__ int besti[1024];
  for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
    A[e] = make_double2(0, 0);
    B[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) {
    int i = p % w, j = p / w;
    int iw = i > 0 ? i - 1 : 1, ie = i < nc ? i + 1 : nc - 1, js = j > 0 ? j - 1 : 1, jn = j < nc ? j + 1 : nc - 1;
    int sides = (i == 0) + (i == nc) + (j == 0) + (j == nc);
    double k = (double)kh[(long long)j * pk + i];
    double2* row = A + (long long)p * m;
    row[p] = make_double2(k * k - 4.0, beta * k * k + 2.0 * sides * k);
    row[j * w + iw].x += 1.0;
    row[j * w + ie].x += 1.0;
    row[js * w + i].x += 1.0;
    row[jn * w + i].x += 1.0;
  }
  __syncthreads();
  for (int k = 0; k < m; ++k) {
    double bv = -1.0;
    int bi = m;
    for (int r = k + threadIdx.x; r < m; r += blockDim.x) {
      double2 a = A[(long long)r * m + k];
      double v = a.x * a.x + a.y * a.y;
      if (v > bv) { bv = v; bi = r; }
    }
    bestv[threadIdx.x] = bv;
    besti[threadIdx.x] = bi;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
      if (threadIdx.x < off) {
        double ov = bestv[threadIdx.x + off];
        int oi = besti[threadIdx.x + off];
        if (ov > bestv[threadIdx.x] || (ov == bestv[threadIdx.x] && oi < besti[threadIdx.x])) {
          bestv[threadIdx.x] = ov;
          besti[threadIdx.x] = oi;
        }
      }
      __syncthreads();
    }
    int piv = besti[0];
    if (!(bestv[0] > 0.0)) {
      if (threadIdx.x == 0) *status = 1;
      return;
    }
    if (piv != k) {
      for (int c = threadIdx.x; c < m; c += blockDim.x) {
        double2 t = A[(long long)k * m + c]; A[(long long)k * m + c] = A[(long long)piv * m + c]; A[(long long)piv * m + c] = t;
        t = B[(long long)k * m + c]; B[(long long)k * m + c] = B[(long long)piv * m + c]; B[(long long)piv * m + c] = t;
      }
    }
    __syncthreads();
    double2 pv = A[(long long)k * m + k];
    double inv = 1.0 / (pv.x * pv.x + pv.y * pv.y);
    double2 ip = make_double2(pv.x * inv, -pv.y * inv);
    __syncthreads();
    for (int c = threadIdx.x; c < m; c += blockDim.x) {
      double2 a = A[(long long)k * m + c];
      A[(long long)k * m + c] = make_double2(a.x * ip.x - a.y * ip.y, a.x * ip.y + a.y * ip.x);
      double2 bb = B[(long long)k * m + c];
      B[(long long)k * m + c] = make_double2(bb.x * ip.x - bb.y * ip.y, bb.x * ip.y + bb.y * ip.x);
    }
    __syncthreads();
    for (int r = threadIdx.x; r < m; r += blockDim.x) fac[r] = A[(long long)r * m + k];
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      int r = (int)(e / m), c = (int)(e % m);
      if (r == k) continue;
      double2 fr = fac[r];
      double2 a = A[(long long)k * m + c];
      double2 x = A[e];
      A[e] = make_double2(x.x - (fr.x * a.x - fr.y * a.y), x.y - (fr.x * a.y + fr.y * a.x));
      double2 bb = B[(long long)k * m + c];
      double2 y = B[e];
      B[e] = make_double2(y.x - (fr.x * bb.x - fr.y * bb.y), y.y - (fr.x * bb.y + fr.y * bb.x));
    }
    __syncthreads();
  }
  for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
    int r = (int)(e / m), c = (int)(e % m);
    double2 v = B[e];
    ainvT[(long long)c * m + r] = mk<T>((T)v.x, (T)v.y);
  }
  if (threadIdx.x == 0) *status = 0;
}

// ---------------------------------------------------------------- layout conversion, set-up

template <class T>
__global__ void import_kernel(c2<T>* __restrict__ dst, int pd, const double2* __restrict__ src, int ps, int n,
                              double scale) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n || j > n) return;
  double2 v = src[(long long)j * ps + i];
  dst[(long long)j * pd + i] = mk<T>((T)(v.x * scale), (T)(v.y * scale));
}

template <class T>
__global__ void export_kernel(double2* __restrict__ dst, int pd, const c2<T>* __restrict__ src, int ps, int n,
                              double scale, const int* __restrict__ stop) {
  pdl_enter();
  if (stop && *stop) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > n || j > n) return;
  c2<T> v = src[(long long)j * ps + i];
  dst[(long long)j * pd + i] = make_double2((double)v.x * scale, (double)v.y * scale);
}

template <class T>
__global__ void inject_kh_kernel(T* __restrict__ kh, int pk, const double* __restrict__ k0, int n0, int stride,
                                 int nl, double H) {
  pdl_enter();
  int I = blockIdx.x * blockDim.x + threadIdx.x;
  int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I > nl || J > nl) return;
  kh[(long long)J * pk + I] = (T)(k0[(long long)stride * J * (n0 + 1) + (long long)stride * I] * H);
}

template <class T, class F2>
cudaError_t gs_colour_t(void* u, int pu, const void* f, int pf, const void* kh, int pk, int n, int colour, double beta,
                        const int* stop, cudaStream_t s, const Inst& bi, double omega) {
  dim3 g = grid2((n + 2) / 2, n + 1);
  g.z = bi.count;
  pdl_launch(gs_colour_kernel<T, F2>, g, dim3(BX, BY), 0, s, (c2<T>*)u, pu, (const F2*)f, pf, (const T*)kh, pk, n, colour,
                                                     (T)beta, (T)omega, stop, bi);
  return cudaGetLastError();
}
template <class T, class F2>
cudaError_t gs_first_t(void* u, int pu, const void* f, int pf, const void* kh, int pk, int n, int colour, double beta,
                       const int* stop, cudaStream_t s, const Inst& bi, double omega) {
  dim3 g = grid2(n + 1, n + 1);
  g.z = bi.count;
  pdl_launch(gs_first_kernel<T, F2>, g, dim3(BX, BY), 0, s, (c2<T>*)u, pu, (const F2*)f, pf, (const T*)kh, pk, n, colour,
                                                    (T)beta, (T)omega, stop, bi);
  return cudaGetLastError();
}
template <class T, class F2>
cudaError_t jacobi_t(void* out, int po, const void* in, int pu, const void* f, int pf, const void* kh, int pk, int n,
                     double beta, double omega, const int* stop, cudaStream_t s, const Inst& bi) {
  dim3 g = grid2(n + 1, n + 1);
  g.z = bi.count;
  pdl_launch(jacobi_kernel<T, F2>, g, dim3(BX, BY), 0, s, (c2<T>*)out, po, (const c2<T>*)in, pu, (const F2*)f, pf,
             (const T*)kh, pk, n, (T)beta, (T)omega, stop, bi);
  return cudaGetLastError();
}
template <class T, class F2>
cudaError_t kacz_colour_t(void* u, int pu, const void* f, int pf, const void* kh, int pk, int n, int colour,
                          double beta, const int* stop, cudaStream_t s, const Inst& bi) {
  dim3 g = grid2((n + 5) / 5, n + 1);
  g.z = bi.count;
  pdl_launch(kacz_colour_kernel<T, F2>, g, dim3(BX, BY), 0, s, (c2<T>*)u, pu, (const F2*)f, pf, (const T*)kh, pk, n, colour,
                                                       (T)beta, stop, bi);
  return cudaGetLastError();
}
template <class T, class F2>
cudaError_t restrict_t(void* fc, int pc, const void* u, int pu, const void* f, int pf, const void* kh, int pk, int n,
                       double beta, const int* stop, cudaStream_t s, const Inst& bi) {
  dim3 g = grid2(n / 2 + 1, n / 2 + 1);
  g.z = bi.count;
  pdl_launch(restrict_residual_kernel<T, F2>, g, dim3(BX, BY), 0, s, (c2<T>*)fc, pc, (const c2<T>*)u, pu, (const F2*)f, pf,
                                                             (const T*)kh, pk, n, (T)beta, stop, bi);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gs_colour(bool fp32, void* u, int pu, const void* f, int pf, bool f64_src, const void* kh, int pk,
                             int n, int colour, double beta, const int* stop, cudaStream_t s, const Inst& bi,
                             double omega) {
  if (!fp32) return gs_colour_t<double, double2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi, omega);
  if (f64_src) return gs_colour_t<float, double2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi, omega);
  return gs_colour_t<float, float2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi, omega);
}

cudaError_t launch_gs_first(bool fp32, void* u, int pu, const void* f, int pf, bool f64_src, const void* kh, int pk,
                            int n, int colour, double beta, const int* stop, cudaStream_t s, const Inst& bi,
                            double omega) {
  if (!fp32) return gs_first_t<double, double2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi, omega);
  if (f64_src) return gs_first_t<float, double2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi, omega);
  return gs_first_t<float, float2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi, omega);
}

cudaError_t launch_jacobi(bool fp32, void* out, int po, const void* in, int pu, const void* f, int pf, bool f64_src,
                          const void* kh, int pk, int n, double beta, double omega, const int* stop, cudaStream_t s,
                          const Inst& bi) {
  if (!fp32) return jacobi_t<double, double2>(out, po, in, pu, f, pf, kh, pk, n, beta, omega, stop, s, bi);
  if (f64_src) return jacobi_t<float, double2>(out, po, in, pu, f, pf, kh, pk, n, beta, omega, stop, s, bi);
  return jacobi_t<float, float2>(out, po, in, pu, f, pf, kh, pk, n, beta, omega, stop, s, bi);
}

cudaError_t launch_kacz_colour(bool fp32, void* u, int pu, const void* f, int pf, bool f64_src, const void* kh, int pk,
                               int n, int colour, double beta, const int* stop, cudaStream_t s, const Inst& bi) {
  if (!fp32) return kacz_colour_t<double, double2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi);
  if (f64_src) return kacz_colour_t<float, double2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi);
  return kacz_colour_t<float, float2>(u, pu, f, pf, kh, pk, n, colour, beta, stop, s, bi);
}

cudaError_t launch_restrict_residual(bool fp32, void* fc, int pc, const void* u, int pu, const void* f, int pf,
                                     bool f64_src, const void* kh, int pk, int n, double beta, const int* stop,
                                     cudaStream_t s, const Inst& bi) {
  if (!fp32) return restrict_t<double, double2>(fc, pc, u, pu, f, pf, kh, pk, n, beta, stop, s, bi);
  if (f64_src) return restrict_t<float, double2>(fc, pc, u, pu, f, pf, kh, pk, n, beta, stop, s, bi);
  return restrict_t<float, float2>(fc, pc, u, pu, f, pf, kh, pk, n, beta, stop, s, bi);
}

cudaError_t launch_prolong_add(bool fp32, void* u, int pu, const void* ec, int pc, int n, const int* stop,
                               cudaStream_t s, const Inst& bi) {
  dim3 g = grid2(n + 1, n + 1);
  g.z = bi.count;
  if (fp32)
    pdl_launch(prolong_add_kernel<float>, g, dim3(BX, BY), 0, s, (float2*)u, pu, (const float2*)ec, pc, n, stop, bi);
  else
    pdl_launch(prolong_add_kernel<double>, g, dim3(BX, BY), 0, s, (double2*)u, pu, (const double2*)ec, pc, n, stop, bi);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(bool fp32, void* u, int pu, const void* f, int pf, const void* ainvT, int nc,
                                const int* stop, cudaStream_t s, const Inst& bi) {
  int m = (nc + 1) * (nc + 1);
  int threads = m < 256 ? ((m + 31) / 32) * 32 : 256;
  dim3 g(1, 1, bi.count);
  if (fp32)
    pdl_launch(coarse_solve_kernel<float>, g, threads, m * sizeof(float2), s, (float2*)u, pu, (const float2*)f, pf,
                                                                       (const float2*)ainvT, nc, stop, bi);
  else
    pdl_launch(coarse_solve_kernel<double>, g, threads, m * sizeof(double2), s, (double2*)u, pu, (const double2*)f, pf,
                                                                         (const double2*)ainvT, nc, stop, bi);
  return cudaGetLastError();
}

cudaError_t launch_import(bool fp32, void* dst, int pd, const double2* src, int ps, int n, double scale,
                          cudaStream_t s) {
  if (fp32)
    pdl_launch(import_kernel<float>, grid2(n + 1, n + 1), dim3(BX, BY), 0, s, (float2*)dst, pd, src, ps, n, scale);
  else
    pdl_launch(import_kernel<double>, grid2(n + 1, n + 1), dim3(BX, BY), 0, s, (double2*)dst, pd, src, ps, n, scale);
  return cudaGetLastError();
}

cudaError_t launch_export(bool fp32, double2* dst, int pd, const void* src, int ps, int n, double scale,
                          const int* stop, cudaStream_t s) {
  if (fp32)
    pdl_launch(export_kernel<float>, grid2(n + 1, n + 1), dim3(BX, BY), 0, s, dst, pd, (const float2*)src, ps, n, scale, stop);
  else
    pdl_launch(export_kernel<double>, grid2(n + 1, n + 1), dim3(BX, BY), 0, s, dst, pd, (const double2*)src, ps, n, scale,
                                                                       stop);
  return cudaGetLastError();
}

cudaError_t launch_inject_kh(bool fp32, void* kh, int pk, const double* k0, int n0, int stride, int nl, double H,
                             cudaStream_t s) {
  if (fp32)
    pdl_launch(inject_kh_kernel<float>, grid2(nl + 1, nl + 1), dim3(BX, BY), 0, s, (float*)kh, pk, k0, n0, stride, nl, H);
  else
    pdl_launch(inject_kh_kernel<double>, grid2(nl + 1, nl + 1), dim3(BX, BY), 0, s, (double*)kh, pk, k0, n0, stride, nl, H);
  return cudaGetLastError();
}

cudaError_t launch_coarse_setup(bool fp32, void* ainvT, double2* work, const void* kh, int pk, int nc, double beta,
                                int* status, cudaStream_t s) {
  if ((nc + 1) * (nc + 1) > 1089) return cudaErrorInvalidValue;
  if (fp32)
    pdl_launch(coarse_setup_kernel<float>, 1, 1024, 0, s, (float2*)ainvT, work, (const float*)kh, pk, nc, beta, status);
  else
    pdl_launch(coarse_setup_kernel<double>, 1, 1024, 0, s, (double2*)ainvT, work, (const double*)kh, pk, nc, beta, status);
  return cudaGetLastError();
}

}  // namespace hz
