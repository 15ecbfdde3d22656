// Device-side helpers shared by the kernels: complex arithmetic in the working precision and
// the 5-point Helmholtz row of the paper's discretisation in h^2-scaled form.
//
// Scaled form: every level stores its equations multiplied by H^2, so a row reads
//   u_E + u_W + u_N + u_S + d_p u_p = f~_p,   f~ = H^2 f,
//   d_p = -4 + (k_p H)^2 (1 + i beta_A) + 2 i s_p (k_p H),
// where s_p is the number of sides of the square the node lies on (0 inside, 1 on an edge,
// 2 at a corner). This is L^H (beta_A = 0) or M^H = L^H + i k^2 beta (Eq. 3) with the
// first-order Sommerfeld condition du/dn - i k u = 0 (Sec. 1) closed by a centred difference:
// the ghost value is u_mirror + 2 i k H u_p, so at the boundary the mirror node's coefficient
// becomes 2 and the diagonal gains 2 i k H per side.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hz {

template <class T> struct cplx_of;
template <> struct cplx_of<double> { using type = double2; };
template <> struct cplx_of<float> { using type = float2; };
template <class T> using c2 = typename cplx_of<T>::type;

template <class T>
__host__ __device__ __forceinline__ c2<T> mk(T re, T im) {
  c2<T> z;
  z.x = re;
  z.y = im;
  return z;
}

// Load a complex element stored as double2 or float2 and convert it to precision T.
template <class T>
__device__ __forceinline__ c2<T> ldc(const double2* p, long long i) {
  double2 v = p[i];
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ __forceinline__ c2<T> ldc(const float2* p, long long i) {
  float2 v = p[i];
  return mk<T>((T)v.x, (T)v.y);
}
template <class T>
__device__ __forceinline__ void stc(double2* p, long long i, c2<T> v) {
  p[i] = make_double2((double)v.x, (double)v.y);
}
template <class T>
__device__ __forceinline__ void stc(float2* p, long long i, c2<T> v) {
  p[i] = make_float2((float)v.x, (float)v.y);
}

template <class T> __device__ __forceinline__ c2<T> cadd(c2<T> a, c2<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <class T> __device__ __forceinline__ c2<T> csub(c2<T> a, c2<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <class T> __device__ __forceinline__ c2<T> cscale(c2<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <class T>
__device__ __forceinline__ c2<T> cmul(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
template <class T>
__device__ __forceinline__ c2<T> cmulc(c2<T> a, c2<T> b) {
  return mk<T>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
template <class T>
__device__ __forceinline__ c2<T> cdiv(c2<T> a, c2<T> b) {
  T inv = (T)1 / (b.x * b.x + b.y * b.y);
  return mk<T>((a.x * b.x + a.y * b.y) * inv, (a.y * b.x - a.x * b.y) * inv);
}
template <class T> __device__ __forceinline__ T cabs2(c2<T> a) { return a.x * a.x + a.y * a.y; }

// Diagonal of the scaled row at a node with kh = k_p H on `sides` sides of the square.
template <class T>
__device__ __forceinline__ c2<T> row_diag(T kh, int sides, T beta) {
  T kh2 = kh * kh;
  return mk<T>(kh2 - (T)4, beta * kh2 + (T)(2 * sides) * kh);
}

// Neighbour indices of node (i, j) on a grid with n intervals, with out-of-domain neighbours
// replaced by their mirror nodes (ghost elimination).
struct Nbr {
  int iw, ie, js, jn, sides;
};
__device__ __forceinline__ Nbr neighbours(int i, int j, int n) {
  Nbr b;
  b.iw = i > 0 ? i - 1 : 1;
  b.ie = i < n ? i + 1 : n - 1;
  b.js = j > 0 ? j - 1 : 1;
  b.jn = j < n ? j + 1 : n - 1;
  b.sides = (i == 0) + (i == n) + (j == 0) + (j == n);
  return b;
}

__device__ __forceinline__ int reflect(int i, int n) {
  i = i < 0 ? -i : i;
  return i > n ? 2 * n - i : i;
}

}  // namespace hz
